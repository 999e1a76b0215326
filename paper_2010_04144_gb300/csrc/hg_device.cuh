// hg_device.cuh -- device code of the stream-collide kernel, shared by the
// translation units that instantiate it (hg_sc_part.cu, compiled once per storage
// type, scheme and launch parity, in parallel) and by hg_kernels.cu,
// whose read-back and boundary kernels use the same lattice tables, storage
// traits and collision.  Everything here has internal linkage, so each
// translation unit owns the instantiations it makes.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "hg_internal.h"

namespace hg {
namespace {


// ---- D3Q19 (rest; +x,-x,+y,-y,+z,-z; 12 diagonals in opposite pairs) ----
__host__ __device__ constexpr int CX(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
         : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int CY(int i) {
    return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
         : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int CZ(int i) {
    return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
         : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
}
__host__ __device__ constexpr int OPP(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr float W(int i) {
    return i == 0 ? (1.0f / 3.0f) : (i <= 6 ? (1.0f / 18.0f) : (1.0f / 36.0f));
}
__host__ __device__ constexpr double WD(int i) {
    return i == 0 ? (1.0 / 3.0) : (i <= 6 ? (1.0 / 18.0) : (1.0 / 36.0));
}

// Lattice weights in FP32 as an unevaluated sum hi + lo (hi = w rounded to FP32,
// lo = the remainder rounded to FP32): a product w x is formed as fma(hi, x, lo x),
// good to about one rounding of the product.  With w rounded once to FP32 every
// product would carry the weight's own relative error (up to 3e-8, the same sign at
// every site and step), so the FP32 equilibrium would gain or lose mass and momentum
// by that fraction in every collision -- a bias that accumulates over thousands of
// steps, where the rounding of the products themselves varies and averages out.
__host__ __device__ constexpr float WLO(int i) { return (float)(WD(i) - (double)W(i)); }
template <int I> __device__ __forceinline__ float mulw(float x) {
    return __fmaf_rn(W(I), x, __fmul_rn(WLO(I), x));
}

// ---- storage traits ----
// ld/st convert between storage and the collision variable: FP32 stores f~ and
// collides on f~; FP16/BF16 store h = f~/w (avoids subnormals) and collide on h
// directly (collide_scaled), so no per-value scaling is executed.  phys gives
// the physical deviation f~ for read-back.
template <int S> struct St;
template <> struct St<kF32> {
    using T = float;
    static constexpr bool kScaled = false;
    template <int I> static __device__ __forceinline__ float ld(T v) { return v; }
    template <int I> static __device__ __forceinline__ T st(float v) { return v; }
    template <int I> static __device__ __forceinline__ float phys(T v) { return v; }
    static __device__ __forceinline__ double ldd(T v, int) { return (double)v; }
};
template <> struct St<kF16> {
    using T = __half;
    static constexpr bool kScaled = true;
    template <int I> static __device__ __forceinline__ float ld(T v) { return __half2float(v); }
    template <int I> static __device__ __forceinline__ T st(float v) { return __float2half_rn(v); }
    template <int I> static __device__ __forceinline__ float phys(T v) { return mulw<I>(__half2float(v)); }
    static __device__ __forceinline__ double ldd(T v, int i) { return __dmul_rn((double)__half2float(v), WD(i)); }
};
template <> struct St<kBF16> {
    using T = __nv_bfloat16;
    static constexpr bool kScaled = true;
    template <int I> static __device__ __forceinline__ float ld(T v) { return __bfloat162float(v); }
    template <int I> static __device__ __forceinline__ T st(float v) { return __float2bfloat16_rn(v); }
    template <int I> static __device__ __forceinline__ float phys(T v) { return mulw<I>(__bfloat162float(v)); }
    static __device__ __forceinline__ double ldd(T v, int i) { return __dmul_rn((double)__bfloat162float(v), WD(i)); }
};

template <int N> struct IC { static constexpr int v = N; };
template <int B, int E, typename F> __device__ __forceinline__ void unroll(F &&f) {
    if constexpr (B < E) {
        f(IC<B>{});
        unroll<B + 1, E>(f);
    }
}

// Iolet rule for link I of a site next to iolet k (boundary slot `slot`); raw =
// the site's own post-collision value leaving towards x - c_I (direction opp(I)),
// in the collision variable.  Scaled storage (h = f~/w) drops the w_I factors
// (w_I = w_opp(I)); its velocity coefficients are stored divided by w_I.
template <int I, bool SC>
__device__ __forceinline__ float iolet_rule(const DomDev &D, int k, int slot, float raw) {
    const float val = D.bcv[k];
    if (D.io_kind[k] == 0) return -raw + (SC ? 2.0f * val : mulw<I>(2.0f * val));  // anti-bounce-back
    return raw + val * D.coef[(int64_t)slot * 18 + (I - 1)];              // moving wall
}

// LBGK collision in deviation form, in place on g[19]; returns (drho, u).
// Every product and sum is written with explicit rounding intrinsics (__fmul_rn,
// __fadd_rn, __fmaf_rn), so the compiler cannot contract them differently in the
// different kernels that inline this: all variants produce the same bits.
#define HG_MUL __fmul_rn
#define HG_ADD __fadd_rn
#define HG_SUB __fsub_rn
#define HG_FMA __fmaf_rn

// SC: the scaled variable h = f~/w (16-bit storage), whose equilibrium carries no
// weight; otherwise f~, whose equilibrium is w times that (split-weight products).
template <bool SC>
__device__ __forceinline__ void relax_pairs(float g[19], float omega, float base, float rho,
                                            float ux, float uy, float uz) {
    const float r45 = HG_MUL(4.5f, rho), r3 = HG_MUL(3.0f, rho);
    auto pair = [&](auto ia, int b, float cu) {
        constexpr int a = decltype(ia)::v;
        const float q = HG_FMA(HG_MUL(r45, cu), cu, base);    // base + 4.5 rho cu^2
        const float c3 = HG_MUL(r3, cu);
        const float sym = SC ? q : mulw<a>(q);
        const float asym = SC ? c3 : mulw<a>(c3);
        g[a] = HG_FMA(omega, HG_SUB(HG_ADD(sym, asym), g[a]), g[a]);
        g[b] = HG_FMA(omega, HG_SUB(HG_SUB(sym, asym), g[b]), g[b]);
    };
    pair(IC<1>{}, 2, ux);
    pair(IC<3>{}, 4, uy);
    pair(IC<5>{}, 6, uz);
    pair(IC<7>{}, 8, HG_ADD(ux, uy));
    pair(IC<9>{}, 10, HG_SUB(ux, uy));
    pair(IC<11>{}, 12, HG_ADD(ux, uz));
    pair(IC<13>{}, 14, HG_SUB(ux, uz));
    pair(IC<15>{}, 16, HG_ADD(uy, uz));
    pair(IC<17>{}, 18, HG_SUB(uy, uz));
}

struct Moments {
    float drho, ux, uy, uz, rho, base;
};

// u, rho and the equilibrium's isotropic part from drho and j.
__device__ __forceinline__ Moments finish_moments(float drho, float jx, float jy, float jz) {
    Moments m;
    m.drho = drho;
    m.rho = HG_ADD(1.0f, drho);
    const float inv = __frcp_rn(m.rho);
    m.ux = HG_MUL(jx, inv);
    m.uy = HG_MUL(jy, inv);
    m.uz = HG_MUL(jz, inv);
    const float usq = HG_FMA(m.ux, m.ux, HG_FMA(m.uy, m.uy, HG_MUL(m.uz, m.uz)));
    m.base = HG_FMA(HG_MUL(-1.5f, m.rho), usq, drho);       // drho - 1.5 rho u.u
    return m;
}

__device__ __forceinline__ float4 collide(float g[19], float omega) {
    float drho = g[0];
#pragma unroll
    for (int i = 1; i < 19; ++i) drho = HG_ADD(drho, g[i]);
    const float d12 = HG_SUB(g[1], g[2]), d34 = HG_SUB(g[3], g[4]), d56 = HG_SUB(g[5], g[6]);
    const float d78 = HG_SUB(g[7], g[8]), d910 = HG_SUB(g[9], g[10]), d1112 = HG_SUB(g[11], g[12]);
    const float d1314 = HG_SUB(g[13], g[14]), d1516 = HG_SUB(g[15], g[16]), d1718 = HG_SUB(g[17], g[18]);
    const float jx = HG_ADD(HG_ADD(HG_ADD(d12, d78), HG_ADD(d910, d1112)), d1314);
    const float jy = HG_ADD(HG_ADD(HG_SUB(HG_ADD(d34, d78), d910), d1516), d1718);
    const float jz = HG_SUB(HG_ADD(HG_SUB(HG_ADD(d56, d1112), d1314), d1516), d1718);
    const Moments m = finish_moments(drho, jx, jy, jz);
    g[0] = HG_FMA(omega, HG_SUB(mulw<0>(m.base), g[0]), g[0]);
    relax_pairs<false>(g, omega, m.base, m.rho, m.ux, m.uy, m.uz);
    return make_float4(m.drho, m.ux, m.uy, m.uz);
}

// The same collision in the scaled variable h_i = f~_i / w_i (16-bit storage):
// moments weight h by w, the equilibrium h~eq_i = drho + rho (3 c.u + 4.5 (c.u)^2
// - 1.5 u.u) carries no w.
__device__ __forceinline__ float4 collide_scaled(float g[19], float omega) {
    const float sa = HG_ADD(HG_ADD(HG_ADD(g[1], g[2]), HG_ADD(g[3], g[4])), HG_ADD(g[5], g[6]));
    const float sd = HG_ADD(HG_ADD(HG_ADD(HG_ADD(g[7], g[8]), HG_ADD(g[9], g[10])),
                                   HG_ADD(HG_ADD(g[11], g[12]), HG_ADD(g[13], g[14]))),
                            HG_ADD(HG_ADD(g[15], g[16]), HG_ADD(g[17], g[18])));
    const float drho = HG_ADD(mulw<0>(g[0]), HG_ADD(mulw<1>(sa), mulw<7>(sd)));
    const float d12 = HG_SUB(g[1], g[2]), d34 = HG_SUB(g[3], g[4]), d56 = HG_SUB(g[5], g[6]);
    const float d78 = HG_SUB(g[7], g[8]), d910 = HG_SUB(g[9], g[10]), d1112 = HG_SUB(g[11], g[12]);
    const float d1314 = HG_SUB(g[13], g[14]), d1516 = HG_SUB(g[15], g[16]), d1718 = HG_SUB(g[17], g[18]);
    const float ex = HG_ADD(HG_ADD(d78, d910), HG_ADD(d1112, d1314));
    const float ey = HG_ADD(HG_SUB(d78, d910), HG_ADD(d1516, d1718));
    const float ez = HG_ADD(HG_SUB(d1112, d1314), HG_SUB(d1516, d1718));
    const float jx = HG_ADD(mulw<1>(d12), mulw<7>(ex));
    const float jy = HG_ADD(mulw<1>(d34), mulw<7>(ey));
    const float jz = HG_ADD(mulw<1>(d56), mulw<7>(ez));
    const Moments m = finish_moments(drho, jx, jy, jz);
    g[0] = HG_FMA(omega, HG_SUB(m.base, g[0]), g[0]);
    relax_pairs<true>(g, omega, m.base, m.rho, m.ux, m.uy, m.uz);
    return make_float4(m.drho, m.ux, m.uy, m.uz);
}

template <int S> __device__ __forceinline__ float4 collide_s(float g[19], float omega) {
    if constexpr (St<S>::kScaled) return collide_scaled(g, omega);
    else return collide(g, omega);
}


// A pointer the compiler cannot see through: loads from it are not merged with
// earlier loads from the same address.
template <typename T> __device__ __forceinline__ const T *opaque_ptr(const T *p) {
    const T *q;
    asm volatile("mov.b64 %0, %1;" : "=l"(q) : "l"(p));
    return q;
}

template <typename T> __device__ __forceinline__ T ldg_nc(const T *p) { return __ldg(p); }
template <> __device__ __forceinline__ __half ldg_nc(const __half *p) {
    return __ushort_as_half(__ldg(reinterpret_cast<const unsigned short *>(p)));
}
template <> __device__ __forceinline__ __nv_bfloat16 ldg_nc(const __nv_bfloat16 *p) {
    return __ushort_as_bfloat16(__ldg(reinterpret_cast<const unsigned short *>(p)));
}

// Loads carrying an L2 prefetch-size hint (256 B): a miss fetches the whole
// 256-byte span, which neighbouring warps' gathers then hit.  ld_ro: read-only
// data (non-coherent path); ld_rw: data this kernel also writes (AA).
template <typename T> struct HintLd;
template <> struct HintLd<float> {
    static __device__ __forceinline__ float ro(const float *p) {
        float v;
        asm("ld.global.nc.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
        return v;
    }
    static __device__ __forceinline__ float rw(const float *p) {
        float v;
        asm("ld.global.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p) : "memory");
        return v;
    }
};
template <> struct HintLd<int32_t> {
    static __device__ __forceinline__ int32_t ro(const int32_t *p) {
        int32_t v;
        asm("ld.global.nc.L2::256B.s32 %0, [%1];" : "=r"(v) : "l"(p));
        return v;
    }
};
template <typename H> struct HintLd16 {
    static __device__ __forceinline__ H ro(const H *p) {
        unsigned short v;
        asm("ld.global.nc.L2::256B.b16 %0, [%1];" : "=h"(v) : "l"(p));
        return *reinterpret_cast<H *>(&v);
    }
    static __device__ __forceinline__ H rw(const H *p) {
        unsigned short v;
        asm("ld.global.L2::256B.b16 %0, [%1];" : "=h"(v) : "l"(p) : "memory");
        return *reinterpret_cast<H *>(&v);
    }
};
template <> struct HintLd<__half> : HintLd16<__half> {};
template <> struct HintLd<__nv_bfloat16> : HintLd16<__nv_bfloat16> {};

template <bool HINT, typename T> __device__ __forceinline__ T load_ro(const T *p) {
    if constexpr (HINT) return HintLd<T>::ro(p);
    else return ldg_nc(p);
}
template <bool HINT> __device__ __forceinline__ int32_t load_nbr(const int32_t *p) {
    if constexpr (HINT) return HintLd<int32_t>::ro(p);
    else return __ldg(p);
}
template <bool HINT, typename T> __device__ __forceinline__ T load_rw(const T *p) {
    if constexpr (HINT) return HintLd<T>::rw(p);
    else return *p;
}

// ---- neighbour entries of a site: the 18-row table or its run encoding ----
// Both give the same int32 entry for link I (1..18): the fluid neighbour's device
// index, or for a non-fluid link the virtual index s + dd np with dd = opp(I) - I
// (A/B) or I - opp(I) (AA).  TabNb reads row I-1 of the table (72 bytes per site
// in all); RunNb reads one word per site (non-fluid flags, run within the chunk),
// the chunk's first run and the run's 80-byte row of offsets, which the run's other
// sites also read (L1 hits): about 4 + 80 / run-length bytes per site.
// RunNb::reload() gives an accessor whose next reads are not merged with earlier
// ones, so a scatter after the collision re-reads (cache hits) instead of keeping
// 18 entries in registers.
template <bool HINT> struct TabNb {
    const int32_t *p;
    int64_t np;
    __device__ __forceinline__ TabNb(const DomDev &D, int64_t s) : p(D.nbr + s), np(D.np) {}
    __device__ __forceinline__ void all(int32_t nb[18]) const {
#pragma unroll
        for (int i = 0; i < 18; ++i) nb[i] = load_nbr<HINT>(p + (int64_t)i * np);
    }
};
template <int SCHEME, bool HINT> struct RunNb {
    uint32_t w;
    const int32_t *rd;
    int32_t s, np;
    __device__ __forceinline__ RunNb(const DomDev &D, int64_t s_) : s((int32_t)s_), np((int32_t)D.np) {
        w = (uint32_t)load_nbr<HINT>(reinterpret_cast<const int32_t *>(D.lword) + s_);
        rd = D.rdelta + (int64_t)(__ldg(D.run0 + (s_ >> 10)) + (int32_t)(w >> 18)) * kRunStride;
    }
    __device__ __forceinline__ RunNb(uint32_t w_, const int32_t *rd_, int32_t s_, int32_t np_)
        : w(w_), rd(rd_), s(s_), np(np_) {}
    // all 18 entries: the run's row as five 16-byte loads
    __device__ __forceinline__ void all(int32_t nb[18]) const {
        int32_t d[kRunStride];
#pragma unroll
        for (int k = 0; k < kRunStride / 4; ++k) {
            const int4 v = __ldg(reinterpret_cast<const int4 *>(rd) + k);
            d[4 * k] = v.x;
            d[4 * k + 1] = v.y;
            d[4 * k + 2] = v.z;
            d[4 * k + 3] = v.w;
        }
        unroll<1, 19>([&](auto ic) {
            constexpr int I = decltype(ic)::v;
            constexpr int dd = SCHEME == kAA ? I - OPP(I) : OPP(I) - I;
            nb[I - 1] = ((w >> (I - 1)) & 1u) ? s + dd * np : s + d[I - 1];
        });
    }
    __device__ __forceinline__ RunNb reload() const { return RunNb(w, opaque_ptr(rd), s, np); }
    // bring the run's row into L1 ahead of all(): its 80 bytes span at most two lines
    __device__ __forceinline__ void prefetch() const {
        asm volatile("prefetch.global.L1 [%0];" ::"l"(rd));
        asm volatile("prefetch.global.L1 [%0];" ::"l"(rd + kRunStride - 1));
    }
};
// The same for a pair of adjacent sites s, s+1 (s even: both in one 1024-site
// chunk): one 8-byte load of both table entries, or of both words; a run shared
// by the two (the usual case) is read once.
template <bool HINT> struct TabNb2 {
    const int32_t *p;
    int64_t np;
    __device__ __forceinline__ TabNb2(const DomDev &D, int64_t s) : p(D.nbr + s), np(D.np) {}
    template <int I> __device__ __forceinline__ int2 at() const {
        return __ldg(reinterpret_cast<const int2 *>(p + (int64_t)(I - 1) * np));
    }
};
template <int SCHEME> struct RunNb2 {
    uint32_t wa, wb;
    const int32_t *ra, *rb;
    int32_t s, np;
    __device__ __forceinline__ RunNb2(const DomDev &D, int64_t s_) : s((int32_t)s_), np((int32_t)D.np) {
        const uint2 w = __ldg(reinterpret_cast<const uint2 *>(D.lword + s_));
        const int32_t r0 = __ldg(D.run0 + (s_ >> 10));
        wa = w.x;
        wb = w.y;
        ra = D.rdelta + (int64_t)(r0 + (int32_t)(w.x >> 18)) * kRunStride;
        rb = D.rdelta + (int64_t)(r0 + (int32_t)(w.y >> 18)) * kRunStride;
    }
    template <int I> __device__ __forceinline__ int2 at() const {
        constexpr int dd = SCHEME == kAA ? I - OPP(I) : OPP(I) - I;
        const int32_t da = __ldg(ra + (I - 1));
        const int32_t db = ra == rb ? da : __ldg(rb + (I - 1));
        return make_int2(((wa >> (I - 1)) & 1u) ? s + dd * np : s + da,
                         ((wb >> (I - 1)) & 1u) ? s + 1 + dd * np : s + 1 + db);
    }
};
template <int SCHEME, bool HINT, bool RUNS>
using NbOf = typename std::conditional<RUNS, RunNb<SCHEME, HINT>, TabNb<HINT>>::type;
template <int SCHEME, bool RUNS>
using Nb2Of = typename std::conditional<RUNS, RunNb2<SCHEME>, TabNb2<false>>::type;

// ---- sites next to an iolet (rare path) ----
// Neighbour table entries of non-fluid links hold a virtual index that makes
// the ordinary address formula land on the site's own opposite slot, so a wall
// needs no code at all.  Sites with a link into an iolet opening are flagged in
// `iomask`; their slot is the rank of the flag (per-32-site prefix + popcount)
// and their canonical link codes sit in io_codes[slot][18].
__device__ __forceinline__ bool site_flag(const DomDev &D, int64_t s, uint32_t &word) {
    word = __ldg(D.iomask + (s >> 5));
    return (word >> (s & 31)) & 1u;
}
__device__ __forceinline__ int site_slot(const DomDev &D, int64_t s, uint32_t word) {
    return __ldg(D.ioprefix + (s >> 5)) + __popc(word & ((1u << (s & 31)) - 1u));
}
template <int S>
__device__ __forceinline__ void apply_iolet_links(const DomDev &D, int slot, float g[19]) {
    const int32_t *codes = D.io_codes + (int64_t)slot * 18;
    unroll<1, 19>([&](auto ic) {
        constexpr int I = decltype(ic)::v;
        const int32_t c = __ldg(codes + (I - 1));
        if (c < -1) g[I] = iolet_rule<I, St<S>::kScaled>(D, -c - 2, slot, g[I]);
    });
}
// A stream-collide launch may start while the previous step's iolet update is
// still running (programmatic dependent launch): everything it reads except the
// boundary values was complete before that update began.  Only the sites with
// an iolet link use those values (and overwrite the moments slot the update
// reads), so only they wait here for the update to finish.  Without an
// overlapping launch the wait returns at once.
__device__ __forceinline__ void wait_for_iolet_update() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <int S>
__device__ __forceinline__ int iolet_fixup(const DomDev &D, int64_t s, float g[19]) {
    uint32_t word;
    if (!site_flag(D, s, word)) return -1;
    wait_for_iolet_update();
    const int slot = site_slot(D, s, word);
    apply_iolet_links<S>(D, slot, g);
    return slot;
}

template <typename T> __device__ __forceinline__ T *opaque(T *p) {
    T *q;
    asm volatile("mov.b64 %0, %1;" : "=l"(q) : "l"(p));
    return q;
}

// ---- A/B pull: F_{t-1} in src, F_t to dst ----
template <int S, bool HINT = false, bool RUNS = false>
__device__ __forceinline__ void site_ab(const DomDev &D, const typename St<S>::T *__restrict__ src,
                                        typename St<S>::T *__restrict__ dst, int64_t s);

// The A/B site update with the site's neighbour accessor already made.
template <int S, bool HINT, typename NB>
__device__ __forceinline__ void site_ab_with(const DomDev &D, const typename St<S>::T *__restrict__ src,
                                             typename St<S>::T *__restrict__ dst, int64_t s, const NB &tab) {
    using Tr = St<S>;
    const int64_t np = D.np;
    int32_t nb[18];
    tab.all(nb);
    float g[19];
    g[0] = Tr::template ld<0>(load_ro<HINT>(src + s));
    unroll<1, 19>([&](auto ic) {  // virtual indices: walls read their own opposite value
        constexpr int I = decltype(ic)::v;
        g[I] = Tr::template ld<I>(load_ro<HINT>(src + ((int64_t)I * np + nb[I - 1])));
    });
    const int slot = iolet_fixup<S>(D, s, g);
    const float4 m = collide_s<S>(g, D.omega);
    unroll<0, 19>([&](auto ic) {
        constexpr int I = decltype(ic)::v;
        dst[(int64_t)I * np + s] = Tr::template st<I>(g[I]);
    });
    if (slot >= 0) D.bnd[slot] = m;
}

template <int S, bool HINT, bool RUNS>
__device__ __forceinline__ void site_ab(const DomDev &D, const typename St<S>::T *__restrict__ src,
                                        typename St<S>::T *__restrict__ dst, int64_t s) {
    site_ab_with<S, HINT>(D, src, dst, s, NbOf<kAB, HINT, RUNS>(D, s));
}

// ---- AA even step: state G_t natural at the own site -> F_t swapped at the own site ----
// The store base is passed through an opaque move so the compiler recomputes
// the 19 store addresses after the collision instead of keeping the load
// addresses alive across it (75 -> ~45 registers).
template <int S, bool HINT = false>
__device__ __forceinline__ void site_aa_even(const DomDev &D, typename St<S>::T *buf, int64_t s) {
    using Tr = St<S>;
    const int64_t np = D.np;
    float g[19];
    unroll<0, 19>([&](auto ic) {
        constexpr int I = decltype(ic)::v;
        g[I] = Tr::template ld<I>(load_rw<HINT>(buf + (int64_t)I * np + s));
    });
    const int slot = iolet_fixup<S>(D, s, g);  // the odd step left raw values on iolet links
    const float4 m = collide_s<S>(g, D.omega);
    typename St<S>::T *wb = opaque(buf + s);
    unroll<0, 19>([&](auto ic) {
        constexpr int I = decltype(ic)::v;
        wb[(int64_t)OPP(I) * np] = Tr::template st<I>(g[I]);
    });
    if (slot >= 0) D.bnd[slot] = m;
}

// ---- AA odd step: gather F_{t-1} (swapped) from x - c_i, scatter F_t to x + c_i ----
// Entry OPP(I) of the site's row is the site at x + c_I; its virtual index for
// a non-fluid link turns the scatter into the raw write to the own slot OPP(I).
template <int S, bool HINT, bool RUNS, bool STASH, typename NB>
__device__ __forceinline__ void site_aa_odd_with(const DomDev &D, typename St<S>::T *buf, int64_t s,
                                                 const NB &tab, int32_t *stash = nullptr) {
    using Tr = St<S>;
    const int64_t np = D.np;
    int32_t nb[18];
    tab.all(nb);
    if constexpr (STASH) {  // 19 words per thread (odd stride: no bank conflicts), 18 used
        stash += 19 * threadIdx.x;
#pragma unroll
        for (int i = 0; i < 18; ++i) stash[i] = nb[i];
        asm volatile("" ::: "memory");  // the stash stores stay ahead of the gathers
    }
    float g[19];
    g[0] = Tr::template ld<0>(load_rw<HINT>(buf + s));
    unroll<1, 19>([&](auto ic) {
        constexpr int I = decltype(ic)::v;
        g[I] = Tr::template ld<I>(load_rw<HINT>(buf + ((int64_t)OPP(I) * np + nb[I - 1])));
    });
    const int slot = iolet_fixup<S>(D, s, g);
    const float4 m = collide_s<S>(g, D.omega);
    typename St<S>::T *wb = opaque(buf);
    // the scatter addresses are the gather addresses (entry OPP(I) of the site at x +
    // c_I): STASH takes the 18 entries back from shared memory, otherwise they are
    // decoded again (cache hits); either frees 18 registers across the collision
    wb[s] = Tr::template st<0>(g[0]);
    if constexpr (RUNS || STASH) {
        if constexpr (STASH) {
            // the stash address is known only once the collision has produced m: the
            // reads cannot move above it, so the entries are not live across it
            int32_t *st2;
            asm volatile("{\n\t.reg .f32 t;\n\tmov.f32 t, %2;\n\tmov.b64 %0, %1;\n\t}"
                         : "=l"(st2) : "l"(stash), "f"(m.x) : "memory");
#pragma unroll
            for (int i = 0; i < 18; ++i) nb[i] = st2[i];
        } else {
            tab.reload().all(nb);
        }
        unroll<1, 19>([&](auto ic) {
            constexpr int I = decltype(ic)::v;
            wb[(int64_t)I * np + nb[OPP(I) - 1]] = Tr::template st<I>(g[I]);
        });
    } else {  // table: each store's entry reread right before it
        const int32_t *nb2 = opaque(D.nbr);
        unroll<1, 19>([&](auto ic) {
            constexpr int I = decltype(ic)::v;
            wb[(int64_t)I * np + __ldg(nb2 + (int64_t)(OPP(I) - 1) * np + s)] = Tr::template st<I>(g[I]);
        });
    }
    if (slot >= 0) D.bnd[slot] = m;
}

template <int S, bool HINT = false, bool RUNS = false, bool STASH = false>
__device__ __forceinline__ void site_aa_odd(const DomDev &D, typename St<S>::T *buf, int64_t s,
                                            int32_t *stash = nullptr) {
    site_aa_odd_with<S, HINT, RUNS, STASH>(D, buf, s, NbOf<kAA, HINT, RUNS>(D, s), stash);
}

// ==== async-staged variant (V = 1) ==========================================
// The 19 gathers of every site a thread owns are issued as cp.async copies into
// a shared-memory stage [SPT][19][blockDim] (4-byte words) before one wait, so
// the loads in flight do not hold registers.  16-bit elements are fetched as
// the aligned 32-bit word that contains them; `sel` remembers which half.
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

template <int S> struct Word;
template <> struct Word<kF32> {
    static __device__ __forceinline__ const void *src(const float *p, uint32_t &sel, int) {
        return p;
    }
    template <int I> static __device__ __forceinline__ float get(uint32_t w, uint32_t) {
        return __uint_as_float(w);
    }
};
template <int S16> struct Word16 {
    using T = typename St<S16>::T;
    static __device__ __forceinline__ const void *src(const T *p, uint32_t &sel, int I) {
        const uintptr_t a = (uintptr_t)p;
        sel |= (uint32_t)((a >> 1) & 1u) << I;
        return (const void *)(a & ~(uintptr_t)3);
    }
    template <int I> static __device__ __forceinline__ float get(uint32_t w, uint32_t sel) {
        const unsigned short h = (unsigned short)(((sel >> I) & 1u) ? (w >> 16) : (w & 0xffffu));
        if constexpr (S16 == kF16) return St<kF16>::template ld<I>(__ushort_as_half(h));
        else return St<kBF16>::template ld<I>(__ushort_as_bfloat16(h));
    }
};
template <> struct Word<kF16> : Word16<kF16> {};
template <> struct Word<kBF16> : Word16<kBF16> {};

// Issue the gathers of site s (virtual indices: one formula for every link).
// A/B pulls slot I from x - c_I; AA odd pulls the swapped slot OPP(I).
template <int S, bool AA>
__device__ __forceinline__ uint32_t issue_gathers(const DomDev &D, const typename St<S>::T *src,
                                                  int64_t s, uint32_t stage, uint32_t rstride) {
    const int64_t np = D.np;
    uint32_t sel = 0;
    int32_t nb[18];
#pragma unroll
    for (int i = 0; i < 18; ++i) nb[i] = __ldg(D.nbr + (int64_t)i * np + s);
    cp_async4(stage, Word<S>::src(src + s, sel, 0));
    unroll<1, 19>([&](auto ic) {
        constexpr int I = decltype(ic)::v;
        const typename St<S>::T *p = src + ((int64_t)(AA ? OPP(I) : I) * np + nb[I - 1]);
        cp_async4(stage + I * rstride, Word<S>::src(p, sel, I));
    });
    return sel;
}

template <int S>
__device__ __forceinline__ void read_staged(const uint32_t *st, uint32_t rwords, uint32_t sel,
                                            float g[19]) {
    unroll<0, 19>([&](auto ic) {
        constexpr int I = decltype(ic)::v;
        g[I] = Word<S>::template get<I>(st[I * rwords], sel);
    });
}

template <int S, int SPT>
__device__ __forceinline__ void tile_ab_async(const DomDev &D, const TileDev &tl, bool odd,
                                              uint32_t *stage_base) {
    using T = typename St<S>::T;
    const T *src = (const T *)D.f[odd ? 0 : 1];  // F_{t-1} sits in f[(t-1) & 1]
    T *dst = (T *)D.f[odd ? 1 : 0];
    const uint32_t B = blockDim.x;
    uint32_t sel[SPT];
#pragma unroll
    for (int j = 0; j < SPT; ++j) {
        const int r = j * B + threadIdx.x;
        sel[j] = r < tl.count ? issue_gathers<S, false>(D, src, tl.start + r,
                                                        smem_addr(stage_base + (j * 19) * B + threadIdx.x), 4 * B)
                              : 0u;
    }
    cp_async_wait_all();
#pragma unroll
    for (int j = 0; j < SPT; ++j) {
        const int r = j * B + threadIdx.x;
        if (r >= tl.count) continue;
        const int64_t s = tl.start + r;
        float g[19];
        read_staged<S>(stage_base + (j * 19) * B + threadIdx.x, B, sel[j], g);
        const int slot = iolet_fixup<S>(D, s, g);
        const float4 m = collide_s<S>(g, D.omega);
        T *wb = opaque(dst + s);
        unroll<0, 19>([&](auto ic) {
            constexpr int I = decltype(ic)::v;
            wb[(int64_t)I * D.np] = St<S>::template st<I>(g[I]);
        });
        if (slot >= 0) D.bnd[slot] = m;
    }
}

template <int S, int SPT>
__device__ __forceinline__ void tile_aa_odd_async(const DomDev &D, const TileDev &tl,
                                                  uint32_t *stage_base) {
    using T = typename St<S>::T;
    T *buf = (T *)D.f[0];
    const uint32_t B = blockDim.x;
    uint32_t sel[SPT];
#pragma unroll
    for (int j = 0; j < SPT; ++j) {
        const int r = j * B + threadIdx.x;
        sel[j] = r < tl.count ? issue_gathers<S, true>(D, buf, tl.start + r,
                                                       smem_addr(stage_base + (j * 19) * B + threadIdx.x), 4 * B)
                              : 0u;
    }
    cp_async_wait_all();
#pragma unroll
    for (int j = 0; j < SPT; ++j) {
        const int r = j * B + threadIdx.x;
        if (r >= tl.count) continue;
        const int64_t s = tl.start + r;
        float g[19];
        read_staged<S>(stage_base + (j * 19) * B + threadIdx.x, B, sel[j], g);
        const int slot = iolet_fixup<S>(D, s, g);
        const float4 m = collide_s<S>(g, D.omega);
        const int32_t *nb2 = opaque(D.nbr);  // fresh (L1-resident) reads for the scatter
        T *wb = opaque(buf);
        const int64_t np = D.np;
        wb[s] = St<S>::template st<0>(g[0]);
        unroll<1, 19>([&](auto ic) {
            constexpr int I = decltype(ic)::v;
            const int32_t tg = __ldg(nb2 + (int64_t)(OPP(I) - 1) * np + s);  // site at x + c_I
            wb[(int64_t)I * np + tg] = St<S>::template st<I>(g[I]);
        });
        if (slot >= 0) D.bnd[slot] = m;
    }
}

// ==== staged-scatter AA odd step (V = 4, one site per thread) ===============
// The odd step stores the value of direction I at x + c_I.  Most of those
// targets lie in the same tile: their values are parked in the gather stage
// (free once every thread has read its gathers) at the target's position and
// then written row by row with coalesced stores.  A target outside the tile
// gets its value directly; a non-fluid target parks the raw value at the own
// site's slot OPP(I).  Position p's row-I value comes from the pull source of
// direction I at p (its own neighbour-table entry I), or from p itself when
// that entry is virtual; entry I is also the target entry of p's own
// direction OPP(I), so the scatter pass records in one bit per row whether the
// tile holds position p's value.  Each location is read and written by one
// site only (the AA property), so the deferred stores race with no other tile.
template <int S>
__device__ __forceinline__ void tile_aa_odd_staged(const DomDev &D, const TileDev &tl, uint32_t *stage) {
    using T = typename St<S>::T;
    T *buf = (T *)D.f[0];
    const uint32_t B = blockDim.x;
    const int r = threadIdx.x;
    const bool live = r < tl.count;
    const int64_t s = tl.start + r;
    const int64_t np = D.np;
    const uint32_t sel = live ? issue_gathers<S, true>(D, buf, s, smem_addr(stage + r), 4 * B) : 0u;
    cp_async_wait_all();
    float g[19];
    int slot = -1;
    float4 m = make_float4(0.f, 0.f, 0.f, 0.f);
    if (live) {
        read_staged<S>(stage + r, B, sel, g);
        slot = iolet_fixup<S>(D, s, g);
        m = collide_s<S>(g, D.omega);
    }
    __syncthreads();  // every gather has been read: the stage now takes outputs
    uint32_t held = 0;  // bit J: the tile holds this position's row-J value
    if (live) {
        const int32_t *nb2 = opaque(D.nbr);
        T *wb = opaque(buf);
        wb[s] = St<S>::template st<0>(g[0]);
        unroll<1, 19>([&](auto ic) {
            constexpr int I = decltype(ic)::v;
            const int32_t tg = __ldg(nb2 + (int64_t)(OPP(I) - 1) * np + s);  // site at x + c_I
            const int64_t rel = (int64_t)tg - tl.start;
            if ((uint64_t)rel < (uint64_t)tl.count) {
                stage[I * B + (uint32_t)rel] = __float_as_uint(g[I]);
                held |= 1u << OPP(I);
            } else if (tg < 0 || tg >= np) {
                stage[OPP(I) * B + r] = __float_as_uint(g[I]);
                held |= 1u << OPP(I);
            } else {
                wb[(int64_t)I * np + tg] = St<S>::template st<I>(g[I]);
            }
        });
        if (slot >= 0) D.bnd[slot] = m;
    }
    __syncthreads();
    if (live) {
        T *wb = opaque(buf);
        unroll<1, 19>([&](auto ic) {
            constexpr int I = decltype(ic)::v;
            if ((held >> I) & 1u)
                wb[(int64_t)I * np + s] = St<S>::template st<I>(__uint_as_float(stage[I * B + r]));
        });
    }
}

// AA even step on pairs of adjacent sites (2 per thread): vector loads/stores.
template <int S> struct Pair;
template <> struct Pair<kF32> {
    template <int I> static __device__ __forceinline__ void ld(const float *p, float &a, float &b) {
        const float2 v = *(const float2 *)p;
        a = v.x;
        b = v.y;
    }
    template <int I> static __device__ __forceinline__ void st(float *p, float a, float b) {
        *(float2 *)p = make_float2(a, b);
    }
};
// Two adjacent 16-bit values move as one 4-byte word and convert with the paired
// intrinsics (same round-to-nearest-even as the scalar conversions, so the bits
// are those of every other variant; fewer instructions for kernels near their
// issue limit).
template <int S16> struct Pair16;
template <> struct Pair16<kF16> {
    template <int I> static __device__ __forceinline__ void ld(const __half *p, float &a, float &b) {
        const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(p));
        a = f.x;
        b = f.y;
    }
    template <int I> static __device__ __forceinline__ void st(__half *p, float a, float b) {
        *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(a, b);
    }
};
template <> struct Pair16<kBF16> {
    template <int I> static __device__ __forceinline__ void ld(const __nv_bfloat16 *p, float &a, float &b) {
        const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
        a = f.x;
        b = f.y;
    }
    template <int I> static __device__ __forceinline__ void st(__nv_bfloat16 *p, float a, float b) {
        *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(a, b);
    }
};
template <> struct Pair<kF16> : Pair16<kF16> {};
template <> struct Pair<kBF16> : Pair16<kBF16> {};

// ---- A/B pull on a pair of adjacent sites (variant 5, 16-bit storage) ----
// Sites s and s+1 (s even) share one 8-byte load per neighbour-table row, one
// 4-byte load of the rest values and one 4-byte store per direction: fewer
// memory instructions per site for a kernel that runs near its issue limit.
template <int S, bool RUNS = false>
__device__ __forceinline__ void site_ab_pair(const DomDev &D, const typename St<S>::T *__restrict__ src,
                                             typename St<S>::T *__restrict__ dst, int64_t s) {
    using Tr = St<S>;
    const int64_t np = D.np;
    const Nb2Of<kAB, RUNS> tab(D, s);
    float ga[19], gb[19];
    Pair<S>::template ld<0>(src + s, ga[0], gb[0]);
    unroll<1, 19>([&](auto ic) {
        constexpr int I = decltype(ic)::v;
        const int2 nb = tab.template at<I>();
        ga[I] = Tr::template ld<I>(ldg_nc(src + ((int64_t)I * np + nb.x)));
        gb[I] = Tr::template ld<I>(ldg_nc(src + ((int64_t)I * np + nb.y)));
    });
    const int slot_a = iolet_fixup<S>(D, s, ga);
    const int slot_b = iolet_fixup<S>(D, s + 1, gb);
    const float4 ma = collide_s<S>(ga, D.omega);
    const float4 mb = collide_s<S>(gb, D.omega);
    typename St<S>::T *wb = opaque(dst + s);
    unroll<0, 19>([&](auto ic) {
        constexpr int I = decltype(ic)::v;
        Pair<S>::template st<I>(wb + (int64_t)I * np, ga[I], gb[I]);
    });
    if (slot_a >= 0) D.bnd[slot_a] = ma;
    if (slot_b >= 0) D.bnd[slot_b] = mb;
}

// ---- AA on a pair of adjacent sites (variant 6 / 7: 7 adds L2 prefetch hints) ----
// Sites s and s+1 (s even) share one 8-byte load per neighbour-table row, both for
// the gathers and for the re-read that addresses the scatter, and one load and one
// store of their two rest values; the 18 gathers and 18 scattered stores stay per
// site.  The odd step reads slot OPP(I) at x - c_I and writes slot I at x + c_I.
template <int S, bool HINT>
__device__ __forceinline__ void site_aa_odd_pair(const DomDev &D, typename St<S>::T *buf, int64_t s) {
    using Tr = St<S>;
    const int64_t np = D.np;
    float ga[19], gb[19];
    Pair<S>::template ld<0>(buf + s, ga[0], gb[0]);
    unroll<1, 19>([&](auto ic) {
        constexpr int I = decltype(ic)::v;
        const int2 nb = __ldg(reinterpret_cast<const int2 *>(D.nbr + (int64_t)(I - 1) * np + s));
        ga[I] = Tr::template ld<I>(load_rw<HINT>(buf + ((int64_t)OPP(I) * np + nb.x)));
        gb[I] = Tr::template ld<I>(load_rw<HINT>(buf + ((int64_t)OPP(I) * np + nb.y)));
    });
    const int slot_a = iolet_fixup<S>(D, s, ga);
    const int slot_b = iolet_fixup<S>(D, s + 1, gb);
    const float4 ma = collide_s<S>(ga, D.omega);
    const float4 mb = collide_s<S>(gb, D.omega);
    typename St<S>::T *wb = opaque(buf);
    const int32_t *nb2 = opaque(D.nbr);  // reread (L1 hits) instead of keeping 36 entries live
    Pair<S>::template st<0>(wb + s, ga[0], gb[0]);
    unroll<1, 19>([&](auto ic) {
        constexpr int I = decltype(ic)::v;
        const int2 tg = __ldg(reinterpret_cast<const int2 *>(nb2 + (int64_t)(OPP(I) - 1) * np + s));
        wb[(int64_t)I * np + tg.x] = Tr::template st<I>(ga[I]);
        wb[(int64_t)I * np + tg.y] = Tr::template st<I>(gb[I]);
    });
    if (slot_a >= 0) D.bnd[slot_a] = ma;
    if (slot_b >= 0) D.bnd[slot_b] = mb;
}

// AA even step on the same pairs: local, vector loads and stores of both sites.
template <int S, bool HINT>
__device__ __forceinline__ void site_aa_even_pair(const DomDev &D, typename St<S>::T *buf, int64_t s) {
    const int64_t np = D.np;
    float ga[19], gb[19];
    unroll<0, 19>([&](auto ic) {
        constexpr int I = decltype(ic)::v;
        Pair<S>::template ld<I>(buf + (int64_t)I * np + s, ga[I], gb[I]);
    });
    const int slot_a = iolet_fixup<S>(D, s, ga);
    const int slot_b = iolet_fixup<S>(D, s + 1, gb);
    const float4 ma = collide_s<S>(ga, D.omega);
    const float4 mb = collide_s<S>(gb, D.omega);
    typename St<S>::T *wb = opaque(buf + s);
    unroll<0, 19>([&](auto ic) {
        constexpr int I = decltype(ic)::v;
        Pair<S>::template st<I>(wb + (int64_t)OPP(I) * np, ga[I], gb[I]);
    });
    if (slot_a >= 0) D.bnd[slot_a] = ma;
    if (slot_b >= 0) D.bnd[slot_b] = mb;
}

template <int S>
__device__ __forceinline__ void tile_aa_even_pairs(const DomDev &D, const TileDev &tl) {
    using T = typename St<S>::T;
    T *buf = (T *)D.f[0];
    const int64_t np = D.np;
    for (int r = 2 * threadIdx.x; r < tl.count; r += 2 * blockDim.x) {
        const int64_t s = tl.start + r;  // even: tiles start at multiples of 64
        if (r + 1 >= tl.count) {         // ragged tail: one site
            site_aa_even<S>(D, buf, s);
            continue;
        }
        float ga[19], gb[19];
        unroll<0, 19>([&](auto ic) {
            constexpr int I = decltype(ic)::v;
            Pair<S>::template ld<I>(buf + (int64_t)I * np + s, ga[I], gb[I]);
        });
        const int slot_a = iolet_fixup<S>(D, s, ga);
        const int slot_b = iolet_fixup<S>(D, s + 1, gb);
        const float4 ma = collide_s<S>(ga, D.omega);
        const float4 mb = collide_s<S>(gb, D.omega);
        T *wb = opaque(buf + s);
        unroll<0, 19>([&](auto ic) {
            constexpr int I = decltype(ic)::v;
            Pair<S>::template st<I>(wb + (int64_t)OPP(I) * np, ga[I], gb[I]);
        });
        if (slot_a >= 0) D.bnd[slot_a] = ma;
        if (slot_b >= 0) D.bnd[slot_b] = mb;
    }
}

// ==== TMA bulk-copy AA even step (V = 2) ======================================
// One thread moves the tile's 19 rows (contiguous segments of the SoA arrays)
// into shared memory with cp.async.bulk, completion tracked by an mbarrier;
// every thread collides its sites from shared memory, writes the swapped
// result back into the same column, and one thread stores the 19 rows with
// bulk copies.  The wait is bounded: on timeout the context error word is set.
constexpr uint32_t kWaitLimit = 1u << 22;

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    for (uint32_t it = 0; it < kWaitLimit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void bulk_g2s(void *sdst, const void *gsrc, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(sdst)),
        "l"(gsrc), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void bulk_s2g(void *gdst, const void *ssrc, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(smem_addr(ssrc)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit_wait_read() {
    asm volatile("cp.async.bulk.commit_group;\ncp.async.bulk.wait_group.read 0;\n" ::: "memory");
}

template <int S>
__device__ __forceinline__ void tile_aa_even_tma(const DomDev &D, const TileDev &tl, uint32_t cap,
                                                 unsigned char *smem) {
    using T = typename St<S>::T;
    constexpr uint32_t E = sizeof(T);
    T *buf = (T *)D.f[0];
    const int64_t np = D.np;
    uint64_t *bar = (uint64_t *)smem;
    T *rows = (T *)(smem + 16);
    const uint32_t bytes = ((uint32_t)tl.count * E + 15u) & ~15u;  // padding keeps it inside the row
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_expect_tx(bar, 19u * bytes);
        for (int I = 0; I < 19; ++I) bulk_g2s(rows + (size_t)I * cap, buf + (int64_t)I * np + tl.start, bytes, bar);
    }
    const bool ok = __syncthreads_and(mbar_wait_bounded(bar, 0));
    if (!ok) {  // never expected: report, let the copies land, leave the tile untouched
        if (threadIdx.x == 0) atomicExch(D.err, 1);
        mbar_wait_bounded(bar, 0);
        return;
    }
    for (int r = threadIdx.x; r < tl.count; r += blockDim.x) {
        const int64_t s = tl.start + r;
        float g[19];
        unroll<0, 19>([&](auto ic) {
            constexpr int I = decltype(ic)::v;
            g[I] = St<S>::template ld<I>(rows[(size_t)I * cap + r]);
        });
        const int slot = iolet_fixup<S>(D, s, g);
        const float4 m = collide_s<S>(g, D.omega);
        unroll<0, 19>([&](auto ic) {
            constexpr int I = decltype(ic)::v;
            rows[(size_t)OPP(I) * cap + r] = St<S>::template st<I>(g[I]);
        });
        if (slot >= 0) D.bnd[slot] = m;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int I = 0; I < 19; ++I) bulk_s2g(buf + (int64_t)I * np + tl.start, rows + (size_t)I * cap, bytes);
        bulk_commit_wait_read();
    }
}

// PAR is the parity of the step this launch executes: 0 = even, 1 = odd (the
// AA step kind), 2 = read from the domain's step counter per block (A/B, and AA
// batches whose domains are at different parities).
// One tile of one domain, after the prologue has located it.
template <int S, int SCHEME, int SPT, int PAR, int V, bool RUNS, bool STASH = false, bool HOIST = false>
__device__ __forceinline__ void stream_collide_tile_impl(const DomDev &D, const TileDev &tl, bool odd,
                                                         uint32_t *stage) {
    using T = typename St<S>::T;
    if constexpr (V == 1 || V == 2 || V == 4) {
        if constexpr (SCHEME == kAB) {
            tile_ab_async<S, SPT>(D, tl, odd, stage);
        } else {
            if (odd) {
                if constexpr (V == 4) tile_aa_odd_staged<S>(D, tl, stage);
                else tile_aa_odd_async<S, SPT>(D, tl, stage);
            } else if constexpr (V == 2) {
                tile_aa_even_tma<S>(D, tl, (uint32_t)(SPT * blockDim.x), (unsigned char *)stage);
            } else {
                tile_aa_even_pairs<S>(D, tl);
            }
        }
    } else if constexpr (V == 6 || V == 7) {
        // AA on adjacent pairs: each thread takes sites 2t and 2t+1 of the tile (SPT = 2)
        static_assert(SCHEME == kAA && SPT == 2, "variants 6 and 7 are the AA pair forms");
        constexpr bool HINT = V == 7;
        T *buf = (T *)D.f[0];
        if (RUNS && odd) {
            // the run-encoded odd step takes one site at a time (decoding two runs at
            // once keeps too many values live), sites t and t + blockDim, so a warp's
            // gathers and scatters cover consecutive sites
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int r = j * blockDim.x + threadIdx.x;
                if (r < tl.count) site_aa_odd<S, HINT, true, STASH>(D, buf, tl.start + r, (int32_t *)stage);
            }
            return;
        }
        const int r = 2 * threadIdx.x;
        const int64_t s = tl.start + r;  // even: tiles start at multiples of 2 * blockDim
        if (r + 1 < tl.count) {
            if (odd) site_aa_odd_pair<S, HINT>(D, buf, s);
            else site_aa_even_pair<S, HINT>(D, buf, s);
        } else if (r < tl.count) {  // ragged tail: one site
            if (odd) site_aa_odd<S, HINT, false>(D, buf, s);
            else site_aa_even<S, HINT>(D, buf, s);
        }
    } else if constexpr (V == 5) {
        // A/B on adjacent pairs: each thread takes sites 2t and 2t+1 of the tile (SPT = 2)
        static_assert(SCHEME == kAB && SPT == 2, "variant 5 is the A/B pair form");
        const int r = 2 * threadIdx.x;
        const int64_t s = tl.start + r;  // even: tiles start at multiples of 2 * blockDim
        const T *src = (const T *)D.f[odd ? 0 : 1];
        T *dst = (T *)D.f[odd ? 1 : 0];
        if (r + 1 < tl.count) site_ab_pair<S, RUNS>(D, src, dst, s);
        else if (r < tl.count) site_ab<S, false, RUNS>(D, src, dst, s);  // ragged tail: one site
    } else if (HOIST && (SCHEME == kAB || odd)) {
        // every site's link word first (and a prefetch of its run row into L1), then the
        // sites one by one: a later site's decode no longer waits on its own word and row
        constexpr bool HINT = V == 3;
        uint32_t ws[SPT];
        const int32_t *rds[SPT];
#pragma unroll
        for (int j = 0; j < SPT; ++j) {
            const int r = j * blockDim.x + threadIdx.x;
            ws[j] = 0;
            rds[j] = D.rdelta;
            if (r < tl.count) {
                const RunNb<SCHEME, HINT> t(D, tl.start + r);
                t.prefetch();
                ws[j] = t.w;
                rds[j] = t.rd;
            }
        }
#pragma unroll
        for (int j = 0; j < SPT; ++j) {
            const int r = j * blockDim.x + threadIdx.x;
            if (r >= tl.count) continue;
            const int64_t s = tl.start + r;
            const RunNb<SCHEME, HINT> t(ws[j], rds[j], (int32_t)s, (int32_t)D.np);
            if constexpr (SCHEME == kAB) {
                site_ab_with<S, HINT>(D, (const T *)D.f[odd ? 0 : 1], (T *)D.f[odd ? 1 : 0], s, t);
            } else {
                site_aa_odd_with<S, HINT, true, false>(D, (T *)D.f[0], s, t);
            }
        }
    } else {
        constexpr bool HINT = V == 3;
#pragma unroll
        for (int j = 0; j < SPT; ++j) {
            const int r = j * blockDim.x + threadIdx.x;
            const int64_t s = tl.start + r;
            const bool live = r < tl.count;
            if constexpr (SCHEME == kAB) {
                if (live) {
                    const T *src = (const T *)D.f[odd ? 0 : 1];
                    T *dst = (T *)D.f[odd ? 1 : 0];
                    site_ab<S, HINT, RUNS>(D, src, dst, s);
                }
            } else {
                T *buf = (T *)D.f[0];
                if (live) {
                    if (odd) site_aa_odd<S, HINT, RUNS, STASH>(D, buf, s, (int32_t *)stage);
                    else site_aa_even<S, HINT>(D, buf, s);
                }
            }
        }
    }
}

// Variants 8..11 are 3, 5, 6, 7 reading the run-encoded neighbour table.  The host
// launches them only on domains that have one (the others get 3, 5, 6, 7); a domain
// without one here is reported through the error word (code 2) and left untouched.
// Variant 12 is 8 for the AA scheme with the odd step's 18 entries stashed in shared
// memory across the collision instead of decoded twice; 14 is 10 with the same stash;
// 13 is 8 with every site's link word loaded (and its run row prefetched) before the
// first site's gathers.
template <int V> constexpr int table_variant() {
    return V == 8 || V == 12 || V == 13 ? 3 : V == 9 ? 5 : V == 10 || V == 14 ? 6 : V == 11 ? 7 : V;
}

template <int S, int SCHEME, int SPT, int PAR, int V>
__device__ __forceinline__ void stream_collide_tile(const DomDev &D, const TileDev &tl, bool odd,
                                                    uint32_t *stage) {
    if constexpr (V >= 8) {
        if (D.lword == nullptr) {
            if (threadIdx.x == 0) atomicExch(D.err, 2);
            return;
        }
        stream_collide_tile_impl<S, SCHEME, SPT, PAR, table_variant<V>(), true, V == 12 || V == 14, V == 13>(D, tl, odd,
                                                                                                 stage);
    } else {
        stream_collide_tile_impl<S, SCHEME, SPT, PAR, V, false>(D, tl, odd, stage);
    }
}

// Many domains per launch: each block finds its tile in the tile table; the
// first threads copy the tile's domain descriptor into shared memory, one
// 8-byte word each, while thread 0 reads the domain's step counter.
template <int S, int SCHEME, int SPT, int PAR, int V>
__global__ void __launch_bounds__(512) k_stream_collide(const DomDev *__restrict__ doms,
                                                        const TileDev *__restrict__ tiles,
                                                        const int64_t *__restrict__ steps, int off) {
    static_assert(sizeof(DomDev) % 8 == 0, "descriptor copied in 8-byte words");
    constexpr int kWords = (int)(sizeof(DomDev) / 8);
    __shared__ DomDev D;
    __shared__ int64_t t_now;
    extern __shared__ __align__(128) uint32_t stage[];
    const TileDev tl = tiles[blockIdx.x];
    if (threadIdx.x < kWords)
        reinterpret_cast<uint64_t *>(&D)[threadIdx.x] =
            __ldg(reinterpret_cast<const uint64_t *>(doms + tl.dom) + threadIdx.x);
    // the step this launch executes (1-based); only its parity matters, and a
    // launch whose domains all share it gets it as a template argument
    if constexpr (PAR == 2)
        if (threadIdx.x == 0) t_now = __ldg(steps + tl.dom) + off + 1;
    __syncthreads();
    const bool odd = PAR == 2 ? (t_now & 1) != 0 : PAR == 1;
    stream_collide_tile<S, SCHEME, SPT, PAR, V>(D, tl, odd, stage);
}

// One domain per launch: the descriptor is a kernel parameter (constant bank)
// and block b takes sites [b*T, b*T + T) with T = SPT * blockDim, so no block
// waits on a table load or a barrier before its first neighbour-table load.
template <int S, int SCHEME, int SPT, int PAR, int V>
__global__ void __launch_bounds__(512) k_stream_collide_one(const __grid_constant__ DomDev D, int64_t n,
                                                            int off) {
    // a launch chained after this one (the next domain of a per-domain launch
    // sequence) may be scheduled once every block here has started; kernels launched
    // without programmatic serialisation ignore the trigger
    asm volatile("griddepcontrol.launch_dependents;");
    extern __shared__ __align__(128) uint32_t stage[];
    const int64_t ts = (int64_t)SPT * blockDim.x;
    TileDev tl;
    tl.dom = 0;
    tl.start = (int64_t)blockIdx.x * ts;
    tl.count = (int32_t)(n - tl.start < ts ? n - tl.start : ts);
    bool odd;
    if constexpr (PAR == 2) odd = ((__ldg(D.step) + off + 1) & 1) != 0;
    else odd = PAR == 1;
    stream_collide_tile<S, SCHEME, SPT, PAR, V>(D, tl, odd, stage);
}


template <int S, int SCHEME, int PAR, int V, int SPT>
cudaError_t launch_sc_one(const CollideCfg &cfg, const DomDev *doms, const TileDev *tiles,
                          int64_t n_tiles, int off, const OneDomain &one, cudaStream_t st) {
    // V1/V4: cp.async stage of 4-byte words (V4 reuses it for the odd step's outputs);
    // V2 also holds the even step's 19 rows + mbarrier
    size_t smem = (V == 1 || V == 2 || V == 4) ? (size_t)SPT * 19 * cfg.block * 4 : 0;
    if (V == 12 || V == 14) smem = (size_t)19 * cfg.block * 4;  // the AA odd step's entry stash
    if (V == 2) smem += 16;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)n_tiles);
    lc.blockDim = dim3((unsigned)cfg.block);
    lc.dynamicSmemBytes = smem;
    lc.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = at;
    lc.numAttrs = one.overlap_previous ? 1 : 0;  // start while the previous iolet update runs
    if (one.d) {
        auto k = k_stream_collide_one<S, SCHEME, SPT, PAR, V>;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        return cudaLaunchKernelEx(&lc, k, *one.d, one.n, off);
    }
    auto k = k_stream_collide<S, SCHEME, SPT, PAR, V>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return cudaLaunchKernelEx(&lc, k, doms, tiles, one.steps, off);
}

template <int S, int SCHEME, int PAR>
cudaError_t launch_sc_spt(const CollideCfg &cfg, const DomDev *doms, const TileDev *tiles,
                          int64_t n_tiles, int off, const OneDomain &one, cudaStream_t st) {
    if (cfg.variant == 1) {
        switch (cfg.spt) {
            case 1: return launch_sc_one<S, SCHEME, PAR, 1, 1>(cfg, doms, tiles, n_tiles, off, one, st);
            case 2: return launch_sc_one<S, SCHEME, PAR, 1, 2>(cfg, doms, tiles, n_tiles, off, one, st);
            default: return cudaErrorInvalidValue;
        }
    }
    if (cfg.variant == 3) {
        switch (cfg.spt) {
            case 1: return launch_sc_one<S, SCHEME, PAR, 3, 1>(cfg, doms, tiles, n_tiles, off, one, st);
            case 2: return launch_sc_one<S, SCHEME, PAR, 3, 2>(cfg, doms, tiles, n_tiles, off, one, st);
            case 4: return launch_sc_one<S, SCHEME, PAR, 3, 4>(cfg, doms, tiles, n_tiles, off, one, st);
            default: return cudaErrorInvalidValue;
        }
    }
    if (cfg.variant == 4) {
        if constexpr (SCHEME == kAB) return cudaErrorInvalidValue;
        else if (cfg.spt != 1) return cudaErrorInvalidValue;
        else return launch_sc_one<S, SCHEME, PAR, 4, 1>(cfg, doms, tiles, n_tiles, off, one, st);
    }
    if (cfg.variant == 5) {
        if constexpr (SCHEME != kAB || S == kF32) return cudaErrorInvalidValue;
        else if (cfg.spt != 2) return cudaErrorInvalidValue;
        else return launch_sc_one<S, SCHEME, PAR, 5, 2>(cfg, doms, tiles, n_tiles, off, one, st);
    }
    if (cfg.variant == 6 || cfg.variant == 7) {
        if constexpr (SCHEME != kAA) return cudaErrorInvalidValue;
        else if (cfg.spt != 2) return cudaErrorInvalidValue;
        else if (cfg.variant == 6) return launch_sc_one<S, SCHEME, PAR, 6, 2>(cfg, doms, tiles, n_tiles, off, one, st);
        else return launch_sc_one<S, SCHEME, PAR, 7, 2>(cfg, doms, tiles, n_tiles, off, one, st);
    }
    if (cfg.variant == 8) {
        switch (cfg.spt) {
            case 1: return launch_sc_one<S, SCHEME, PAR, 8, 1>(cfg, doms, tiles, n_tiles, off, one, st);
            case 2: return launch_sc_one<S, SCHEME, PAR, 8, 2>(cfg, doms, tiles, n_tiles, off, one, st);
            case 4: return launch_sc_one<S, SCHEME, PAR, 8, 4>(cfg, doms, tiles, n_tiles, off, one, st);
            default: return cudaErrorInvalidValue;
        }
    }
    if (cfg.variant == 14) {
        if constexpr (SCHEME != kAA) return cudaErrorInvalidValue;
        else if (cfg.spt != 2) return cudaErrorInvalidValue;
        else return launch_sc_one<S, SCHEME, PAR, 14, 2>(cfg, doms, tiles, n_tiles, off, one, st);
    }
    if (cfg.variant == 13) {
        switch (cfg.spt) {
            case 2: return launch_sc_one<S, SCHEME, PAR, 13, 2>(cfg, doms, tiles, n_tiles, off, one, st);
            case 4: return launch_sc_one<S, SCHEME, PAR, 13, 4>(cfg, doms, tiles, n_tiles, off, one, st);
            default: return cudaErrorInvalidValue;
        }
    }
    if (cfg.variant == 12) {
        if constexpr (SCHEME != kAA) return cudaErrorInvalidValue;
        else switch (cfg.spt) {
            case 1: return launch_sc_one<S, SCHEME, PAR, 12, 1>(cfg, doms, tiles, n_tiles, off, one, st);
            case 2: return launch_sc_one<S, SCHEME, PAR, 12, 2>(cfg, doms, tiles, n_tiles, off, one, st);
            default: return cudaErrorInvalidValue;
        }
    }
    if (cfg.variant == 9) {
        if constexpr (SCHEME != kAB || S == kF32) return cudaErrorInvalidValue;
        else if (cfg.spt != 2) return cudaErrorInvalidValue;
        else return launch_sc_one<S, SCHEME, PAR, 9, 2>(cfg, doms, tiles, n_tiles, off, one, st);
    }
    if (cfg.variant == 10 || cfg.variant == 11) {
        if constexpr (SCHEME != kAA) return cudaErrorInvalidValue;
        else if (cfg.spt != 2) return cudaErrorInvalidValue;
        else if (cfg.variant == 10) return launch_sc_one<S, SCHEME, PAR, 10, 2>(cfg, doms, tiles, n_tiles, off, one, st);
        else return launch_sc_one<S, SCHEME, PAR, 11, 2>(cfg, doms, tiles, n_tiles, off, one, st);
    }
    if (cfg.variant == 2) {
        if (SCHEME == kAB) return cudaErrorInvalidValue;
        switch (cfg.spt) {
            case 1: return launch_sc_one<S, SCHEME, PAR, 2, 1>(cfg, doms, tiles, n_tiles, off, one, st);
            case 2: return launch_sc_one<S, SCHEME, PAR, 2, 2>(cfg, doms, tiles, n_tiles, off, one, st);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (cfg.spt) {
        case 1: return launch_sc_one<S, SCHEME, PAR, 0, 1>(cfg, doms, tiles, n_tiles, off, one, st);
        case 2: return launch_sc_one<S, SCHEME, PAR, 0, 2>(cfg, doms, tiles, n_tiles, off, one, st);
        case 4: return launch_sc_one<S, SCHEME, PAR, 0, 4>(cfg, doms, tiles, n_tiles, off, one, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

}  // namespace hg
