// hg_kernels.cu -- sm_103a kernels of the sparse D3Q19 LBGK hot path.
//
// Method (arXiv 2010.04144, Section 2): D3Q19 lattice, single-relaxation-time
// collision, rigid walls, pressure/velocity conditions at inlets/outlets, on
// a sparse list of fluid sites.  Section 2.3 / Section 3: averaged iolet
// values drive the paired inlets of a coupled domain.
//
// Kernels
//   k_stream_collide   fused streaming + boundary rules + LBGK collision for
//                      every site of one or many domains (tile table), A/B pull
//                      or AA in-place, FP32 / FP16 / BF16 storage.  HBM-bound.
//   k_iolet_update     per iolet: FP64 mean of u.n and drho over its adjacent
//                      sites (fixed order), then the boundary value of the next
//                      step (pulse, or coupled factor x source mean).
//   k_advance          bumps the per-domain completed-step counters.
//   k_macroscopic / k_export_state / k_import_state / k_mass*: read-back.
//
// The step parity is read from a device counter, so one captured CUDA graph
// replays any number of times without re-recording kernel arguments.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

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
__host__ __device__ constexpr float INVW(int i) { return i == 0 ? 3.0f : (i <= 6 ? 18.0f : 36.0f); }
__host__ __device__ constexpr double WD(int i) {
    return i == 0 ? (1.0 / 3.0) : (i <= 6 ? (1.0 / 18.0) : (1.0 / 36.0));
}

// ---- storage traits ----
template <int S> struct St;
template <> struct St<kF32> {
    using T = float;
    template <int I> static __device__ __forceinline__ float ld(T v) { return v; }
    template <int I> static __device__ __forceinline__ T st(float v) { return v; }
    static __device__ __forceinline__ double ldd(T v, int) { return (double)v; }
};
template <> struct St<kF16> {
    using T = __half;
    template <int I> static __device__ __forceinline__ float ld(T v) { return __half2float(v) * W(I); }
    template <int I> static __device__ __forceinline__ T st(float v) { return __float2half_rn(v * INVW(I)); }
    static __device__ __forceinline__ double ldd(T v, int i) { return (double)__half2float(v) * WD(i); }
};
template <> struct St<kBF16> {
    using T = __nv_bfloat16;
    template <int I> static __device__ __forceinline__ float ld(T v) { return __bfloat162float(v) * W(I); }
    template <int I> static __device__ __forceinline__ T st(float v) { return __float2bfloat16_rn(v * INVW(I)); }
    static __device__ __forceinline__ double ldd(T v, int i) { return (double)__bfloat162float(v) * WD(i); }
};

template <int N> struct IC { static constexpr int v = N; };
template <int B, int E, typename F> __device__ __forceinline__ void unroll(F &&f) {
    if constexpr (B < E) {
        f(IC<B>{});
        unroll<B + 1, E>(f);
    }
}

// Boundary rule for a non-fluid link in direction I whose device code is v < 0;
// raw = the site's own post-collision value leaving towards x - c_I (direction opp(I)).
template <int I>
__device__ __forceinline__ float link_rule(const DomDev &D, int32_t v, float raw, int &slot) {
    if (v == -1) return raw;  // half-way bounce-back
    const int c = -v - 2;
    const int k = c & (kMaxIolets - 1);
    slot = c >> 8;
    const float val = D.bcv[k];
    if (D.io_kind[k] == 0) return -raw + 2.0f * W(I) * val;  // anti-bounce-back, drho_k
    return raw + val * D.coef[(int64_t)slot * 18 + (I - 1)];  // moving wall, u_w = U phi (-a)
}

// LBGK collision in deviation form, in place on g[19]; returns (drho, u).
__device__ __forceinline__ float4 collide(float g[19], float omega) {
    float drho = 0.f;
#pragma unroll
    for (int i = 0; i < 19; ++i) drho += g[i];
    const float d12 = g[1] - g[2], d34 = g[3] - g[4], d56 = g[5] - g[6];
    const float d78 = g[7] - g[8], d910 = g[9] - g[10], d1112 = g[11] - g[12];
    const float d1314 = g[13] - g[14], d1516 = g[15] - g[16], d1718 = g[17] - g[18];
    const float jx = d12 + d78 + d910 + d1112 + d1314;
    const float jy = d34 + d78 - d910 + d1516 + d1718;
    const float jz = d56 + d1112 - d1314 + d1516 - d1718;
    const float rho = 1.0f + drho;
    const float inv = 1.0f / rho;
    const float ux = jx * inv, uy = jy * inv, uz = jz * inv;
    const float usq = ux * ux + uy * uy + uz * uz;
    const float base = drho - 1.5f * rho * usq;
    const float r45 = 4.5f * rho, r3 = 3.0f * rho;
    g[0] += omega * (W(0) * base - g[0]);
    auto pair = [&](int a, int b, float w, float cu) {
        const float sym = w * (base + r45 * cu * cu);
        const float asym = w * r3 * cu;
        g[a] += omega * (sym + asym - g[a]);
        g[b] += omega * (sym - asym - g[b]);
    };
    pair(1, 2, W(1), ux);
    pair(3, 4, W(3), uy);
    pair(5, 6, W(5), uz);
    pair(7, 8, W(7), ux + uy);
    pair(9, 10, W(9), ux - uy);
    pair(11, 12, W(11), ux + uz);
    pair(13, 14, W(13), ux - uz);
    pair(15, 16, W(15), uy + uz);
    pair(17, 18, W(17), uy - uz);
    return make_float4(drho, ux, uy, uz);
}

template <typename T> __device__ __forceinline__ T ldg_nc(const T *p) { return __ldg(p); }
template <> __device__ __forceinline__ __half ldg_nc(const __half *p) {
    unsigned short r;
    asm volatile("ld.global.nc.u16 %0, [%1];" : "=h"(r) : "l"(p));
    return __ushort_as_half(r);
}
template <> __device__ __forceinline__ __nv_bfloat16 ldg_nc(const __nv_bfloat16 *p) {
    unsigned short r;
    asm volatile("ld.global.nc.u16 %0, [%1];" : "=h"(r) : "l"(p));
    return __ushort_as_bfloat16(r);
}

// ---- A/B pull: F_{t-1} in src, F_t to dst ----
template <int S>
__device__ __forceinline__ void site_ab(const DomDev &D, const typename St<S>::T *__restrict__ src,
                                        typename St<S>::T *__restrict__ dst, int64_t s) {
    using Tr = St<S>;
    const int64_t np = D.np;
    int32_t nb[18];
#pragma unroll
    for (int i = 0; i < 18; ++i) nb[i] = __ldg(D.nbr + (int64_t)i * np + s);
    float g[19];
    g[0] = Tr::template ld<0>(ldg_nc(src + s));
    int slot = -1;
    unroll<1, 19>([&](auto ic) {
        constexpr int I = decltype(ic)::v;
        const int32_t v = nb[I - 1];
        if (v >= 0) {
            g[I] = Tr::template ld<I>(ldg_nc(src + (int64_t)I * np + v));
        } else {
            const float raw = Tr::template ld<OPP(I)>(ldg_nc(src + (int64_t)OPP(I) * np + s));
            g[I] = link_rule<I>(D, v, raw, slot);
        }
    });
    const float4 m = collide(g, D.omega);
    unroll<0, 19>([&](auto ic) {
        constexpr int I = decltype(ic)::v;
        dst[(int64_t)I * np + s] = Tr::template st<I>(g[I]);
    });
    if (slot >= 0) D.bnd[slot] = m;
}

// ---- AA even step: state G_t natural at the own site -> F_t swapped at the own site ----
template <int S>
__device__ __forceinline__ void site_aa_even(const DomDev &D, typename St<S>::T *buf, int64_t s,
                                             bool flagged) {
    using Tr = St<S>;
    const int64_t np = D.np;
    float g[19];
    unroll<0, 19>([&](auto ic) {
        constexpr int I = decltype(ic)::v;
        g[I] = Tr::template ld<I>(buf[(int64_t)I * np + s]);
    });
    int slot = -1;
    if (flagged) {  // rare: the previous odd step left raw values on iolet links
        unroll<1, 19>([&](auto ic) {
            constexpr int I = decltype(ic)::v;
            const int32_t v = __ldg(D.nbr + (int64_t)(I - 1) * np + s);
            if (v < -1) g[I] = link_rule<I>(D, v, g[I], slot);
        });
    }
    const float4 m = collide(g, D.omega);
    unroll<0, 19>([&](auto ic) {
        constexpr int I = decltype(ic)::v;
        buf[(int64_t)OPP(I) * np + s] = Tr::template st<I>(g[I]);
    });
    if (slot >= 0) D.bnd[slot] = m;
}

// ---- AA odd step: gather F_{t-1} (swapped) from x - c_i, scatter F_t to x + c_i ----
template <int S>
__device__ __forceinline__ void site_aa_odd(const DomDev &D, typename St<S>::T *buf, int64_t s) {
    using Tr = St<S>;
    const int64_t np = D.np;
    int32_t nb[18];
#pragma unroll
    for (int i = 0; i < 18; ++i) nb[i] = __ldg(D.nbr + (int64_t)i * np + s);
    float g[19];
    g[0] = Tr::template ld<0>(buf[s]);
    int slot = -1;
    unroll<1, 19>([&](auto ic) {
        constexpr int I = decltype(ic)::v;
        const int32_t v = nb[I - 1];
        if (v >= 0) {
            g[I] = Tr::template ld<I>(buf[(int64_t)OPP(I) * np + v]);
        } else {
            const float raw = Tr::template ld<OPP(I)>(buf[(int64_t)I * np + s]);
            g[I] = link_rule<I>(D, v, raw, slot);
        }
    });
    const float4 m = collide(g, D.omega);
    buf[s] = Tr::template st<0>(g[0]);
    unroll<1, 19>([&](auto ic) {
        constexpr int I = decltype(ic)::v;
        const int32_t t = nb[OPP(I) - 1];  // site at x + c_I
        if (t >= 0) buf[(int64_t)I * np + t] = Tr::template st<I>(g[I]);
        else buf[(int64_t)OPP(I) * np + s] = Tr::template st<I>(g[I]);  // raw, rule applied on read
    });
    if (slot >= 0) D.bnd[slot] = m;
}

template <int S, int SCHEME, int SPT>
__global__ void __launch_bounds__(512) k_stream_collide(const DomDev *__restrict__ doms,
                                                         const TileDev *__restrict__ tiles,
                                                         int off) {
    using T = typename St<S>::T;
    __shared__ DomDev D;
    __shared__ int64_t t_now;
    const TileDev tl = tiles[blockIdx.x];
    if (threadIdx.x == 0) {
        D = doms[tl.dom];
        t_now = *D.step + off + 1;  // the step this launch executes (1-based)
    }
    __syncthreads();
    const int64_t t = t_now;
#pragma unroll
    for (int j = 0; j < SPT; ++j) {
        const int r = j * blockDim.x + threadIdx.x;
        const int64_t s = tl.start + r;
        const bool live = r < tl.count;
        if constexpr (SCHEME == kAB) {
            if (live) {
                const T *src = (const T *)D.f[(t - 1) & 1];
                T *dst = (T *)D.f[t & 1];
                site_ab<S>(D, src, dst, s);
            }
        } else {
            T *buf = (T *)D.f[0];
            if (t & 1) {
                if (live) site_aa_odd<S>(D, buf, s);
            } else {
                const uint32_t word = live ? __ldg(D.iomask + (s >> 5)) : 0u;
                if (live) site_aa_even<S>(D, buf, s, (word >> (s & 31)) & 1u);
            }
        }
    }
}

// ---- iolet update: FP64 means in fixed order, next boundary value ----
__device__ __forceinline__ void block_sum2(double &a, double &b) {
    __shared__ double sa[32], sb[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) {
        sa[w] = a;
        sb[w] = b;
    }
    __syncthreads();
    const int nw = blockDim.x >> 5;
    if (w == 0) {
        a = l < nw ? sa[l] : 0.0;
        b = l < nw ? sb[l] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
    }
}

__device__ __forceinline__ void reduce_iolet(const int32_t *slots, const float4 *bnd, int n,
                                             double nx, double ny, double nz, double &su,
                                             double &sr) {
    su = 0.0;
    sr = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const float4 m = bnd[slots[j]];
        su += (double)m.y * nx + (double)m.z * ny + (double)m.w * nz;
        sr += (double)m.x;
    }
    block_sum2(su, sr);
}

__global__ void __launch_bounds__(256) k_iolet_update(const IoDev *__restrict__ ios, int off) {
    const IoDev &I = ios[blockIdx.x];
    double su, sr;
    reduce_iolet(I.slots, I.bnd, I.n_slots, I.nx, I.ny, I.nz, su, sr);
    if (threadIdx.x == 0) {
        const double cnt = (double)I.n_slots;
        I.M[0] = I.n_slots ? su / cnt : 0.0;
        I.M[1] = I.n_slots ? sr / cnt : 0.0;
        I.M[2] = cnt;
    }
    double val;
    if (I.coupled) {
        double cu, cr;
        reduce_iolet(I.src_slots, I.src_bnd, I.src_n_slots, I.src_nx, I.src_ny, I.src_nz, cu, cr);
        val = I.factor * (I.src_n_slots ? cu / (double)I.src_n_slots : 0.0);
    } else {
        const double tn = (double)(*I.step + off + 2);  // the next step
        double p = 1.0;
        if (I.pulse == 1) p = 0.5 * (1.0 - cos(2.0 * 3.141592653589793 * tn / I.period));
        else if (I.pulse == 2) p = sin(2.0 * 3.141592653589793 * tn / I.period);
        val = I.value * p;
    }
    if (threadIdx.x == 0) *I.bcv = (float)val;
}

__global__ void k_advance_list(int64_t *base, const int32_t *idx, int n, int64_t by) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) base[idx[i]] += by;
}

// ---- read-back: F_t of site s, direction I (raw storage value) ----
template <int S, int SCHEME, int I>
__device__ __forceinline__ typename St<S>::T stored_F(const DomDev &D, int64_t t, int64_t s) {
    using T = typename St<S>::T;
    const int64_t np = D.np;
    if constexpr (SCHEME == kAB) {
        return ((const T *)D.f[t & 1])[(int64_t)I * np + s];
    } else {
        const T *buf = (const T *)D.f[0];
        if (!(t & 1) || I == 0) return buf[(int64_t)OPP(I) * np + s];
        const int32_t tg = D.nbr[(int64_t)(OPP(I) - 1) * np + s];
        return tg >= 0 ? buf[(int64_t)I * np + tg] : buf[(int64_t)OPP(I) * np + s];
    }
}

template <int S, int SCHEME, int I>
__device__ __forceinline__ typename St<S>::T *stored_F_ptr(const DomDev &D, int64_t t, int64_t s) {
    using T = typename St<S>::T;
    const int64_t np = D.np;
    if constexpr (SCHEME == kAB) {
        return ((T *)D.f[t & 1]) + (int64_t)I * np + s;
    } else {
        T *buf = (T *)D.f[0];
        if (!(t & 1) || I == 0) return buf + (int64_t)OPP(I) * np + s;
        const int32_t tg = D.nbr[(int64_t)(OPP(I) - 1) * np + s];
        return tg >= 0 ? buf + (int64_t)I * np + tg : buf + (int64_t)OPP(I) * np + s;
    }
}

template <int S, int SCHEME>
__global__ void k_macroscopic(const DomDev *__restrict__ dd, int64_t n, const int64_t *canon_of,
                              float4 *out) {
    using Tr = St<S>;
    const DomDev D = *dd;
    const int64_t t = *D.step;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        float g[19];
        unroll<0, 19>([&](auto ic) {
            constexpr int I = decltype(ic)::v;
            g[I] = Tr::template ld<I>(stored_F<S, SCHEME, I>(D, t, s));
        });
        float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
        unroll<0, 19>([&](auto ic) {
            constexpr int I = decltype(ic)::v;
            drho += g[I];
            if (CX(I)) jx += CX(I) * g[I];
            if (CY(I)) jy += CY(I) * g[I];
            if (CZ(I)) jz += CZ(I) * g[I];
        });
        const float inv = 1.0f / (1.0f + drho);
        out[canon_of ? canon_of[s] : s] = make_float4(drho, jx * inv, jy * inv, jz * inv);
    }
}

template <int S, int SCHEME>
__global__ void k_export_state(const DomDev *__restrict__ dd, int64_t n, const int64_t *canon_of,
                               typename St<S>::T *out) {
    const DomDev D = *dd;
    const int64_t t = *D.step;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = canon_of ? canon_of[s] : s;
        unroll<0, 19>([&](auto ic) {
            constexpr int I = decltype(ic)::v;
            out[(int64_t)I * n + c] = stored_F<S, SCHEME, I>(D, t, s);
        });
    }
}

template <int S, int SCHEME>
__global__ void k_import_state(const DomDev *__restrict__ dd, int64_t n, const int64_t *canon_of,
                               const typename St<S>::T *in) {
    const DomDev D = *dd;
    const int64_t t = *D.step;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = canon_of ? canon_of[s] : s;
        unroll<0, 19>([&](auto ic) {
            constexpr int I = decltype(ic)::v;
            *stored_F_ptr<S, SCHEME, I>(D, t, s) = in[(int64_t)I * n + c];
        });
    }
}

constexpr int kMassChunk = 8192;
constexpr int kMassThreads = 256;

template <int S>
__global__ void __launch_bounds__(kMassThreads) k_mass_partials(const DomDev *__restrict__ dd,
                                                                int64_t n, double *partials) {
    using T = typename St<S>::T;
    const DomDev D = *dd;
    const int64_t t = *D.step;
    const T *buf = (const T *)D.f[(D.f[1] != nullptr) ? (t & 1) : 0];
    const int64_t lo = (int64_t)blockIdx.x * kMassChunk;
    const int64_t hi = lo + kMassChunk < n ? lo + kMassChunk : n;
    double a = 0.0, b = 0.0;
    for (int64_t s = lo + threadIdx.x; s < hi; s += blockDim.x) {
#pragma unroll
        for (int i = 0; i < 19; ++i) a += St<S>::ldd(buf[(int64_t)i * D.np + s], i);
    }
    block_sum2(a, b);
    if (threadIdx.x == 0) partials[blockIdx.x] = a;
}

__global__ void __launch_bounds__(kMassThreads) k_mass_final(const double *partials, int64_t np_,
                                                             double *out) {
    double a = 0.0, b = 0.0;
    for (int64_t j = threadIdx.x; j < np_; j += blockDim.x) a += partials[j];
    block_sum2(a, b);
    if (threadIdx.x == 0) *out = a;
}

template <int S, int SCHEME>
cudaError_t launch_sc_spt(const CollideCfg &cfg, const DomDev *doms, const TileDev *tiles,
                          int64_t n_tiles, int off, cudaStream_t st) {
    switch (cfg.spt) {
        case 1: k_stream_collide<S, SCHEME, 1><<<(unsigned)n_tiles, cfg.block, 0, st>>>(doms, tiles, off); break;
        case 2: k_stream_collide<S, SCHEME, 2><<<(unsigned)n_tiles, cfg.block, 0, st>>>(doms, tiles, off); break;
        case 4: k_stream_collide<S, SCHEME, 4><<<(unsigned)n_tiles, cfg.block, 0, st>>>(doms, tiles, off); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

inline unsigned rb_grid(int64_t n) {
    int64_t g = (n + 255) / 256;
    if (g > 152 * 64) g = 152 * 64;
    return (unsigned)(g > 0 ? g : 1);
}

}  // namespace

cudaError_t launch_stream_collide(const CollideCfg &cfg, const DomDev *doms, const TileDev *tiles,
                                  int64_t n_tiles, int off, cudaStream_t st) {
    if (n_tiles <= 0) return cudaSuccess;
    if (cfg.scheme == kAB) {
        if (cfg.storage == kF32) return launch_sc_spt<kF32, kAB>(cfg, doms, tiles, n_tiles, off, st);
        if (cfg.storage == kF16) return launch_sc_spt<kF16, kAB>(cfg, doms, tiles, n_tiles, off, st);
        if (cfg.storage == kBF16) return launch_sc_spt<kBF16, kAB>(cfg, doms, tiles, n_tiles, off, st);
    } else {
        if (cfg.storage == kF32) return launch_sc_spt<kF32, kAA>(cfg, doms, tiles, n_tiles, off, st);
        if (cfg.storage == kF16) return launch_sc_spt<kF16, kAA>(cfg, doms, tiles, n_tiles, off, st);
        if (cfg.storage == kBF16) return launch_sc_spt<kBF16, kAA>(cfg, doms, tiles, n_tiles, off, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_iolet_update(const IoDev *ios, int n_ios, int off, cudaStream_t st) {
    if (n_ios <= 0) return cudaSuccess;
    k_iolet_update<<<n_ios, 256, 0, st>>>(ios, off);
    return cudaGetLastError();
}

cudaError_t launch_advance_list(int64_t *steps_base, const int32_t *idx, int n, int64_t by,
                                cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_advance_list<<<(n + 127) / 128, 128, 0, st>>>(steps_base, idx, n, by);
    return cudaGetLastError();
}

#define HG_DISPATCH_SS(storage, scheme, CALL)                                  \
    do {                                                                       \
        if (scheme == kAB) {                                                   \
            if (storage == kF32) { constexpr int S_ = kF32, C_ = kAB; CALL; }  \
            else if (storage == kF16) { constexpr int S_ = kF16, C_ = kAB; CALL; } \
            else { constexpr int S_ = kBF16, C_ = kAB; CALL; }                 \
        } else {                                                               \
            if (storage == kF32) { constexpr int S_ = kF32, C_ = kAA; CALL; }  \
            else if (storage == kF16) { constexpr int S_ = kF16, C_ = kAA; CALL; } \
            else { constexpr int S_ = kBF16, C_ = kAA; CALL; }                 \
        }                                                                      \
    } while (0)

cudaError_t launch_macroscopic(int storage, int scheme, const DomDev *dom_dev, int64_t n,
                               const int64_t *canon_of, float4 *out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    HG_DISPATCH_SS(storage, scheme,
                   (k_macroscopic<S_, C_><<<rb_grid(n), 256, 0, st>>>(dom_dev, n, canon_of, out)));
    return cudaGetLastError();
}

cudaError_t launch_export_state(int storage, int scheme, const DomDev *dom_dev, int64_t n,
                                const int64_t *canon_of, void *out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    HG_DISPATCH_SS(storage, scheme,
                   (k_export_state<S_, C_><<<rb_grid(n), 256, 0, st>>>(
                       dom_dev, n, canon_of, (typename St<S_>::T *)out)));
    return cudaGetLastError();
}

cudaError_t launch_import_state(int storage, int scheme, const DomDev *dom_dev, int64_t n,
                                const int64_t *canon_of, const void *in, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    HG_DISPATCH_SS(storage, scheme,
                   (k_import_state<S_, C_><<<rb_grid(n), 256, 0, st>>>(
                       dom_dev, n, canon_of, (const typename St<S_>::T *)in)));
    return cudaGetLastError();
}

int64_t mass_partials_needed(int64_t n) { return n > 0 ? (n + kMassChunk - 1) / kMassChunk : 1; }

cudaError_t launch_mass(int storage, const DomDev *dom_dev, int64_t n, int64_t /*np*/,
                        double *partials, double *out, cudaStream_t st) {
    const int64_t P = mass_partials_needed(n);
    if (n <= 0) {
        return cudaMemsetAsync(out, 0, sizeof(double), st);
    }
    if (storage == kF32) k_mass_partials<kF32><<<(unsigned)P, kMassThreads, 0, st>>>(dom_dev, n, partials);
    else if (storage == kF16) k_mass_partials<kF16><<<(unsigned)P, kMassThreads, 0, st>>>(dom_dev, n, partials);
    else k_mass_partials<kBF16><<<(unsigned)P, kMassThreads, 0, st>>>(dom_dev, n, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_mass_final<<<1, kMassThreads, 0, st>>>(partials, P, out);
    return cudaGetLastError();
}

}  // namespace hg
