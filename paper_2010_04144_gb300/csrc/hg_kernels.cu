// hg_kernels.cu -- sm_103a kernels of the sparse D3Q19 LBGK hot path.
//
// Method (arXiv 2010.04144, Section 2): D3Q19 lattice, single-relaxation-time
// collision, rigid walls, pressure/velocity conditions at inlets/outlets, on
// a sparse list of fluid sites.  Section 2.3 / Section 3: averaged iolet
// values drive the paired inlets of a coupled domain.
//
// Kernels
//   k_stream_collide_one / k_stream_collide (hg_device.cuh, instantiated per
//                      storage type, scheme and launch parity in hg_sc_part.cu):
//                      fused streaming + boundary rules + LBGK collision for
//                      every site of one domain, or of many through a tile
//                      table; A/B pull or AA in place; FP32 / FP16 / BF16
//                      storage.  HBM-bound.
//   k_guo_force        body force on the sites next to forced arterial outlets
//                      (alternating coupling exchanges only).
//   k_iolet_update     per iolet: FP64 mean of u.n and drho over its adjacent
//                      sites (fixed order), then the boundary values of the
//                      next step (pulse, coupled factor x source mean, or the
//                      reverse exchange's outlet force).  It lets the next
//                      step's stream-collide start early (programmatic
//                      dependent launch).
//   k_advance_list     bumps the per-domain completed-step counters.
//   k_macroscopic / k_export_state / k_import_state / k_mass*: read-back.
//
// AA launches whose domains all share the parity of the step they execute get
// it as a template argument (graphs hold an even number of steps, so replays
// keep it); A/B launches and mixed AA batches read it from the step counters.
//
// Neighbour table on the device: entry i-1 of site s is the index of the pull
// source x_s - c_i when it is fluid, else a virtual index s + d*np (d = +-1)
// chosen so that the scheme's usual address formula reaches the site's own
// opposite slot -- the bounce-back value -- with no branch.  Links into iolet
// openings are fixed up on a rare path (iomask, ioprefix, io_codes).
#include "hg_device.cuh"

namespace hg {
namespace {

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

// One CTA per (iolet, chunk of kIoChunk slots): thread t takes slot t of the
// chunk, a fixed shuffle tree sums the block, the partial goes to
// partials[part0 + chunk].  The CTA that completes an iolet (atomic ticket, no
// waiting) sums its partials in chunk order -> M; the CTA that completes the
// last iolet sets every iolet's boundary value for the next step.  The result
// depends only on the slot lists, never on scheduling.
__global__ void __launch_bounds__(kIoChunk) k_iolet_update(const IoDev *__restrict__ ios, int n_ios,
                                                           const int2 *__restrict__ chunks,
                                                           double2 *partials, unsigned *counters,
                                                           int off) {
    // the next step's stream-collide may launch now: it waits for this grid
    // only where it needs the boundary values this grid produces
    asm volatile("griddepcontrol.launch_dependents;");
    __shared__ int s_last;
    const int2 ck = chunks[blockIdx.x];
    const IoDev &I = ios[ck.x];
    double su = 0.0, sr = 0.0;
    const int j = ck.y * kIoChunk + threadIdx.x;
    if (j < I.n_slots) {
        const float4 m = I.bnd[__ldg(I.slots + j)];
        su = (double)m.y * I.nx + (double)m.z * I.ny + (double)m.w * I.nz;
        sr = (double)m.x;
    }
    block_sum2(su, sr);
    if (threadIdx.x == 0) {
        partials[I.part0 + ck.y] = make_double2(su, sr);
        __threadfence();
        s_last = atomicAdd(&counters[ck.x], 1u) == (unsigned)(I.n_chunks - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    __shared__ double2 s_part[kIoChunk];
    double a = 0.0, b = 0.0;
    for (int c0 = 0; c0 < I.n_chunks; c0 += kIoChunk) {  // all loads in flight, then an ordered sum
        const int c = c0 + threadIdx.x;
        if (c < I.n_chunks) s_part[threadIdx.x] = __ldcg(partials + I.part0 + c);
        __syncthreads();
        if (threadIdx.x == 0) {
            const int m = min(kIoChunk, I.n_chunks - c0);
            for (int q = 0; q < m; ++q) {
                a += s_part[q].x;
                b += s_part[q].y;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double cnt = (double)I.n_slots;
        I.M[0] = I.n_slots ? a / cnt : 0.0;
        I.M[1] = I.n_slots ? b / cnt : 0.0;
        I.M[2] = cnt;
        counters[ck.x] = 0u;
        __threadfence();
        s_last = atomicAdd(&counters[n_ios], 1u) == (unsigned)(n_ios - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int k = threadIdx.x; k < n_ios; k += blockDim.x) {
        const IoDev &J = ios[k];
        // the exchange after step e is forward unless exchanges alternate and e is odd
        const int64_t e = *J.step + off + 1;
        const bool forward = !J.alternate || (e & 1) == 0;
        if (J.coupled) {
            if (forward) *J.bcv = (float)(J.factor * __ldcg(J.src_M));
        } else {
            // phase of the next step in [0, 1): exact remainder first, so the FP64
            // cosine only ever sees an argument in [0, 2 pi)
            const double tn = (double)(e + 1);
            const double ph = J.pulse ? fmod(tn, J.period) / J.period : 0.0;
            double p = 1.0;
            if (J.pulse == 1) p = 0.5 * (1.0 - cos(2.0 * 3.141592653589793 * ph));
            else if (J.pulse == 2) p = sin(2.0 * 3.141592653589793 * ph);
            *J.bcv = (float)(J.value * p);
        }
        if (!forward && J.n_rev > 0) {
            // reverse: mean over the fed inlets of inflow speed / factor; the outlet's force
            // density is the dynamic pressure of that speed, against the outward axis
            double v = 0.0;
            for (int r = 0; r < J.n_rev; ++r) v += -__ldcg(J.rev[r].M) / J.rev[r].factor;
            v /= (double)J.n_rev;
            const double q = -0.5 * v * fabs(v);
            *J.force = make_float4((float)(q * J.nx), (float)(q * J.ny), (float)(q * J.nz), 0.0f);
        }
    }
    if (threadIdx.x == 0) counters[n_ios] = 0u;
}

__global__ void k_advance_list(int64_t *base, const int32_t *idx, int n, int64_t by) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) base[idx[i]] += by;
}

// ---- body force next to forced iolets (reverse coupling direction) ----
// Guo, Zheng and Shi forcing: with force density F the velocity is
// u_F = (j + F/2)/rho, the equilibrium is taken at u_F and the collision adds
// (1 - omega/2) S_i, S_i = w_i [3 (c_i - u_F) + 9 (c_i.u_F) c_i] . F.  The
// forced result differs from the unforced one, which the stream-collide kernel
// has just stored, by omega (feq(u_F) - feq(u)) + (1 - omega/2) S_i(u_F): a
// function of (drho, u, F) alone.  This pass runs right after stream-collide,
// one thread per boundary slot listed as forced, adds that difference to the
// 19 stored values where the step left them (scaled storage drops the w_i) and
// rewrites the slot's moments with u_F, before the iolet reductions read them.
// Keeping it out of stream-collide leaves that kernel's registers untouched.
// A site takes the summed force of the distinct iolets it touches.
template <bool SC>
__device__ __forceinline__ void guo_delta(float4 m, float fx, float fy, float fz, float omega, float d[19],
                                          float4 &mf) {
    const float rho = HG_ADD(1.0f, m.x);
    const float h = HG_MUL(0.5f, __frcp_rn(rho));
    const float vx = HG_FMA(h, fx, m.y), vy = HG_FMA(h, fy, m.z), vz = HG_FMA(h, fz, m.w);
    const float usq = HG_FMA(m.y, m.y, HG_FMA(m.z, m.z, HG_MUL(m.w, m.w)));
    const float vsq = HG_FMA(vx, vx, HG_FMA(vy, vy, HG_MUL(vz, vz)));
    const float vf = HG_FMA(vx, fx, HG_FMA(vy, fy, HG_MUL(vz, fz)));
    const float a = HG_MUL(omega, rho);
    const float b = HG_FMA(-0.5f, omega, 1.0f);
    // isotropic part shared by every direction: a (-1.5 (u_F^2 - u^2)) + b (-3 u_F.F)
    const float iso = HG_FMA(a, HG_MUL(-1.5f, HG_SUB(vsq, usq)), HG_MUL(b, HG_MUL(-3.0f, vf)));
    d[0] = SC ? iso : mulw<0>(iso);
    auto pair = [&](auto iA, int B, float cu, float cv, float cf) {
        constexpr int A = decltype(iA)::v;
        const float sym = HG_FMA(a, HG_MUL(4.5f, HG_SUB(HG_MUL(cv, cv), HG_MUL(cu, cu))),
                                 HG_FMA(b, HG_MUL(9.0f, HG_MUL(cv, cf)), iso));
        const float asym = HG_MUL(3.0f, HG_FMA(a, HG_SUB(cv, cu), HG_MUL(b, cf)));
        const float p = HG_ADD(sym, asym), q = HG_SUB(sym, asym);
        d[A] = SC ? p : mulw<A>(p);
        d[B] = SC ? q : mulw<A>(q);
    };
    pair(IC<1>{}, 2, m.y, vx, fx);
    pair(IC<3>{}, 4, m.z, vy, fy);
    pair(IC<5>{}, 6, m.w, vz, fz);
    pair(IC<7>{}, 8, HG_ADD(m.y, m.z), HG_ADD(vx, vy), HG_ADD(fx, fy));
    pair(IC<9>{}, 10, HG_SUB(m.y, m.z), HG_SUB(vx, vy), HG_SUB(fx, fy));
    pair(IC<11>{}, 12, HG_ADD(m.y, m.w), HG_ADD(vx, vz), HG_ADD(fx, fz));
    pair(IC<13>{}, 14, HG_SUB(m.y, m.w), HG_SUB(vx, vz), HG_SUB(fx, fz));
    pair(IC<15>{}, 16, HG_ADD(m.z, m.w), HG_ADD(vy, vz), HG_ADD(fy, fz));
    pair(IC<17>{}, 18, HG_SUB(m.z, m.w), HG_SUB(vy, vz), HG_SUB(fy, fz));
    mf = make_float4(m.x, vx, vy, vz);
}

template <int S, int SCHEME>
__global__ void __launch_bounds__(128) k_guo_force(const DomDev *__restrict__ doms,
                                                   const int2 *__restrict__ fslots, int n, int off) {
    using T = typename St<S>::T;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int2 e = fslots[q];
    const DomDev &D = doms[e.x];
    const int slot = e.y;
    const int32_t *codes = D.io_codes + (int64_t)slot * 18;
    float fx = 0.0f, fy = 0.0f, fz = 0.0f;
    for (int i = 0; i < 18; ++i) {
        const int32_t c = codes[i];
        if (c >= -1) continue;
        bool first = true;
        for (int j = 0; j < i; ++j) first = first && (codes[j] != c);
        if (!first) continue;
        const float4 f = D.io_force[-c - 2];
        fx = HG_ADD(fx, f.x);
        fy = HG_ADD(fy, f.y);
        fz = HG_ADD(fz, f.z);
    }
    if (fx == 0.0f && fy == 0.0f && fz == 0.0f) return;
    float d[19];
    float4 mf;
    guo_delta<St<S>::kScaled>(D.bnd[slot], fx, fy, fz, D.omega, d, mf);
    const int64_t s = D.slot_site[slot];
    const int64_t np = D.np;
    const int64_t t = *D.step + off + 1;  // the step stream-collide just ran
    T *base;
    if constexpr (SCHEME == kAB) base = (T *)D.f[t & 1];
    else base = (T *)D.f[0];
    unroll<0, 19>([&](auto ic) {
        constexpr int I = decltype(ic)::v;
        int64_t at;
        if constexpr (SCHEME == kAB) {
            at = (int64_t)I * np + s;                            // own slot I
        } else if (I == 0) {
            at = s;
        } else if ((t & 1) == 0) {
            at = (int64_t)OPP(I) * np + s;                       // even: swapped, own site
        } else {
            at = (int64_t)I * np + D.nbr[(int64_t)(OPP(I) - 1) * np + s];  // odd: at x + c_I
        }
        const float v = St<S>::template ld<I>(base[at]);
        base[at] = St<S>::template st<I>(HG_ADD(v, d[I]));
    });
    D.bnd[slot] = mf;
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
        return buf[(int64_t)I * np + D.nbr[(int64_t)(OPP(I) - 1) * np + s]];  // x + c_I, or own raw
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
        return buf + ((int64_t)I * np + D.nbr[(int64_t)(OPP(I) - 1) * np + s]);
    }
}

template <int S, int SCHEME>
__global__ void k_macroscopic(const DomDev *__restrict__ dd, int64_t n, const int32_t *canon_of,
                              float4 *out) {
    using Tr = St<S>;
    const DomDev D = *dd;
    const int64_t t = *D.step;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        float g[19];
        unroll<0, 19>([&](auto ic) {
            constexpr int I = decltype(ic)::v;
            g[I] = Tr::template phys<I>(stored_F<S, SCHEME, I>(D, t, s));
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
__global__ void k_export_state(const DomDev *__restrict__ dd, int64_t n, const int32_t *canon_of,
                               typename St<S>::T *out, int64_t row) {
    const DomDev D = *dd;
    const int64_t t = *D.step;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = canon_of ? canon_of[s] : s;
        unroll<0, 19>([&](auto ic) {
            constexpr int I = decltype(ic)::v;
            out[(int64_t)I * row + c] = stored_F<S, SCHEME, I>(D, t, s);
        });
    }
}

template <int S, int SCHEME>
__global__ void k_import_state(const DomDev *__restrict__ dd, int64_t n, const int32_t *canon_of,
                               const typename St<S>::T *in, int64_t row) {
    const DomDev D = *dd;
    const int64_t t = *D.step;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = canon_of ? canon_of[s] : s;
        unroll<0, 19>([&](auto ic) {
            constexpr int I = decltype(ic)::v;
            *stored_F_ptr<S, SCHEME, I>(D, t, s) = in[(int64_t)I * row + c];
        });
    }
}

// ---- halo exchange of a split domain (A/B scheme: F_t sits in f[t & 1]) ----
template <typename W>
__global__ void k_halo_pack(const DomDev *__restrict__ doms, const int64_t *__restrict__ steps,
                            const HaloDev *__restrict__ ent, int64_t n, W *send, int off) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const HaloDev h = ent[e];
        const int64_t t = steps[h.dom] + off + 1;
        send[e] = ((const W *)doms[h.dom].f[t & 1])[h.off];
    }
}

template <typename W>
__global__ void k_halo_unpack(const DomDev *__restrict__ doms, const int64_t *__restrict__ steps,
                              const HaloDev *__restrict__ ent, int64_t n, const W *recv, int off) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const HaloDev h = ent[e];
        const int64_t t = steps[h.dom] + off + 1;
        ((W *)doms[h.dom].f[t & 1])[h.off] = recv[e];
    }
}

template <typename W>
__global__ void k_halo_direct(const DomDev *__restrict__ doms, const int64_t *__restrict__ steps,
                              const HaloMove *__restrict__ mv, int64_t n, int off) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const HaloMove m = mv[e];
        const int64_t t = steps[m.src_dom] + off + 1;
        ((W *)doms[m.dst_dom].f[t & 1])[m.dst_off] = ((const W *)doms[m.src_dom].f[t & 1])[m.src_off];
    }
}

constexpr int kMassChunk = 8192;
constexpr int kMassThreads = 256;

// Block b sums F_t of canonical sites [8192 b, 8192 (b+1)) in FP64, each site's
// 19 values in direction order 0..18 wherever the scheme keeps them (thread t
// takes every 256th site, then a fixed shuffle tree), reading each site at its
// device index, and counts the values that are not finite.  The sum is a
// function of the state F_t alone: the same bits for A/B and AA and for every
// device ordering.  Explicit rounding intrinsics keep every operation's order
// fixed against compiler contraction.
template <int S, int SCHEME>
__global__ void __launch_bounds__(kMassThreads) k_mass_partials(const DomDev *__restrict__ dd,
                                                                int64_t n, const int32_t *dev_of,
                                                                double2 *partials) {
    const DomDev D = *dd;
    const int64_t t = *D.step;
    const int64_t lo = (int64_t)blockIdx.x * kMassChunk;
    const int64_t hi = lo + kMassChunk < n ? lo + kMassChunk : n;
    double a = 0.0, b = 0.0;
    for (int64_t c = lo + threadIdx.x; c < hi; c += blockDim.x) {
        const int64_t s = dev_of ? (int64_t)dev_of[c] : c;
        unroll<0, 19>([&](auto ic) {
            constexpr int I = decltype(ic)::v;
            const double v = St<S>::ldd(stored_F<S, SCHEME, I>(D, t, s), I);
            a = __dadd_rn(a, v);
            if (!isfinite(v)) b = __dadd_rn(b, 1.0);
        });
    }
    block_sum2(a, b);
    if (threadIdx.x == 0) partials[blockIdx.x] = make_double2(a, b);
}

// The same sum over a state already in canonical order ([19][stride]).
template <int S>
__global__ void __launch_bounds__(kMassThreads) k_mass_partials_flat(const typename St<S>::T *f, int64_t n,
                                                                     int64_t stride, double2 *partials) {
    const int64_t lo = (int64_t)blockIdx.x * kMassChunk;
    const int64_t hi = lo + kMassChunk < n ? lo + kMassChunk : n;
    double a = 0.0, b = 0.0;
    for (int64_t c = lo + threadIdx.x; c < hi; c += blockDim.x) {
        unroll<0, 19>([&](auto ic) {
            constexpr int I = decltype(ic)::v;
            const double v = St<S>::ldd(f[(int64_t)I * stride + c], I);
            a = __dadd_rn(a, v);
            if (!isfinite(v)) b = __dadd_rn(b, 1.0);
        });
    }
    block_sum2(a, b);
    if (threadIdx.x == 0) partials[blockIdx.x] = make_double2(a, b);
}

__global__ void __launch_bounds__(kMassThreads) k_mass_final(const double2 *partials, int64_t np_,
                                                             double2 *out) {
    double a = 0.0, b = 0.0;
    for (int64_t j = threadIdx.x; j < np_; j += blockDim.x) {
        a = __dadd_rn(a, partials[j].x);
        b = __dadd_rn(b, partials[j].y);
    }
    block_sum2(a, b);
    if (threadIdx.x == 0) *out = make_double2(a, b);
}

inline unsigned rb_grid(int64_t n) {
    int64_t g = (n + 255) / 256;
    if (g > 152 * 64) g = 152 * 64;
    return (unsigned)(g > 0 ? g : 1);
}

}  // namespace

cudaError_t launch_stream_collide(const CollideCfg &cfg, const DomDev *doms, const TileDev *tiles,
                                  int64_t n_tiles, int off, int parity, const OneDomain &one,
                                  cudaStream_t st) {
    if (n_tiles <= 0) return cudaSuccess;
    // A/B reads its buffer parity per block: specialising it measured slower (the
    // compile-time buffer choice raised the variant-3 kernel from 52 to 58 registers)
    const int par = cfg.scheme == kAB ? 2 : (parity == 0 || parity == 1 ? parity : 2);
#define HG_PART(S_, C_, P_)                                                                    \
    if (cfg.storage == S_ && cfg.scheme == C_ && par == P_)                                   \
        return launch_sc_part<S_, C_, P_>(cfg, doms, tiles, n_tiles, off, one, st);
    HG_PART(kF32, kAB, 2) HG_PART(kF32, kAA, 0) HG_PART(kF32, kAA, 1) HG_PART(kF32, kAA, 2)
    HG_PART(kF16, kAB, 2) HG_PART(kF16, kAA, 0) HG_PART(kF16, kAA, 1) HG_PART(kF16, kAA, 2)
    HG_PART(kBF16, kAB, 2) HG_PART(kBF16, kAA, 0) HG_PART(kBF16, kAA, 1) HG_PART(kBF16, kAA, 2)
#undef HG_PART
    return cudaErrorInvalidValue;
}

cudaError_t launch_iolet_update(const IoDev *ios, int n_ios, const int2 *chunks, int n_chunks,
                                double2 *partials, unsigned *counters, int off, cudaStream_t st) {
    if (n_ios <= 0 || n_chunks <= 0) return cudaSuccess;
    k_iolet_update<<<n_chunks, kIoChunk, 0, st>>>(ios, n_ios, chunks, partials, counters, off);
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

cudaError_t launch_guo_force(int storage, int scheme, const DomDev *doms, const int2 *fslots, int n,
                             int off, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)((n + 127) / 128);
    HG_DISPATCH_SS(storage, scheme, (k_guo_force<S_, C_><<<grid, 128, 0, st>>>(doms, fslots, n, off)));
    return cudaGetLastError();
}

cudaError_t launch_macroscopic(int storage, int scheme, const DomDev *dom_dev, int64_t n,
                               const int32_t *canon_of, float4 *out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    HG_DISPATCH_SS(storage, scheme,
                   (k_macroscopic<S_, C_><<<rb_grid(n), 256, 0, st>>>(dom_dev, n, canon_of, out)));
    return cudaGetLastError();
}

cudaError_t launch_export_state(int storage, int scheme, const DomDev *dom_dev, int64_t n,
                                const int32_t *canon_of, void *out, cudaStream_t st, int64_t row) {
    if (n <= 0) return cudaSuccess;
    if (row == 0) row = n;
    HG_DISPATCH_SS(storage, scheme,
                   (k_export_state<S_, C_><<<rb_grid(n), 256, 0, st>>>(
                       dom_dev, n, canon_of, (typename St<S_>::T *)out, row)));
    return cudaGetLastError();
}

cudaError_t launch_import_state(int storage, int scheme, const DomDev *dom_dev, int64_t n,
                                const int32_t *canon_of, const void *in, cudaStream_t st, int64_t row) {
    if (n <= 0) return cudaSuccess;
    if (row == 0) row = n;
    HG_DISPATCH_SS(storage, scheme,
                   (k_import_state<S_, C_><<<rb_grid(n), 256, 0, st>>>(
                       dom_dev, n, canon_of, (const typename St<S_>::T *)in, row)));
    return cudaGetLastError();
}

cudaError_t launch_halo_pack(int elem, const DomDev *doms, const int64_t *steps, const HaloDev *ent,
                             int64_t n, void *send, int off, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (elem == 4) k_halo_pack<uint32_t><<<rb_grid(n), 256, 0, st>>>(doms, steps, ent, n, (uint32_t *)send, off);
    else k_halo_pack<uint16_t><<<rb_grid(n), 256, 0, st>>>(doms, steps, ent, n, (uint16_t *)send, off);
    return cudaGetLastError();
}

cudaError_t launch_halo_unpack(int elem, const DomDev *doms, const int64_t *steps, const HaloDev *ent,
                               int64_t n, const void *recv, int off, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (elem == 4)
        k_halo_unpack<uint32_t><<<rb_grid(n), 256, 0, st>>>(doms, steps, ent, n, (const uint32_t *)recv, off);
    else
        k_halo_unpack<uint16_t><<<rb_grid(n), 256, 0, st>>>(doms, steps, ent, n, (const uint16_t *)recv, off);
    return cudaGetLastError();
}

cudaError_t launch_halo_direct(int elem, const DomDev *doms, const int64_t *steps, const HaloMove *mv,
                               int64_t n, int off, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (elem == 4) k_halo_direct<uint32_t><<<rb_grid(n), 256, 0, st>>>(doms, steps, mv, n, off);
    else k_halo_direct<uint16_t><<<rb_grid(n), 256, 0, st>>>(doms, steps, mv, n, off);
    return cudaGetLastError();
}

cudaError_t launch_mass_flat(int storage, const void *f, int64_t n, int64_t stride, double2 *partials,
                             double2 *out, cudaStream_t st) {
    const int64_t P = mass_partials_needed(n);
    if (n <= 0) return cudaMemsetAsync(out, 0, sizeof(double2), st);
    if (storage == kF32)
        k_mass_partials_flat<kF32><<<(unsigned)P, kMassThreads, 0, st>>>((const float *)f, n, stride, partials);
    else if (storage == kF16)
        k_mass_partials_flat<kF16><<<(unsigned)P, kMassThreads, 0, st>>>((const __half *)f, n, stride, partials);
    else
        k_mass_partials_flat<kBF16><<<(unsigned)P, kMassThreads, 0, st>>>((const __nv_bfloat16 *)f, n, stride,
                                                                           partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_mass_final<<<1, kMassThreads, 0, st>>>(partials, P, out);
    return cudaGetLastError();
}

int64_t mass_partials_needed(int64_t n) { return n > 0 ? (n + kMassChunk - 1) / kMassChunk : 1; }

cudaError_t launch_mass(int storage, int scheme, const DomDev *dom_dev, int64_t n, const int32_t *dev_of,
                        double2 *partials, double2 *out, cudaStream_t st) {
    const int64_t P = mass_partials_needed(n);
    if (n <= 0) {
        return cudaMemsetAsync(out, 0, sizeof(double2), st);
    }
    HG_DISPATCH_SS(storage, scheme,
                   (k_mass_partials<S_, C_><<<(unsigned)P, kMassThreads, 0, st>>>(dom_dev, n, dev_of, partials)));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_mass_final<<<1, kMassThreads, 0, st>>>(partials, P, out);
    return cudaGetLastError();
}

}  // namespace hg
