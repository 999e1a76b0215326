// hg_internal.h -- device-side tables shared by the host runtime (hg_host.cpp)
// and the kernels (hg_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hg {

// Device neighbour table: entry i-1 of site s holds the device index of the
// pull source when it is fluid, else a virtual index chosen so the scheme's
// gather address lands on the site's own opposite slot (bounce-back):
//   A/B:  s + (opp(i) - i) * np      (src row i  + v  ==  row opp(i) + s)
//   AA:   s + (i - opp(i)) * np      (buf row opp(i) + v  ==  row i + s)
// Virtual indices lie outside [0, n).  Links into iolet openings are told apart
// through iomask / ioprefix / io_codes (canonical codes per boundary slot).
constexpr int kMaxIolets = 4096;

enum Storage : int { kF32 = 0, kF16 = 1, kBF16 = 2 };
enum Scheme : int { kAB = 0, kAA = 1 };

// Per-domain descriptor read by the stream-collide and read-back kernels.
constexpr int kRunStride = 20;  // int32 entries per run of a run-encoded neighbour table

struct DomDev {
    void *f[2];               // distributions, SoA [19][np]; AA uses f[0] only
    const int32_t *nbr;       // [18][np] device codes
    // The same table run-length encoded (null when it does not compress): per site
    // a word whose bits 0..17 flag the non-fluid links (their entry is the virtual
    // index) and whose bits 18..27 give the site's run relative to the run of its
    // 1024-site chunk (run0); per run the 18 offsets (entry minus site index) its
    // fluid links share.
    const uint32_t *lword;
    const int32_t *run0;
    const int32_t *rdelta;    // kRunStride entries per run: 18 offsets, 2 zeros (16-byte rows)
    const uint32_t *iomask;   // bit s: site s has an iolet link
    const int32_t *ioprefix;  // per 32-site word: flagged sites before it (slot = rank of the flag)
    const int32_t *io_codes;  // per slot x 18: canonical codes (-1 wall, -(2+k) iolet, >= 0 fluid)
    float4 *bnd;              // per adjacent slot: (drho, ux, uy, uz) of the step's G_t
    const float *coef;        // per adjacent slot x 18: velocity-link coefficient 6 w_i c_i.(-a) phi
    const float *bcv;         // per iolet: boundary value of the step being run
    const int8_t *io_kind;    // per iolet: 0 pressure, 1 velocity
    const int64_t *step;      // completed steps before the current launch group
    int32_t *err;             // context error word: set when a bounded device wait gives up
    int64_t n;                // sites
    int64_t np;               // row stride (n padded)
    float omega;              // 1 / tau
    int32_t n_io;
    // read by the body-force pass only (kept after the fields stream-collide reads)
    const int32_t *slot_site; // per slot: the site's device index
    const float4 *io_force;   // per iolet: body-force density on its adjacent sites (null = none)
};

// A launch over one domain only: its descriptor (host copy, passed by value as a
// kernel parameter) and site count; d == nullptr means "use the tile table".
// steps: the context's per-domain step counters (indexed by TileDev::dom).
// overlap_previous: the launch directly follows the previous step's iolet update
// on the stream and may start before it ends (programmatic dependent launch);
// only sites with iolet links wait for it.
struct OneDomain {
    const DomDev *d;
    int64_t n;
    const int64_t *steps;
    bool overlap_previous;
};

// One block of the stream-collide grid: `count` sites of domain `dom` from `start`.
struct TileDev {
    int32_t dom;
    int32_t count;
    int64_t start;
};

// A venous inlet fed by an arterial outlet, seen from the outlet (reverse exchange).
struct RevSrc {
    const double *M;          // the inlet's means (mean u.n first)
    double factor;            // the pair's velocity factor
};

// Per-iolet work of the iolet-update kernel (reduction + next boundary value).
struct IoDev {
    const int32_t *slots;     // adjacent-site slots of this iolet, canonical order
    const float4 *bnd;        // owner's per-slot moments
    const double *src_M;      // coupled source iolet's means (or null)
    double *M;                // out: (mean u.n, mean drho, count)
    float *bcv;               // out: boundary value for the next step
    const int64_t *step;      // owner's completed-step counter
    const RevSrc *rev;        // inlets this outlet feeds (reverse exchange), n_rev of them
    float4 *force;            // out (reverse exchange): this iolet's body-force density
    double nx, ny, nz;        // unit outward axis
    double value, period, factor;
    int32_t n_slots;
    int32_t n_chunks;         // ceil(n_slots / kIoChunk), at least 1
    int32_t part0;            // first partial of this iolet in the plan's partials array
    int32_t pulse;
    int32_t coupled;
    int32_t n_rev;
    int32_t alternate;        // 1: exchanges alternate forward (even step) / reverse (odd step)
    int32_t pad;
};

// Slots reduced by one CTA of the iolet-update kernel.
constexpr int kIoChunk = 256;

// Launch configuration of the stream-collide kernel.
struct CollideCfg {
    int storage;
    int scheme;
    int block;
    int spt;
    int variant;  // 0 = gathers into registers, 1 = gathers staged by cp.async (spt 1 or 2),
                  // 2 = as 1, and the AA even step moves whole rows with TMA bulk copies,
                  // 3 = as 0 with L2 prefetch hints, 4 = as 1 with the AA odd step's
                  // stores staged in shared memory (spt 1), 5 = A/B on adjacent site
                  // pairs (16-bit storage, spt 2)
};

// parity (AA only): 0 = every domain runs an even step, 1 = odd, 2 = per-domain
// parity read from the step counters.
cudaError_t launch_stream_collide(const CollideCfg &cfg, const DomDev *doms, const TileDev *tiles,
                                  int64_t n_tiles, int off, int parity, const OneDomain &one,
                                  cudaStream_t st);
// The stream-collide kernels of one storage type S (0 f32, 1 f16, 2 bf16), scheme
// (0 A/B, 1 AA) and launch parity PAR (0 even, 1 odd, 2 read from the step counter;
// A/B always 2): every variant and shape, instantiated in a translation unit of its
// own (hg_sc_part.cu, compiled once per combination, so the twelve build in parallel).
template <int S, int SCHEME, int PAR>
cudaError_t launch_sc_part(const CollideCfg &cfg, const DomDev *doms, const TileDev *tiles, int64_t n_tiles,
                           int off, const OneDomain &one, cudaStream_t st);
#define HG_SC_PART_DECL(S_, C_, P_)                                                                  \
    template <>                                                                                     \
    cudaError_t launch_sc_part<S_, C_, P_>(const CollideCfg &, const DomDev *, const TileDev *, int64_t, int, \
                                           const OneDomain &, cudaStream_t);
HG_SC_PART_DECL(0, 0, 2) HG_SC_PART_DECL(0, 1, 0) HG_SC_PART_DECL(0, 1, 1) HG_SC_PART_DECL(0, 1, 2)
HG_SC_PART_DECL(1, 0, 2) HG_SC_PART_DECL(1, 1, 0) HG_SC_PART_DECL(1, 1, 1) HG_SC_PART_DECL(1, 1, 2)
HG_SC_PART_DECL(2, 0, 2) HG_SC_PART_DECL(2, 1, 0) HG_SC_PART_DECL(2, 1, 1) HG_SC_PART_DECL(2, 1, 2)
#undef HG_SC_PART_DECL
// One CTA per (iolet, chunk) in `chunks`; partials: 2 doubles per chunk;
// counters: n_ios + 1 zeroed unsigned ints (left zeroed on return).
cudaError_t launch_iolet_update(const IoDev *ios, int n_ios, const int2 *chunks, int n_chunks,
                                double2 *partials, unsigned *counters, int off, cudaStream_t st);
cudaError_t launch_advance_list(int64_t *steps_base, const int32_t *idx, int n, int64_t by,
                                cudaStream_t st);
// Body force on the listed boundary slots ((domain, slot) pairs), right after the
// stream-collide launch of step offset `off` and before the iolet update.
cudaError_t launch_guo_force(int storage, int scheme, const DomDev *doms, const int2 *fslots, int n,
                             int off, cudaStream_t st);
// Reconstruct F_t of one domain (device order) and write macroscopic fields
// (drho, ux, uy, uz) to out[canon_of ? canon_of[s] : s] (device -> canonical index).
cudaError_t launch_macroscopic(int storage, int scheme, const DomDev *dom_dev, int64_t n,
                               const int32_t *canon_of, float4 *out, cudaStream_t st);
// Raw state export/import of F_t of device sites [0, n) in canonical order
// (storage type, [19][row] with row = n, or `row` when non-zero: the sites of a
// partition written into the whole domain's rows).
cudaError_t launch_export_state(int storage, int scheme, const DomDev *dom_dev, int64_t n,
                                const int32_t *canon_of, void *out, cudaStream_t st, int64_t row = 0);
cudaError_t launch_import_state(int storage, int scheme, const DomDev *dom_dev, int64_t n,
                                const int32_t *canon_of, const void *in, cudaStream_t st, int64_t row = 0);

// One value of the halo exchange between partitions of a split domain: direction
// row and site of one partition's distributions (offset = row * np + site in the
// buffer holding F_t).
struct HaloDev {
    int32_t dom;    // descriptor (context domain table index) of the partition
    int32_t pad;
    int64_t off;
};
// After the stream-collide launch of step offset `off`: copy F_t values of the
// owning partitions into a send buffer (pack), or from a receive buffer into the
// ghost positions of the reading partitions (unpack); elem = 4 or 2 bytes.
cudaError_t launch_halo_pack(int elem, const DomDev *doms, const int64_t *steps, const HaloDev *ent,
                             int64_t n, void *send, int off, cudaStream_t st);
cudaError_t launch_halo_unpack(int elem, const DomDev *doms, const int64_t *steps, const HaloDev *ent,
                               int64_t n, const void *recv, int off, cudaStream_t st);
// One halo value moved straight from the sender's F_t to the receiver's ghost (both
// partitions on one device): element offsets into the partitions' distribution
// buffers, below 19 * np < 2^32 (a split holds at most 200 * 2^20 sites).
struct HaloMove {
    int32_t src_dom, dst_dom;
    uint32_t src_off, dst_off;
};
cudaError_t launch_halo_direct(int elem, const DomDev *doms, const int64_t *steps, const HaloMove *mv,
                               int64_t n, int off, cudaStream_t st);
// Mass of a state held in canonical order ([19][stride], sites [0, n)): the same
// chunks, order and rounding as launch_mass.
cudaError_t launch_mass_flat(int storage, const void *f, int64_t n, int64_t stride, double2 *partials,
                             double2 *out, cudaStream_t st);
// Mass check: FP64 partial sums of F_t over fixed chunks of 8192 sites in
// canonical order, each site's values in direction order (dev_of: canonical ->
// device index, null = identity), then a fixed-order final sum.  Each partial
// also counts the non-finite values (NaN/Inf watchdog).  partials needs
// mass_partials_needed(n) entries; out receives (mass, non-finite count).
int64_t mass_partials_needed(int64_t n);
cudaError_t launch_mass(int storage, int scheme, const DomDev *dom_dev, int64_t n, const int32_t *dev_of,
                        double2 *partials, double2 *out, cudaStream_t st);

}  // namespace hg
