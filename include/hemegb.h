/*
 * hemegb.h -- C ABI of the GB300 sparse lattice-Boltzmann hot path.
 *
 * Method: "Towards Blood Flow in the Virtual Human: Efficient Self-Coupling of
 * HemeLB" (arXiv 2010.04144).  Section 2 fixes the solver: D3Q19 lattice,
 * single-relaxation-time (LBGK) collision, rigid walls, pressure and velocity
 * boundary conditions at inlets and outlets, Newtonian fluid on a sparse
 * vascular geometry.  Section 2.3 and Section 3 fix the self-coupling: only
 * averaged macroscopic values cross between coupled boundaries, and the
 * arterial outlet's average velocity, times a per-pair scale factor (the
 * velocity-scale equation after Eq. (1)), becomes the velocity boundary
 * condition of the paired venous inlet.
 *
 * Conventions (every function):
 *   - returns HG_OK (0) or a negative HG_ERR_* code; hg_last_error(ctx) then
 *     holds a message for the calling thread (valid until its next call);
 *   - sizes and counts are int64_t; handles are opaque;
 *   - host arrays passed in are owned by the caller and copied during the
 *     call; host arrays passed out are caller-allocated;
 *   - the library owns all device memory it allocates (through the context's
 *     allocator callback, else cudaMalloc);
 *   - work is ordered on the context's CUDA stream; hg_step* only enqueue,
 *     hg_read_* / hg_save_state / hg_mass synchronise the stream;
 *   - one thread at a time drives a context and its domains, except that
 *     hg_domain_create may run on a second thread meanwhile (its host build
 *     and uploads overlap the first thread's steps; the new domain joins the
 *     context only when complete); hg_ctx_destroy must not overlap a build.
 *
 * Lattice conventions (identical on every entry point):
 *   - velocities: i = 0 rest; 1..6 = +x,-x,+y,-y,+z,-z; 7..18 = (1,1,0),
 *     (-1,-1,0),(1,-1,0),(-1,1,0),(1,0,1),(-1,0,-1),(1,0,-1),(-1,0,1),(0,1,1),
 *     (0,-1,-1),(0,1,-1),(0,-1,1); weights 1/3, 1/18, 1/36;
 *   - canonical site order: ascending 3-D Morton key (x in bit 0);
 *   - neighbour table nbr[18][N]: nbr[i-1][s] = canonical index of the fluid
 *     site at x_s - c_i (pull source), else -(2+k) when that lattice point
 *     lies in the opening of iolet k, else -1 (wall);
 *   - distributions are stored as deviations from the lattice weights
 *     (f~ = f - w); FP16/BF16 storage keeps f~_i / w_i.
 */
#ifndef HEMEGB_H
#define HEMEGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define HG_OK 0
#define HG_ERR_ARG (-1)     /* invalid argument (sizes, ranges, handles) */
#define HG_ERR_OOM (-2)     /* device or host allocation failed */
#define HG_ERR_CUDA (-3)    /* a CUDA call failed (message holds the CUDA error) */
#define HG_ERR_TIMEOUT (-4) /* a bounded device wait gave up: the state is not trusted */
#define HG_ERR_STATE (-5)   /* call not valid in the object's current state */

/* ---- distribution storage ---- */
#define HG_STORE_F32 0  /* f~ in FP32 */
#define HG_STORE_F16 1  /* f~/w in FP16 (round to nearest even), collision in FP32 */
#define HG_STORE_BF16 2 /* f~/w in BF16 (round to nearest even), collision in FP32 */

/* ---- propagation scheme ---- */
#define HG_SCHEME_AB 0 /* two buffers, pull streaming every step */
#define HG_SCHEME_AA 1 /* one buffer, in place: even steps local, odd steps gather+scatter */

/* ---- iolets ---- */
#define HG_PRESSURE 0  /* anti-bounce-back: f~_i = -f~*_opp + 2 w_i drho_k */
#define HG_VELOCITY 1  /* moving-wall bounce-back: f~_i = f~*_opp + 6 w_i c_i.u_w */
#define HG_PLUG 0      /* velocity profile: uniform */
#define HG_PARABOLIC 1 /* velocity profile: peak on the axis, zero at the radius */
#define HG_PULSE_CONST 0  /* value(t) = value */
#define HG_PULSE_COSINE 1 /* value(t) = value * (1 - cos(2 pi t / period)) / 2 */
#define HG_PULSE_SINE 2   /* value(t) = value * sin(2 pi t / period) */

/* ---- site orderings (device layout; exported data is always canonical) ----
 * Every ordering gives bit-identical fields, iolet means and mass: the per-site
 * arithmetic does not depend on it, each iolet's FP64 sums and the mass sum
 * run in canonical order.  Only the memory access pattern changes. */
#define HG_ORDER_MORTON 0 /* canonical order */
#define HG_ORDER_ROWS 1   /* lexicographic: x fastest, then y, then z */
#define HG_ORDER_BRICKS 2 /* x-fastest rows inside 32 x 8 x 8 bricks, bricks in Morton order */

/* ---- host-side fault injection (hg_ctx_inject_fault) ---- */
#define HG_FAULT_ALLOC 1       /* the arg-th device allocation from now on fails (0 cancels) */
#define HG_FAULT_DEVICE_WAIT 2 /* set the device error word as a bounded wait that gave up does */

/* Coupling exchange direction (Section 3 alternates forward and reverse). */
#define HG_COUPLE_FORWARD 0   /* forward after every step (default) */
#define HG_COUPLE_ALTERNATE 1 /* forward after even steps, reverse after odd steps */

typedef struct hg_ctx hg_ctx;
typedef struct hg_domain hg_domain;
typedef struct hg_split hg_split;

/* Device allocator hook: returns a device pointer of at least `bytes` bytes
 * (256-byte aligned) or NULL; `free` receives the pointer and size. */
typedef void *(*hg_alloc_fn)(size_t bytes, void *user);
typedef void (*hg_free_fn)(void *ptr, size_t bytes, void *user);

typedef struct {
    int32_t device;           /* CUDA device ordinal */
    int32_t storage;          /* HG_STORE_* */
    int32_t scheme;           /* HG_SCHEME_* */
    int32_t block_size;       /* stream-collide threads per block (multiple of 32, <= 512); 0 = 256 */
    int32_t sites_per_thread; /* 1, 2 or 4; 0 = 1 */
    int32_t graph_steps;      /* steps captured per CUDA graph; 0 = 16; negative = no graphs */
    int32_t kernel_variant;   /* stream-collide form; every form gives bit-identical results:
                                 0 = gathers into registers;
                                 1 = gathers staged in shared memory by cp.async, AA even step
                                     on site pairs (sites_per_thread 1 or 2);
                                 2 = 1, with the AA even step moved by TMA bulk copies (AA only,
                                     sites_per_thread 1 or 2);
                                 3 = 0, with L2 256-byte prefetch hints on every load;
                                 4 = 1, with the AA odd step's stores staged in shared memory
                                     and written coalesced (AA only, sites_per_thread 1);
                                 5 = 0 on pairs of adjacent sites sharing table loads and
                                     packed stores (A/B with FP16/BF16 storage,
                                     sites_per_thread 2);
                                 6 = AA on pairs of adjacent sites: shared table loads for
                                     the gathers and the scatter, packed rest values, the
                                     even step on vector pairs (sites_per_thread 2);
                                 7 = 6 with L2 256-byte prefetch hints on the loads;
                                 8, 9, 10, 11 = 3, 5, 6, 7 reading the run-encoded
                                     neighbour table (hg_domain_runs) instead of the
                                     18 table rows; a launch over a domain without
                                     one runs 3, 5, 6, 7; same shapes as 3, 5, 6, 7;
                                 12 = 8 for AA (1 or 2 sites per thread) with the odd
                                     step's 18 entries stashed in shared memory
                                     across the collision instead of decoded twice;
                                 13 = 8 (2 or 4 sites per thread) with every site's
                                     link word loaded, and its run row prefetched,
                                     before the first site's gathers;
                                 14 = 10 with the stash of 12 (AA, 2 sites per
                                     thread) */
    void *stream;             /* cudaStream_t to order work on; NULL = a stream the context creates */
    hg_alloc_fn alloc;        /* NULL = cudaMalloc */
    hg_free_fn free;          /* NULL = cudaFree */
    void *alloc_user;
} hg_ctx_params;

/* Iolet descriptor.  Section 3.1: vessel tips are cut flat, perpendicular to
 * the centreline; the cut disc is the opening.  Fixed point: 1 lattice unit =
 * 1024.  A non-fluid lattice point q is in the opening when it lies beyond the
 * plane through `centre` normal to `axis` (axis points out of the fluid) by at
 * most 2 lattice units and within `radius` of the axis line; the test is exact
 * integer arithmetic, the lowest iolet index wins.  Limits: |centre| <= 2^31,
 * |axis| components <= 2^20 (not all zero), 0 <= radius <= 2^31. */
typedef struct {
    int32_t kind;    /* HG_PRESSURE / HG_VELOCITY */
    int32_t profile; /* HG_PLUG / HG_PARABOLIC (velocity iolets) */
    int32_t pulse;   /* HG_PULSE_* */
    int32_t reserved;
    double value;    /* density deviation drho (pressure) or peak inward speed (velocity) */
    double period;   /* pulse period in steps (pulsed iolets) */
    int64_t centre[3];
    int64_t axis[3];
    int64_t radius;
} hg_iolet;

typedef struct {
    double tau;       /* relaxation time, 0.5 < tau (Section 3.3 quotes tau in (0.5, 1]) */
    int32_t ordering; /* HG_ORDER_* device site layout */
    int32_t reserved;
} hg_lb_params;

/* One forward coupling pair (Section 3): from now on the velocity iolet
 * dst_iolet of the destination domain takes, at time t, the value
 * factor * (mean of u.n over the sites next to src_iolet of the source domain
 * at time t-1), n the source iolet's unit outward axis. */
typedef struct {
    int32_t src_iolet;
    int32_t dst_iolet;
    double factor;
} hg_pair;

/* ---- context ---- */

/* Create a context on p->device.  Storage and scheme apply to every domain of
 * the context.  Errors: HG_ERR_ARG (bad field), HG_ERR_CUDA.
 * Passage: infrastructure: no passage (device, stream and memory set-up). */
int hg_ctx_create(const hg_ctx_params *p, hg_ctx **out);

/* Destroy a context and every domain still attached to it.
 * Passage: infrastructure: no passage. */
int hg_ctx_destroy(hg_ctx *ctx);

/* Message of the calling thread's last failed call, if that call concerned
 * this context (or its domains); "" otherwise.
 * Passage: infrastructure: no passage. */
const char *hg_last_error(hg_ctx *ctx);

/* Wait for all work enqueued on the context's stream.  Returns HG_ERR_TIMEOUT
 * (and clears the flag) when a bounded device wait gave up since the last
 * call, HG_ERR_STATE when a run-encoded kernel variant met a domain without a
 * run encoding (the host never launches one so): the state is then not trusted.
 * Passage: infrastructure: no passage. */
int hg_sync(hg_ctx *ctx);

/* ---- domains ---- */

/* Build a domain from fluid voxels (Section 2.2: sparse geometry, only fluid
 * sites stored).  xyz: n_fluid x 3 int32 lattice coordinates, any order, no
 * duplicates, each in [0, 2^21).  iolets: n_iolets descriptors (<= 4096).
 * Builds the canonical site order and neighbour table, classifies iolet links,
 * uploads everything and initialises the rest state f~ = 0 at step 0.
 * Errors: HG_ERR_ARG (range, duplicate, too many iolets, tau <= 0.5),
 * HG_ERR_OOM, HG_ERR_CUDA.
 * Passage: Section 2.2 (sparse blocks, fluid sites only) and Section 2
 * (D3Q19, rigid walls, pressure/velocity iolets). */
int hg_domain_create(hg_ctx *ctx, const int32_t *xyz, int64_t n_fluid, const hg_iolet *iolets,
                     int32_t n_iolets, const hg_lb_params *lb, hg_domain **out);

/* Free a domain's device memory and detach it from its context.  Coupling
 * pairs that involve it are dropped.
 * Passage: infrastructure: no passage. */
int hg_domain_destroy(hg_domain *d);

/* Sizes: sites, iolets, sites next to any iolet, completed steps, device
 * bytes held.  Any out pointer may be NULL.
 * Passage: infrastructure: no passage. */
int hg_domain_info(hg_domain *d, int64_t *n_sites, int32_t *n_iolets, int64_t *n_adjacent,
                   int64_t *step, int64_t *device_bytes);

/* Runs of the run-encoded neighbour table (0: none built).  Every domain keeps
 * its 18-row table (72 bytes per site, what the gathers of a pull step read
 * besides the populations); where it compresses (runs of at least 4.5 sites on
 * average) the build also encodes it as runs: maximal ranges of consecutive
 * device sites whose fluid links share one offset per direction (each 2^20-site
 * span starting a new run), plus a 4-byte word per site flagging its non-fluid
 * links.  In rows ordering a run covers most of an x-row of a vessel, so the
 * encoding costs about 4 + 80 / run-length bytes per site (80-byte rows).
 * Kernel variants 8..14 read it; the results are the same bits.
 * Passage: Section 2.2 (indirect addressing of the sparse fluid-site list). */
int hg_domain_runs(hg_domain *d, int64_t *n_runs);

/* Host only: the run encoding hg_domain_create builds, for a device neighbour
 * table nbr[18][row_stride] of sites [0, n) whose fluid entries lie in
 * [0, n_ref) and whose other entries are the scheme's virtual indices
 * (q + (opp(i) - i) row_stride for A/B, q + (i - opp(i)) row_stride for AA).
 * Outputs: lword_out[row_stride] (bits 0..17: link i+1 non-fluid; bits 18..27:
 * run minus run0_out[q >> 10]), run0_out[(row_stride + 1023) / 1024],
 * rdelta_out[n_runs * 18] (at most n * 16 / 72 + 1 runs); any output may be
 * NULL.  *n_runs_out = 0 when the table does not compress (average run below
 * 4.5 sites) or an entry is not of that form.  Errors: HG_ERR_ARG.
 * Passage: Section 2.2 (indirect addressing of the sparse fluid-site list). */
int hg_encode_runs(const int32_t *nbr, int64_t n, int64_t n_ref, int64_t row_stride, int32_t scheme,
                   uint32_t *lword_out, int32_t *run0_out, int32_t *rdelta_out, int64_t *n_runs_out);

/* Canonical site coordinates, n_sites x 3 int32 (host), whatever the
 * device ordering.
 * Passage: Section 2.2 (sites stored by blocks; canonical order = ascending
 * Morton key, which visits every aligned 8^3 block contiguously). */
int hg_domain_sites(hg_domain *d, int32_t *xyz_out);

/* Canonical neighbour table as used on the device, nbr[18][n_sites] int32
 * (host), decoded to the conventions above whatever the device ordering.
 * Passage: Section 2.2 (sparse geometry: streaming follows the links between
 * stored fluid sites). */
int hg_domain_neighbours(hg_domain *d, int32_t *nbr_out);

/* Host only (no context, no device): the canonical site order and neighbour
 * table hg_domain_create builds for the same input, with the same checks.
 * xyz_out: n_fluid x 3 in canonical order (may be NULL); nbr_out:
 * nbr[18][n_fluid] in the conventions above.  Errors: HG_ERR_ARG (bad sizes,
 * coordinates, duplicates or iolets).
 * Passage: Section 2.2 (sparse blocks of fluid sites). */
int hg_build_neighbours(const int32_t *xyz, int64_t n_fluid, const hg_iolet *iolets, int32_t n_iolets,
                        int32_t *xyz_out, int32_t *nbr_out);

/* ---- coupling (Section 2.3, Section 3) ---- */

/* Add forward coupling pairs from src to dst (both in ctx, src != dst).  Each
 * dst_iolet must be a velocity iolet and may appear once; the pairs take
 * effect from the next step.  Both domains must then be stepped together.
 * Errors: HG_ERR_ARG.
 * Passage: Section 2.3 (only averaged values cross) and Section 3 (the
 * velocity-scale equation after Eq. (1)). */
int hg_couple(hg_ctx *ctx, hg_domain *src, hg_domain *dst, const hg_pair *pairs, int32_t n_pairs);

/* Exchange schedule of every coupling pair of the context (Section 3: the
 * exchange alternates between the forward and the reverse direction).
 * HG_COUPLE_FORWARD: after every step each coupled venous inlet takes factor
 * x the mean u.n of its arterial outlet.  HG_COUPLE_ALTERNATE: the exchange
 * after step e is that forward one when e is even; when e is odd it is the
 * reverse one instead: every arterial outlet k that feeds inlets J_k gets
 * v_k = mean over j in J_k of (inflow speed at j, i.e. -mean u.n) / factor_j
 * and the body-force density F_k = -(1/2) v_k |v_k| n_k (n_k its unit outward
 * axis), which acts on every site next to outlet k through Guo, Zheng and Shi
 * forcing (u = (j + F/2)/rho, source (1 - 1/(2 tau)) w_i [3 (c_i - u) +
 * 9 (c_i.u) c_i].F) until the next reverse exchange.  Each exchange leaves
 * the other direction's values unchanged.  The paper describes the reverse
 * direction in words only; this is the library's reading of it.  Setting a
 * mode zeroes every force.  Synchronises the stream.  Errors: HG_ERR_ARG.
 * Passage: Section 3 (alternating exchange; Guo forcing from the dynamic
 * pressure at the arterial outlets). */
int hg_set_coupling_mode(hg_ctx *ctx, int32_t mode);

/* Host helper for Section 3's coupling map and scale factors.
 * Map: arteries in ascending order each take the closest venous inlet not yet
 * taken; every venous inlet left joins its closest artery (ties: lowest
 * index; distances compared exactly on the fixed-point centres).  Pressure
 * drops: dP_v/P_0 = 0.3 + 0.4 * uniforms[v] (uniform in [0.3, 0.7]).
 * Factors: the velocity-scale equation after Eq. (1),
 *   v_i/v_0 = (A_0/A_i) r_i / sum_j r_j,  r_i = dP_i L_1 A_i / (dP_1 L_i A_1).
 * Inputs: art_centres n_art x 3 and ven_centres n_ven x 3 (fixed point 2^-10),
 * areas in lattice units^2, uniforms n_ven values in [0, 1).  Outputs (n_ven
 * each): assign (artery index), dist (lattice units), dp, factor.
 * Errors: HG_ERR_ARG (n_art < 1, zero distance, non-positive area).
 * Passage: Section 3 (greedy nearest-neighbour map; dP/P_0 ~ U(0.3, 0.7);
 * Eq. (1) and the velocity-scale equation after it). */
int hg_coupling_factors(const int64_t *art_centres, const double *art_areas, int32_t n_art,
                        const int64_t *ven_centres, const double *ven_areas, int32_t n_ven,
                        const double *uniforms, int32_t *assign, double *dist, double *dp,
                        double *factor);

/* ---- stepping ---- */

/* Advance every domain of the context by n_steps LB steps (split domains are
 * advanced by hg_split_step).  Step t streams the
 * post-collision state F_{t-1} (pull from x - c_i; wall, pressure and velocity
 * rules on non-fluid links, with boundary values of time t), collides (LBGK,
 * tau) into F_t, then reduces the iolet means of time t in FP64 and sets the
 * boundary values of time t+1 (pulses; coupled inlets from the means).
 * Groups of steps run as captured CUDA graphs.  Asynchronous.
 * Passage: Section 2 (the LB step: D3Q19 streaming, LBGK collision, walls,
 * iolets) and Section 2.3 (coupled values exchanged every step). */
int hg_step(hg_ctx *ctx, int64_t n_steps);

/* Same for a subset of the context's domains (coupled partners included);
 * the domains may be at different step counts.
 * Passage: Section 2 and Section 2.3, as hg_step. */
int hg_step_domains(hg_ctx *ctx, hg_domain *const *doms, int32_t n_doms, int64_t n_steps);

/* Like hg_step but without graphs and with CUDA events around every kernel:
 * total milliseconds spent in the stream-collide kernel and in the iolet
 * update kernel; per_step (2 x n_steps floats, may be NULL) receives each
 * step's (stream-collide ms, iolet-update ms).  Any pointer may be NULL.
 * Synchronises.
 * Passage: Section 2 (the LB step), timed per kernel (infrastructure). */
int hg_step_profiled(hg_ctx *ctx, int64_t n_steps, double *ms_stream_collide,
                     double *ms_iolet, float *per_step);

/* Change the stream-collide launch shape of an existing context (threads per
 * block: multiple of 32, <= 512; sites per thread: 1, 2 or 4; kernel variant
 * as in hg_ctx_params).  Results do not depend on it (each site's arithmetic
 * is the same); used by the autotuner.  Errors: HG_ERR_ARG.
 * Passage: infrastructure: no passage. */
int hg_ctx_set_launch(hg_ctx *ctx, int32_t block_size, int32_t sites_per_thread,
                      int32_t kernel_variant);

/* ---- read-back ---- */

/* Macroscopic fields of the current state F_t, canonical order, n_sites x 4
 * FP32 host array: (drho, ux, uy, uz), drho = rho - 1, u = j / rho.
 * Passage: Section 2 (the macroscopic density and velocity of the LB state). */
int hg_read_macroscopic(hg_domain *d, float *out, int64_t *step_out);

/* Same into a caller-owned device array (n_sites x 4 FP32, 16-byte aligned);
 * asynchronous on the context stream.
 * Passage: Section 2, as hg_read_macroscopic. */
int hg_read_macroscopic_device(hg_domain *d, float *dev_out);

/* Iolet means of the last completed step, n_iolets x 3 FP64 host array:
 * (mean u.n over the sites next to the iolet, mean drho there, site count);
 * n is the iolet's unit outward axis.  Sums in FP64 in canonical order.
 * Passage: Section 2.3 (only the average value of macroscopic properties is
 * passed between coupled instances). */
int hg_read_iolet_stats(hg_domain *d, double *out);

/* Boundary values the next step will use, n_iolets FP32 (host).
 * Passage: Section 2 (iolet conditions) and Section 3 (coupled inlets). */
int hg_read_boundary_values(hg_domain *d, float *out);

/* Body-force densities the next step applies next to each iolet (reverse
 * coupling exchange, see hg_set_coupling_mode), n_iolets x 3 FP32 (host).
 * Passage: Section 3 (reverse direction: arterial-outlet boundary force). */
int hg_read_iolet_forces(hg_domain *d, float *out);

/* Total mass deviation sum_s sum_i f~_i(s) of the current state, FP64: fixed
 * chunks of 8192 sites in canonical order, each summed by a fixed tree, the
 * chunk sums added in order (the same bits for every device ordering).
 * Passage: infrastructure: no passage (mass check of the LB state; the paper
 * describes none). */
int hg_mass(hg_domain *d, double *out);

/* Total mass deviation of a caller-owned distribution array, without any
 * device allocation.  The paper has no counterpart: this exists for callers
 * that may not allocate device memory -- an application whose own pool
 * already owns the whole device heap, or a monitoring thread that must not
 * call cudaMalloc/cudaFree because they can synchronise the device and stall
 * the solver.  f_dev: 19 rows of row_stride values of the given storage type
 * (HG_STORE_*; FP16/BF16 rows hold f~/w), sites 0..n-1 of each row are summed
 * (FP64, fixed chunks of 8192 sites, same order as hg_mass); out_dev: one
 * double in device memory; stream: cudaStream_t (NULL = legacy default).
 * Scratch: a fixed 16384-double array inside the library, held on every GPU
 * that loads it until the process exits, so n is limited to 134,217,728 sites
 * (HG_ERR_ARG beyond).  The first call on a device looks up that array's
 * device address (cudaGetSymbolAddress) with the device current; make that
 * first call before any stream capture.  The address is kept for the rest of
 * the process: it belongs to the device's primary context as it was at that
 * first call, so after cudaDeviceReset (or any teardown of that context) this
 * entry point must not be called again in the same process.  All calls share the array: calls
 * whose kernels overlap on the GPU race and may return wrong sums; calls
 * ordered on one stream are safe.  Asynchronous.  Errors: HG_ERR_ARG,
 * HG_ERR_CUDA.
 * Passage: no counterpart in the paper (see above). */
int hg_mass_noalloc(const void *f_dev, int32_t storage, int64_t n, int64_t row_stride,
                    double *out_dev, void *stream);

/* Mass check with a NaN/Inf watchdog: the FP64 mass of the current state
 * (as hg_mass) and the number of stored values that are not finite.  Returns
 * HG_ERR_STATE when that number is non-zero (both outputs are still filled).
 * Either pointer may be NULL.  Synchronises.
 * Passage: infrastructure: no passage (state watchdog). */
int hg_state_check(hg_domain *d, double *mass, int64_t *nonfinite);

/* The per-site moments the last step's iolet reductions took as input: for
 * every site next to any iolet, in canonical order, its canonical index
 * (sites_out, n_adjacent int64) and (drho, ux, uy, uz) FP32 (mom_out,
 * n_adjacent x 4) of that step's collision.  hg_read_iolet_stats holds the FP64
 * means of exactly these values.  Synchronises.
 * Passage: Section 2.3 (the averaged macroscopic values passed between coupled
 * instances are averages of these per-site values). */
int hg_read_adjacent_moments(hg_domain *d, int64_t *sites_out, float *mom_out);

/* Host-side fault injection for tests of the error paths (no GPU fault is
 * made).  HG_FAULT_ALLOC: the arg-th device allocation the context makes from
 * now on (1 = the next) fails as if the allocator returned NULL; the call that
 * makes it returns HG_ERR_OOM and releases what it had set up; arg = 0 cancels.
 * HG_FAULT_DEVICE_WAIT: writes code arg (0 -> 1) to the context's device error
 * word, stream-ordered, exactly as a bounded device wait that gave up would;
 * the next hg_sync returns HG_ERR_TIMEOUT.  Errors: HG_ERR_ARG, HG_ERR_CUDA.
 * Passage: infrastructure: no passage (failure detection). */
int hg_ctx_inject_fault(hg_ctx *ctx, int32_t kind, int64_t arg);

/* ---- split (partitioned) domains ----
 * Section 2.2 decomposes the sparse domain over ranks and ends every step with a
 * non-blocking exchange of the populations that cross the cuts; Section 2.2.1
 * balances the cut.  A split domain cuts the canonical site list into n_parts
 * contiguous ranges of equal cost (a site costs 1, a site with a link into an
 * iolet opening costs boundary_weight); each partition holds its own
 * distributions and neighbour table plus ghost copies of the sites it pulls
 * from, and after every stream-collide the crossing values move into the
 * receivers' ghosts: directly, by one kernel, or staged as messages (packed per
 * (sender, receiver) pair, copied into the receiver's buffer, unpacked).  Iolet means are reduced over the whole domain in canonical
 * order, so a split run is bit-identical to the same domain unsplit.  All
 * partitions of a split live on the context's device; the A/B scheme only; a
 * split takes no part in coupling, and hg_step does not advance it. */
#define HG_EXCHANGE_DIRECT 0 /* one kernel moves every halo value from sender to receiver */
#define HG_EXCHANGE_STAGED 1 /* pack per (sender, receiver) block, one copy per block, unpack:
                                the message form of a transport between devices */
typedef struct {
    int32_t n_parts;        /* 1 <= n_parts <= min(n_fluid, 1024) */
    int32_t exchange;       /* HG_EXCHANGE_DIRECT or HG_EXCHANGE_STAGED (same bits either way) */
    double boundary_weight; /* cost of a site next to an iolet relative to a bulk site (<= 0: 1) */
} hg_split_params;

/* Host only: the cut (first_out, n_parts + 1 canonical indices), the ghost
 * count of every partition (ghosts_out, n_parts) and the halo values each pair
 * exchanges per step (halo_out[q * n_parts + p]: values partition p pulls from
 * partition q), for the same input hg_split_create takes.  Any output may be
 * NULL.  Errors: HG_ERR_ARG.
 * Passage: Section 2.2 (domain decomposition, neighbour exchange) and Section
 * 2.2.1 (load balancing). */
int hg_split_layout(const int32_t *xyz, int64_t n_fluid, const hg_iolet *iolets, int32_t n_iolets,
                    const hg_split_params *sp, int64_t *first_out, int64_t *ghosts_out, int64_t *halo_out);

/* Build a split domain (same inputs and checks as hg_domain_create; the context
 * must use the A/B scheme).  The cut is always taken on the canonical order;
 * lb->ordering (as for hg_domain_create) sets the device order of each
 * partition's owned sites, its ghosts following them.  Errors:
 * HG_ERR_ARG, HG_ERR_STATE (context full), HG_ERR_OOM, HG_ERR_CUDA.
 * Passage: Section 2.2 and Section 2.2.1. */
int hg_split_create(hg_ctx *ctx, const int32_t *xyz, int64_t n_fluid, const hg_iolet *iolets, int32_t n_iolets,
                    const hg_lb_params *lb, const hg_split_params *sp, hg_split **out);

/* Free a split domain.
 * Passage: infrastructure: no passage. */
int hg_split_destroy(hg_split *s);

/* Partition `part`: first canonical site, owned sites, ghost sites, halo values
 * it receives per step.  Any out pointer may be NULL.
 * Passage: Section 2.2 (decomposition). */
int hg_split_info(hg_split *s, int32_t part, int64_t *first, int64_t *owned, int64_t *ghosts, int64_t *halo_in);

/* Advance a split domain by n_steps (as hg_step, with the halo exchange after
 * every stream-collide).  Asynchronous.
 * Passage: Section 2 (the LB step) and Section 2.2 (neighbour exchange). */
int hg_split_step(hg_split *s, int64_t n_steps);

/* Read-back of a split domain, whole domain in canonical order, as the
 * hg_read_macroscopic / hg_read_state / hg_read_iolet_stats /
 * hg_read_boundary_values / hg_mass of an unsplit domain.  Synchronise.
 * Passage: Section 2 (macroscopic fields) and Section 2.3 (iolet averages). */
int hg_split_read_macroscopic(hg_split *s, float *out);
/* Passage: infrastructure: no passage (raw state read-back). */
int hg_split_read_state(hg_split *s, void *out);
/* Passage: Section 2.3 (averaged iolet values). */
int hg_split_read_iolet_stats(hg_split *s, double *out);
/* Passage: Section 2 (iolet conditions). */
int hg_split_read_boundary_values(hg_split *s, float *out);
/* Passage: infrastructure: no passage (mass check). */
int hg_split_mass(hg_split *s, double *out);

/* ---- checkpoint / resume ---- */

/* Bytes needed by hg_save_state for this domain.
 * Passage: infrastructure: no passage (checkpointing; the paper excludes data
 * output from its timings, Section 2.2). */
int hg_state_bytes(hg_domain *d, int64_t *bytes);

/* Save the current state to a host buffer.  Layout (version 2): a 40-byte
 * header (magic "HEMEGB1\0", n_sites, step, n_iolets, storage, scheme,
 * version), boundary values (n_iolets FP32), iolet means (n_iolets x 3 FP64),
 * F_t in canonical order in the storage type (19 x n_sites), iolet forces
 * (n_iolets x 4 FP32).
 * Passage: infrastructure: no passage (checkpoint). */
int hg_save_state(hg_domain *d, void *host_buf, int64_t bytes);

/* Restore a state written by hg_save_state of a domain with the same
 * geometry, storage and scheme; stepping then continues bit-identically.
 * Passage: infrastructure: no passage (resume). */
int hg_load_state(hg_domain *d, const void *host_buf, int64_t bytes);

/* Raw state of the current time level F_t as 19 x n_sites values of the
 * storage type (FP32, or f~/w in FP16/BF16), canonical order (host).
 * Passage: infrastructure: no passage (raw state read-back). */
int hg_read_state(hg_domain *d, void *host_out);

#ifdef __cplusplus
}
#endif

#endif /* HEMEGB_H */
