// hg_host.cpp -- host runtime behind the C ABI in include/hemegb.h.
//
// Geometry (Section 2.2: sparse vascular geometry, only non-empty blocks
// stored): fluid voxels are sorted into canonical Morton order; a sparse set
// of 8^3 blocks, each with a 512-bit occupancy map, answers "which site sits
// at lattice point q" in O(1) via popcount rank.  Non-fluid link targets are
// classified against the iolet openings in exact 128-bit integer arithmetic.
//
// Stepping: per set of domains a plan holds the stream-collide tile table,
// the per-iolet update table and a captured CUDA graph of G steps; kernels
// read the step parity from device counters, so the graph replays unchanged.
//
// Threads: hg_domain_create may run on one thread while another drives the
// same context (steps, reads, destroys).  The context's mutex guards the slot
// table and the coupling map; a build uploads on a stream of its own and
// publishes its slot only once every copy has landed.  Error messages are kept
// per thread.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/hemegb.h"
#include "hg_internal.h"

using namespace hg;

namespace {

// ---------------------------------------------------------------- lattice
const int kC[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
                       {0, 0, 1},  {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                       {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                       {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
inline double wgt(int i) { return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }

// ---------------------------------------------------------------- threads
// Phase timing of a build, printed to stderr when HEMEGB_TRACE_BUILD is set.
struct PhaseTrace {
    bool on;
    std::chrono::steady_clock::time_point t;
    int64_t n;
    explicit PhaseTrace(int64_t n_) : on(getenv("HEMEGB_TRACE_BUILD") != nullptr), t(std::chrono::steady_clock::now()), n(n_) {}
    void mark(const char *phase) {
        if (!on) return;
        const auto t2 = std::chrono::steady_clock::now();
        fprintf(stderr, "hemegb build n=%lld %s %.3f s\n", (long long)n, phase,
                std::chrono::duration<double>(t2 - t).count());
        t = t2;
    }
};

int n_threads() {
    unsigned h = std::thread::hardware_concurrency();
    if (h == 0) h = 4;
    return (int)std::min<unsigned>(h, 64);
}

template <typename F> void parallel_for(int64_t n, F &&fn, int64_t grain = 1 << 14) {
    int T = n_threads();
    int64_t chunks = (n + grain - 1) / grain;
    if (T <= 1 || chunks <= 1) {
        fn((int64_t)0, n);
        return;
    }
    std::atomic<int64_t> next{0};
    std::vector<std::thread> th;
    for (int t = 0; t < std::min<int64_t>(T, chunks); ++t)
        th.emplace_back([&] {
            for (;;) {
                int64_t c = next.fetch_add(1);
                if (c >= chunks) break;
                int64_t lo = c * grain, hi = std::min(n, lo + grain);
                fn(lo, hi);
            }
        });
    for (auto &x : th) x.join();
}

// A table whose elements are left uninitialised on resize, so a large table is
// first written (and its pages first touched) by the parallel loop that fills it.
template <class T> struct NoInitAlloc : std::allocator<T> {
    using std::allocator<T>::allocator;
    template <class U> struct rebind { using other = NoInitAlloc<U>; };
    template <class U, class... A> void construct(U *p, A &&...a) {
        if constexpr (sizeof...(A) == 0) ::new ((void *)p) U;
        else ::new ((void *)p) U(std::forward<A>(a)...);
    }
};
using I32Table = std::vector<int32_t, NoInitAlloc<int32_t>>;
using U32Table = std::vector<uint32_t, NoInitAlloc<uint32_t>>;
using U64Table = std::vector<uint64_t, NoInitAlloc<uint64_t>>;
using I64Table = std::vector<int64_t, NoInitAlloc<int64_t>>;

// ---------------------------------------------------------------- Morton
inline uint64_t spread21(uint64_t v) {
    v &= 0x1fffffULL;
    v = (v | (v << 32)) & 0x1f00000000ffffULL;
    v = (v | (v << 16)) & 0x1f0000ff0000ffULL;
    v = (v | (v << 8)) & 0x100f00f00f00f00fULL;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ULL;
    v = (v | (v << 2)) & 0x1249249249249249ULL;
    return v;
}
inline uint64_t morton3(uint32_t x, uint32_t y, uint32_t z) {
    return spread21(x) | (spread21(y) << 1) | (spread21(z) << 2);
}

// ---------------------------------------------------------------- iolets
bool iolet_ok(const hg_iolet &io) {
    const int64_t lim = (int64_t)1 << 31;
    bool nz = false;
    for (int d = 0; d < 3; ++d) {
        if (io.centre[d] < -lim || io.centre[d] > lim) return false;
        if (io.axis[d] < -(1 << 20) || io.axis[d] > (1 << 20)) return false;
        nz = nz || io.axis[d] != 0;
    }
    if (!nz || io.radius < 0 || io.radius > lim) return false;
    if (io.kind != HG_PRESSURE && io.kind != HG_VELOCITY) return false;
    if (io.profile != HG_PLUG && io.profile != HG_PARABOLIC) return false;
    if (io.pulse < HG_PULSE_CONST || io.pulse > HG_PULSE_SINE) return false;
    if (io.pulse != HG_PULSE_CONST && !(io.period > 0)) return false;
    return true;
}

struct IoletGeom {
    hg_iolet d;
    double cx, cy, cz, reach2;  // centre (lattice units) and a bounding radius^2
};

// Exact opening test: 0 < (q-c).a <= 2|a| and |(q-c) x a|^2 <= r^2 |a|^2 (fixed point).
bool in_opening(const hg_iolet &io, int64_t qx, int64_t qy, int64_t qz) {
    typedef __int128 i128;
    const i128 dx = (i128)qx * 1024 - io.centre[0];
    const i128 dy = (i128)qy * 1024 - io.centre[1];
    const i128 dz = (i128)qz * 1024 - io.centre[2];
    const i128 ax = io.axis[0], ay = io.axis[1], az = io.axis[2];
    const i128 dot = dx * ax + dy * ay + dz * az;
    if (dot <= 0) return false;
    const i128 aa = ax * ax + ay * ay + az * az;
    if (dot * dot > (i128)(2048 * 2048) * aa) return false;
    const i128 c0 = dy * az - dz * ay, c1 = dz * ax - dx * az, c2 = dx * ay - dy * ax;
    const i128 r = io.radius;
    return c0 * c0 + c1 * c1 + c2 * c2 <= r * r * aa;
}

int32_t classify(const std::vector<IoletGeom> &io, int64_t qx, int64_t qy, int64_t qz) {
    for (size_t k = 0; k < io.size(); ++k) {
        const IoletGeom &g = io[k];
        const double ddx = qx - g.cx, ddy = qy - g.cy, ddz = qz - g.cz;
        if (ddx * ddx + ddy * ddy + ddz * ddz > g.reach2) continue;
        if (in_opening(g.d, qx, qy, qz)) return -(2 + (int32_t)k);
    }
    return -1;
}

// ---------------------------------------------------------------- sparse blocks
// Blocks of 8^3 lattice points in Morton order: block key = morton >> 9.
struct BlockIndex {
    std::vector<uint64_t> bkey;    // sorted block keys
    std::vector<int64_t> first;    // canonical index of the block's first site
    std::vector<uint64_t> bits;    // 8 words per block: occupancy by in-block Morton offset
    std::vector<uint16_t> prefix;  // 8 per block: sites in words before w
    std::vector<int32_t> table;    // open-addressing hash: block key -> block id
    uint64_t mask = 0;

    static inline uint64_t hash(uint64_t k) { return (k * 0x9E3779B97F4A7C15ULL) >> 17; }

    void build(const U64Table &keys) {
        const int64_t n = (int64_t)keys.size();
        for (int64_t s = 0; s < n; ++s) {
            const uint64_t b = keys[s] >> 9;
            if (bkey.empty() || bkey.back() != b) {
                bkey.push_back(b);
                first.push_back(s);
            }
        }
        const int64_t nb = (int64_t)bkey.size();
        bits.assign(nb * 8, 0);
        prefix.assign(nb * 8, 0);
        for (int64_t b = 0; b < nb; ++b) {
            const int64_t hi = (b + 1 < nb) ? first[b + 1] : n;
            for (int64_t s = first[b]; s < hi; ++s) {
                const unsigned o = (unsigned)(keys[s] & 511);
                bits[b * 8 + (o >> 6)] |= 1ULL << (o & 63);
            }
            uint16_t acc = 0;
            for (int w = 0; w < 8; ++w) {
                prefix[b * 8 + w] = acc;
                acc += (uint16_t)__builtin_popcountll(bits[b * 8 + w]);
            }
        }
        uint64_t cap = 16;
        while (cap < (uint64_t)nb * 2) cap <<= 1;
        mask = cap - 1;
        table.assign(cap, -1);
        for (int64_t b = 0; b < nb; ++b) {
            uint64_t h = hash(bkey[b]) & mask;
            while (table[h] >= 0) h = (h + 1) & mask;
            table[h] = (int32_t)b;
        }
    }

    // block id of block key b, or -1
    inline int64_t block_id(uint64_t b) const {
        uint64_t h = hash(b) & mask;
        for (;;) {
            const int32_t id = table[h];
            if (id < 0 || bkey[id] == b) return id;
            h = (h + 1) & mask;
        }
    }
    // canonical index of the site with Morton key `key` in block `id`, or -1
    inline int64_t rank(int64_t id, uint64_t key) const {
        const unsigned o = (unsigned)(key & 511);
        const uint64_t w = bits[id * 8 + (o >> 6)];
        const uint64_t bit = 1ULL << (o & 63);
        if (!(w & bit)) return -1;
        return first[id] + prefix[id * 8 + (o >> 6)] + __builtin_popcountll(w & (bit - 1));
    }
};

// A thread's lookups with the last block seen in each of the eight slots that the
// 2x2x2 neighbourhood of blocks maps to (the low bit of each block coordinate): the
// 18 neighbours of consecutive canonical sites mostly fall in the same few blocks.
struct BlockCache {
    const BlockIndex &bi;
    uint64_t tag[8];
    int64_t id[8];
    explicit BlockCache(const BlockIndex &b) : bi(b) {
        for (int k = 0; k < 8; ++k) tag[k] = ~0ULL, id[k] = -1;
    }
    inline int64_t find(uint64_t key) {
        const uint64_t b = key >> 9;
        const int slot = (int)(b & 7);
        if (tag[slot] != b) {
            tag[slot] = b;
            id[slot] = bi.block_id(b);
        }
        return id[slot] < 0 ? -1 : bi.rank(id[slot], key);
    }
};

// Morton key of the lattice point one unit along +-axis from the point with key k
// (dilated-integer increment: the other axes' bits are held at one / zero so the
// carry or borrow runs through the axis' own bits only); the caller keeps the
// coordinate inside [0, 2^21).
inline uint64_t morton_step(uint64_t k, int axis, int d) {
    const uint64_t M = 0x1249249249249249ULL << axis;
    if (d > 0) return (((k | ~M) + 1) & M) | (k & ~M);
    if (d < 0) return (((k & M) - 1) & M) | (k & ~M);
    return k;
}

// Canonical order: sort (key, index) pairs by key -- bucket by the leading key
// bits, then sort each bucket, buckets in parallel.
void sort_keys(U64Table &key, I64Table &idx) {
    const int64_t n = (int64_t)key.size();
    if (n <= 1) return;
    // bucket by the top 12 bits of the key range (counting sort, in parallel over
    // contiguous site chunks), then sort each bucket; keys are distinct, so the
    // result does not depend on the thread count
    const int T = (int)std::max<int64_t>(1, std::min<int64_t>(n_threads(), n / 65536 + 1));
    const int64_t per = (n + T - 1) / T;
    std::vector<uint64_t> mxs(T, 0);
    parallel_for(T, [&](int64_t lo, int64_t hi) {
        for (int64_t t = lo; t < hi; ++t)
            for (int64_t s = t * per; s < std::min(n, (t + 1) * per); ++s) mxs[t] = std::max(mxs[t], key[s]);
    }, 1);
    uint64_t mx = 0;
    for (uint64_t m : mxs) mx = std::max(mx, m);
    int bl = 64 - (mx ? __builtin_clzll(mx) : 63);
    const int nbits = 12;
    const int shift = std::max(0, bl - nbits);
    const int64_t nbk = (int64_t)1 << nbits;
    std::vector<int64_t> hist((size_t)T * nbk, 0);  // [chunk][bucket]
    parallel_for(T, [&](int64_t lo, int64_t hi) {
        for (int64_t t = lo; t < hi; ++t)
            for (int64_t s = t * per; s < std::min(n, (t + 1) * per); ++s) hist[(size_t)t * nbk + (key[s] >> shift)]++;
    }, 1);
    std::vector<int64_t> cnt(nbk + 1, 0);
    {
        int64_t acc = 0;
        for (int64_t b = 0; b < nbk; ++b) {
            cnt[b] = acc;
            for (int t = 0; t < T; ++t) {
                const int64_t h = hist[(size_t)t * nbk + b];
                hist[(size_t)t * nbk + b] = acc;  // this chunk's first position in bucket b
                acc += h;
            }
        }
        cnt[nbk] = acc;
    }
    struct KeyIdx {
        uint64_t first;
        int64_t second;
        bool operator<(const KeyIdx &o) const { return first < o.first || (first == o.first && second < o.second); }
    };
    std::vector<KeyIdx, NoInitAlloc<KeyIdx>> tmp(n);  // every element written by the scatter
    parallel_for(T, [&](int64_t lo, int64_t hi) {
        for (int64_t t = lo; t < hi; ++t) {
            int64_t *pos = hist.data() + (size_t)t * nbk;
            for (int64_t s = t * per; s < std::min(n, (t + 1) * per); ++s) tmp[pos[key[s] >> shift]++] = {key[s], idx[s]};
        }
    }, 1);
    parallel_for(nbk, [&](int64_t lo, int64_t hi) {
        for (int64_t b = lo; b < hi; ++b) std::sort(tmp.begin() + cnt[b], tmp.begin() + cnt[b + 1]);
    }, 1);
    parallel_for(n, [&](int64_t lo, int64_t hi) {
        for (int64_t s = lo; s < hi; ++s) {
            key[s] = tmp[s].first;
            idx[s] = tmp[s].second;
        }
    });
}

// Device layout of a domain's sites (the canonical order is always Morton):
//   HG_ORDER_ROWS   lexicographic, x fastest, then y, then z: a warp's 32
//                   consecutive sites mostly form one x-row, and the same row
//                   shifted by one lattice unit is again a run of consecutive
//                   sites, so gathers and the AA scatter touch few sectors;
//   HG_ORDER_BRICKS rows inside 32 x 8 x 8 bricks, the bricks in Morton order
//                   (row locality with block locality for very large domains).
// canon_of[q] = canonical index of the site at device position q.
int device_order(const std::vector<int32_t> &xyz, int64_t n, int ordering, std::vector<int32_t> &canon_of,
                 std::string &why) {
    int32_t lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int e = 0; e < 3; ++e) {
        lo[e] = n ? xyz[e] : 0;
        hi[e] = lo[e];
    }
    for (int64_t s = 0; s < n; ++s)
        for (int e = 0; e < 3; ++e) {
            lo[e] = std::min(lo[e], xyz[3 * s + e]);
            hi[e] = std::max(hi[e], xyz[3 * s + e]);
        }
    U64Table key(n);  // both written in full by the parallel loop below
    I64Table idx(n);
    if (ordering == HG_ORDER_ROWS) {
        parallel_for(n, [&](int64_t a, int64_t b) {
            for (int64_t s = a; s < b; ++s) {
                const uint64_t x = (uint64_t)(xyz[3 * s] - lo[0]), y = (uint64_t)(xyz[3 * s + 1] - lo[1]),
                               z = (uint64_t)(xyz[3 * s + 2] - lo[2]);
                key[s] = (z << 42) | (y << 21) | x;
                idx[s] = s;
            }
        });
    } else {  // HG_ORDER_BRICKS: 32 x 8 x 8
        uint32_t mx = 0;
        for (int e = 0; e < 3; ++e)
            mx = std::max<uint32_t>(mx, (uint32_t)(hi[e] - lo[e]) >> (e == 0 ? 5 : 3));
        int w = 0;
        while (w < 21 && (mx >> w)) ++w;
        if (3 * w + 11 > 64) {
            why = "domain extent too large for the brick ordering";
            return HG_ERR_ARG;
        }
        parallel_for(n, [&](int64_t a, int64_t b) {
            for (int64_t s = a; s < b; ++s) {
                const uint32_t x = (uint32_t)(xyz[3 * s] - lo[0]), y = (uint32_t)(xyz[3 * s + 1] - lo[1]),
                               z = (uint32_t)(xyz[3 * s + 2] - lo[2]);
                const uint64_t brick = morton3(x >> 5, y >> 3, z >> 3);
                const uint64_t inner = ((uint64_t)(z & 7) << 8) | ((uint64_t)(y & 7) << 5) | (x & 31);
                key[s] = (brick << 11) | inner;
                idx[s] = s;
            }
        });
    }
    sort_keys(key, idx);
    canon_of.resize(n);
    parallel_for(n, [&](int64_t lo, int64_t hi) {
        for (int64_t q = lo; q < hi; ++q) canon_of[q] = (int32_t)idx[q];
    });
    return HG_OK;
}

// Velocity-iolet link coefficient of link i of the site at xyz (Section 2: velocity
// condition at inlets): 6 w_i c_i.u_w / U, u_w the inward profile velocity per unit
// peak speed at the link midpoint x - c_i/2 (parabolic: peak on the axis, zero at
// the radius; plug: uniform).  16-bit storage holds f~/w and collides on it, so
// its coefficient drops w_i.  Zero for pressure iolets.
float link_coef(const hg_iolet &io, const int32_t *xyz, int i, int storage) {
    if (io.kind != HG_VELOCITY) return 0.0f;
    const double an = std::sqrt((double)io.axis[0] * io.axis[0] + (double)io.axis[1] * io.axis[1] +
                                (double)io.axis[2] * io.axis[2]);
    const double ah[3] = {io.axis[0] / an, io.axis[1] / an, io.axis[2] / an};
    double phi = 1.0;
    if (io.profile == HG_PARABOLIC) {
        double rel[3], along = 0.0;
        for (int e = 0; e < 3; ++e) {
            rel[e] = (xyz[e] - 0.5 * kC[i][e]) - io.centre[e] / 1024.0;
            along += rel[e] * ah[e];
        }
        double p2 = 0.0;
        for (int e = 0; e < 3; ++e) {
            const double t = rel[e] - along * ah[e];
            p2 += t * t;
        }
        const double r = io.radius / 1024.0;
        phi = r > 0 ? std::max(0.0, 1.0 - p2 / (r * r)) : 0.0;
    }
    const double cdot = -(kC[i][0] * ah[0] + kC[i][1] * ah[1] + kC[i][2] * ah[2]);
    const double wi = storage == HG_STORE_F32 ? wgt(i) : 1.0;
    return (float)(6.0 * wi * cdot * phi);
}

double pulse(int kind, double t, double period) {
    const double ph = kind == HG_PULSE_CONST ? 0.0 : std::fmod(t, period) / period;
    if (kind == HG_PULSE_COSINE) return 0.5 * (1.0 - std::cos(2.0 * 3.141592653589793 * ph));
    if (kind == HG_PULSE_SINE) return std::sin(2.0 * 3.141592653589793 * ph);
    return 1.0;
}

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace

// ================================================================ objects
// In a plan over several domains, up to this many domains of at least this many
// sites get a stream-collide launch of their own (the single-domain kernel reads its
// descriptor from the parameter bank at fixed offsets; the tile-table kernel copies
// it into shared memory behind a barrier, measured 15-20 % slower per launch); the
// smaller domains share one tile-table launch.
constexpr int kSeparateMaxDoms = 16;
constexpr int64_t kSeparateMinSites = (int64_t)1 << 20;

struct PlanKey {
    std::vector<int32_t> doms;
    bool operator<(const PlanKey &o) const { return doms < o.doms; }
};

struct Plan {
    std::vector<int32_t> doms;
    DevBuf tiles, ios, adv, chunks, partials, counters, rev, fslots;
    // halo exchange of a split domain (after stream-collide, before the iolet update):
    // direct (one kernel moves every value from sender to receiver) or staged (pack
    // into `send`, copy each (sender, receiver) block to `recv`, unpack)
    DevBuf halo_pack, halo_unpack, send, recv, halo_moves;
    int64_t n_halo = 0;
    int halo_elem = 4;
    bool halo_staged = false;
    std::vector<std::pair<size_t, size_t>> halo_blocks;  // (byte offset, bytes) per partition pair
    DomDev one{};       // single-domain plans: the descriptor passed by value to stream-collide
    bool single = false;
    bool tiles_runs = true;  // every domain of the tile-table (or single) launch has a run encoding
    // a few large domains (a coupled pair, a split's partitions): one single-domain
    // launch each instead of one tile-table launch, chained by programmatic dependent
    // launch; descriptor and sites stepped per launch
    std::vector<DomDev> sep;
    std::vector<int64_t> sep_n;
    int64_t n_tiles = 0;
    int n_fslots = 0;  // (domain, slot) pairs the body-force pass visits
    int n_ios = 0;
    int n_chunks = 0;
    cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};  // by parity mode
    int graph_steps = 0;
};

struct CoupleSrc {
    int32_t src_dom, src_k;
    double factor;
};

struct hg_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int storage = 0, scheme = 0, block = 256, spt = 1, variant = 0, graph_steps = 16;
    hg_alloc_fn alloc = nullptr;
    hg_free_fn free_fn = nullptr;
    void *alloc_user = nullptr;
    std::mutex mu;                  // guards doms, reserved, coupled
    std::vector<hg_domain *> doms;  // by index (nullptr = free slot)
    std::vector<char> reserved;     // slots held by builds in progress
    DevBuf dom_table;               // DomDev[capacity]
    DevBuf errw;                    // device error word (bounded waits that gave up)
    DevBuf steps;                   // int64[capacity]
    int capacity = 0;
    std::map<std::pair<int32_t, int32_t>, CoupleSrc> coupled;  // (dst dom, dst k) -> source
    std::atomic<int> couple_mode{HG_COUPLE_FORWARD};  // read by builds on another thread
    std::map<PlanKey, std::unique_ptr<Plan>> plans;
    DevBuf scratch;                 // mass partials, read-back staging
    std::atomic<int64_t> device_bytes{0};
    std::atomic<int64_t> fail_alloc_in{0};  // injected fault: the k-th next allocation fails (0 = none)
    std::vector<hg_split *> splits;         // split domains (destroyed with the context)
};

// One partition of a split domain: a contiguous range of the canonical site list
// (owned, device positions [0, n_own)) followed by its ghosts (sites of other
// partitions it pulls from, [n_own, n_loc)), with its own distributions, neighbour
// table (local indices) and iolet mask; boundary slots are numbered globally.
struct SplitPart {
    int32_t idx = -1;                  // context domain-table slot (descriptor, step counter)
    int64_t first = 0, n_own = 0, n_loc = 0, np = 0;
    std::vector<int64_t> ghosts;       // global canonical indices of the ghost sites
    DevBuf f[2], nbr, iomask, ioprefix, gidx;  // gidx: local -> global canonical index
    DevBuf lword, run0, rdelta;                // run-length encoded table (empty: not built)
    int64_t n_runs = 0;
    DomDev dev{};
};

struct hg_split {
    hg_ctx *ctx = nullptr;
    int64_t n = 0, n_adj = 0, step = 0;
    int32_t nio = 0;
    double tau = 0.8;
    std::vector<hg_iolet> io;
    std::vector<int32_t> io_ptr;
    std::vector<SplitPart> parts;
    bool staged = false;                            // halo transport (hg_split_params.exchange)
    std::vector<HaloDev> pack, unpack;              // grouped by (sender, receiver) pair
    std::vector<std::pair<size_t, size_t>> blocks;  // element (offset, count) per pair
    DevBuf bnd, io_codes, coef, slot_site, bcv, io_kind, M, slots, force;  // shared by the parts
};

struct hg_domain {
    hg_ctx *ctx = nullptr;
    int32_t idx = -1;
    int64_t n = 0, np = 0;
    int32_t nio = 0;
    double tau = 0.8;
    int64_t n_adj = 0;
    int64_t step = 0;  // host mirror of completed steps
    std::vector<int32_t> xyz;           // canonical coordinates
    std::vector<hg_iolet> io;
    std::vector<int32_t> io_ptr;        // CSR over slots per iolet
    DevBuf f[2], nbr, iomask, ioprefix, io_codes, bnd, coef, bcv, io_kind, M, slots;
    DevBuf force;                        // per iolet: body-force density (float4), reverse exchange
    DevBuf slot_site;                    // per slot: device site index
    std::vector<int32_t> slots_host;     // per-iolet CSR of slots (io_ptr), host copy
    std::vector<int32_t> io_codes_host;  // per slot x 18, canonical codes
    std::vector<int32_t> slot_of_dev;    // device site -> slot or -1
    int32_t ordering = HG_ORDER_MORTON;  // device layout of the sites
    std::vector<int32_t> canon_of_host;  // device -> canonical index (empty: identity)
    std::vector<int32_t> dev_of_host;    // canonical -> device index (empty: identity)
    DevBuf canon_of, dev_of;             // device copies of the two permutations
    DevBuf lword, run0, rdelta;          // run-length encoded neighbour table (empty: not built)
    int64_t n_runs = 0;
    int64_t bytes = 0;
};

namespace {

std::vector<DevBuf *> domain_buffers(hg_domain *d) {
    return {&d->f[0], &d->f[1], &d->nbr, &d->iomask, &d->ioprefix, &d->io_codes, &d->bnd, &d->coef,
            &d->bcv, &d->io_kind, &d->M, &d->slots, &d->force, &d->slot_site, &d->canon_of, &d->dev_of,
            &d->lword, &d->run0, &d->rdelta};
}

// last failure of the calling thread and the context it concerned
thread_local const hg_ctx *t_err_ctx = nullptr;
thread_local std::string t_err;

int fail(hg_ctx *ctx, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err_ctx = ctx;
    t_err = buf;
    return code;
}

#define CU(ctx, call)                                                                       \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail(ctx, HG_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));  \
    } while (0)

int dev_alloc(hg_ctx *ctx, DevBuf &b, size_t bytes) {
    if (bytes == 0) bytes = 256;
    bytes = (bytes + 255) & ~(size_t)255;
    int64_t k = ctx->fail_alloc_in.load();
    while (k > 0 && !ctx->fail_alloc_in.compare_exchange_weak(k, k - 1)) {
    }
    if (k == 1) return fail(ctx, HG_ERR_OOM, "injected allocation failure (%zu bytes)", bytes);
    void *p = nullptr;
    if (ctx->alloc) {
        p = ctx->alloc(bytes, ctx->alloc_user);
        if (!p) return fail(ctx, HG_ERR_OOM, "allocator callback returned NULL for %zu bytes", bytes);
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, HG_ERR_OOM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
        }
    }
    b.p = p;
    b.bytes = bytes;
    ctx->device_bytes += (int64_t)bytes;
    return HG_OK;
}

void dev_free(hg_ctx *ctx, DevBuf &b) {
    if (!b.p) return;
    if (ctx->free_fn) ctx->free_fn(b.p, b.bytes, ctx->alloc_user);
    else cudaFree(b.p);
    ctx->device_bytes -= (int64_t)b.bytes;
    b.p = nullptr;
    b.bytes = 0;
}

void drop_plans(hg_ctx *ctx) {
    for (auto &kv : ctx->plans) {
        Plan &p = *kv.second;
        for (auto &g : p.graph)
            if (g) cudaGraphExecDestroy(g);
        for (DevBuf *b : {&p.tiles, &p.ios, &p.adv, &p.chunks, &p.partials, &p.counters, &p.rev, &p.fslots,
                          &p.halo_pack, &p.halo_unpack, &p.send, &p.recv, &p.halo_moves})
            dev_free(ctx, *b);
    }
    ctx->plans.clear();
}

DomDev make_domdev(hg_ctx *ctx, hg_domain *d) {
    DomDev D;
    memset(&D, 0, sizeof D);
    D.f[0] = d->f[0].p;
    D.f[1] = d->f[1].p;
    D.nbr = (const int32_t *)d->nbr.p;
    D.lword = (const uint32_t *)d->lword.p;
    D.run0 = (const int32_t *)d->run0.p;
    D.rdelta = (const int32_t *)d->rdelta.p;
    D.iomask = (const uint32_t *)d->iomask.p;
    D.ioprefix = (const int32_t *)d->ioprefix.p;
    D.io_codes = (const int32_t *)d->io_codes.p;
    D.slot_site = (const int32_t *)d->slot_site.p;
    D.bnd = (float4 *)d->bnd.p;
    D.coef = (const float *)d->coef.p;
    D.bcv = (const float *)d->bcv.p;
    D.io_kind = (const int8_t *)d->io_kind.p;
    D.io_force = nullptr;
    if (ctx->couple_mode == HG_COUPLE_ALTERNATE) {
        std::lock_guard<std::mutex> lk(ctx->mu);
        for (const auto &kv : ctx->coupled)
            if (kv.second.src_dom == d->idx) D.io_force = (const float4 *)d->force.p;
    }
    D.step = (const int64_t *)ctx->steps.p + d->idx;
    D.err = (int32_t *)ctx->errw.p;
    D.n = d->n;
    D.np = d->np;
    D.omega = (float)(1.0 / d->tau);
    D.n_io = d->nio;
    return D;
}

// Rewrite every live domain's descriptor (stream-ordered): after a change of
// coupling or coupling mode, which decides whether a domain is forced.
cudaError_t refresh_domdevs(hg_ctx *ctx) {
    std::vector<hg_domain *> live;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        for (hg_domain *d : ctx->doms)
            if (d) live.push_back(d);
    }
    for (hg_domain *d : live) {
        const DomDev D = make_domdev(ctx, d);
        cudaError_t e = cudaMemcpyAsync((DomDev *)ctx->dom_table.p + d->idx, &D, sizeof D,
                                        cudaMemcpyHostToDevice, ctx->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaStreamSynchronize(ctx->stream);
}

const DomDev *domdev_ptr(hg_domain *d) {
    return (const DomDev *)d->ctx->dom_table.p + d->idx;
}

size_t elem_bytes(int storage) { return storage == HG_STORE_F32 ? 4 : 2; }

// Kernel variants and the launch shapes each supports (see hg_ctx_params).
bool variant_ok(int storage, int scheme, int spt, int variant) {
    switch (variant) {
        case 0: case 3: return true;
        case 1: return spt != 4;
        case 2: return spt != 4 && scheme == HG_SCHEME_AA;
        case 4: return spt == 1 && scheme == HG_SCHEME_AA;
        case 5: return spt == 2 && scheme == HG_SCHEME_AB && storage != HG_STORE_F32;
        case 6: case 7: return spt == 2 && scheme == HG_SCHEME_AA;
        case 8: return true;  // 8..11: variants 3, 5, 6, 7 reading the run-encoded table
        case 9: return spt == 2 && scheme == HG_SCHEME_AB && storage != HG_STORE_F32;
        case 10: case 11: return spt == 2 && scheme == HG_SCHEME_AA;
        case 12: return spt != 4 && scheme == HG_SCHEME_AA;
        case 13: return spt != 1;
        case 14: return spt == 2 && scheme == HG_SCHEME_AA;
        default: return false;
    }
}

int ensure_scratch(hg_ctx *ctx, size_t bytes) {
    if (ctx->scratch.bytes >= bytes) return HG_OK;
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    dev_free(ctx, ctx->scratch);
    return dev_alloc(ctx, ctx->scratch, bytes);
}

// Run-length encoding of a device neighbour table ([18][np], sites [0, n); fluid
// entries in [0, n_ref), every other entry the virtual index q + dd_i np with
// dd_i = vdir * (opp(i) - i)).  A run is a maximal range of consecutive sites in
// which each direction's fluid links share one offset (entry - site); non-fluid
// links do not break a run, a per-site bit marks them instead; every 2^20-site span
// starts a run (the spans are encoded in parallel).  rdelta holds
// kRunStride entries per run (the 18 offsets, then zeros), so a run's row is one
// aligned 80-byte block the kernels read with 16-byte loads.  Rows ordering
// makes a run cover most of an x-row of a vessel.  Returns false (nothing built)
// when an entry does not fit that form or the encoding would not save enough
// traffic (runs shorter than 4.5 sites on average: more than 16 bytes per site).
bool build_runs(const int32_t *nbr, int64_t n, int64_t n_ref, int64_t np, int vdir, U32Table &lword,
                std::vector<int32_t> &run0, std::vector<int32_t> &rdelta) {
    if (n <= 0) return false;
    lword.resize((size_t)np);  // [0, n) is written by the spans below, in parallel
    std::fill(lword.begin() + n, lword.end(), 0u);
    run0.assign((size_t)((np + 1023) / 1024), 0);
    rdelta.clear();
    // Spans of 2^20 sites (whole 1024-site chunks) are encoded in parallel, each starting
    // a run of its own; run0 and the rows then move by the runs of the spans before.
    constexpr int64_t kSpan = (int64_t)1 << 20;
    const int64_t n_span = (n + kSpan - 1) / kSpan;
    std::vector<std::vector<int32_t>> rows(n_span);
    std::vector<int64_t> runs(n_span, 0);
    std::atomic<bool> bad{false};             // an entry of the wrong form, or too many runs
    std::atomic<int64_t> counted{0};          // runs so far, all spans: stop once it cannot pay
    parallel_for(n_span, [&](int64_t lo, int64_t hi) {
        for (int64_t sp = lo; sp < hi && !bad; ++sp) {
            const int64_t a = sp * kSpan, b = std::min(n, a + kSpan);
            std::vector<int32_t> &rd = rows[sp];
            int32_t cur[18] = {0};
            bool have[18] = {false};
            int64_t run = -1;  // local to the span
            for (int64_t q = a; q < b && !bad; ++q) {
                uint32_t miss = 0;
                bool brk = run < 0;
                for (int i = 0; i < 18; ++i) {
                    const int32_t v = nbr[(size_t)i * np + q];
                    if (v >= 0 && v < n_ref) {
                        if (have[i] && cur[i] != v - (int32_t)q) brk = true;
                    } else {
                        const int dir = i + 1, opp = (dir & 1) ? dir + 1 : dir - 1;
                        if ((int64_t)v != q + (int64_t)vdir * (opp - dir) * np) {
                            bad = true;
                            return;
                        }
                        miss |= 1u << i;
                    }
                }
                if (brk) {
                    ++run;
                    if ((counted.fetch_add(1) + 1) * 72 > 16 * n) {
                        bad = true;
                        return;
                    }
                    rd.resize((size_t)(run + 1) * kRunStride, 0);
                    for (int i = 0; i < 18; ++i) have[i] = false;
                }
                if ((q & 1023) == 0) run0[(size_t)(q >> 10)] = (int32_t)run;  // local until shifted
                for (int i = 0; i < 18; ++i)
                    if (!((miss >> i) & 1u) && !have[i]) {
                        have[i] = true;
                        cur[i] = nbr[(size_t)i * np + q] - (int32_t)q;
                        rd[(size_t)run * kRunStride + i] = cur[i];
                    }
                lword[(size_t)q] = miss | ((uint32_t)(run - run0[(size_t)(q >> 10)]) << 18);
            }
            runs[sp] = run + 1;
        }
    }, 1);
    if (bad) return false;
    int64_t total = 0;
    std::vector<int64_t> first(n_span, 0);
    for (int64_t sp = 0; sp < n_span; ++sp) {
        first[sp] = total;
        total += runs[sp];
    }
    if (total * 72 > 16 * n || total > INT32_MAX) return false;
    rdelta.resize((size_t)total * kRunStride);
    parallel_for(n_span, [&](int64_t lo, int64_t hi) {
        for (int64_t sp = lo; sp < hi; ++sp) {
            std::copy(rows[sp].begin(), rows[sp].end(), rdelta.begin() + first[sp] * kRunStride);
            const int64_t c0 = sp * (kSpan >> 10), c1 = std::min<int64_t>((int64_t)run0.size(), c0 + (kSpan >> 10));
            for (int64_t c = c0; c < c1 && c * 1024 < n; ++c) run0[(size_t)c] += (int32_t)first[sp];
        }
    }, 1);
    return true;
}

// Canonical site order (ascending 3-D Morton key) and neighbour table in
// canonical codes (Section 2.2: sparse geometry, fluid sites only): entry i-1 of
// site s is the canonical index of the fluid site at x_s - c_i, else -(2+k) if
// that lattice point lies in the opening of iolet k (lowest k wins), else -1.
// nbr has 18 rows of `stride` entries (>= n; the padding is -1).  Returns HG_OK
// or HG_ERR_ARG with the reason in `why`.
int build_canonical(const int32_t *xyz, int64_t n, const hg_iolet *iolets, int32_t nio, int64_t stride,
                    std::vector<int32_t> &xyz_sorted, I32Table &nbr, std::string &why) {
    U64Table key(n);  // both written in full by the parallel loop below
    I64Table idx(n);
    std::atomic<int> bad{0};
    parallel_for(n, [&](int64_t lo, int64_t hi) {
        for (int64_t s = lo; s < hi; ++s) {
            const int32_t x = xyz[3 * s], y = xyz[3 * s + 1], z = xyz[3 * s + 2];
            if (x < 0 || y < 0 || z < 0 || x >= (1 << 21) || y >= (1 << 21) || z >= (1 << 21)) bad = 1;
            key[s] = morton3((uint32_t)x, (uint32_t)y, (uint32_t)z);
            idx[s] = s;
        }
    });
    if (bad) {
        why = "site coordinate outside [0, 2^21)";
        return HG_ERR_ARG;
    }
    sort_keys(key, idx);
    for (int64_t s = 1; s < n; ++s)
        if (key[s] == key[s - 1]) {
            char buf[96];
            snprintf(buf, sizeof buf, "duplicate site at canonical index %lld", (long long)s);
            why = buf;
            return HG_ERR_ARG;
        }
    xyz_sorted.resize(3 * n);
    parallel_for(n, [&](int64_t lo, int64_t hi) {
        for (int64_t s = lo; s < hi; ++s)
            for (int c = 0; c < 3; ++c) xyz_sorted[3 * s + c] = xyz[3 * idx[s] + c];
    });
    I64Table().swap(idx);
    BlockIndex bi;
    bi.build(key);
    std::vector<IoletGeom> geo(nio);
    for (int k = 0; k < nio; ++k) {
        geo[k].d = iolets[k];
        geo[k].cx = iolets[k].centre[0] / 1024.0;
        geo[k].cy = iolets[k].centre[1] / 1024.0;
        geo[k].cz = iolets[k].centre[2] / 1024.0;
        const double r = iolets[k].radius / 1024.0 + 3.0;
        geo[k].reach2 = r * r + 1.0;
    }
    nbr.resize((size_t)18 * stride);  // every entry is written below, in parallel
    if (stride > n)
        for (int i = 0; i < 18; ++i) std::fill(nbr.begin() + (size_t)i * stride + n, nbr.begin() + (size_t)(i + 1) * stride, -1);
    parallel_for(n, [&](int64_t lo, int64_t hi) {
        BlockCache cache(bi);
        for (int64_t s = lo; s < hi; ++s) {
            const int64_t x = xyz_sorted[3 * s], y = xyz_sorted[3 * s + 1], z = xyz_sorted[3 * s + 2];
            const uint64_t ks = key[s];  // the site's own Morton key (sorted order)
            for (int i = 1; i < 19; ++i) {
                const int64_t qx = x - kC[i][0], qy = y - kC[i][1], qz = z - kC[i][2];
                int64_t v = -1;
                if (qx >= 0 && qy >= 0 && qz >= 0 && qx < (1 << 21) && qy < (1 << 21) && qz < (1 << 21))
                    v = cache.find(morton_step(morton_step(morton_step(ks, 0, -kC[i][0]), 1, -kC[i][1]), 2,
                                               -kC[i][2]));
                nbr[(size_t)(i - 1) * stride + s] = v >= 0 ? (int32_t)v : classify(geo, qx, qy, qz);
            }
        }
    });
    return HG_OK;
}

}  // namespace

// ================================================================ C ABI
extern "C" {

int hg_ctx_create(const hg_ctx_params *p, hg_ctx **out) {
    if (!p || !out) return HG_ERR_ARG;
    *out = nullptr;
    if (p->storage < HG_STORE_F32 || p->storage > HG_STORE_BF16) return HG_ERR_ARG;
    if (p->scheme != HG_SCHEME_AB && p->scheme != HG_SCHEME_AA) return HG_ERR_ARG;
    int block = p->block_size ? p->block_size : 256;
    int spt = p->sites_per_thread ? p->sites_per_thread : 1;
    if (block < 32 || block > 512 || block % 32) return HG_ERR_ARG;
    if (spt != 1 && spt != 2 && spt != 4) return HG_ERR_ARG;
    if (!variant_ok(p->storage, p->scheme, spt, p->kernel_variant)) return HG_ERR_ARG;
    if ((p->alloc == nullptr) != (p->free == nullptr)) return HG_ERR_ARG;
    std::unique_ptr<hg_ctx> c(new hg_ctx);
    c->device = p->device;
    c->storage = p->storage;
    c->scheme = p->scheme;
    c->block = block;
    c->spt = spt;
    c->variant = p->kernel_variant;
    c->graph_steps = p->graph_steps == 0 ? 16 : p->graph_steps;
    c->alloc = p->alloc;
    c->free_fn = p->free;
    c->alloc_user = p->alloc_user;
    if (cudaSetDevice(p->device) != cudaSuccess) {
        cudaGetLastError();
        return HG_ERR_CUDA;
    }
    if (p->stream) {
        c->stream = (cudaStream_t)p->stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess)
            return HG_ERR_CUDA;
        c->own_stream = true;
    }
    c->capacity = 4096;
    // on any failure below, release what was set up so far
    auto undo = [&](int code) {
        if (c->stream) cudaStreamSynchronize(c->stream);
        dev_free(c.get(), c->dom_table);
        dev_free(c.get(), c->steps);
        dev_free(c.get(), c->errw);
        if (c->own_stream) cudaStreamDestroy(c->stream);
        cudaGetLastError();
        return code;
    };
    int rc = dev_alloc(c.get(), c->dom_table, sizeof(DomDev) * c->capacity);
    if (rc == HG_OK) rc = dev_alloc(c.get(), c->steps, sizeof(int64_t) * c->capacity);
    if (rc == HG_OK) rc = dev_alloc(c.get(), c->errw, 256);
    if (rc != HG_OK) return undo(rc);
    if (cudaMemsetAsync(c->steps.p, 0, c->steps.bytes, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->errw.p, 0, c->errw.bytes, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return undo(HG_ERR_CUDA);
    c->doms.assign(c->capacity, nullptr);
    c->reserved.assign(c->capacity, 0);
    *out = c.release();
    return HG_OK;
}

int hg_domain_destroy(hg_domain *d);
int hg_split_destroy(hg_split *sp);

int hg_ctx_destroy(hg_ctx *ctx) {
    if (!ctx) return HG_ERR_ARG;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    while (!ctx->splits.empty()) hg_split_destroy(ctx->splits.back());
    for (auto *d : ctx->doms)
        if (d) hg_domain_destroy(d);
    drop_plans(ctx);
    dev_free(ctx, ctx->scratch);
    dev_free(ctx, ctx->dom_table);
    dev_free(ctx, ctx->errw);
    dev_free(ctx, ctx->steps);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return HG_OK;
}

const char *hg_last_error(hg_ctx *ctx) {
    if (!ctx) return "null context";
    return t_err_ctx == ctx ? t_err.c_str() : "";
}

int hg_sync(hg_ctx *ctx) {
    if (!ctx) return HG_ERR_ARG;
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    int32_t e = 0;
    CU(ctx, cudaMemcpyAsync(&e, ctx->errw.p, sizeof e, cudaMemcpyDeviceToHost, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    if (e) {
        CU(ctx, cudaMemsetAsync(ctx->errw.p, 0, sizeof e, ctx->stream));
        CU(ctx, cudaStreamSynchronize(ctx->stream));
        if (e == 2)
            return fail(ctx, HG_ERR_STATE, "a run-encoded kernel variant met a domain without a run encoding; "
                                           "the state is not trusted");
        return fail(ctx, HG_ERR_TIMEOUT, "a bounded device wait gave up (code %d); the state is not trusted", e);
    }
    return HG_OK;
}

int hg_domain_create(hg_ctx *ctx, const int32_t *xyz, int64_t n, const hg_iolet *iolets,
                     int32_t nio, const hg_lb_params *lb, hg_domain **out) {
    if (!ctx) return HG_ERR_ARG;
    if (!out) return fail(ctx, HG_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 0 || (n > 0 && !xyz)) return fail(ctx, HG_ERR_ARG, "bad site array");
    if (n > ((int64_t)200 << 20))  // 32-bit row offsets in the AA kernels need 19 * np < 2^32
        return fail(ctx, HG_ERR_ARG, "too many sites in one domain (%lld > 209715200)", (long long)n);
    if (nio < 0 || nio > kMaxIolets || (nio > 0 && !iolets))
        return fail(ctx, HG_ERR_ARG, "n_iolets must be in [0, %d]", kMaxIolets);
    const double tau = lb ? lb->tau : 0.8;
    if (!(tau > 0.5)) return fail(ctx, HG_ERR_ARG, "tau must exceed 1/2");
    const int32_t ordering = lb ? lb->ordering : HG_ORDER_MORTON;
    if (ordering < HG_ORDER_MORTON || ordering > HG_ORDER_BRICKS)
        return fail(ctx, HG_ERR_ARG, "unknown ordering %d", ordering);
    for (int k = 0; k < nio; ++k)
        if (!iolet_ok(iolets[k])) return fail(ctx, HG_ERR_ARG, "iolet %d out of range", k);
    CU(ctx, cudaSetDevice(ctx->device));
    int slot_idx = -1;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        for (int i = 0; i < ctx->capacity; ++i)
            if (!ctx->doms[i] && !ctx->reserved[i]) {
                slot_idx = i;
                ctx->reserved[i] = 1;
                break;
            }
    }
    if (slot_idx < 0) return fail(ctx, HG_ERR_STATE, "context holds too many domains");
    // the slot returns to the pool unless the build publishes it
    struct SlotGuard {
        hg_ctx *ctx;
        int idx;
        ~SlotGuard() {
            std::lock_guard<std::mutex> lk(ctx->mu);
            ctx->reserved[idx] = 0;
        }
    } slot_guard{ctx, slot_idx};

    std::unique_ptr<hg_domain> d(new hg_domain);
    d->ctx = ctx;
    d->n = n;
    d->np = std::max<int64_t>(128, (n + 127) / 128 * 128);
    d->nio = nio;
    d->tau = tau;
    d->ordering = ordering;
    d->io.assign(iolets, iolets + nio);

    PhaseTrace trace(n);
    // --- canonical order and neighbour table (canonical codes)
    const int64_t np = d->np;
    I32Table nbr;
    {
        std::string why;
        const int brc = build_canonical(xyz, n, iolets, nio, np, d->xyz, nbr, why);
        if (brc != HG_OK) return fail(ctx, brc, "%s", why.c_str());
    }

    trace.mark("canonical order and table");
    // --- device ordering: a permutation of the canonical order (none for Morton).
    // The table's columns move to their device positions and fluid entries are
    // renumbered; every other table is built in device order below, except the
    // per-iolet slot lists, which stay in canonical order of the sites so each
    // iolet's FP64 sums run in the same order whatever the layout.
    std::vector<int32_t> canon_of, dev_of;  // device -> canonical, canonical -> device
    if (d->ordering != HG_ORDER_MORTON) {
        std::string why;
        if (device_order(d->xyz, n, d->ordering, canon_of, why) != HG_OK)
            return fail(ctx, HG_ERR_ARG, "%s", why.c_str());
        dev_of.assign(n, 0);
        parallel_for(n, [&](int64_t lo, int64_t hi) {
            for (int64_t q = lo; q < hi; ++q) dev_of[canon_of[q]] = (int32_t)q;
        });
        I32Table row(n);
        for (int i = 0; i < 18; ++i) {
            int32_t *r = nbr.data() + (size_t)i * np;
            parallel_for(n, [&](int64_t lo, int64_t hi) {
                for (int64_t q = lo; q < hi; ++q) {
                    const int32_t v = r[canon_of[q]];
                    row[q] = v >= 0 ? dev_of[v] : v;
                }
            });
            parallel_for(n, [&](int64_t lo, int64_t hi) { std::copy(row.begin() + lo, row.begin() + hi, r + lo); });
        }
    }
    auto canon = [&](int64_t q) -> int64_t { return canon_of.empty() ? q : canon_of[q]; };

    trace.mark("device ordering");
    // --- iolet adjacency: slots numbered in device order (the kernels find a
    // site's slot as the rank of its flag), per-iolet CSR lists in canonical order
    I32Table slot_of(n);
    parallel_for(n, [&](int64_t lo, int64_t hi) { std::fill(slot_of.begin() + lo, slot_of.begin() + hi, -1); });
    int64_t n_adj = 0;
    std::vector<int64_t> per_io(nio + 1, 0);
    auto distinct_iolets = [&](int64_t q, int seen[18]) {
        int n_seen = 0;
        for (int i = 0; i < 18; ++i) {
            const int32_t v = nbr[(size_t)i * np + q];
            if (v < -1) {
                const int k = -v - 2;
                bool dup = false;
                for (int t = 0; t < n_seen; ++t) dup = dup || seen[t] == k;
                if (!dup) seen[n_seen++] = k;
            }
        }
        return n_seen;
    };
    // which sites have a link into an opening (parallel), then their slots in device order
    std::vector<uint8_t> touches((size_t)n, 0);
    if (nio > 0)
        parallel_for(n, [&](int64_t lo, int64_t hi) {
            for (int64_t q = lo; q < hi; ++q)
                for (int i = 0; i < 18; ++i)
                    if (nbr[(size_t)i * np + q] < -1) {
                        touches[(size_t)q] = 1;
                        break;
                    }
        });
    std::vector<int64_t> flagged;  // device positions of those sites, ascending
    for (int64_t q = 0; q < n; ++q)
        if (touches[(size_t)q]) {
            int seen[18];
            const int ns = distinct_iolets(q, seen);
            for (int t = 0; t < ns; ++t) per_io[seen[t] + 1]++;
            slot_of[q] = (int32_t)n_adj++;
            flagged.push_back(q);
        }
    std::vector<uint8_t>().swap(touches);
    d->n_adj = n_adj;
    for (int k = 0; k < nio; ++k) per_io[k + 1] += per_io[k];
    d->io_ptr.assign(per_io.begin(), per_io.end());
    std::vector<int32_t> slots(std::max<int64_t>(1, per_io[nio]));
    {
        std::vector<std::pair<int64_t, int64_t>> by_canon;  // (canonical index, device position)
        by_canon.reserve(flagged.size());
        for (int64_t q : flagged) by_canon.push_back({canon(q), q});
        std::sort(by_canon.begin(), by_canon.end());
        std::vector<int64_t> fill(per_io.begin(), per_io.end() - 1);
        for (const auto &cq : by_canon) {
            int seen[18];
            const int ns = distinct_iolets(cq.second, seen);
            for (int t = 0; t < ns; ++t) slots[fill[seen[t]]++] = slot_of[cq.second];
        }
    }
    std::vector<float> coef((size_t)std::max<int64_t>(1, n_adj) * 18, 0.0f);
    std::vector<uint32_t> mask((size_t)(np / 32), 0u);
    std::vector<int32_t> codes((size_t)std::max<int64_t>(1, n_adj) * 18, -1);
    for (int64_t q : flagged) {
        const int32_t sl = slot_of[q];
        mask[q >> 5] |= 1u << (q & 31);
        const int64_t c = canon(q);
        for (int i = 1; i < 19; ++i) {  // canonical codes: fluid links hold the canonical source
            const int32_t v = nbr[(size_t)(i - 1) * np + q];
            codes[(size_t)sl * 18 + (i - 1)] = v >= 0 ? (int32_t)canon(v) : v;
        }
        for (int i = 1; i < 19; ++i) {
            const int32_t v = nbr[(size_t)(i - 1) * np + q];
            if (v >= -1) continue;
            coef[(size_t)sl * 18 + (i - 1)] = link_coef(iolets[-v - 2], &d->xyz[3 * c], i, ctx->storage);
        }
    }
    // per-32-site prefix counts of flagged sites: slot = rank of the site's flag
    std::vector<int32_t> prefix(mask.size(), 0);
    {
        int32_t acc = 0;
        for (size_t w = 0; w < mask.size(); ++w) {
            prefix[w] = acc;
            acc += __builtin_popcount(mask[w]);
        }
    }
    trace.mark("iolet slots");
    // virtual indices for every non-fluid link (walls and iolet links alike)
    const bool aa = ctx->scheme == HG_SCHEME_AA;
    parallel_for(n, [&](int64_t lo, int64_t hi) {
        for (int64_t q = lo; q < hi; ++q)
            for (int i = 1; i < 19; ++i) {
                int32_t &v = nbr[(size_t)(i - 1) * np + q];
                if (v >= 0) continue;
                const int opp = (i & 1) ? i + 1 : i - 1;
                const int64_t dd = aa ? (int64_t)(i - opp) : (int64_t)(opp - i);
                v = (int32_t)(q + dd * np);
            }
    });
    std::vector<int32_t> slot_site((size_t)std::max<int64_t>(1, n_adj), 0);
    for (int64_t q = 0; q < n; ++q)
        if (slot_of[q] >= 0) slot_site[slot_of[q]] = (int32_t)q;
    trace.mark("virtual indices");
    U32Table lword;
    std::vector<int32_t> run0, rdelta;
    if (build_runs(nbr.data(), n, n, np, aa ? -1 : 1, lword, run0, rdelta))
        d->n_runs = (int64_t)rdelta.size() / kRunStride;
    d->io_codes_host = codes;
    d->slot_of_dev.assign(slot_of.begin(), slot_of.end());
    d->slots_host = slots;
    d->canon_of_host = canon_of;
    d->dev_of_host = dev_of;

    trace.mark("run encoding");
    // --- device buffers
    hg_ctx *c = ctx;
    const size_t eb = elem_bytes(ctx->storage);
    int rc = HG_OK;
    d->idx = slot_idx;
    auto A = [&](DevBuf &b, size_t bytes) {
        if (rc == HG_OK) rc = dev_alloc(c, b, bytes);
    };
    A(d->f[0], 19 * (size_t)np * eb);
    if (ctx->scheme == HG_SCHEME_AB) A(d->f[1], 19 * (size_t)np * eb);
    A(d->nbr, 18 * (size_t)np * 4);
    A(d->iomask, (size_t)np / 8);
    A(d->ioprefix, (size_t)np / 8);
    A(d->io_codes, codes.size() * 4);
    A(d->bnd, (size_t)std::max<int64_t>(1, n_adj) * 16);
    A(d->coef, coef.size() * 4);
    A(d->bcv, (size_t)std::max(1, nio) * 4);
    A(d->io_kind, (size_t)std::max(1, nio));
    A(d->M, (size_t)std::max(1, nio) * 24);
    A(d->slots, slots.size() * 4);
    A(d->force, (size_t)std::max(1, nio) * 16);
    A(d->slot_site, slot_site.size() * 4);
    if (!canon_of.empty()) {
        A(d->canon_of, (size_t)n * 4);
        A(d->dev_of, (size_t)n * 4);
    }
    if (d->n_runs) {
        A(d->lword, lword.size() * 4);
        A(d->run0, run0.size() * 4);
        A(d->rdelta, rdelta.size() * 4);
    }
    auto cleanup = [&] {
        for (DevBuf *b : domain_buffers(d.get())) dev_free(c, *b);
    };
    if (rc != HG_OK) {
        cleanup();
        return rc;
    }
    for (DevBuf *b : domain_buffers(d.get())) d->bytes += (int64_t)b->bytes;
    std::vector<float> bcv(std::max(1, nio), 0.0f);
    std::vector<int8_t> kinds(std::max(1, nio), 0);
    for (int k = 0; k < nio; ++k) {
        bcv[k] = (float)(iolets[k].value * pulse(iolets[k].pulse, 1.0, iolets[k].period));
        kinds[k] = (int8_t)iolets[k].kind;
    }
    trace.mark("allocation");
    // uploads run on a stream of this build, so a build on another thread
    // neither waits for nor races with the context's stream
    cudaStream_t up = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&up, cudaStreamNonBlocking);
    auto H2D = [&](DevBuf &b, const void *src, size_t bytes) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, up);
    };
    H2D(d->nbr, nbr.data(), nbr.size() * 4);
    H2D(d->iomask, mask.data(), mask.size() * 4);
    H2D(d->ioprefix, prefix.data(), prefix.size() * 4);
    H2D(d->io_codes, codes.data(), codes.size() * 4);
    H2D(d->coef, coef.data(), coef.size() * 4);
    H2D(d->bcv, bcv.data(), bcv.size() * 4);
    H2D(d->io_kind, kinds.data(), kinds.size());
    H2D(d->slots, slots.data(), slots.size() * 4);
    H2D(d->slot_site, slot_site.data(), slot_site.size() * 4);
    if (!canon_of.empty()) {
        H2D(d->canon_of, canon_of.data(), (size_t)n * 4);
        H2D(d->dev_of, dev_of.data(), (size_t)n * 4);
    }
    if (d->n_runs) {
        H2D(d->lword, lword.data(), lword.size() * 4);
        H2D(d->run0, run0.data(), run0.size() * 4);
        H2D(d->rdelta, rdelta.data(), rdelta.size() * 4);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(d->f[0].p, 0, d->f[0].bytes, up);
    if (e == cudaSuccess && d->f[1].p) e = cudaMemsetAsync(d->f[1].p, 0, d->f[1].bytes, up);
    if (e == cudaSuccess) e = cudaMemsetAsync(d->bnd.p, 0, d->bnd.bytes, up);
    if (e == cudaSuccess) e = cudaMemsetAsync(d->M.p, 0, d->M.bytes, up);
    if (e == cudaSuccess) e = cudaMemsetAsync(d->force.p, 0, d->force.bytes, up);
    if (e == cudaSuccess) e = cudaMemsetAsync((int64_t *)ctx->steps.p + slot_idx, 0, sizeof(int64_t), up);
    DomDev D = make_domdev(ctx, d.get());
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((DomDev *)ctx->dom_table.p + slot_idx, &D, sizeof D, cudaMemcpyHostToDevice, up);
    if (up) {
        const cudaError_t es = cudaStreamSynchronize(up);
        if (e == cudaSuccess) e = es;
        cudaStreamDestroy(up);
    }
    if (e != cudaSuccess) {
        cleanup();
        return fail(ctx, HG_ERR_CUDA, "upload failed: %s", cudaGetErrorString(e));
    }
    trace.mark("upload");
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->doms[slot_idx] = d.get();
    }
    *out = d.release();
    return HG_OK;
}

int hg_domain_destroy(hg_domain *d) {
    if (!d) return HG_ERR_ARG;
    hg_ctx *ctx = d->ctx;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    drop_plans(ctx);
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        for (auto it = ctx->coupled.begin(); it != ctx->coupled.end();) {
            if (it->first.first == d->idx || it->second.src_dom == d->idx) it = ctx->coupled.erase(it);
            else ++it;
        }
        ctx->doms[d->idx] = nullptr;
    }
    for (DevBuf *b : domain_buffers(d)) dev_free(ctx, *b);
    if (ctx->couple_mode == HG_COUPLE_ALTERNATE) refresh_domdevs(ctx);  // a source may have lost its pairs
    delete d;
    return HG_OK;
}

int hg_domain_info(hg_domain *d, int64_t *n_sites, int32_t *n_iolets, int64_t *n_adjacent,
                   int64_t *step, int64_t *device_bytes) {
    if (!d) return HG_ERR_ARG;
    if (n_sites) *n_sites = d->n;
    if (n_iolets) *n_iolets = d->nio;
    if (n_adjacent) *n_adjacent = d->n_adj;
    if (step) *step = d->step;
    if (device_bytes) *device_bytes = d->bytes;
    return HG_OK;
}

int hg_encode_runs(const int32_t *nbr, int64_t n, int64_t n_ref, int64_t row_stride, int32_t scheme,
                   uint32_t *lword_out, int32_t *run0_out, int32_t *rdelta_out, int64_t *n_runs_out) {
    if (!nbr || !n_runs_out || n < 1 || n_ref < n || row_stride < n || row_stride > ((int64_t)1 << 30) ||
        (scheme != HG_SCHEME_AB && scheme != HG_SCHEME_AA))
        return HG_ERR_ARG;
    U32Table lw;
    std::vector<int32_t> r0, rd;
    *n_runs_out = 0;
    if (!build_runs(nbr, n, n_ref, row_stride, scheme == HG_SCHEME_AA ? -1 : 1, lw, r0, rd)) return HG_OK;
    *n_runs_out = (int64_t)rd.size() / kRunStride;
    if (lword_out) std::copy(lw.begin(), lw.end(), lword_out);
    if (run0_out) std::copy(r0.begin(), r0.end(), run0_out);
    if (rdelta_out)
        for (int64_t r = 0; r < *n_runs_out; ++r)
            std::copy(rd.begin() + r * kRunStride, rd.begin() + r * kRunStride + 18, rdelta_out + r * 18);
    return HG_OK;
}

int hg_domain_runs(hg_domain *d, int64_t *n_runs) {
    if (!d || !n_runs) return HG_ERR_ARG;
    *n_runs = d->n_runs;
    return HG_OK;
}

int hg_domain_sites(hg_domain *d, int32_t *xyz_out) {
    if (!d || (!xyz_out && d->n)) return HG_ERR_ARG;
    if (d->n) memcpy(xyz_out, d->xyz.data(), sizeof(int32_t) * 3 * d->n);
    return HG_OK;
}

int hg_domain_neighbours(hg_domain *d, int32_t *nbr_out) {
    if (!d || (!nbr_out && d->n)) return HG_ERR_ARG;
    hg_ctx *ctx = d->ctx;
    CU(ctx, cudaSetDevice(ctx->device));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    std::vector<int32_t> row(std::max<int64_t>(1, d->n));
    const std::vector<int32_t> &co = d->canon_of_host, &dv = d->dev_of_host;
    for (int i = 0; i < 18; ++i) {
        CU(ctx, cudaMemcpy(row.data(), (const int32_t *)d->nbr.p + (size_t)i * d->np,
                           sizeof(int32_t) * d->n, cudaMemcpyDeviceToHost));
        // back to canonical positions and indices; virtual indices (outside [0, n)) mark
        // non-fluid links: wall, or the iolet code of the site's slot
        for (int64_t c = 0; c < d->n; ++c) {
            const int64_t q = dv.empty() ? c : dv[c];
            const int32_t v = row[q];
            int32_t &o = nbr_out[(size_t)i * d->n + c];
            if (v >= 0 && v < d->n) {
                o = co.empty() ? v : co[v];
            } else {
                const int32_t sl = d->slot_of_dev[q];
                o = sl >= 0 ? d->io_codes_host[(size_t)sl * 18 + i] : -1;
            }
        }
    }
    return HG_OK;
}

int hg_couple(hg_ctx *ctx, hg_domain *src, hg_domain *dst, const hg_pair *pairs, int32_t n) {
    if (!ctx) return HG_ERR_ARG;
    if (!src || !dst || src->ctx != ctx || dst->ctx != ctx || src == dst)
        return fail(ctx, HG_ERR_ARG, "coupling needs two distinct domains of this context");
    if (n < 0 || (n > 0 && !pairs)) return fail(ctx, HG_ERR_ARG, "bad pair array");
    for (int j = 0; j < n; ++j) {
        const hg_pair &p = pairs[j];
        if (p.src_iolet < 0 || p.src_iolet >= src->nio || p.dst_iolet < 0 || p.dst_iolet >= dst->nio)
            return fail(ctx, HG_ERR_ARG, "pair %d: iolet index out of range", j);
        if (dst->io[p.dst_iolet].kind != HG_VELOCITY)
            return fail(ctx, HG_ERR_ARG, "pair %d: destination iolet is not a velocity iolet", j);
        bool taken;
        {
            std::lock_guard<std::mutex> lk(ctx->mu);
            taken = ctx->coupled.count({dst->idx, p.dst_iolet}) != 0;
        }
        if (taken) return fail(ctx, HG_ERR_ARG, "pair %d: destination iolet already coupled", j);
        for (int q = 0; q < j; ++q)
            if (pairs[q].dst_iolet == p.dst_iolet)
                return fail(ctx, HG_ERR_ARG, "pair %d: destination iolet repeated", j);
        if (!std::isfinite(p.factor)) return fail(ctx, HG_ERR_ARG, "pair %d: factor not finite", j);
    }
    CU(ctx, cudaSetDevice(ctx->device));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    // the next step's value follows the source's current mean at once
    std::vector<double> Ms((size_t)std::max(1, src->nio) * 3);
    CU(ctx, cudaMemcpyAsync(Ms.data(), src->M.p, Ms.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    std::vector<float> v(std::max(1, n));
    for (int j = 0; j < n; ++j) {
        const hg_pair &p = pairs[j];
        {
            std::lock_guard<std::mutex> lk(ctx->mu);
            ctx->coupled[{dst->idx, p.dst_iolet}] = {src->idx, p.src_iolet, p.factor};
        }
        v[j] = (float)(p.factor * Ms[3 * p.src_iolet]);
        CU(ctx, cudaMemcpyAsync((float *)dst->bcv.p + p.dst_iolet, &v[j], 4, cudaMemcpyHostToDevice, ctx->stream));
    }
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    drop_plans(ctx);
    CU(ctx, refresh_domdevs(ctx));
    return HG_OK;
}

int hg_set_coupling_mode(hg_ctx *ctx, int32_t mode) {
    if (!ctx) return HG_ERR_ARG;
    if (mode != HG_COUPLE_FORWARD && mode != HG_COUPLE_ALTERNATE)
        return fail(ctx, HG_ERR_ARG, "unknown coupling mode %d", mode);
    CU(ctx, cudaSetDevice(ctx->device));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    std::vector<hg_domain *> live;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        for (hg_domain *d : ctx->doms)
            if (d) live.push_back(d);
    }
    for (hg_domain *d : live) CU(ctx, cudaMemsetAsync(d->force.p, 0, d->force.bytes, ctx->stream));
    ctx->couple_mode = mode;
    drop_plans(ctx);
    CU(ctx, refresh_domdevs(ctx));
    return HG_OK;
}

int hg_build_neighbours(const int32_t *xyz, int64_t n, const hg_iolet *iolets, int32_t nio, int32_t *xyz_out,
                        int32_t *nbr_out) {
    if (n < 0 || (n > 0 && (!xyz || !nbr_out))) return HG_ERR_ARG;
    if (nio < 0 || nio > kMaxIolets || (nio > 0 && !iolets)) return HG_ERR_ARG;
    for (int k = 0; k < nio; ++k)
        if (!iolet_ok(iolets[k])) return HG_ERR_ARG;
    std::vector<int32_t> xs;
    I32Table nbr;
    std::string why;
    const int rc = build_canonical(xyz, n, iolets, nio, n, xs, nbr, why);
    if (rc != HG_OK) return fail(nullptr, rc, "%s", why.c_str());
    if (n > 0) {
        memcpy(nbr_out, nbr.data(), (size_t)18 * n * sizeof(int32_t));
        if (xyz_out) memcpy(xyz_out, xs.data(), (size_t)3 * n * sizeof(int32_t));
    }
    return HG_OK;
}

int hg_coupling_factors(const int64_t *art_c, const double *art_a, int32_t na, const int64_t *ven_c,
                        const double *ven_a, int32_t nv, const double *uni, int32_t *assign,
                        double *dist, double *dp, double *factor) {
    if (na < 1 || nv < 0 || !art_c || !art_a || (nv > 0 && (!ven_c || !ven_a || !uni || !assign ||
                                                          !dist || !dp || !factor)))
        return HG_ERR_ARG;
    typedef __int128 i128;
    auto d2 = [&](int a, int v) {
        i128 s = 0;
        for (int c = 0; c < 3; ++c) {
            const i128 t = (i128)art_c[3 * a + c] - ven_c[3 * v + c];
            s += t * t;
        }
        return s;
    };
    std::vector<char> taken(nv, 0);
    for (int v = 0; v < nv; ++v) assign[v] = -1;
    for (int a = 0; a < na; ++a) {
        int best = -1;
        i128 bd = 0;
        for (int v = 0; v < nv; ++v) {
            if (taken[v]) continue;
            const i128 dd = d2(a, v);
            if (best < 0 || dd < bd) {
                best = v;
                bd = dd;
            }
        }
        if (best < 0) break;
        taken[best] = 1;
        assign[best] = a;
    }
    for (int v = 0; v < nv; ++v) {
        if (taken[v]) continue;
        int best = 0;
        i128 bd = d2(0, v);
        for (int a = 1; a < na; ++a) {
            const i128 dd = d2(a, v);
            if (dd < bd) {
                best = a;
                bd = dd;
            }
        }
        assign[v] = best;
    }
    for (int v = 0; v < nv; ++v) {
        dist[v] = std::sqrt((double)d2(assign[v], v)) / 1024.0;
        dp[v] = 0.3 + 0.4 * uni[v];
        if (!(dist[v] > 0) || !(ven_a[v] > 0)) return HG_ERR_ARG;
    }
    for (int a = 0; a < na; ++a) {
        if (!(art_a[a] > 0)) return HG_ERR_ARG;
        int first = -1;
        for (int v = 0; v < nv; ++v)
            if (assign[v] == a) {
                first = v;
                break;
            }
        if (first < 0) continue;
        // ratio_i = dP_i L_1 A_i / (dP_1 L_i A_1); factor_i = (A_0 / A_i) ratio_i / sum ratio
        double total = 0.0;
        for (int v = 0; v < nv; ++v)
            if (assign[v] == a)
                total += dp[v] * dist[first] * ven_a[v] / (dp[first] * dist[v] * ven_a[first]);
        for (int v = 0; v < nv; ++v)
            if (assign[v] == a) {
                const double r = dp[v] * dist[first] * ven_a[v] / (dp[first] * dist[v] * ven_a[first]);
                factor[v] = (art_a[a] / ven_a[v]) * r / total;
            }
    }
    return HG_OK;
}

}  // extern "C"

// ================================================================ stepping
namespace {

int build_plan(hg_ctx *ctx, const std::vector<int32_t> &doms, Plan *&out) {
    PlanKey key{doms};
    auto it = ctx->plans.find(key);
    if (it != ctx->plans.end()) {
        out = it->second.get();
        return HG_OK;
    }
    std::unique_ptr<Plan> p(new Plan);
    p->doms = doms;
    const int64_t ts = (int64_t)ctx->block * ctx->spt;
    std::vector<TileDev> tiles;
    std::vector<IoDev> ios;
    std::vector<int2> chunks;
    std::vector<std::pair<int32_t, int32_t>> io_key;  // (domain, iolet) of each IoDev
    std::vector<RevSrc> rev;
    std::vector<int2> forced;                          // (domain, slot) under a body force
    std::vector<std::pair<size_t, int32_t>> rev_of;    // per IoDev: (first RevSrc, count)
    std::map<std::pair<int32_t, int32_t>, std::vector<std::pair<int32_t, int32_t>>> fed;  // source -> inlets
    if (ctx->couple_mode == HG_COUPLE_ALTERNATE) {
        std::lock_guard<std::mutex> lk(ctx->mu);
        for (const auto &kv : ctx->coupled)
            fed[{kv.second.src_dom, kv.second.src_k}].push_back(kv.first);
    }
    // large domains get a single-domain launch each (chained); the rest share one
    // tile-table launch
    std::vector<char> separate(doms.size(), 0);
    if (doms.size() > 1) {
        int n_sep = 0;
        for (size_t j = 0; j < doms.size() && n_sep < kSeparateMaxDoms; ++j)
            if (ctx->doms[doms[j]]->n >= kSeparateMinSites) {
                separate[j] = 1;
                ++n_sep;
            }
    }
    for (size_t j = 0; j < doms.size(); ++j) {
        const int32_t di = doms[j];
        hg_domain *d = ctx->doms[di];
        if (separate[j]) {
            p->sep.push_back(make_domdev(ctx, d));
            p->sep_n.push_back(d->n);
        } else if (doms.size() > 1) {
            p->tiles_runs = p->tiles_runs && d->n_runs > 0;
            for (int64_t s = 0; s < d->n; s += ts) {
                TileDev t;
                t.dom = di;
                t.count = (int32_t)std::min(ts, d->n - s);
                t.start = s;
                tiles.push_back(t);
            }
        }
        for (int k = 0; k < d->nio; ++k) {
            IoDev I;
            memset(&I, 0, sizeof I);
            const hg_iolet &io = d->io[k];
            I.slots = (const int32_t *)d->slots.p + d->io_ptr[k];
            I.n_slots = (int32_t)(d->io_ptr[k + 1] - d->io_ptr[k]);
            I.bnd = (const float4 *)d->bnd.p;
            I.M = (double *)d->M.p + 3 * k;
            I.bcv = (float *)d->bcv.p + k;
            I.step = (const int64_t *)ctx->steps.p + di;
            const double an = std::sqrt((double)io.axis[0] * io.axis[0] + (double)io.axis[1] * io.axis[1] +
                                        (double)io.axis[2] * io.axis[2]);
            I.nx = io.axis[0] / an;
            I.ny = io.axis[1] / an;
            I.nz = io.axis[2] / an;
            I.value = io.value;
            I.period = io.period;
            I.pulse = io.pulse;
            I.n_chunks = std::max(1, (I.n_slots + kIoChunk - 1) / kIoChunk);
            I.part0 = (int32_t)chunks.size();
            for (int c = 0; c < I.n_chunks; ++c) chunks.push_back(make_int2((int)ios.size(), c));
            bool is_coupled = false;
            CoupleSrc cs{};
            {
                std::lock_guard<std::mutex> lk(ctx->mu);
                auto cp = ctx->coupled.find({di, k});
                if (cp != ctx->coupled.end()) {
                    is_coupled = true;
                    cs = cp->second;
                }
            }
            if (is_coupled) {
                hg_domain *sd = ctx->doms[cs.src_dom];
                if (std::find(doms.begin(), doms.end(), cs.src_dom) == doms.end())
                    return fail(ctx, HG_ERR_ARG, "a coupled source domain is not being stepped");
                I.coupled = 1;
                I.factor = cs.factor;
                I.src_M = (const double *)sd->M.p + 3 * cs.src_k;
            }
            I.force = (float4 *)d->force.p + k;
            I.alternate = ctx->couple_mode == HG_COUPLE_ALTERNATE;
            auto fd = fed.find({di, k});
            size_t r0 = rev.size();
            if (fd != fed.end()) {
                for (const auto &dst : fd->second) {
                    if (std::find(doms.begin(), doms.end(), dst.first) == doms.end())
                        return fail(ctx, HG_ERR_ARG, "a coupled destination domain is not being stepped");
                    double f;
                    {
                        std::lock_guard<std::mutex> lk(ctx->mu);
                        f = ctx->coupled.at(dst).factor;
                    }
                    rev.push_back(RevSrc{(const double *)ctx->doms[dst.first]->M.p + 3 * dst.second, f});
                }
            }
            rev_of.push_back({r0, (int32_t)(rev.size() - r0)});
            if (fd != fed.end())  // the outlet's adjacent slots take its body force
                for (int64_t q = d->io_ptr[k]; q < d->io_ptr[k + 1]; ++q)
                    forced.push_back(make_int2(di, d->slots_host[q]));
            ios.push_back(I);
        }
    }
    std::sort(forced.begin(), forced.end(),
              [](int2 a, int2 b) { return a.x != b.x ? a.x < b.x : a.y < b.y; });
    forced.erase(std::unique(forced.begin(), forced.end(),
                             [](int2 a, int2 b) { return a.x == b.x && a.y == b.y; }),
                 forced.end());
    p->n_tiles = (int64_t)tiles.size();
    p->n_ios = (int)ios.size();
    if (doms.size() == 1) {
        p->single = true;
        p->one = make_domdev(ctx, ctx->doms[doms[0]]);
        p->tiles_runs = ctx->doms[doms[0]]->n_runs > 0;
        const int64_t n1 = ctx->doms[doms[0]]->n;
        p->n_tiles = (n1 + ts - 1) / ts;
    }
    p->n_chunks = (int)chunks.size();
    int rc = dev_alloc(ctx, p->tiles, std::max<size_t>(1, tiles.size()) * sizeof(TileDev));
    if (rc == HG_OK) rc = dev_alloc(ctx, p->ios, std::max<size_t>(1, ios.size()) * sizeof(IoDev));
    if (rc == HG_OK) rc = dev_alloc(ctx, p->adv, std::max<size_t>(1, doms.size()) * 4);
    if (rc == HG_OK) rc = dev_alloc(ctx, p->chunks, std::max<size_t>(1, chunks.size()) * sizeof(int2));
    if (rc == HG_OK) rc = dev_alloc(ctx, p->partials, std::max<size_t>(1, chunks.size()) * sizeof(double2));
    if (rc == HG_OK) rc = dev_alloc(ctx, p->counters, (ios.size() + 1) * sizeof(unsigned));
    if (rc == HG_OK) rc = dev_alloc(ctx, p->rev, std::max<size_t>(1, rev.size()) * sizeof(RevSrc));
    if (rc == HG_OK) rc = dev_alloc(ctx, p->fslots, std::max<size_t>(1, forced.size()) * sizeof(int2));
    p->n_fslots = (int)forced.size();
    if (rc != HG_OK) {
        for (DevBuf *b : {&p->tiles, &p->ios, &p->adv, &p->chunks, &p->partials, &p->counters, &p->rev, &p->fslots})
            dev_free(ctx, *b);
        return rc;
    }
    for (size_t q = 0; q < ios.size(); ++q) {
        ios[q].rev = (const RevSrc *)p->rev.p + rev_of[q].first;
        ios[q].n_rev = rev_of[q].second;
    }
    // stream-ordered before the plan's first launch (pageable sources are staged on the call)
    cudaStream_t st = ctx->stream;
    cudaError_t e = cudaMemsetAsync(p->counters.p, 0, p->counters.bytes, st);
    if (e == cudaSuccess && !tiles.empty())
        e = cudaMemcpyAsync(p->tiles.p, tiles.data(), tiles.size() * sizeof(TileDev), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !ios.empty())
        e = cudaMemcpyAsync(p->ios.p, ios.data(), ios.size() * sizeof(IoDev), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->adv.p, doms.data(), doms.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !chunks.empty())
        e = cudaMemcpyAsync(p->chunks.p, chunks.data(), chunks.size() * sizeof(int2), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !rev.empty())
        e = cudaMemcpyAsync(p->rev.p, rev.data(), rev.size() * sizeof(RevSrc), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !forced.empty())
        e = cudaMemcpyAsync(p->fslots.p, forced.data(), forced.size() * sizeof(int2), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(st);
        for (DevBuf *b : {&p->tiles, &p->ios, &p->adv, &p->chunks, &p->partials, &p->counters, &p->rev, &p->fslots})
            dev_free(ctx, *b);
        return fail(ctx, HG_ERR_CUDA, "plan upload failed: %s", cudaGetErrorString(e));
    }
    out = p.get();
    ctx->plans[key] = std::move(p);
    return HG_OK;
}

// Parity mode of a domain set: 0 / 1 = every domain has completed an even / odd
// number of steps (AA kernels specialised per step kind), 2 = mixed.
int parity_mode(hg_ctx *ctx, const std::vector<int32_t> &doms) {
    int m = -1;
    for (int32_t di : doms) {
        const int q = (int)(ctx->doms[di]->step & 1);
        if (m < 0) m = q;
        else if (m != q) return 2;
    }
    return m < 0 ? 0 : m;
}

// Kernel parity argument for the step at offset `off` of a group starting in `mode`.
inline int step_parity(hg_ctx *ctx, int mode, int64_t off) {
    if (ctx->scheme == HG_SCHEME_AB || mode == 2) return 2;
    return (int)((mode + off + 1) & 1);  // 1 when the executed step is odd
}

// Halo exchange of a split domain after step offset `off`: every partition's F_t
// values that another partition pulls are packed per (sender, receiver) pair,
// each pair's block is copied into the receiver's buffer (on one device a plain
// device-to-device copy; between devices this is the one transfer that changes),
// and unpacked into the receiver's ghost positions.
cudaError_t enqueue_halo(hg_ctx *ctx, Plan *p, int off) {
    if (p->n_halo == 0) return cudaSuccess;
    const DomDev *doms = (const DomDev *)ctx->dom_table.p;
    const int64_t *steps = (const int64_t *)ctx->steps.p;
    if (!p->halo_staged)
        return launch_halo_direct(p->halo_elem, doms, steps, (const HaloMove *)p->halo_moves.p, p->n_halo, off,
                                  ctx->stream);
    cudaError_t e = launch_halo_pack(p->halo_elem, doms, steps, (const HaloDev *)p->halo_pack.p, p->n_halo,
                                     p->send.p, off, ctx->stream);
    for (const auto &b : p->halo_blocks) {
        if (e != cudaSuccess) return e;
        e = cudaMemcpyAsync((char *)p->recv.p + b.first, (const char *)p->send.p + b.first, b.second,
                            cudaMemcpyDeviceToDevice, ctx->stream);
    }
    if (e != cudaSuccess) return e;
    return launch_halo_unpack(p->halo_elem, doms, steps, (const HaloDev *)p->halo_unpack.p, p->n_halo,
                              p->recv.p, off, ctx->stream);
}

// The stream-collide launch(es) of step offset `off`.  overlap: the first launch may
// start while the previous step's iolet update runs; separate per-domain launches
// after the first may start while the previous one runs (they share no data within
// a step; sites with iolet links still wait, through the chain, for that update).
// The run-encoded variants (8..11) step only domains that have a run encoding;
// a launch over any other domain takes the table form of the same variant.
CollideCfg collide_cfg(hg_ctx *ctx, bool runs) {
    CollideCfg cfg{ctx->storage, ctx->scheme, ctx->block, ctx->spt, ctx->variant};
    if (cfg.variant >= 8 && !runs)
        cfg.variant = cfg.variant == 8 || cfg.variant == 12 || cfg.variant == 13 ? 3
                      : cfg.variant == 9                                      ? 5
                      : cfg.variant == 10 || cfg.variant == 14                ? 6
                                                                              : 7;
    return cfg;
}

cudaError_t launch_sc(hg_ctx *ctx, Plan *p, int off, int parity, bool overlap) {
    const int64_t *steps = (const int64_t *)ctx->steps.p;
    const DomDev *table = (const DomDev *)ctx->dom_table.p;
    const int64_t ts = (int64_t)ctx->block * ctx->spt;
    bool chained = overlap;
    for (size_t j = 0; j < p->sep.size(); ++j) {
        if (p->sep_n[j] == 0) continue;
        const OneDomain one{&p->sep[j], p->sep_n[j], steps, chained};
        const cudaError_t e = launch_stream_collide(collide_cfg(ctx, p->sep[j].lword != nullptr), table, nullptr,
                                                    (p->sep_n[j] + ts - 1) / ts, off, parity, one, ctx->stream);
        if (e != cudaSuccess) return e;
        chained = true;
    }
    if (p->n_tiles == 0) return cudaSuccess;
    const OneDomain one{p->single ? &p->one : nullptr, p->single ? ctx->doms[p->doms[0]]->n : 0, steps, chained};
    return launch_stream_collide(collide_cfg(ctx, p->tiles_runs), table, (const TileDev *)p->tiles.p, p->n_tiles,
                                 off, parity, one, ctx->stream);
}

cudaError_t enqueue_steps(hg_ctx *ctx, Plan *p, int64_t k, int mode) {
    for (int64_t off = 0; off < k; ++off) {
        // after the first step of a group the previous kernel is this group's iolet update
        // (the first follows the step-counter advance, which the parity read needs)
        cudaError_t e = launch_sc(ctx, p, (int)off, step_parity(ctx, mode, off), off > 0 && p->n_ios > 0);
        if (e != cudaSuccess) return e;
        e = launch_guo_force(ctx->storage, ctx->scheme, (const DomDev *)ctx->dom_table.p,
                             (const int2 *)p->fslots.p, p->n_fslots, (int)off, ctx->stream);
        if (e != cudaSuccess) return e;
        e = enqueue_halo(ctx, p, (int)off);
        if (e != cudaSuccess) return e;
        e = launch_iolet_update((const IoDev *)p->ios.p, p->n_ios, (const int2 *)p->chunks.p, p->n_chunks,
                                (double2 *)p->partials.p, (unsigned *)p->counters.p, (int)off, ctx->stream);
        if (e != cudaSuccess) return e;
    }
    return launch_advance_list((int64_t *)ctx->steps.p, (const int32_t *)p->adv.p, (int)p->doms.size(), k,
                               ctx->stream);
}

int ensure_graph(hg_ctx *ctx, Plan *p, int mode) {
    if (p->graph[mode] || ctx->graph_steps <= 0) return HG_OK;
    cudaGraph_t g = nullptr;
    CU(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue_steps(ctx, p, ctx->graph_steps, mode);
    cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return fail(ctx, HG_ERR_CUDA, "graph capture failed: %s",
                    cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&p->graph[mode], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        p->graph[mode] = nullptr;
        return fail(ctx, HG_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
    }
    p->graph_steps = ctx->graph_steps;
    return HG_OK;
}

// n steps of a plan: whole groups as graph replays, the rest launched directly.
int run_plan(hg_ctx *ctx, Plan *p, int64_t n, int mode) {
    int64_t left = n;
    if (ctx->graph_steps > 0 && n >= ctx->graph_steps) {
        while (left >= ctx->graph_steps) {
            const int rc = ensure_graph(ctx, p, mode);
            if (rc != HG_OK) return rc;
            CU(ctx, cudaGraphLaunch(p->graph[mode], ctx->stream));
            left -= ctx->graph_steps;
            if (mode != 2) mode = (int)((mode + ctx->graph_steps) & 1);
        }
    }
    if (left > 0) CU(ctx, enqueue_steps(ctx, p, left, mode));
    return HG_OK;
}

int step_set(hg_ctx *ctx, std::vector<int32_t> doms, int64_t n) {
    if (n < 0) return fail(ctx, HG_ERR_ARG, "negative step count");
    std::sort(doms.begin(), doms.end());
    doms.erase(std::unique(doms.begin(), doms.end()), doms.end());
    if (doms.empty() || n == 0) return HG_OK;
    CU(ctx, cudaSetDevice(ctx->device));
    Plan *p = nullptr;
    int rc = build_plan(ctx, doms, p);
    if (rc != HG_OK) return rc;
    rc = run_plan(ctx, p, n, parity_mode(ctx, doms));
    if (rc != HG_OK) return rc;
    for (int32_t di : doms) ctx->doms[di]->step += n;
    return HG_OK;
}

}  // namespace

extern "C" {

int hg_step(hg_ctx *ctx, int64_t n) {
    if (!ctx) return HG_ERR_ARG;
    std::vector<int32_t> doms;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        for (int i = 0; i < ctx->capacity; ++i)
            if (ctx->doms[i]) doms.push_back(i);
    }
    return step_set(ctx, doms, n);
}

int hg_step_domains(hg_ctx *ctx, hg_domain *const *ds, int32_t nd, int64_t n) {
    if (!ctx) return HG_ERR_ARG;
    if (nd < 0 || (nd > 0 && !ds)) return fail(ctx, HG_ERR_ARG, "bad domain list");
    std::vector<int32_t> doms;
    for (int j = 0; j < nd; ++j) {
        if (!ds[j] || ds[j]->ctx != ctx) return fail(ctx, HG_ERR_ARG, "domain %d not in this context", j);
        doms.push_back(ds[j]->idx);
    }
    return step_set(ctx, doms, n);
}

int hg_step_profiled(hg_ctx *ctx, int64_t n, double *ms_sc, double *ms_io, float *per_step) {
    if (!ctx) return HG_ERR_ARG;
    if (n < 0) return fail(ctx, HG_ERR_ARG, "negative step count");
    std::vector<int32_t> doms;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        for (int i = 0; i < ctx->capacity; ++i)
            if (ctx->doms[i]) doms.push_back(i);
    }
    if (ms_sc) *ms_sc = 0.0;
    if (ms_io) *ms_io = 0.0;
    if (doms.empty() || n == 0) return HG_OK;
    CU(ctx, cudaSetDevice(ctx->device));
    Plan *p = nullptr;
    int rc = build_plan(ctx, doms, p);
    if (rc != HG_OK) return rc;
    std::vector<cudaEvent_t> ev((size_t)3 * n);
    for (auto &x : ev) CU(ctx, cudaEventCreate(&x));
    const int mode = parity_mode(ctx, doms);
    cudaError_t e = cudaSuccess;
    for (int64_t j = 0; j < n && e == cudaSuccess; ++j) {
        cudaEventRecord(ev[3 * j], ctx->stream);
        e = launch_sc(ctx, p, (int)j, step_parity(ctx, mode, j), false);  // timed launches stay serial
        cudaEventRecord(ev[3 * j + 1], ctx->stream);
        if (e == cudaSuccess)  // the body-force pass (if any) is timed with the iolet update
            e = launch_guo_force(ctx->storage, ctx->scheme, (const DomDev *)ctx->dom_table.p,
                                 (const int2 *)p->fslots.p, p->n_fslots, (int)j, ctx->stream);
        if (e == cudaSuccess)
            e = launch_iolet_update((const IoDev *)p->ios.p, p->n_ios, (const int2 *)p->chunks.p, p->n_chunks,
                                    (double2 *)p->partials.p, (unsigned *)p->counters.p, (int)j, ctx->stream);
        cudaEventRecord(ev[3 * j + 2], ctx->stream);
    }
    if (e == cudaSuccess)
        e = launch_advance_list((int64_t *)ctx->steps.p, (const int32_t *)p->adv.p, (int)doms.size(), n,
                                ctx->stream);
    cudaError_t es = cudaStreamSynchronize(ctx->stream);
    double a = 0.0, b = 0.0;
    for (int64_t j = 0; j < n && e == cudaSuccess && es == cudaSuccess; ++j) {
        float x = 0.f, y = 0.f;
        cudaEventElapsedTime(&x, ev[3 * j], ev[3 * j + 1]);
        cudaEventElapsedTime(&y, ev[3 * j + 1], ev[3 * j + 2]);
        a += x;
        b += y;
        if (per_step) {
            per_step[2 * j] = x;
            per_step[2 * j + 1] = y;
        }
    }
    for (auto &x : ev) cudaEventDestroy(x);
    if (e != cudaSuccess) return fail(ctx, HG_ERR_CUDA, "launch failed: %s", cudaGetErrorString(e));
    if (es != cudaSuccess) return fail(ctx, HG_ERR_CUDA, "step failed: %s", cudaGetErrorString(es));
    for (int32_t di : doms) ctx->doms[di]->step += n;
    if (ms_sc) *ms_sc = a;
    if (ms_io) *ms_io = b;
    return HG_OK;
}

int hg_ctx_set_launch(hg_ctx *ctx, int32_t block, int32_t spt, int32_t variant) {
    if (!ctx) return HG_ERR_ARG;
    if (block < 32 || block > 512 || block % 32) return fail(ctx, HG_ERR_ARG, "block size must be a multiple of 32 in [32, 512]");
    if (spt != 1 && spt != 2 && spt != 4) return fail(ctx, HG_ERR_ARG, "sites per thread must be 1, 2 or 4");
    if (!variant_ok(ctx->storage, ctx->scheme, spt, variant))
        return fail(ctx, HG_ERR_ARG, "kernel variant must be 0 or 3, 1 or 2 with 1 or 2 sites per thread "
                                     "(2: AA only), 4 with 1 site per thread (AA only), 5 with 2 sites "
                                     "per thread (A/B, 16-bit storage only), 6 or 7 with 2 sites per "
                                     "thread (AA only), 8..11 with the shapes of 3, 5, 6, 7, 12 with 1 or "
                                     "2 sites per thread (AA only), 13 with 2 or 4 sites per thread, or 14 "
                                     "with 2 sites per thread (AA only)");
    if (block == ctx->block && spt == ctx->spt && variant == ctx->variant) return HG_OK;
    CU(ctx, cudaSetDevice(ctx->device));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->block = block;
    ctx->spt = spt;
    ctx->variant = variant;
    drop_plans(ctx);
    return HG_OK;
}

int hg_read_macroscopic_device(hg_domain *d, float *dev_out) {
    if (!d || (!dev_out && d->n)) return HG_ERR_ARG;
    hg_ctx *ctx = d->ctx;
    if (((uintptr_t)dev_out) & 15) return fail(ctx, HG_ERR_ARG, "output must be 16-byte aligned");
    CU(ctx, cudaSetDevice(ctx->device));
    CU(ctx, launch_macroscopic(ctx->storage, ctx->scheme, domdev_ptr(d), d->n, (const int32_t *)d->canon_of.p,
                               (float4 *)dev_out, ctx->stream));
    return HG_OK;
}

int hg_read_macroscopic(hg_domain *d, float *out, int64_t *step_out) {
    if (!d || (!out && d->n)) return HG_ERR_ARG;
    hg_ctx *ctx = d->ctx;
    CU(ctx, cudaSetDevice(ctx->device));
    int rc = ensure_scratch(ctx, (size_t)std::max<int64_t>(1, d->n) * 16);
    if (rc != HG_OK) return rc;
    rc = hg_read_macroscopic_device(d, (float *)ctx->scratch.p);
    if (rc != HG_OK) return rc;
    if (d->n) CU(ctx, cudaMemcpyAsync(out, ctx->scratch.p, (size_t)d->n * 16, cudaMemcpyDeviceToHost, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    if (step_out) *step_out = d->step;
    return HG_OK;
}

int hg_read_iolet_stats(hg_domain *d, double *out) {
    if (!d || (!out && d->nio)) return HG_ERR_ARG;
    hg_ctx *ctx = d->ctx;
    CU(ctx, cudaSetDevice(ctx->device));
    if (d->nio) CU(ctx, cudaMemcpyAsync(out, d->M.p, (size_t)d->nio * 24, cudaMemcpyDeviceToHost, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    return HG_OK;
}

int hg_read_iolet_forces(hg_domain *d, float *out) {
    if (!d || (!out && d->nio)) return HG_ERR_ARG;
    hg_ctx *ctx = d->ctx;
    CU(ctx, cudaSetDevice(ctx->device));
    std::vector<float4> f((size_t)std::max(1, d->nio));
    if (d->nio) CU(ctx, cudaMemcpyAsync(f.data(), d->force.p, (size_t)d->nio * 16, cudaMemcpyDeviceToHost, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < d->nio; ++k) {
        out[3 * k] = f[k].x;
        out[3 * k + 1] = f[k].y;
        out[3 * k + 2] = f[k].z;
    }
    return HG_OK;
}

int hg_read_boundary_values(hg_domain *d, float *out) {
    if (!d || (!out && d->nio)) return HG_ERR_ARG;
    hg_ctx *ctx = d->ctx;
    CU(ctx, cudaSetDevice(ctx->device));
    if (d->nio) CU(ctx, cudaMemcpyAsync(out, d->bcv.p, (size_t)d->nio * 4, cudaMemcpyDeviceToHost, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    return HG_OK;
}

// FP64 mass of the current state in canonical order, and its count of non-finite values.
static int mass_pass(hg_domain *d, double *mass, int64_t *nonfinite) {
    hg_ctx *ctx = d->ctx;
    CU(ctx, cudaSetDevice(ctx->device));
    const int64_t P = mass_partials_needed(d->n);
    int rc = ensure_scratch(ctx, (size_t)(P + 1) * sizeof(double2));
    if (rc != HG_OK) return rc;
    double2 *part = (double2 *)ctx->scratch.p;
    CU(ctx, launch_mass(ctx->storage, ctx->scheme, domdev_ptr(d), d->n, (const int32_t *)d->dev_of.p, part,
                        part + P, ctx->stream));
    double2 r;
    CU(ctx, cudaMemcpyAsync(&r, part + P, sizeof r, cudaMemcpyDeviceToHost, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    if (mass) *mass = r.x;
    if (nonfinite) *nonfinite = (int64_t)r.y;
    return HG_OK;
}

int hg_mass(hg_domain *d, double *out) {
    if (!d || !out) return HG_ERR_ARG;
    return mass_pass(d, out, nullptr);
}

int hg_state_check(hg_domain *d, double *mass, int64_t *nonfinite) {
    if (!d) return HG_ERR_ARG;
    double m = 0.0;
    int64_t bad = 0;
    const int rc = mass_pass(d, &m, &bad);
    if (rc != HG_OK) return rc;
    if (mass) *mass = m;
    if (nonfinite) *nonfinite = bad;
    if (bad) return fail(d->ctx, HG_ERR_STATE, "the state holds %lld non-finite values", (long long)bad);
    return HG_OK;
}

int hg_read_adjacent_moments(hg_domain *d, int64_t *sites_out, float *mom_out) {
    if (!d || (d->n_adj && (!sites_out || !mom_out))) return HG_ERR_ARG;
    hg_ctx *ctx = d->ctx;
    CU(ctx, cudaSetDevice(ctx->device));
    std::vector<float4> b((size_t)std::max<int64_t>(1, d->n_adj));
    if (d->n_adj)
        CU(ctx, cudaMemcpyAsync(b.data(), d->bnd.p, (size_t)d->n_adj * 16, cudaMemcpyDeviceToHost, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    int64_t j = 0;
    for (int64_t c = 0; c < d->n; ++c) {  // canonical order of the sites
        const int64_t q = d->dev_of_host.empty() ? c : d->dev_of_host[c];
        const int32_t sl = d->slot_of_dev[q];
        if (sl < 0) continue;
        sites_out[j] = c;
        mom_out[4 * j] = b[sl].x;
        mom_out[4 * j + 1] = b[sl].y;
        mom_out[4 * j + 2] = b[sl].z;
        mom_out[4 * j + 3] = b[sl].w;
        ++j;
    }
    return HG_OK;
}

int hg_ctx_inject_fault(hg_ctx *ctx, int32_t kind, int64_t arg) {
    if (!ctx) return HG_ERR_ARG;
    if (kind == HG_FAULT_ALLOC) {
        if (arg < 0) return fail(ctx, HG_ERR_ARG, "allocation index must be >= 0");
        ctx->fail_alloc_in = arg;
        return HG_OK;
    }
    if (kind == HG_FAULT_DEVICE_WAIT) {
        const int32_t code = arg ? (int32_t)arg : 1;
        CU(ctx, cudaSetDevice(ctx->device));
        CU(ctx, cudaMemcpyAsync(ctx->errw.p, &code, sizeof code, cudaMemcpyHostToDevice, ctx->stream));
        CU(ctx, cudaStreamSynchronize(ctx->stream));
        return HG_OK;
    }
    return fail(ctx, HG_ERR_ARG, "unknown fault kind %d", kind);
}

// checkpoint layout: header | bcv[nio] f32 | M[nio*3] f64 | F[19][n] storage |
// force[nio] float4 (body-force densities of the reverse coupling exchange)
struct StateHeader {
    char magic[8];
    int64_t n, step;
    int32_t nio, storage, scheme, version;
};

int hg_state_bytes(hg_domain *d, int64_t *bytes) {
    if (!d || !bytes) return HG_ERR_ARG;
    *bytes = (int64_t)sizeof(StateHeader) + (int64_t)d->nio * 4 + (int64_t)d->nio * 24 +
             19 * d->n * (int64_t)elem_bytes(d->ctx->storage) + (int64_t)d->nio * 16;
    return HG_OK;
}

int hg_read_state(hg_domain *d, void *host_out) {
    if (!d || (!host_out && d->n)) return HG_ERR_ARG;
    hg_ctx *ctx = d->ctx;
    CU(ctx, cudaSetDevice(ctx->device));
    const size_t fb = 19 * (size_t)d->n * elem_bytes(ctx->storage);
    int rc = ensure_scratch(ctx, std::max<size_t>(fb, 16));
    if (rc != HG_OK) return rc;
    CU(ctx, launch_export_state(ctx->storage, ctx->scheme, domdev_ptr(d), d->n, (const int32_t *)d->canon_of.p,
                                ctx->scratch.p, ctx->stream));
    if (fb) CU(ctx, cudaMemcpyAsync(host_out, ctx->scratch.p, fb, cudaMemcpyDeviceToHost, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    return HG_OK;
}

int hg_save_state(hg_domain *d, void *buf, int64_t bytes) {
    if (!d || !buf) return HG_ERR_ARG;
    hg_ctx *ctx = d->ctx;
    int64_t need = 0;
    hg_state_bytes(d, &need);
    if (bytes < need) return fail(ctx, HG_ERR_ARG, "buffer too small (%lld < %lld)", (long long)bytes, (long long)need);
    StateHeader h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, "HEMEGB1", 8);
    h.n = d->n;
    h.step = d->step;
    h.nio = d->nio;
    h.storage = ctx->storage;
    h.scheme = ctx->scheme;
    h.version = 2;
    char *p = (char *)buf;
    memcpy(p, &h, sizeof h);
    p += sizeof h;
    CU(ctx, cudaSetDevice(ctx->device));
    const size_t fb = 19 * (size_t)d->n * elem_bytes(ctx->storage);
    if (d->nio) {
        CU(ctx, cudaMemcpyAsync(p, d->bcv.p, (size_t)d->nio * 4, cudaMemcpyDeviceToHost, ctx->stream));
        p += (size_t)d->nio * 4;
        CU(ctx, cudaMemcpyAsync(p, d->M.p, (size_t)d->nio * 24, cudaMemcpyDeviceToHost, ctx->stream));
        p += (size_t)d->nio * 24;
        CU(ctx, cudaMemcpyAsync(p + fb, d->force.p, (size_t)d->nio * 16, cudaMemcpyDeviceToHost, ctx->stream));
    }
    return hg_read_state(d, p);  // synchronises the stream
}

int hg_load_state(hg_domain *d, const void *buf, int64_t bytes) {
    if (!d || !buf) return HG_ERR_ARG;
    hg_ctx *ctx = d->ctx;
    int64_t need = 0;
    hg_state_bytes(d, &need);
    if (bytes < need) return fail(ctx, HG_ERR_ARG, "buffer too small");
    StateHeader h;
    memcpy(&h, buf, sizeof h);
    if (memcmp(h.magic, "HEMEGB1", 8) != 0 || h.version != 2)
        return fail(ctx, HG_ERR_ARG, "not a hemegb state");
    if (h.n != d->n || h.nio != d->nio || h.storage != ctx->storage || h.scheme != ctx->scheme)
        return fail(ctx, HG_ERR_ARG, "state does not match this domain (sites, iolets, storage or scheme)");
    if (h.step < 0) return fail(ctx, HG_ERR_ARG, "negative step");
    const char *p = (const char *)buf + sizeof h;
    CU(ctx, cudaSetDevice(ctx->device));
    const size_t fb = 19 * (size_t)d->n * elem_bytes(ctx->storage);
    int rc = ensure_scratch(ctx, std::max<size_t>(fb, 16));
    if (rc != HG_OK) return rc;
    // every copy is ordered on the context's stream ahead of the import kernel
    if (d->nio) {
        CU(ctx, cudaMemcpyAsync(d->bcv.p, p, (size_t)d->nio * 4, cudaMemcpyHostToDevice, ctx->stream));
        p += (size_t)d->nio * 4;
        CU(ctx, cudaMemcpyAsync(d->M.p, p, (size_t)d->nio * 24, cudaMemcpyHostToDevice, ctx->stream));
        p += (size_t)d->nio * 24;
        CU(ctx, cudaMemcpyAsync(d->force.p, p + fb, (size_t)d->nio * 16, cudaMemcpyHostToDevice, ctx->stream));
    }
    const int64_t step = h.step;
    CU(ctx, cudaMemcpyAsync((int64_t *)ctx->steps.p + d->idx, &step, 8, cudaMemcpyHostToDevice, ctx->stream));
    d->step = h.step;
    if (fb) CU(ctx, cudaMemcpyAsync(ctx->scratch.p, p, fb, cudaMemcpyHostToDevice, ctx->stream));
    CU(ctx, launch_import_state(ctx->storage, ctx->scheme, domdev_ptr(d), d->n, (const int32_t *)d->canon_of.p,
                                ctx->scratch.p, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    return HG_OK;
}

}  // extern "C"

// ================================================================ split domains
// Section 2.2: the sparse domain is decomposed over ranks and every step ends with
// a non-blocking exchange of the populations that cross the cuts; Section 2.2.1:
// the cut balances the work.  Here the canonical (Morton) site list is cut into
// contiguous ranges of equal cost; each partition keeps ghost copies of the sites
// it pulls from, and after every stream-collide the crossing values are packed per
// (sender, receiver) pair, copied into the receiver's buffer and unpacked into its
// ghosts.  All partitions of one split live on the context's device (the copy of
// each block is a device-to-device copy).  Boundary slots are numbered globally in
// canonical order and the per-slot and per-iolet arrays are shared, so each
// iolet's FP64 reduction sees the same values in the same order as for the whole
// domain: a split run is bit-identical to the unsplit one.
namespace {

struct SplitLayout {
    std::vector<int64_t> first;                              // k + 1 cuts (canonical indices)
    std::vector<std::vector<int64_t>> ghosts;                // per partition, sorted
    std::vector<std::vector<std::pair<int32_t, int64_t>>> need;  // [q * k + p]: (direction i, site) p pulls from q
};

inline bool has_iolet_link(const I32Table &nbr, int64_t stride, int64_t s) {
    for (int i = 0; i < 18; ++i)
        if (nbr[(size_t)i * stride + s] < -1) return true;
    return false;
}

// Cuts with equal cost per partition (a site costs 1, a site with an iolet link
// `bw`), every partition non-empty; ghosts and the halo each partition needs.
void split_layout(const I32Table &nbr, int64_t stride, int64_t n, int k, double bw, SplitLayout &L) {
    std::vector<double> pre(n + 1, 0.0);
    for (int64_t s = 0; s < n; ++s) pre[s + 1] = pre[s] + (has_iolet_link(nbr, stride, s) ? bw : 1.0);
    L.first.assign(k + 1, 0);
    for (int p = 1; p < k; ++p) {
        int64_t c = std::lower_bound(pre.begin(), pre.end(), pre[n] * p / k) - pre.begin();
        c = std::max<int64_t>(c, L.first[p - 1] + 1);
        L.first[p] = std::min<int64_t>(c, n - (k - p));
    }
    L.first[k] = n;
    L.ghosts.assign(k, {});
    L.need.assign((size_t)k * k, {});
    for (int p = 0; p < k; ++p) {
        const int64_t a = L.first[p], b = L.first[p + 1];
        std::vector<std::pair<int32_t, int64_t>> pulls;
        for (int i = 0; i < 18; ++i)
            for (int64_t s = a; s < b; ++s) {
                const int32_t v = nbr[(size_t)i * stride + s];
                if (v >= 0 && (v < a || v >= b)) pulls.push_back({i, v});
            }
        std::vector<int64_t> &g = L.ghosts[p];
        for (const auto &e : pulls) g.push_back(e.second);
        std::sort(g.begin(), g.end());
        g.erase(std::unique(g.begin(), g.end()), g.end());
        // (direction, site) pairs are distinct: site v + c_i is the only puller of (i, v)
        for (const auto &e : pulls) {
            const int q = (int)(std::upper_bound(L.first.begin(), L.first.end(), e.second) - L.first.begin()) - 1;
            L.need[(size_t)q * k + p].push_back(e);
        }
    }
}

void free_split(hg_ctx *ctx, hg_split *sp) {
    for (SplitPart &P : sp->parts)
        for (DevBuf *b : {&P.f[0], &P.f[1], &P.nbr, &P.iomask, &P.ioprefix, &P.gidx, &P.lword, &P.run0, &P.rdelta})
            dev_free(ctx, *b);
    for (DevBuf *b : {&sp->bnd, &sp->io_codes, &sp->coef, &sp->slot_site, &sp->bcv, &sp->io_kind, &sp->M,
                      &sp->slots, &sp->force})
        dev_free(ctx, *b);
    std::lock_guard<std::mutex> lk(ctx->mu);
    for (SplitPart &P : sp->parts)
        if (P.idx >= 0) ctx->reserved[P.idx] = 0;
}

int split_plan(hg_split *sp, Plan *&out) {
    hg_ctx *ctx = sp->ctx;
    PlanKey key;
    for (const SplitPart &P : sp->parts) key.doms.push_back(P.idx);
    auto it = ctx->plans.find(key);
    if (it != ctx->plans.end()) {
        out = it->second.get();
        return HG_OK;
    }
    std::unique_ptr<Plan> p(new Plan);
    p->doms = key.doms;
    const int64_t ts = (int64_t)ctx->block * ctx->spt;
    std::vector<TileDev> tiles;
    for (const SplitPart &P : sp->parts) {
        p->tiles_runs = p->tiles_runs && P.n_runs > 0;
        for (int64_t s = 0; s < P.n_own; s += ts) tiles.push_back(TileDev{P.idx, (int32_t)std::min(ts, P.n_own - s), s});
    }
    std::vector<IoDev> ios;
    std::vector<int2> chunks;
    for (int k = 0; k < sp->nio; ++k) {
        IoDev I;
        memset(&I, 0, sizeof I);
        const hg_iolet &io = sp->io[k];
        I.slots = (const int32_t *)sp->slots.p + sp->io_ptr[k];
        I.n_slots = sp->io_ptr[k + 1] - sp->io_ptr[k];
        I.bnd = (const float4 *)sp->bnd.p;
        I.M = (double *)sp->M.p + 3 * k;
        I.bcv = (float *)sp->bcv.p + k;
        I.step = (const int64_t *)ctx->steps.p + sp->parts[0].idx;
        const double an = std::sqrt((double)io.axis[0] * io.axis[0] + (double)io.axis[1] * io.axis[1] +
                                    (double)io.axis[2] * io.axis[2]);
        I.nx = io.axis[0] / an;
        I.ny = io.axis[1] / an;
        I.nz = io.axis[2] / an;
        I.value = io.value;
        I.period = io.period;
        I.pulse = io.pulse;
        I.n_chunks = std::max(1, (I.n_slots + kIoChunk - 1) / kIoChunk);
        I.part0 = (int32_t)chunks.size();
        for (int c = 0; c < I.n_chunks; ++c) chunks.push_back(make_int2((int)ios.size(), c));
        I.force = (float4 *)sp->force.p + k;
        ios.push_back(I);
    }
    p->n_tiles = (int64_t)tiles.size();
    p->n_ios = (int)ios.size();
    p->n_chunks = (int)chunks.size();
    if (sp->parts.size() <= 64) {  // one single-domain launch per partition, no tile table
        for (const SplitPart &P : sp->parts) {
            p->sep.push_back(P.dev);
            p->sep_n.push_back(P.n_own);
        }
        p->n_tiles = 0;
    }
    p->n_halo = (int64_t)sp->pack.size();
    p->halo_elem = (int)elem_bytes(ctx->storage);
    p->halo_staged = sp->staged;
    if (p->halo_staged)
        for (const auto &b : sp->blocks)
            p->halo_blocks.push_back({b.first * p->halo_elem, b.second * p->halo_elem});
    int rc = HG_OK;
    auto A = [&](DevBuf &b, size_t bytes) {
        if (rc == HG_OK) rc = dev_alloc(ctx, b, bytes);
    };
    A(p->tiles, std::max<size_t>(1, tiles.size()) * sizeof(TileDev));
    A(p->ios, std::max<size_t>(1, ios.size()) * sizeof(IoDev));
    A(p->adv, std::max<size_t>(1, key.doms.size()) * 4);
    A(p->chunks, std::max<size_t>(1, chunks.size()) * sizeof(int2));
    A(p->partials, std::max<size_t>(1, chunks.size()) * sizeof(double2));
    A(p->counters, (ios.size() + 1) * sizeof(unsigned));
    A(p->rev, sizeof(RevSrc));
    A(p->fslots, sizeof(int2));
    const size_t n_staged = p->halo_staged ? sp->pack.size() : 0, n_moves = p->halo_staged ? 0 : sp->pack.size();
    A(p->halo_pack, std::max<size_t>(1, n_staged) * sizeof(HaloDev));
    A(p->halo_unpack, std::max<size_t>(1, n_staged) * sizeof(HaloDev));
    A(p->send, std::max<size_t>(1, n_staged) * p->halo_elem);
    A(p->recv, std::max<size_t>(1, n_staged) * p->halo_elem);
    A(p->halo_moves, std::max<size_t>(1, n_moves) * sizeof(HaloMove));
    auto release = [&] {
        for (DevBuf *b : {&p->tiles, &p->ios, &p->adv, &p->chunks, &p->partials, &p->counters, &p->rev,
                          &p->fslots, &p->halo_pack, &p->halo_unpack, &p->send, &p->recv, &p->halo_moves})
            dev_free(ctx, *b);
    };
    if (rc != HG_OK) {
        release();
        return rc;
    }
    cudaStream_t st = ctx->stream;
    cudaError_t e = cudaMemsetAsync(p->counters.p, 0, p->counters.bytes, st);
    auto H2D = [&](DevBuf &b, const void *src, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, st);
    };
    H2D(p->tiles, tiles.data(), tiles.size() * sizeof(TileDev));
    H2D(p->ios, ios.data(), ios.size() * sizeof(IoDev));
    H2D(p->adv, key.doms.data(), key.doms.size() * 4);
    H2D(p->chunks, chunks.data(), chunks.size() * sizeof(int2));
    std::vector<HaloMove> moves(n_moves);
    for (size_t j = 0; j < n_moves; ++j)
        moves[j] = HaloMove{sp->pack[j].dom, sp->unpack[j].dom, (uint32_t)sp->pack[j].off, (uint32_t)sp->unpack[j].off};
    H2D(p->halo_pack, sp->pack.data(), n_staged * sizeof(HaloDev));
    H2D(p->halo_unpack, sp->unpack.data(), n_staged * sizeof(HaloDev));
    H2D(p->halo_moves, moves.data(), n_moves * sizeof(HaloMove));
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host tables above are temporaries
    if (e != cudaSuccess) {
        cudaStreamSynchronize(st);
        release();
        return fail(ctx, HG_ERR_CUDA, "split plan upload failed: %s", cudaGetErrorString(e));
    }
    out = p.get();
    ctx->plans[key] = std::move(p);
    return HG_OK;
}

const DomDev *part_dev(hg_split *sp, int p) { return (const DomDev *)sp->ctx->dom_table.p + sp->parts[p].idx; }

}  // namespace

extern "C" {

int hg_split_layout(const int32_t *xyz, int64_t n, const hg_iolet *iolets, int32_t nio, const hg_split_params *sp,
                    int64_t *first_out, int64_t *ghosts_out, int64_t *halo_out) {
    if (!sp || n < 1 || !xyz || (nio > 0 && !iolets) || nio < 0 || nio > kMaxIolets) return HG_ERR_ARG;
    const int k = sp->n_parts;
    if (k < 1 || k > 1024 || k > n) return HG_ERR_ARG;
    for (int q = 0; q < nio; ++q)
        if (!iolet_ok(iolets[q])) return HG_ERR_ARG;
    std::vector<int32_t> xs;
    I32Table nbr;
    std::string why;
    if (build_canonical(xyz, n, iolets, nio, n, xs, nbr, why) != HG_OK) return fail(nullptr, HG_ERR_ARG, "%s", why.c_str());
    SplitLayout L;
    split_layout(nbr, n, n, k, sp->boundary_weight > 0 ? sp->boundary_weight : 1.0, L);
    for (int p = 0; p <= k; ++p)
        if (first_out) first_out[p] = L.first[p];
    for (int p = 0; p < k; ++p) {
        if (ghosts_out) ghosts_out[p] = (int64_t)L.ghosts[p].size();
        for (int q = 0; q < k; ++q)
            if (halo_out) halo_out[(size_t)q * k + p] = (int64_t)L.need[(size_t)q * k + p].size();
    }
    return HG_OK;
}

int hg_split_create(hg_ctx *ctx, const int32_t *xyz, int64_t n, const hg_iolet *iolets, int32_t nio,
                    const hg_lb_params *lb, const hg_split_params *spar, hg_split **out) {
    if (!ctx) return HG_ERR_ARG;
    if (!out || !spar) return fail(ctx, HG_ERR_ARG, "out or params is NULL");
    *out = nullptr;
    if (ctx->scheme != HG_SCHEME_AB) return fail(ctx, HG_ERR_ARG, "split domains use the A/B scheme");
    if (n < 1 || !xyz || n > ((int64_t)200 << 20)) return fail(ctx, HG_ERR_ARG, "bad site array");
    const int k = spar->n_parts;
    if (k < 1 || k > 1024 || k > n) return fail(ctx, HG_ERR_ARG, "n_parts must be in [1, min(n, 1024)]");
    if (nio < 0 || nio > kMaxIolets || (nio > 0 && !iolets)) return fail(ctx, HG_ERR_ARG, "bad iolet array");
    const double tau = lb ? lb->tau : 0.8;
    if (!(tau > 0.5)) return fail(ctx, HG_ERR_ARG, "tau must exceed 1/2");
    const int32_t ordering = lb ? lb->ordering : HG_ORDER_MORTON;
    if (ordering < HG_ORDER_MORTON || ordering > HG_ORDER_BRICKS)
        return fail(ctx, HG_ERR_ARG, "unknown ordering %d", ordering);
    if (spar->exchange != HG_EXCHANGE_DIRECT && spar->exchange != HG_EXCHANGE_STAGED)
        return fail(ctx, HG_ERR_ARG, "unknown halo exchange %d", spar->exchange);
    for (int q = 0; q < nio; ++q)
        if (!iolet_ok(iolets[q])) return fail(ctx, HG_ERR_ARG, "iolet %d out of range", q);
    CU(ctx, cudaSetDevice(ctx->device));
    std::unique_ptr<hg_split> sp(new hg_split);
    sp->ctx = ctx;
    sp->n = n;
    sp->nio = nio;
    sp->tau = tau;
    sp->staged = spar->exchange == HG_EXCHANGE_STAGED;
    sp->io.assign(iolets, iolets + nio);
    std::vector<int32_t> xs;
    I32Table nbr;
    {
        std::string why;
        if (build_canonical(xyz, n, iolets, nio, n, xs, nbr, why) != HG_OK)
            return fail(ctx, HG_ERR_ARG, "%s", why.c_str());
    }
    SplitLayout L;
    split_layout(nbr, n, n, k, spar->boundary_weight > 0 ? spar->boundary_weight : 1.0, L);
    // reserve one context slot (descriptor + step counter) per partition
    sp->parts.resize(k);
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        int got = 0;
        for (int i = 0; i < ctx->capacity && got < k; ++i)
            if (!ctx->doms[i] && !ctx->reserved[i]) {
                ctx->reserved[i] = 1;
                sp->parts[got++].idx = i;
            }
        if (got < k) {
            for (int j = 0; j < got; ++j) ctx->reserved[sp->parts[j].idx] = 0;
            return fail(ctx, HG_ERR_STATE, "context holds too many domains");
        }
    }
    // Device order of each partition's owned sites: canonical (Morton) or, like a
    // whole domain, rows or bricks of the partition's own sites.  perm[p][q] = offset
    // (from the partition's first canonical site) of the site at device position q;
    // inv[p] is the inverse.  Empty: identity.
    std::vector<std::vector<int32_t>> perm(k), inv(k);
    if (ordering != HG_ORDER_MORTON)
        for (int p = 0; p < k; ++p) {
            const int64_t a = L.first[p], m = L.first[p + 1] - a;
            std::vector<int32_t> sub(xs.begin() + 3 * a, xs.begin() + 3 * (a + m));
            std::string why;
            if (device_order(sub, m, ordering, perm[p], why) != HG_OK) {
                free_split(ctx, sp.get());
                return fail(ctx, HG_ERR_ARG, "%s", why.c_str());
            }
            inv[p].resize(m);
            for (int64_t q = 0; q < m; ++q) inv[p][perm[p][q]] = (int32_t)q;
        }
    auto canon_at = [&](int p, int64_t q) -> int64_t { return L.first[p] + (perm[p].empty() ? q : perm[p][q]); };
    auto dev_pos = [&](int p, int64_t c) -> int64_t {
        const int64_t o = c - L.first[p];
        return inv[p].empty() ? o : inv[p][o];
    };
    // Global boundary slots: partition by partition, in each partition's device order
    // (so a partition's slots are one consecutive run its iomask/ioprefix address);
    // the per-iolet slot lists below stay in canonical site order, which keeps the
    // iolet reductions' summation order, and so their bits, independent of the
    // partitioning and the ordering.
    std::vector<int32_t> slot_of(n, -1);
    std::vector<int64_t> per_io(nio + 1, 0);
    int64_t n_adj = 0;
    auto distinct = [&](int64_t c, int seen[18]) {
        int ns = 0;
        for (int i = 0; i < 18; ++i) {
            const int32_t v = nbr[(size_t)i * n + c];
            if (v >= -1) continue;
            bool dup = false;
            for (int t = 0; t < ns; ++t) dup = dup || seen[t] == -v - 2;
            if (!dup) seen[ns++] = -v - 2;
        }
        return ns;
    };
    for (int p = 0; p < k; ++p)
        for (int64_t q = 0; q < L.first[p + 1] - L.first[p]; ++q) {
            const int64_t c = canon_at(p, q);
            int seen[18];
            const int ns = distinct(c, seen);
            for (int t = 0; t < ns; ++t) per_io[seen[t] + 1]++;
            if (ns) slot_of[c] = (int32_t)n_adj++;
        }
    sp->n_adj = n_adj;
    for (int q = 0; q < nio; ++q) per_io[q + 1] += per_io[q];
    sp->io_ptr.assign(per_io.begin(), per_io.end());
    std::vector<int32_t> slots(std::max<int64_t>(1, per_io[nio]));
    std::vector<int32_t> codes((size_t)std::max<int64_t>(1, n_adj) * 18, -1);
    std::vector<float> coef((size_t)std::max<int64_t>(1, n_adj) * 18, 0.0f);
    std::vector<int32_t> slot_site((size_t)std::max<int64_t>(1, n_adj), 0);
    {
        std::vector<int64_t> fill(per_io.begin(), per_io.end() - 1);
        for (int p = 0; p < k; ++p)
            for (int64_t c = L.first[p]; c < L.first[p + 1]; ++c) {
                const int32_t sl = slot_of[c];
                if (sl < 0) continue;
                int seen[18];
                const int ns = distinct(c, seen);
                for (int t = 0; t < ns; ++t) slots[fill[seen[t]]++] = sl;
                slot_site[sl] = (int32_t)dev_pos(p, c);
                for (int i = 1; i < 19; ++i) {
                    const int32_t v = nbr[(size_t)(i - 1) * n + c];
                    codes[(size_t)sl * 18 + (i - 1)] = v;
                    if (v < -1) coef[(size_t)sl * 18 + (i - 1)] = link_coef(iolets[-v - 2], &xs[3 * c], i, ctx->storage);
                }
            }
    }
    const size_t eb = elem_bytes(ctx->storage);
    int rc = HG_OK;
    auto A = [&](DevBuf &b, size_t bytes) {
        if (rc == HG_OK) rc = dev_alloc(ctx, b, bytes);
    };
    A(sp->bnd, (size_t)std::max<int64_t>(1, n_adj) * 16);
    A(sp->io_codes, codes.size() * 4);
    A(sp->coef, coef.size() * 4);
    A(sp->slot_site, slot_site.size() * 4);
    A(sp->bcv, (size_t)std::max(1, nio) * 4);
    A(sp->io_kind, (size_t)std::max(1, nio));
    A(sp->M, (size_t)std::max(1, nio) * 24);
    A(sp->slots, slots.size() * 4);
    A(sp->force, (size_t)std::max(1, nio) * 16);
    // per partition: local tables (owned sites first, then ghosts)
    std::vector<std::vector<int32_t>> tab(k), mask(k), pref(k), gidx(k), r0(k), rd(k);
    std::vector<U32Table> lw(k);
    for (int p = 0; p < k && rc == HG_OK; ++p) {
        SplitPart &P = sp->parts[p];
        P.first = L.first[p];
        P.n_own = L.first[p + 1] - L.first[p];
        P.ghosts = L.ghosts[p];
        P.n_loc = P.n_own + (int64_t)P.ghosts.size();
        P.np = std::max<int64_t>(128, (P.n_loc + 127) / 128 * 128);
        const int64_t a = P.first, b = L.first[p + 1], np = P.np;
        auto local = [&](int64_t v) -> int64_t {
            if (v >= a && v < b) return dev_pos(p, v);
            return P.n_own + (std::lower_bound(P.ghosts.begin(), P.ghosts.end(), v) - P.ghosts.begin());
        };
        std::vector<int32_t> &T = tab[p];
        T.assign((size_t)18 * np, 0);
        for (int i = 1; i < 19; ++i) {
            const int opp = (i & 1) ? i + 1 : i - 1;
            for (int64_t q = 0; q < np; ++q) {
                const int32_t v = q < P.n_own ? nbr[(size_t)(i - 1) * n + canon_at(p, q)] : -1;
                T[(size_t)(i - 1) * np + q] = v >= 0 ? (int32_t)local(v) : (int32_t)(q + (int64_t)(opp - i) * np);
            }
        }
        mask[p].assign((size_t)np / 32, 0u);
        pref[p].assign((size_t)np / 32, 0);
        int32_t acc = 0, base = -1;
        for (int64_t q = 0; q < P.n_own; ++q) {
            const int32_t sl = slot_of[canon_at(p, q)];
            if (sl < 0) continue;
            mask[p][q >> 5] |= 1u << (q & 31);
            if (base < 0) base = sl;
        }
        base = std::max(base, 0);
        for (size_t w = 0; w < mask[p].size(); ++w) {
            pref[p][w] = base + acc;
            acc += __builtin_popcount(mask[p][w]);
        }
        gidx[p].resize(P.n_loc);
        for (int64_t q = 0; q < P.n_own; ++q) gidx[p][q] = (int32_t)canon_at(p, q);
        for (size_t g = 0; g < P.ghosts.size(); ++g) gidx[p][P.n_own + g] = (int32_t)P.ghosts[g];
        A(P.f[0], 19 * (size_t)np * eb);
        A(P.f[1], 19 * (size_t)np * eb);
        A(P.nbr, T.size() * 4);
        A(P.iomask, mask[p].size() * 4);
        A(P.ioprefix, pref[p].size() * 4);
        A(P.gidx, gidx[p].size() * 4);
        // owned sites only (ghost rows are never read); entries may point at ghosts
        if (build_runs(T.data(), P.n_own, P.n_loc, np, 1, lw[p], r0[p], rd[p])) {
            P.n_runs = (int64_t)rd[p].size() / kRunStride;
            A(P.lword, lw[p].size() * 4);
            A(P.run0, r0[p].size() * 4);
            A(P.rdelta, rd[p].size() * 4);
        }
    }
    if (rc != HG_OK) {
        free_split(ctx, sp.get());
        return rc;
    }
    // halo blocks, one per (sender, receiver) pair
    for (int q = 0; q < k; ++q)
        for (int p = 0; p < k; ++p) {
            const auto &need = L.need[(size_t)q * k + p];
            if (need.empty()) continue;
            const size_t off = sp->pack.size();
            const SplitPart &Q = sp->parts[q], &P = sp->parts[p];
            for (const auto &e : need) {
                const int64_t g = P.n_own + (std::lower_bound(P.ghosts.begin(), P.ghosts.end(), e.second) -
                                             P.ghosts.begin());
                sp->pack.push_back(HaloDev{Q.idx, 0, (int64_t)(e.first + 1) * Q.np + dev_pos(q, e.second)});
                sp->unpack.push_back(HaloDev{P.idx, 0, (int64_t)(e.first + 1) * P.np + g});
            }
            sp->blocks.push_back({off, need.size()});
        }
    std::vector<float> bcv(std::max(1, nio), 0.0f);
    std::vector<int8_t> kinds(std::max(1, nio), 0);
    for (int q = 0; q < nio; ++q) {
        bcv[q] = (float)(iolets[q].value * pulse(iolets[q].pulse, 1.0, iolets[q].period));
        kinds[q] = (int8_t)iolets[q].kind;
    }
    cudaStream_t st = ctx->stream;
    cudaError_t e = cudaSuccess;
    auto H2D = [&](DevBuf &b, const void *src, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, st);
    };
    H2D(sp->io_codes, codes.data(), codes.size() * 4);
    H2D(sp->coef, coef.data(), coef.size() * 4);
    H2D(sp->slot_site, slot_site.data(), slot_site.size() * 4);
    H2D(sp->bcv, bcv.data(), bcv.size() * 4);
    H2D(sp->io_kind, kinds.data(), kinds.size());
    H2D(sp->slots, slots.data(), slots.size() * 4);
    for (DevBuf *b : {&sp->bnd, &sp->M, &sp->force})
        if (e == cudaSuccess) e = cudaMemsetAsync(b->p, 0, b->bytes, st);
    for (int p = 0; p < k; ++p) {
        SplitPart &P = sp->parts[p];
        H2D(P.nbr, tab[p].data(), tab[p].size() * 4);
        H2D(P.iomask, mask[p].data(), mask[p].size() * 4);
        H2D(P.ioprefix, pref[p].data(), pref[p].size() * 4);
        H2D(P.gidx, gidx[p].data(), gidx[p].size() * 4);
        if (P.n_runs) {
            H2D(P.lword, lw[p].data(), lw[p].size() * 4);
            H2D(P.run0, r0[p].data(), r0[p].size() * 4);
            H2D(P.rdelta, rd[p].data(), rd[p].size() * 4);
        }
        for (DevBuf *b : {&P.f[0], &P.f[1]})
            if (e == cudaSuccess) e = cudaMemsetAsync(b->p, 0, b->bytes, st);
        if (e == cudaSuccess) e = cudaMemsetAsync((int64_t *)ctx->steps.p + P.idx, 0, sizeof(int64_t), st);
        DomDev &D = P.dev;
        memset(&D, 0, sizeof D);
        D.f[0] = P.f[0].p;
        D.f[1] = P.f[1].p;
        D.nbr = (const int32_t *)P.nbr.p;
        D.lword = (const uint32_t *)P.lword.p;
        D.run0 = (const int32_t *)P.run0.p;
        D.rdelta = (const int32_t *)P.rdelta.p;
        D.iomask = (const uint32_t *)P.iomask.p;
        D.ioprefix = (const int32_t *)P.ioprefix.p;
        D.io_codes = (const int32_t *)sp->io_codes.p;
        D.bnd = (float4 *)sp->bnd.p;
        D.coef = (const float *)sp->coef.p;
        D.bcv = (const float *)sp->bcv.p;
        D.io_kind = (const int8_t *)sp->io_kind.p;
        D.step = (const int64_t *)ctx->steps.p + P.idx;
        D.err = (int32_t *)ctx->errw.p;
        D.n = P.n_loc;
        D.np = P.np;
        D.omega = (float)(1.0 / tau);
        D.n_io = nio;
        D.slot_site = (const int32_t *)sp->slot_site.p;
        D.io_force = nullptr;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync((DomDev *)ctx->dom_table.p + P.idx, &D, sizeof D, cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // host tables are released below
    if (e != cudaSuccess) {
        cudaStreamSynchronize(st);
        free_split(ctx, sp.get());
        return fail(ctx, HG_ERR_CUDA, "split upload failed: %s", cudaGetErrorString(e));
    }
    ctx->splits.push_back(sp.get());
    *out = sp.release();
    return HG_OK;
}

int hg_split_destroy(hg_split *sp) {
    if (!sp) return HG_ERR_ARG;
    hg_ctx *ctx = sp->ctx;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    drop_plans(ctx);
    free_split(ctx, sp);
    ctx->splits.erase(std::remove(ctx->splits.begin(), ctx->splits.end(), sp), ctx->splits.end());
    delete sp;
    return HG_OK;
}

int hg_split_info(hg_split *sp, int32_t part, int64_t *first, int64_t *owned, int64_t *ghosts, int64_t *halo_in) {
    if (!sp || part < 0 || part >= (int32_t)sp->parts.size()) return HG_ERR_ARG;
    const SplitPart &P = sp->parts[part];
    if (first) *first = P.first;
    if (owned) *owned = P.n_own;
    if (ghosts) *ghosts = (int64_t)P.ghosts.size();
    if (halo_in) {
        int64_t h = 0;
        for (const HaloDev &u : sp->unpack) h += u.dom == P.idx;
        *halo_in = h;
    }
    return HG_OK;
}

int hg_split_step(hg_split *sp, int64_t n) {
    if (!sp) return HG_ERR_ARG;
    hg_ctx *ctx = sp->ctx;
    if (n < 0) return fail(ctx, HG_ERR_ARG, "negative step count");
    if (n == 0) return HG_OK;
    CU(ctx, cudaSetDevice(ctx->device));
    Plan *p = nullptr;
    int rc = split_plan(sp, p);
    if (rc == HG_OK) rc = run_plan(ctx, p, n, 2);
    if (rc != HG_OK) return rc;
    sp->step += n;
    return HG_OK;
}

int hg_split_read_macroscopic(hg_split *sp, float *out) {
    if (!sp || !out) return HG_ERR_ARG;
    hg_ctx *ctx = sp->ctx;
    CU(ctx, cudaSetDevice(ctx->device));
    int rc = ensure_scratch(ctx, (size_t)sp->n * 16);
    if (rc != HG_OK) return rc;
    for (size_t p = 0; p < sp->parts.size(); ++p)
        CU(ctx, launch_macroscopic(ctx->storage, ctx->scheme, part_dev(sp, (int)p), sp->parts[p].n_own,
                                   (const int32_t *)sp->parts[p].gidx.p, (float4 *)ctx->scratch.p, ctx->stream));
    CU(ctx, cudaMemcpyAsync(out, ctx->scratch.p, (size_t)sp->n * 16, cudaMemcpyDeviceToHost, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    return HG_OK;
}

// F_t of every partition's owned sites, canonical order, into the context scratch.
static int split_export(hg_split *sp, size_t extra) {
    hg_ctx *ctx = sp->ctx;
    const size_t fb = 19 * (size_t)sp->n * elem_bytes(ctx->storage);
    int rc = ensure_scratch(ctx, ((fb + 255) & ~(size_t)255) + extra);
    if (rc != HG_OK) return rc;
    for (size_t p = 0; p < sp->parts.size(); ++p)
        CU(ctx, launch_export_state(ctx->storage, ctx->scheme, part_dev(sp, (int)p), sp->parts[p].n_own,
                                    (const int32_t *)sp->parts[p].gidx.p, ctx->scratch.p, ctx->stream, sp->n));
    return HG_OK;
}

int hg_split_read_state(hg_split *sp, void *out) {
    if (!sp || !out) return HG_ERR_ARG;
    hg_ctx *ctx = sp->ctx;
    CU(ctx, cudaSetDevice(ctx->device));
    int rc = split_export(sp, 0);
    if (rc != HG_OK) return rc;
    CU(ctx, cudaMemcpyAsync(out, ctx->scratch.p, 19 * (size_t)sp->n * elem_bytes(ctx->storage),
                            cudaMemcpyDeviceToHost, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    return HG_OK;
}

int hg_split_mass(hg_split *sp, double *out) {
    if (!sp || !out) return HG_ERR_ARG;
    hg_ctx *ctx = sp->ctx;
    CU(ctx, cudaSetDevice(ctx->device));
    const int64_t P = mass_partials_needed(sp->n);
    int rc = split_export(sp, (size_t)(P + 1) * sizeof(double2));
    if (rc != HG_OK) return rc;
    const size_t fb = (19 * (size_t)sp->n * elem_bytes(ctx->storage) + 255) & ~(size_t)255;
    double2 *part = (double2 *)((char *)ctx->scratch.p + fb);
    CU(ctx, launch_mass_flat(ctx->storage, ctx->scratch.p, sp->n, sp->n, part, part + P, ctx->stream));
    double2 r;
    CU(ctx, cudaMemcpyAsync(&r, part + P, sizeof r, cudaMemcpyDeviceToHost, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    *out = r.x;
    return HG_OK;
}

int hg_split_read_iolet_stats(hg_split *sp, double *out) {
    if (!sp || (!out && sp->nio)) return HG_ERR_ARG;
    hg_ctx *ctx = sp->ctx;
    CU(ctx, cudaSetDevice(ctx->device));
    if (sp->nio) CU(ctx, cudaMemcpyAsync(out, sp->M.p, (size_t)sp->nio * 24, cudaMemcpyDeviceToHost, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    return HG_OK;
}

int hg_split_read_boundary_values(hg_split *sp, float *out) {
    if (!sp || (!out && sp->nio)) return HG_ERR_ARG;
    hg_ctx *ctx = sp->ctx;
    CU(ctx, cudaSetDevice(ctx->device));
    if (sp->nio) CU(ctx, cudaMemcpyAsync(out, sp->bcv.p, (size_t)sp->nio * 4, cudaMemcpyDeviceToHost, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    return HG_OK;
}

}  // extern "C"
