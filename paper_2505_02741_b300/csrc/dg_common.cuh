// dg_common.cuh -- device types and helpers shared by the dyGRASS CUDA kernels.
//
// Slack-slot CSR (generalises the dynamic CSR of Section III-F, Fig. 4):
//   per vertex x:  off[x]  first entry of x's adjacency list in the pool
//                  deg[x]  number of neighbours
//                  cap[x]  slots reserved at off[x] (deg <= cap)
//   pool:          32-byte entries, each list sorted by ascending neighbour id.
// Each entry caches the neighbour's (off, deg) and the position of x inside the
// neighbour's list, so one walk step is one dependent 32-byte load: the entry
// just read names the next list and where the previous vertex sits in it,
// which is all the non-backtracking pick (Section III-B) needs.
#pragma once
#include <cooperative_groups.h>
#include <cooperative_groups/reduce.h>
#include <cooperative_groups/scan.h>
#include <cstdint>
#include <cuda_runtime.h>

namespace dg {

struct __align__(32) Ent {
    uint32_t nbr;   // neighbour id
    uint32_t noff;  // off[nbr] (cached), or HUBREF when nbr is a hub
    uint32_t ndeg;  // deg[nbr] (cached); 0 only in an entry not yet refreshed
    uint32_t rev;   // position of this list's owner inside nbr's list (for HUBREF: its position
                    // when the entry was last written, a hint that may have drifted since)
    double r;       // resistance 1 / w (Section II-A, computed once, IEEE RN)
    double w;       // weight
};
static_assert(sizeof(Ent) == 32, "entry must be one 32-byte sector");

// Hubs (high-degree vertices, power-law graphs): entries pointing at a hub do
// not cache its list, so a hub's list can change without rewriting the back-
// entries held by its (many) neighbours.  A walker arriving at a hub reads
// off/deg from the vertex arrays and skips the previous vertex by id.
// Hysteresis keeps a vertex near the threshold from flipping every batch.
// Meshes never reach the threshold; on a power-law graph a low one keeps the
// per-batch refresh of cached fields small (R-MAT scale 22, 50k-update
// batches: 4.3 ms per batch at 1024, 2.2 ms at 32) for a slightly slower walk.
constexpr uint32_t HUBREF = 0xFFFFFFFFu;
constexpr uint32_t HUB_HI = 32;  // becomes a hub at this degree
constexpr uint32_t HUB_LO = 24;  // stays a hub down to this degree

__host__ __device__ inline bool hub_next(bool was_hub, uint32_t deg) {
    return deg >= HUB_HI || (was_hub && deg >= HUB_LO);
}

// device view of one slack-slot CSR
struct CSRView {
    uint32_t* off;
    uint32_t* deg;
    uint32_t* cap;
    uint8_t* hub;             // 1 = entries pointing here hold HUBREF
    uint32_t* nhub;           // number of hubs (device word)
    uint32_t* twin;           // a hub's second region of cap entries (the next list execution
                              // writes the list there and keeps this one), or 0xFFFFFFFF
    Ent* pool;
    unsigned long long* top;  // entries in use (bump pointer)
    unsigned long long* minr; // a lower bound of every entry's resistance (FP64 bits; positive
                              // doubles order like their bits): the minimum at build, lowered by
                              // every insertion or weight change, never raised
    uint64_t pool_cap;        // entries allocated
    int32_t n;
};

// Warp-aggregated atomics for counters many threads bump at once: the threads
// that arrive together combine their amounts and one of them issues a single
// atomic (one L2 operation per warp instead of one per thread).  agg_add
// returns each caller's own starting offset, as atomicAdd would.
__device__ __forceinline__ uint32_t agg_add(uint32_t* ctr, uint32_t v) {
    namespace cg = cooperative_groups;
    cg::coalesced_group g = cg::coalesced_threads();
    const uint32_t incl = cg::inclusive_scan(g, v);
    uint32_t base = 0;
    if (g.thread_rank() == g.size() - 1) base = atomicAdd(ctr, incl);
    base = g.shfl(base, g.size() - 1);
    return base + incl - v;
}
__device__ __forceinline__ void agg_count(unsigned long long* ctr, unsigned long long v) {
    namespace cg = cooperative_groups;
    cg::coalesced_group g = cg::coalesced_threads();
    const unsigned long long s = cg::reduce(g, v, cg::plus<unsigned long long>());
    if (g.thread_rank() == 0 && s) atomicAdd(ctr, s);
}

// change kinds applied to a CSR
enum : uint8_t { CHG_INS = 0, CHG_DEL = 1, CHG_SETW = 2 };

// per-update status codes (mirror of the C ABI)
enum : int32_t {
    ST_OK = 0, ST_SELF_LOOP = 1, ST_BAD_VERTEX = 2, ST_DUP_INSERT = 3,
    ST_MISSING_DELETE = 4, ST_BAD_WEIGHT = 5, ST_BAD_OP = 6
};
enum : uint8_t { WALK_NONE = 0, WALK_INS = 1, WALK_DEL = 2 };

// abort / error bits raised on the device and read back by the host
enum : uint32_t {
    ERR_POOL_G = 1u << 0,       // G pool short before any write (batch retried after growth)
    ERR_POOL_H = 1u << 1,       // H pool short at commit (commit retried after growth)
    ERR_BAD_INPUT = 1u << 2,    // load/init input invalid
    ERR_DUP_EDGE = 1u << 3,     // load input has a repeated edge
    ERR_NOT_IN_G = 1u << 4,     // init-sparsifier edge missing from G
    ERR_CAP_PRE = 1u << 5,      // staging space short before the walks (batch retried)
    ERR_CAP_COMMIT = 1u << 6,   // candidate / staging space short at commit (commit retried)
    ERR_INTERNAL = 1u << 7,     // consistency check failed (lookup of an edge that must exist)
    ERR_SPIN = 1u << 8,         // a bounded look-back wait gave up (same bit as PRIM_ERR_SPIN)
};
constexpr uint32_t ABORT_MASK = ERR_POOL_G | ERR_POOL_H | ERR_CAP_PRE | ERR_CAP_COMMIT;

__host__ __device__ inline uint32_t cap_for(uint32_t d, float slack) {
    if (d == 0) return 0;
    uint32_t extra = (uint32_t)((double)d * (double)(slack - 1.0f) + 0.999999);
    if (extra < 2) extra = 2;
    return d + extra;
}

// -------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Counter words
// (c0, c1, c2, c3), key (k0, k1); returns output word 0.
// -------------------------------------------------------------------------
__device__ __forceinline__ uint32_t philox_word0(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                 uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int rnd = 0; rnd < 10; ++rnd) {
        const uint32_t m0lo = 0xD2511F53u * c0;
        const uint32_t m0hi = __umulhi(0xD2511F53u, c0);
        const uint32_t m1lo = 0xCD9E8D57u * c2;
        const uint32_t m1hi = __umulhi(0xCD9E8D57u, c2);
        const uint32_t t0 = m1hi ^ c1 ^ k0;
        const uint32_t t2 = m0hi ^ c3 ^ k1;
        c0 = t0;
        c1 = m1lo;
        c2 = t2;
        c3 = m0lo;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c0;
}

// 128-bit loads of an entry (two halves of the sector)
__device__ __forceinline__ void load_ent(const Ent* p, uint4& head, double2& tail) {
    const uint4* q = reinterpret_cast<const uint4*>(p);
    head = __ldg(q);
    tail = __ldg(reinterpret_cast<const double2*>(q + 1));
}

// One non-backtracking step (Section III-B) on list (off, deg) of vertex c:
// j = floor(x * n_eff / 2^32), then the j-th neighbour other than the previous
// vertex.  prev is the previous vertex's slot in this list (pid = false, from a
// cached entry) or its id (pid = true, after arriving at a hub through HUBREF:
// lists are sorted, so L[j] is taken when its id is below prev, else L[j+1]).
// Returns 1 and advances (c, off, deg, prev, pid), 0 at a leaf (n_eff = 0),
// -1 if an offset leaves the pool (a broken mutation; the caller reports it).
__device__ __forceinline__ int nb_step(const CSRView& g, uint32_t x, uint32_t& c, uint32_t& off, uint32_t& deg,
                                       uint32_t& prev, bool& pid, uint4& h, double2& tl) {
    const uint32_t neff = deg - (prev != 0xFFFFFFFFu ? 1u : 0u);
    if (neff == 0) return 0;
    const uint32_t jj = __umulhi(x, neff);
    uint32_t idx = pid ? jj : jj + (jj >= prev ? 1u : 0u);
    if ((uint64_t)off + idx >= g.pool_cap) return -1;
    const uint4* q = reinterpret_cast<const uint4*>(g.pool + off + idx);
    h = __ldg(q);
    if (pid && h.x >= prev) {
        ++idx;
        if ((uint64_t)off + idx >= g.pool_cap) return -1;
        q = reinterpret_cast<const uint4*>(g.pool + off + idx);
        h = __ldg(q);
    }
    tl = __ldg(reinterpret_cast<const double2*>(q + 1));
    const uint32_t from = c;
    c = h.x;
    if (h.y == HUBREF) {
        off = g.off[c];
        deg = g.deg[c];
        prev = from;
        pid = true;
    } else {
        off = h.y;
        deg = h.z;
        prev = h.w;
        pid = false;
    }
    return 1;
}

// first position in list L[0..d) whose neighbour id >= y
__device__ __forceinline__ uint32_t lower_bound_nbr(const Ent* L, uint32_t d, uint32_t y) {
    uint32_t lo = 0, hi = d;
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (L[mid].nbr < y) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// The same lower bound, searched outward from position h (a slot that has
// drifted by a few positions since it was recorded): the probes start next to
// h and double their distance until they bracket y, then a binary search
// inside the bracket.  Any h gives the same result as lower_bound_nbr.
__device__ __forceinline__ uint32_t lower_bound_nbr_near(const Ent* L, uint32_t d, uint32_t y, uint32_t h) {
    if (d == 0) return 0;
    if (h >= d) h = d - 1;
    uint32_t lo, hi, s = 1;  // the bound lies in [lo, hi]
    if (L[h].nbr < y) {
        lo = h + 1;
        hi = lo;
        while (hi < d && L[hi].nbr < y) {
            lo = hi + 1;
            s <<= 1;
            hi = (d - lo > s) ? lo + s : d;
        }
    } else {
        hi = h;
        lo = h;
        while (lo > 0 && !(L[lo - 1].nbr < y)) {
            hi = lo - 1;
            s <<= 1;
            lo = hi > s ? hi - s : 0;
        }
    }
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (L[mid].nbr < y) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// position of y in x's list or 0xFFFFFFFF
__device__ __forceinline__ uint32_t find_nbr(const CSRView& g, uint32_t x, uint32_t y) {
    const Ent* L = g.pool + g.off[x];
    const uint32_t d = g.deg[x];
    const uint32_t p = lower_bound_nbr(L, d, y);
    return (p < d && L[p].nbr == y) ? p : 0xFFFFFFFFu;
}

// edge membership using the shorter of the two lists
__device__ __forceinline__ bool has_edge(const CSRView& g, uint32_t a, uint32_t b, double* w = nullptr) {
    uint32_t x = a, y = b;
    if (g.deg[b] < g.deg[a]) { x = b; y = a; }
    const uint32_t p = find_nbr(g, x, y);
    if (p == 0xFFFFFFFFu) return false;
    if (w) *w = g.pool[g.off[x] + p].w;
    return true;
}

// first index i in [lo, hi) of a sorted array with a[i] > key (upper bound)
template <typename T>
__device__ __forceinline__ uint32_t upper_bound_arr(const T* a, uint32_t lo, uint32_t hi, T key) {
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (a[mid] <= key) lo = mid + 1; else hi = mid;
    }
    return lo;
}
template <typename T>
__device__ __forceinline__ uint32_t lower_bound_arr(const T* a, uint32_t lo, uint32_t hi, T key) {
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

}  // namespace dg
