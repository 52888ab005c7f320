// dg_walk.cuh -- the non-backtracking random-walk kernels (Section III-B/C):
// walkers, per-update reduction (Eq. 12), path replay for recovery and the
// fallback edges.
#pragma once
#include "dg_common.cuh"
#include "dg_host.h"

namespace dg {

// batch header on the device (copied per batch so captured graphs replay it)
struct BatchHdr {
    uint32_t nu;     // updates in the batch
    uint32_t pad;
    uint64_t id0;    // sequence number of the batch's first update
};

struct WalkTasks {
    uint32_t* u;     // start vertex
    uint32_t* v;     // target vertex
    uint32_t* idx;   // update index in the batch
    double* wpq;     // insertion weight (0 for deletions)
    uint64_t* rmax;  // insertion: FP64 bit pattern of the largest R with w_pq * R <= K (all ones for deletions)
    uint8_t* kind;   // WALK_INS / WALK_DEL
    uint32_t* kstar; // insertion: first hitting step (early exit); deletion: minimum high word
                     // of a hit's FP64 resistance seen so far (pruning); 0xFFFFFFFF if none yet
    uint32_t* count; // device: number of walked updates W
};

struct WalkParams {
    double K;
    uint32_t T;
    uint32_t s;
    uint32_t early_exit;
    uint32_t del_prune;   // deletion walkers stop once R exceeds a hit's R of their update
    uint32_t key0, key1;  // Philox key = seed
};

// per-walker record: meta = steps | reason << 16, R = accumulated resistance
struct WalkRecs {
    uint32_t* meta;
    double* R;
    int32_t* paths;  // optional: rows of T+1 vertices per walker (debug)
};

enum : uint32_t { R_NONE = 0, R_HIT = 1, R_OVER_K = 2, R_AT_T = 3, R_LEAF = 4, R_CUT = 5 };

struct WalkShape {
    int block = 256;
    int ilp = 2;
    int blocks_per_sm = 0;  // 0 = occupancy maximum
    int cut = 1;            // persistent launches the walked updates are split over
    int refill = 16;        // empty walker slots a warp with walkers left waits for before refilling
    int lanes = 1;          // lanes per walker (1, 2, 4, 8, 32); above 1 the tiled launch runs
    int tile = 0;           // walked updates a block claims at once, staged in shared memory (0: the
                            // walker queue of the persistent launch; 1..16: the tiled launch)
};

// the tiled launch over walked updates [j_lo, j_hi): shape.tile updates per
// block claim, shape.lanes lanes per walker; walker records only (the
// reduction and emission kernels follow)
void launch_walk_tiled(const CSRView& H, const CSRView& G, const WalkTasks& t, const WalkParams& p,
                       const WalkRecs& r, const BatchHdr* d_hdr, unsigned long long* d_next, uint32_t j_lo,
                       uint32_t j_hi, const WalkShape& shape, const uint32_t* d_err, cudaStream_t st);

// one launch per walked update j (block of s threads), the paper's scheme
void launch_walk_one(const CSRView& H, const CSRView& G, const WalkTasks& t, const WalkParams& p,
                     const WalkRecs& r, const BatchHdr* d_hdr, uint32_t j, const uint32_t* d_err,
                     cudaStream_t st);

struct UpdRes;  // dg_update_result on the device
struct BatchCounters {
    unsigned long long steps;
    unsigned long long accepted;
    unsigned long long recovered;
    unsigned long long walked;
    unsigned long long valid;
    unsigned long long hits;
};

// per-update reduction of walked updates [j_lo, j_hi); writes results, best
// walker per walked update (G: the deletion walks' snapshot, replayed for the
// exact pruned step counts)
void launch_walk_reduce(const CSRView& G, const WalkTasks& t, const WalkParams& p, const WalkRecs& r,
                        const BatchHdr* d_hdr, dg_update_result* res, int32_t* best, BatchCounters* ctr,
                        int32_t* dbg_reason, int32_t* dbg_steps, uint32_t j_lo, uint32_t j_hi, uint32_t* d_err,
                        cudaStream_t st);

// commit candidates (half-edges, keys x*n+y) with G_b weights
struct Cands {
    uint64_t* keys;
    uint32_t* vals;
    double* w;
    uint32_t* count;
    uint32_t cap;
};

// replayed argmin paths of walked deletions: vertices (T+1 per walked update),
// edge weights (T per walked update), path length
struct PathBufs {
    uint32_t* v;
    double* w;
    uint32_t* len;
    uint32_t* fb_list;   // walked deletions without a hit (fallback), appended
    uint32_t* fb_count;  // [0] fallback count; [2..3] u64 (slots << 32 | chunks) of the split scan
    // Split scan of long endpoint lists (claimed when a deletion is queued for
    // the fallback; k_fb_chunks, k_fallback): every distinct endpoint with more
    // than FB_WARP_MAX neighbours gets a slot and ceil(deg / FB_CHUNK) chunks,
    // scanned by one block each.
    uint32_t* fb_slot;   // per vertex: its slot, 0xFFFFFFFF when unclaimed (cleared again by k_fallback)
    uint32_t* fb_big;    // per slot: the vertex
    uint32_t* fb_cbase;  // per slot: its first chunk (ascends with the slot)
    uint32_t* fb_done;   // per slot: 1 when the first look resolved the list (k_fb_quick)
    uint32_t* fb_dslot;  // per fallback deletion and endpoint: the slot, or 0xFFFFFFFF
    double* fb_pr;       // per chunk: minimum resistance found, its weight and neighbour
    double* fb_pw;
    uint32_t* fb_py;
};
constexpr uint32_t FB_CHUNK = 2048;          // list entries per chunk of the split scan
constexpr uint32_t FB_CHUNK_CAP = 1u << 16;  // chunks kept per batch; slots beyond are scanned whole

// Per-update finalization done by the batched walk itself: the walker that
// finishes last for an update queues it, and warps left without walkers take
// queued updates and run the reduction (Eq. 12), the replay of the argmin
// path, the recovered, kept and fallback edges while the walk's long tail is
// still running.  Fallbacks at an endpoint with more than FB_WARP_MAX
// neighbours are left to the block-wide fallback kernel.
constexpr uint32_t FB_WARP_MAX = 1024;
struct FinArgs {
    dg_update_result* res;
    int32_t* best;
    BatchCounters* ctr;
    int32_t* dbg_reason;  // optional debug records
    int32_t* dbg_steps;
    uint32_t* fin;        // per walked update: walkers finished
    uint32_t* queue;      // walked updates in order of completion (0xFFFFFFFF until written)
    uint32_t* qctr;       // [0] next queue slot to take, [1] next queue slot to fill
    const double* fin_w;  // final G_b weight of a kept insertion (NaN if not in G_b)
    Cands c;
    PathBufs pb;
    // resume points of deletion walkers (nullable): the state (vertex, list
    // offset, degree, previous slot or id | hub flag << 31) after every
    // 2^cp_shift steps, ncp per walker, so an argmin path replays as parallel
    // segments instead of one chain of dependent loads
    uint4* cp;
    uint32_t cp_shift, ncp;
    // step records of deletion walkers (nullable; when present no resume
    // points are kept): the resistance accumulated after each step and the
    // pool index of the entry taken (which names the vertex reached), at
    // [(j * T + step) * s + walker] (the walkers of one update side by side,
    // so a warp's records of one step are contiguous)
    double* pr;
    uint32_t* pe;
    uint32_t on;          // 0: records only (reduction and emission run as separate kernels)
    uint32_t spin_limit;  // polls of the finalize queue before ERR_SPIN (FIN_SPIN_LIMIT unless set for tests)
};
constexpr uint32_t FIN_SPIN_LIMIT = 1u << 22;  // about 0.5 s of polling

// checkpoint spacing for step limit T: a power of two >= 16 giving at most 7 per walker
inline uint32_t walk_cp_shift(uint32_t T) {
    uint32_t sh = 4;
    while (((T + (1u << sh) - 1) >> sh) > 8u) ++sh;
    return sh;
}
inline uint32_t walk_ncp(uint32_t T) { return T == 0 ? 0 : (T - 1) >> walk_cp_shift(T); }

// batched persistent walk over walked updates [j_lo, j_hi) of the task list;
// with f.on (one launch over all updates) it also finalizes every update
void launch_walk_batched(const CSRView& H, const CSRView& G, const WalkTasks& t, const WalkParams& p,
                         const WalkRecs& r, const BatchHdr* d_hdr, unsigned long long* d_next,
                         uint32_t j_lo, uint32_t j_hi, const WalkShape& shape, const FinArgs& f,
                         const uint32_t* d_err, cudaStream_t st, cudaStream_t side = nullptr,
                         cudaEvent_t fork = nullptr, cudaEvent_t join = nullptr);

// the fallback edges of deletions the finalizing walk left to the block-wide kernel
void launch_fallback(const CSRView& H, const CSRView& G, const WalkTasks& t, dg_update_result* res,
                     BatchCounters* ctr, Cands c, PathBufs pb, uint32_t w_max, uint32_t* d_err, cudaStream_t st);

// recovered path edges / fallback edges of walked deletions, kept insertions
void launch_emit(const CSRView& H, const CSRView& G, const WalkTasks& t, const WalkParams& p,
                 const WalkRecs& r, const BatchHdr* d_hdr, const int32_t* best, const double* fin_w,
                 dg_update_result* res, BatchCounters* ctr, Cands c, PathBufs pb, uint32_t w_max,
                 uint32_t* d_err, cudaStream_t st);

int device_sms();

// L2 set-aside for H during walks (bytes reserved for persisting lines, max window size)
void walk_set_l2_persist(size_t persist_bytes, size_t max_window);

}  // namespace dg
