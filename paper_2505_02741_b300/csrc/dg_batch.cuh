// dg_batch.cuh -- one resident dynamic graph (G, H in slack-slot CSRs) and
// the batch step of Algorithm 1 under the batch-snapshot semantics.
#pragma once
#include <map>
#include <mutex>
#include <vector>

#include "dg_csr.cuh"
#include "dg_walk.cuh"

namespace dg {

struct Config {
    uint64_t seed = 0;
    double K = 100.0;
    int32_t T = 100;
    int32_t s = 32;
    int32_t early_exit = 1;
    int32_t del_prune = 1;
    int32_t walk_mode = DG_WALK_BATCHED;
    double slack = 1.25;
    double overflow = 0.5;
    uint64_t budget = 0;
    int32_t autotune = 1;
    int32_t timeout_ms = 60000;
    int32_t use_graphs = 1;
    int32_t record = 0;
};

// One walked update's outcome as a shard of a sharded batch exports it: its
// task index j (the same on every replica), the argmin walker and its step
// count (the recorded path length a replica replays), and the update's result.
struct ShardRec {
    uint32_t j;
    int32_t best;
    uint32_t best_steps;
    uint32_t reserved;
    dg_update_result r;
};
static_assert(sizeof(ShardRec) == 48, "shard record is 48 bytes");

// device workspace for batches of at most b_max updates
struct BatchWS {
    uint32_t b_max = 0;
    uint32_t cand_cap = 0;
    DBuf<dg_update> ups;
    DBuf<dg_update_result> res;
    DBuf<BatchHdr> hdr;
    DBuf<uint32_t> err;
    DBuf<BatchCounters> ctr;
    DBuf<unsigned long long> next;
    // validation
    DBuf<uint64_t> vkeys, vkeys_alt;
    DBuf<unsigned long long> vtab;  // edge-key table (vtab_slots) + one word for the repeated-edge flag
    uint32_t vtab_slots = 0;
    DBuf<uint32_t> vvals, vvals_alt, vhist, vscan;
    DBuf<uint8_t> wkind;
    DBuf<double> fin_w;
    DBuf<uint32_t> wflag, wpos, wflag2, wpos2;
    // G changes (and the H removals among them)
    DBuf<uint64_t> gkeys, gkeys_alt, hkeys;
    DBuf<uint32_t> gvals, gvals_alt, ghist, gscan, gcount, hpos, hvals, hcount;
    DBuf<uint8_t> gkind, ghrem, kind_del;
    DBuf<double> gw;
    // walks
    DBuf<uint32_t> t_u, t_v, t_idx, t_kstar, t_count, meta;
    DBuf<uint32_t> t_fin, t_queue, qctr;  // finalization inside the walk: per-update counts, queue, cursors
    DBuf<uint4> cp;                       // deletion walkers' resume points (walk_ncp(T) per walker)
    DBuf<double> step_r;                  // deletion walkers' step records: resistance after the step,
    DBuf<uint32_t> step_e;                //   entry taken (when they fit the budget below)
    DBuf<double> t_wpq, recR;
    DBuf<uint64_t> t_rmax;
    DBuf<uint8_t> t_kind;
    DBuf<int32_t> best;
    // commit
    DBuf<uint64_t> ckeys, ckeys_alt, ck2;
    DBuf<uint32_t> cvals, cvals_alt, chist, cscan, ccount, cflag, cpos, cv2, ccount2;
    DBuf<double> cw;
    DBuf<uint8_t> kind_ins;
    DBuf<uint32_t> path_buf, path_len, fb_list, fb_count;
    DBuf<uint32_t> fb_slot, fb_big, fb_cbase, fb_done, fb_dslot, fb_py;
    DBuf<double> fb_pr, fb_pw;
    DBuf<double> path_w;
    // debug
    DBuf<int32_t> dbg_reason, dbg_steps, dbg_paths;
    // sharded batches: this replica's records, then every replica's
    DBuf<ShardRec> shard_recs;
    ApplyScratch apG, apH, apC;
    uint64_t bytes() const;
};

struct HostStage {  // pinned staging for host-API batches
    dg_update* ups = nullptr;
    dg_update_result* res = nullptr;
    BatchHdr* hdr = nullptr;
    uint32_t* err = nullptr;
    BatchCounters* ctr = nullptr;
    unsigned long long* tops = nullptr;  // [G top, H top]
    uint32_t* counts = nullptr;          // [W, ccount, G's merge: work items, insertions, deletions, changes]
    // device addresses of err, ctr, tops, counts (pinned, written by k_readback)
    uint32_t* d_err = nullptr;
    BatchCounters* d_ctr = nullptr;
    unsigned long long* d_tops = nullptr;
    uint32_t* d_counts = nullptr;
    size_t cap = 0;
};

struct CapturedStep {
    cudaGraphExec_t exec = nullptr;
    uint64_t layout_gen = 0;
    bool device_io = false;
    uint64_t kernels = 0;  // kernel nodes in the captured step
};

struct DGraph {
    int32_t id = 0;
    int32_t n = 0;
    CSR G, H;
    bool has_h = false;
    uint64_t next_id = 0;
    DBuf<uint32_t> touched;    // generation-stamped marks of changed G lists (H lists at commit), see csr_exec
    DBuf<uint32_t> touched_h;  // the same for H while G and H are mutated side by side
    BatchWS ws;
    HostStage hs;
    WalkShape shape;
    bool tuned = false;
    std::vector<std::pair<WalkShape, float>> tune_log;  // the autotuner's trials: shape, median walk ms
    uint64_t layout_gen = 1;  // bumped whenever a buffer baked into a captured step moves
    std::map<uint32_t, CapturedStep> steps;  // by batch-size class
    // a sharded batch between its walks and its commit (graph_shard_*)
    struct {
        bool active = false;
        uint32_t nu = 0, W = 0, j_lo = 0, j_hi = 0;
        cudaStream_t st = nullptr;
    } shard;
    cudaStream_t stream = nullptr;           // private stream (serving)
    // timing events: 0/1 walk, 2/3 batch, 4 end of mutation, 5 end of reduction, 6 end of emission,
    // 7/8 the merge of G's touched lists
    cudaEvent_t ev[9] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    // second stream of the mutation (H side, walk tasks) and its fork/join events
    cudaStream_t side = nullptr;
    cudaEvent_t fk[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // fork / join of the two streams
    dg_batch_stats stats{};
    // ordering against dg_walk_estimate_noalloc (which runs on the caller's
    // stream and returns at once): ev_mut is recorded after every change of G
    // or H and the estimate's stream waits on it; ev_est is recorded after the
    // estimate's kernels and every change of G or H waits on it
    cudaEvent_t ev_mut = nullptr;
    cudaEvent_t ev_est = nullptr;
    std::mutex mu;
    uint64_t bytes() const { return G.bytes() + H.bytes() + touched.bytes() + touched_h.bytes() + ws.bytes(); }
};

struct Ctx;  // context (dg_api.cu)

// batch entry points (stream = caller stream or the context stream)
void graph_load(Ctx& c, DGraph& g, int32_t n, int64_t m, const int32_t* u, const int32_t* v, const double* w);
// H(0) from an edge list (host arrays, or device arrays with device_arrays)
void graph_init_h(Ctx& c, DGraph& g, int64_t mh, const int32_t* u, const int32_t* v, bool device_arrays = false);
// GRASS-like H(0): the given spanning forest plus the n_off off-tree edges of
// largest stretch (dg_grass.cu); stretch_out (host, nullable) receives every
// edge's stretch in canonical edge order
void graph_init_grass(Ctx& c, DGraph& g, int64_t nt, const int32_t* tu, const int32_t* tv, int64_t n_off,
                      double* stretch_out);
void graph_apply(Ctx& c, DGraph& g, int64_t nu, const dg_update* ups, dg_update_result* res, bool device_io,
                 cudaStream_t st);
void graph_release(Ctx& c, DGraph& g);
void graph_release_ws(Ctx& c, DGraph& g, cudaStream_t st);  // batch workspace only
void graph_compact(Ctx& c, DGraph& g, cudaStream_t st);
void graph_export(Ctx& c, DGraph& g, bool which_h, int64_t cap, int32_t* u, int32_t* v, double* w,
                  int64_t* count, cudaStream_t st);
// Sharded batch (Section III-F: the walked updates of one batch are
// independent walk tasks on one snapshot).  Every replica validates and
// mutates identically; shard `rank` of `world` walks the contiguous range
// [W rank / world, W (rank + 1) / world) of the W walked updates and keeps one
// ShardRec per walked update of its range; after the records of every shard
// are gathered, each replica applies the same deterministic commit.
void graph_shard_begin(Ctx& c, DGraph& g, int64_t nu, const dg_update* ups, int32_t rank, int32_t world,
                       cudaStream_t st, uint64_t* nrec_out);
void graph_shard_export(Ctx& c, DGraph& g, ShardRec* host, uint64_t cap, uint64_t* n_out);
void graph_shard_commit(Ctx& c, DGraph& g, const ShardRec* recs, uint64_t nrec, dg_update_result* res);

// Size the batch workspace and pinned staging for batches of up to max_batch
// updates and capture the batch step of every size class up to it, so that
// later batches (served requests of any size) find them ready.
void graph_prepare(Ctx& c, DGraph& g, int64_t max_batch, cudaStream_t st);

// the two halves of the ordering against walk estimates (see DGraph::ev_est)
void graph_wait_estimates(DGraph& g, cudaStream_t st);
void graph_mark_mutation(DGraph& g, cudaStream_t st);

}  // namespace dg
