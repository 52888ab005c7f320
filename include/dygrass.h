/*
 * dygrass.h -- C ABI of libdygrass.so: batched localized non-backtracking
 * random walks that keep a spectral sparsifier H of a dynamic graph G up to
 * date, after dyGRASS (Yuan, Aghdaei, Feng, arXiv:2505.02741).
 *
 * What each call computes, in the paper's terms:
 *   dg_load_graph        -- G(0), the original graph (Section II-A: weighted,
 *                           undirected; r_e = 1 / w_e).
 *   dg_init_sparsifier   -- H(0), the initial sparsifier (Section III-A; the
 *                           paper takes it from GRASS, here the caller passes it).
 *   dg_apply_updates     -- one batch of the EdgeStream of Algorithm 1, with the
 *                           batch-deferred semantics of Section III-F:
 *                           insertions run s NBRW walkers from u toward v on H
 *                           with distortion threshold K and step limit T, and
 *                           the edge is added to H iff no walker reaches v
 *                           (Section III-B, Eq. 12); deletions of an H edge run
 *                           s walkers on the updated G up to T steps and recover
 *                           the edges of the minimum-resistance path that
 *                           reaches v, or a few local edges when none does
 *                           (Section III-C).
 *   dg_query_sparsifier  -- H(t), the output of Algorithm 1.
 *
 * Batch semantics (the paper defers GPU updates to the end of a batch,
 * Section III-F; the order of phases inside a batch is this library's reading):
 *   1. updates are validated in order against a batch-local view of G;
 *   2. G_b = G with every valid change; H' = H minus every deleted edge that
 *      was in H at batch start;
 *   3. insertion walks run on H', deletion walks on G_b, all on that snapshot;
 *   4. H_b = H' U {kept insertions whose edge is in G_b} U recovered edges,
 *      with weights from G_b.  A batch of one update is Algorithm 1 exactly.
 *
 * Randomness: Philox4x32-10 with counter (step, walker, lo32(id), hi32(id))
 * and key (lo32(seed), hi32(seed)); id is the graph's 0-based sequence number
 * of the update over all updates ever submitted to that graph (rejected ones
 * included).  Results therefore do not depend on how a stream is cut into
 * batches of walks, on launch shapes, or on other graphs sharing the device.
 *
 * Conventions for every call:
 *   - Return value: DG_OK (0) or a negative dg_status; no exception crosses
 *     the ABI.  dg_last_error() describes the last failure on this thread.
 *   - Host arrays are owned by the caller and only read (or written) during the
 *     call.  All device memory is owned by the library (allocated through the
 *     caller's hooks in dg_config when given).
 *   - A dg_ctx is bound to one CUDA device; calls on one context must not be
 *     made concurrently from several threads, except dg_submit_updates /
 *     dg_wait, which are thread-safe.
 */
#ifndef DYGRASS_H
#define DYGRASS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dg_ctx dg_ctx;
typedef int32_t dg_status;

#define DG_OK 0
#define DG_E_INVALID (-1) /* bad argument or input (see dg_last_error) */
#define DG_E_NOMEM (-2)   /* device allocation failed or HBM budget exceeded */
#define DG_E_CUDA (-3)    /* CUDA runtime error */
#define DG_E_TIMEOUT (-4) /* device work did not finish within timeout_ms */
#define DG_E_STATE (-5)   /* call not valid in this state (e.g. no sparsifier yet) */
#define DG_E_BUSY (-6)    /* serving queue full */

/* per-update status codes (dg_update_result.status) */
#define DG_UPD_OK 0
#define DG_UPD_SELF_LOOP 1      /* u == v */
#define DG_UPD_BAD_VERTEX 2     /* u or v outside [0, n) */
#define DG_UPD_DUP_INSERT 3     /* insertion of an edge present in the batch-local view of G */
#define DG_UPD_MISSING_DELETE 4 /* deletion of an edge absent from the batch-local view of G */
#define DG_UPD_BAD_WEIGHT 5     /* insertion weight not finite or not > 0 */
#define DG_UPD_BAD_OP 6         /* op not DG_OP_INSERT / DG_OP_DELETE */
/* Checks run in this order: op, vertex range, self-loop, weight, presence. */

#define DG_OP_INSERT 0
#define DG_OP_DELETE 1

/* walk execution forms (dg_config.walk_mode) */
#define DG_WALK_BATCHED 0    /* one persistent launch runs every walker of the batch */
#define DG_WALK_PER_UPDATE 1 /* one launch per walked update, one block of s threads (the paper's GPU scheme) */

typedef struct {
    uint64_t seed;          /* Philox key */
    double K;               /* distortion threshold (Section III-B); >= 0 */
    int32_t T;              /* step limit per walker (Section III-B; the paper fixes 100); 1..65535 */
    int32_t s;              /* walkers per update (Section III-B); 1..1024 */
    int32_t ins_early_exit; /* 1: an insertion's walkers stop at the first step index at which
                               any of them reaches v (decisions unchanged; R~ and step counts
                               refer to the truncated walks); 0: every walker runs to its own stop */
    int32_t del_prune;      /* 1: a deletion's walker may stop once its resistance exceeds that of
                               a walker of the same update that already reached v: it can no
                               longer give the minimum of Eq. 12, so hit, best_walker, r_est and
                               the recovered edges are unchanged.  The counts reported follow the
                               exact rule -- every walker of a deletion with a hit stops at its
                               first step whose resistance exceeds R~ -- so they do not depend on
                               when a walker was actually cut: steps sums those stops and nhits
                               counts the walkers at R~.  0: every deletion walker runs to its own
                               stop (steps and nhits of the full walks) */
    int32_t walk_mode;      /* DG_WALK_BATCHED or DG_WALK_PER_UPDATE */
    double slack;           /* per-vertex capacity = deg + max(2, ceil(deg*(slack-1))); >= 1 */
    double overflow_frac;   /* pool headroom for relocated lists, fraction of the initial pool */
    uint64_t hbm_budget_bytes; /* serving admission budget in bytes; 0 = no limit */
    int32_t autotune;       /* 1: tune walk launch shape per graph on its first large batch */
    int32_t timeout_ms;     /* bound on every host wait for device work; <= 0 means 60000 */
    int32_t use_cuda_graphs;/* 1: capture each batch step as a CUDA graph, replayed per batch size class */
    int32_t record_walkers; /* debug: keep per-walker records (and paths if T <= 256) of the last batch */
    int32_t device;         /* CUDA device ordinal */
    /* optional device allocator (NULL = cudaMallocAsync / cudaFreeAsync on the library stream) */
    void* (*alloc)(size_t bytes, void* cuda_stream, void* user);
    void (*free)(void* ptr, size_t bytes, void* cuda_stream, void* user);
    void* alloc_user;
} dg_config;

/* one streamed edge update, 24 bytes */
typedef struct {
    int32_t u, v;   /* endpoints; walks run from u toward v */
    double w;       /* weight of an insertion (> 0, finite); ignored for a deletion */
    int32_t op;     /* DG_OP_INSERT or DG_OP_DELETE */
    int32_t reserved;
} dg_update;

/* per-update result, 32 bytes */
typedef struct {
    int32_t status;      /* DG_UPD_* */
    uint8_t walked;      /* walkers ran (valid insertion, or deletion of an edge in H) */
    uint8_t hit;         /* some walker reached v (within K for insertions) */
    uint8_t accepted;    /* insertion kept for H (no walker reached v); committed if the edge is in G_b */
    uint8_t fallback;    /* deletion walked but no walker reached v: local fallback edges recovered */
    int32_t nhits;       /* walkers that reached v (after the early-exit cut for insertions; with
                            del_prune, for deletions: the walkers at the minimum resistance R~) */
    int32_t best_walker; /* walker index of R~ (lowest index among equal resistances), -1 if none */
    int32_t nrecovered;  /* distinct edges this deletion returned to H (path or fallback) */
    int32_t steps;       /* walk steps of this update's walkers under the early-exit cut
                            (insertions) or the exact pruning rule of del_prune (deletions) */
    double r_est;        /* R~ = minimum path resistance over hitting walkers (Eq. 12); +inf if none */
} dg_update_result;

/* statistics of the last completed batch on a graph */
typedef struct {
    int64_t updates;         /* updates in the batch */
    int64_t valid;           /* updates with status DG_UPD_OK */
    int64_t walked;          /* walked updates */
    int64_t steps;           /* useful walk steps (sum of dg_update_result.steps) */
    int64_t accepted;        /* kept insertions */
    int64_t recovered;       /* edges returned to H by deletions */
    int64_t h_edges;         /* |E(H)| now (after the batch; counted when the statistics are read) */
    int64_t g_edges;         /* |E(G)| now (after the batch; counted when the statistics are read) */
    double walk_ms;          /* device time of the walk phase (CUDA events on the batch stream) */
    double batch_ms;         /* device time of the whole batch step */
    int64_t walk_launches;   /* kernel launches in the walk phase */
    int64_t launches;        /* kernel launches of the batch step */
    int64_t retries;         /* pool growth / scratch growth retries */
    int32_t walk_block;      /* launch shape used by the walk phase */
    int32_t walk_ilp;
    int32_t walk_blocks_per_sm;
    int32_t graph_replayed;  /* 1 if the step ran as a replayed CUDA graph */
    double mutate_ms;        /* validation + G/H mutation (device time) */
    double reduce_ms;        /* per-update reduction after the walks */
    double emit_ms;          /* path replay and candidate emission */
    double commit_ms;        /* sort, filter and merge into H, result copy-out */
    int32_t walk_cut;        /* persistent walk launches per batch */
    int32_t autotuned;       /* 1 if this batch ran the walk-shape autotuner */
    int32_t walk_refill;     /* empty walker slots a warp waits for before refilling */
    int32_t walk_lanes;      /* lanes per walker (1: one walker per lane) */
    int32_t walk_tile;       /* walked updates per block claim (0: the persistent walker queue) */
    int32_t reserved0;
    double merge_ms;         /* device time of the merge of G's touched lists (-1 when not timed) */
    int64_t merge_entries;   /* 32-byte entries that merge read (old lists) and wrote (new lists) */
} dg_batch_stats;

/* default configuration: seed 0, K 100, T 100, s 32, early exit on, batched walks,
   slack 1.25, overflow 0.5, no budget, autotune on, timeout 60 s, CUDA graphs on */
void dg_config_default(dg_config* cfg);

/* Create a context on cfg->device (cfg may be NULL for defaults). */
dg_status dg_create(const dg_config* cfg, dg_ctx** out);

/* Destroy a context and free all its device memory. NULL is ignored. */
dg_status dg_destroy(dg_ctx* ctx);

/* Text for a status code (static storage). */
const char* dg_status_str(dg_status st);

/* Description of the last error raised on the calling thread (static storage). */
const char* dg_last_error(void);

/*
 * G(0) (Section II-A).  n vertices, m undirected edges (u[i], v[i], w[i]),
 * host arrays of length m.  The graph must be simple: 0 <= u, v < n, u != v,
 * no pair listed twice (in either orientation), w finite and > 0.  Violations
 * return DG_E_INVALID and load nothing.  The graph starts with an empty
 * sparsifier and update sequence number 0.  *graph_id_out receives the id.
 */
dg_status dg_load_graph(dg_ctx* ctx, int32_t n, int64_t m, const int32_t* u, const int32_t* v,
                        const double* w, int32_t* graph_id_out);

/* Free a graph and its sparsifier. */
dg_status dg_unload_graph(dg_ctx* ctx, int32_t graph_id);

/*
 * H(0) (Section III-A: an input of Algorithm 1).  mh edges (u[i], v[i]) that
 * must be edges of the current G (DG_E_INVALID otherwise); weights are taken
 * from G; repeated pairs are kept once.  Replaces the current sparsifier.
 */
dg_status dg_init_sparsifier(dg_ctx* ctx, int32_t graph_id, int64_t mh, const int32_t* u,
                             const int32_t* v);

/*
 * GRASS-like H(0) (Section III-A; the paper precomputes H(0) with GRASS: a
 * spanning tree plus spectrally critical off-tree edges).  The nt edges
 * (tu[i], tv[i]) (host arrays) must be edges of G forming a forest
 * (DG_E_INVALID otherwise: a non-edge, a cycle, a repeated edge).  Every other
 * edge e = (p, q) of G gets the stretch w_e * R_F(p, q), R_F the resistance of
 * the forest path (+inf when p and q lie in different trees): the distortion
 * the insertion test of Section III-B measures, exact on a tree.  H(0) = the
 * forest + the n_off off-tree edges of largest stretch (ties: the smaller edge
 * in lexicographic (min, max) order).  stretch_out (nullable, host) receives
 * the stretch of every edge of G in lexicographic order (0 for forest edges).
 * R_F is formed from root distances: each tree is rooted at its smallest
 * vertex, D[child] = D[parent] + 1/w, R_F = (D[p] - D[l]) + (D[q] - D[l]) with
 * l the lowest common ancestor.  Replaces the current sparsifier.
 */
dg_status dg_init_sparsifier_grass(dg_ctx* ctx, int32_t graph_id, int64_t nt, const int32_t* tu,
                                   const int32_t* tv, int64_t n_off, double* stretch_out);

/*
 * One batch of nu updates (Algorithm 1, batch semantics above).  ups: host
 * array of nu records; res: host array of nu results, or NULL.  cuda_stream:
 * stream to run on (NULL = the context's stream); the call returns after the
 * results are on the host, waiting at most timeout_ms.  nu == 0 is a no-op.
 * Per-update problems are reported in res[i].status; the batch still applies.
 * Pinned host arrays (cudaMallocHost / cudaHostRegister; both, or ups with
 * res NULL) are copied straight to and from the device; other host memory goes
 * through the graph's pinned staging buffers.
 */
dg_status dg_apply_updates(dg_ctx* ctx, int32_t graph_id, int64_t nu, const dg_update* ups,
                           dg_update_result* res, void* cuda_stream);

/*
 * Same as dg_apply_updates with device-resident inputs and outputs: d_ups and
 * d_res are device pointers (d_res may be NULL).  Returns once the batch is
 * complete on the device.
 */
dg_status dg_apply_updates_device(dg_ctx* ctx, int32_t graph_id, int64_t nu, const dg_update* d_ups,
                                  dg_update_result* d_res, void* cuda_stream);

/*
 * Edges of H: u[i] < v[i], lexicographic order, weights from G.  Writes at most
 * cap entries; *count_out receives |E(H)|.  cap < |E(H)| returns DG_E_INVALID
 * with *count_out set.  With u, v and w all NULL the call only sets *count_out
 * and returns DG_OK (size query).
 */
dg_status dg_query_sparsifier(dg_ctx* ctx, int32_t graph_id, int64_t cap, int32_t* u, int32_t* v,
                              double* w, int64_t* count_out);

/* Edges of the current G, same conventions as dg_query_sparsifier. */
dg_status dg_query_graph(dg_ctx* ctx, int32_t graph_id, int64_t cap, int32_t* u, int32_t* v,
                         double* w, int64_t* count_out);

/* Statistics of the graph's last batch. */
dg_status dg_get_batch_stats(dg_ctx* ctx, int32_t graph_id, dg_batch_stats* out);

/*
 * Debug records of the last batch (needs cfg.record_walkers = 1): for every
 * update i and walker k, row i*s+k of reason (1 hit, 2 over K, 3 step limit,
 * 4 leaf, 5 cut by the early exit; 0 if the update was not walked) and steps;
 * paths (nullable, rows of T+1 vertex ids, -1 padded) when T <= 256.
 * cap = number of rows the arrays hold (must be >= nu of that batch).
 */
dg_status dg_get_walker_records(dg_ctx* ctx, int32_t graph_id, int64_t cap, int32_t* reason,
                                int32_t* steps, int32_t* paths);

/* Force a compaction of G's and H's slack-slot pools (normally automatic). */
dg_status dg_compact(dg_ctx* ctx, int32_t graph_id);

/* Device bytes held by a graph (both pools and their vertex arrays). */
dg_status dg_graph_bytes(dg_ctx* ctx, int32_t graph_id, uint64_t* bytes_out);

/* Kernel launches issued by this context so far (all graphs). */
uint64_t dg_launch_count(dg_ctx* ctx);

/* Set / get a graph's next update sequence number (checkpoint / resume). */
dg_status dg_set_next_update_id(dg_ctx* ctx, int32_t graph_id, uint64_t next_id);
dg_status dg_get_next_update_id(dg_ctx* ctx, int32_t graph_id, uint64_t* next_id);

/* Walk launch shape for a graph (threads per block, walkers per thread, blocks per SM);
   0 fields keep the current value.  Outputs never depend on the shape. */
dg_status dg_set_walk_shape(dg_ctx* ctx, int32_t graph_id, int32_t block, int32_t ilp,
                            int32_t blocks_per_sm);

/* Refill threshold of the batched walk (1..32): a warp that still has walkers
   starts new ones only when at least this many of its walker slots are empty
   (or none is busy).  Starting walkers stalls the warp for three dependent
   reads, and the walkers of one update tend to stop together, so waiting for
   several empty slots trades a few idle lanes for fewer stalls.  Outputs never
   depend on it; DG_E_INVALID outside 1..32. */
dg_status dg_set_walk_refill(dg_ctx* ctx, int32_t graph_id, int32_t refill_min);

/*
 * The batching engine's other work shapes: lanes per walker (1, 2, 4, 8 or
 * 32: the lanes of a group draw the Philox words of the next `lanes` steps
 * side by side and take the walker's steps together) and the frontier tile
 * (0: the persistent launch's walker queue; 1..16: a block claims that many
 * walked updates at a time and stages their fields in shared memory; the
 * walks are then followed by separate reduction and emission kernels).
 * Outputs never depend on them.  Marks the graph tuned; DG_E_INVALID
 * outside those values.
 */
dg_status dg_set_walk_coop(dg_ctx* ctx, int32_t graph_id, int32_t lanes, int32_t tile);

/*
 * The autotuner's trials on this graph (from its last run): per trial the
 * shape {block, walkers per thread, refill, lanes, tile, cut} into shapes
 * (6 int32 each) and its median walk time (ms) into ms; host arrays of cap
 * trials; *count_out = the number of trials (cap too small: DG_E_INVALID).
 */
dg_status dg_get_tune_log(dg_ctx* ctx, int32_t graph_id, int64_t cap, int32_t* shapes, float* ms,
                          int64_t* count_out);

/*
 * Sharded batch over replicas (Section III-F: the walked updates of one batch
 * are independent walk tasks on one snapshot).  Every replica -- a context
 * holding the same G, H and update sequence number, typically one per GPU or
 * per process -- calls the three steps with the same batch:
 *
 *   dg_shard_begin   validates and mutates G and H (identically everywhere),
 *                    then walks only this replica's share of the W walked
 *                    updates: the contiguous task range
 *                    [W rank / world, W (rank + 1) / world) (deletions first,
 *                    then insertions, each in update order), and reduces them
 *                    (Eq. 12).  *nrec_out receives the number of records this
 *                    replica exports.  rank in [0, world); record_walkers must
 *                    be off and walk_mode DG_WALK_BATCHED.
 *   dg_shard_export  copies those records (DG_SHARD_RECORD_BYTES each) into
 *                    the caller's host buffer of cap records (recs NULL: only
 *                    *nrec_out is set).
 *   dg_shard_commit  takes the records of every replica gathered in any order
 *                    (nrec in total; each walked update exactly once, else
 *                    DG_E_INVALID and nothing is committed), replays each
 *                    deletion's argmin path from its Philox counters on G_b,
 *                    forms the kept, recovered and fallback edges and commits
 *                    them to H; res (nullable, nu entries of the batch)
 *                    receives every update's result.
 *
 * The gathering is the caller's (for instance an all-gather over processes
 * after exchanging the record counts).  Results, G and H then equal, byte for
 * byte, those of dg_apply_updates on the same batch, on every replica.  Until
 * dg_shard_commit returns, the graph accepts no other batch (DG_E_STATE).
 */
#define DG_SHARD_RECORD_BYTES 48

dg_status dg_shard_begin(dg_ctx* ctx, int32_t graph_id, int64_t nu, const dg_update* ups, int32_t rank,
                         int32_t world, void* cuda_stream, uint64_t* nrec_out);
dg_status dg_shard_export(dg_ctx* ctx, int32_t graph_id, void* recs, uint64_t cap, uint64_t* nrec_out);
dg_status dg_shard_commit(dg_ctx* ctx, int32_t graph_id, uint64_t nrec, const void* recs,
                          dg_update_result* res);

/*
 * Debug: the number of times the finalizing warps of the batched walk poll
 * for the next completed update before they give up (polls >= 0; < 0 restores
 * the default of 2^22 polls, about half a second).  When a wait gives up, the
 * walk kernel records the failure and returns normally; the batch call then
 * returns DG_E_TIMEOUT and the graph's state is unspecified (unload it), while
 * the CUDA context stays usable.  With polls = 0 every batch with a walked
 * update gives up, which is how the tests exercise that path.  Applies to
 * later batches of every graph of the context.
 */
dg_status dg_debug_set_wait_limit(dg_ctx* ctx, int64_t polls);

/*
 * Serving (continuous batching over resident graphs).  dg_submit_updates
 * copies the request and queues it; requests on one graph run in submission
 * order, one at a time; requests on different graphs run concurrently on
 * separate streams when the HBM budget (cfg.hbm_budget_bytes) admits their
 * working set.  res (nullable) must stay valid until dg_wait returns for the
 * ticket.  Each request is one batch: its results equal those of
 * dg_apply_updates on the same graph state.  Thread-safe.
 */
dg_status dg_submit_updates(dg_ctx* ctx, int32_t graph_id, int64_t nu, const dg_update* ups,
                            dg_update_result* res, uint64_t* ticket_out);

/* Wait for a ticket (timeout_ms < 0: the context timeout).  Returns the request's status;
   *latency_ms (nullable) receives submit-to-completion time. */
dg_status dg_wait(dg_ctx* ctx, uint64_t ticket, int32_t timeout_ms, double* latency_ms);

/* dg_wait that also reports, in *queue_ms (nullable), the part of the latency the
   request spent queued before a worker started it (behind earlier requests of its
   graph, or waiting for the HBM budget). */
dg_status dg_wait_ex(dg_ctx* ctx, uint64_t ticket, int32_t timeout_ms, double* latency_ms, double* queue_ms);

/* Prepare a graph for batches (or served requests) of up to max_batch updates:
   sizes its batch workspace and pinned staging, compacts its pools with room
   for several batches of that size, and, with CUDA graphs on, captures the
   batch step of every size class up to max_batch, so that no later batch pays
   for them.  The walk-shape autotuner still runs on the first batch
   of >= 4096 updates unless a shape was set with dg_set_walk_shape. */
dg_status dg_prepare(dg_ctx* ctx, int32_t graph_id, int64_t max_batch);

/*
 * Allocation-free walk estimate.  The paper has no counterpart: this entry
 * point exists for callers of this library that must not allocate device
 * memory while they run -- for instance code that issues work while a stream
 * is being captured, a latency-critical thread on which an allocation could
 * stall the device, or a host application that has handed the GPU's memory to
 * its own pool and cannot afford a call that grows it.
 *
 * It runs the s walkers of each query on a graph that is already resident
 * (loaded earlier with dg_load_graph) and writes one estimate per query; it
 * changes neither G nor H.  kind DG_OP_INSERT walks the current H from u
 * toward v with the distortion threshold K and weight w; kind DG_OP_DELETE
 * walks the current G from u toward v without K and without pruning (every
 * walker runs to its own stop; if (u, v) is still an edge of G a walker may
 * take it directly).  id is the update sequence number the Philox counter
 * uses, so a query with the id, endpoints and weight of an insertion that
 * dg_apply_updates is about to walk on the same H gets the same hit, nhits,
 * best_walker, steps and r_est; a DELETE query on the G a deletion batch left
 * behind (that batch's G_b) with the id of one of its deletions gets that
 * deletion's hit, best_walker and r_est, and the nhits and steps it has with
 * del_prune = 0.
 *
 * d_queries and d_out are device pointers owned by the caller (nq records
 * each).  The walkers' scratch is a static device array inside the library
 * sized for DG_NOALLOC_MAX_QUERIES queries and DG_NOALLOC_MAX_WALKERS walkers
 * (about 1.6 MB); every GPU that loads the library keeps it until the process
 * exits.  nq > DG_NOALLOC_MAX_QUERIES or nq * s > DG_NOALLOC_MAX_WALKERS
 * returns DG_E_INVALID without touching the device.  The call enqueues its
 * kernels on cuda_stream (NULL = the context's stream) and returns without
 * waiting; d_out is ready once that stream reaches this point.  It calls no
 * device allocator.  The first call on a device looks up the static array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  All calls share the one array, which
 * keeps the last call's contents: calls whose work overlaps on the GPU (other
 * streams, other contexts on the same device) race and must be serialized by
 * the caller.  Outside a stream capture the call is ordered against changes
 * of the same graph: its kernels wait for the last dg_apply_updates /
 * dg_submit_updates batch, dg_init_sparsifier or dg_compact of that graph,
 * and the next such call waits for its kernels.  While cuda_stream is being
 * captured that ordering is the caller's: no such change of the graph may
 * run between the capture's launch and the completion of its kernels.
 * nq == 0 returns DG_OK and launches nothing.
 */
#define DG_NOALLOC_MAX_QUERIES 4096
#define DG_NOALLOC_MAX_WALKERS 131072

typedef struct {
    int32_t u, v;     /* walk from u toward v */
    double w;         /* weight of the inserted edge (kind DG_OP_INSERT) */
    int32_t kind;     /* DG_OP_INSERT (walk H, threshold K) or DG_OP_DELETE (walk G, no K) */
    int32_t reserved;
    uint64_t id;      /* update sequence number keying the Philox counters */
} dg_walk_query;      /* 32 bytes */

typedef struct {
    int32_t status;      /* DG_UPD_OK, DG_UPD_BAD_VERTEX, DG_UPD_SELF_LOOP, DG_UPD_BAD_WEIGHT or DG_UPD_BAD_OP */
    int32_t nhits;       /* as dg_update_result */
    int32_t best_walker;
    int32_t steps;
    double r_est;
    uint8_t hit;
    uint8_t reserved[7];
} dg_walk_estimate;      /* 32 bytes */

dg_status dg_walk_estimate_noalloc(dg_ctx* ctx, int32_t graph_id, int64_t nq, const dg_walk_query* d_queries,
                                   dg_walk_estimate* d_out, void* cuda_stream);

/*
 * The updates applied one at a time, as Algorithm 1 states it: every update
 * walks the G and H all earlier updates of the stream left, instead of the
 * snapshot of its batch (Section III-F's deferral).  Results equal applying
 * each update as a batch of one, in order.  The call cuts the stream into
 * prefixes whose batched execution provably gives those results -- no walk of
 * an update of the prefix stands on a vertex whose adjacency another update
 * of the prefix changes (G: the endpoints of every valid update; H: the
 * endpoints of kept insertions and deleted H edges, the vertices of a
 * recovered path), no edge occurs twice, and a deletion whose walkers all
 * missed ends its prefix -- found by a dry run of each window's walks on the
 * current G and H, and runs each prefix as a batch.  ups / res: host arrays
 * of nu records (res nullable).  *prefixes_out (nullable): the number of
 * prefixes (batches) it took.  Errors as dg_apply_updates; the prefixes run
 * before an error stay applied (their results are in res, *prefixes_out
 * counts them, and dg_get_next_update_id tells how far the stream got).
 */
dg_status dg_apply_updates_sequential(dg_ctx* ctx, int32_t graph_id, int64_t nu, const dg_update* ups,
                                      dg_update_result* res, int64_t* prefixes_out);

/* ------------------------------------------------------------------------
 * Quality of the sparsifier (Section IV: the off-tree density d_H, the
 * relative condition number kappa(L_G, L_H) of Eqs. 6-10, and PCG on
 * L_G x = b with L_H as the preconditioner, Table IV).  These calls read G and
 * H as they stand after the last batch; they run on the context's stream,
 * hold the graph (no batch of it runs meanwhile) and return when done.  Every
 * step runs on the device; the host only decides when to stop iterating.
 * ------------------------------------------------------------------------ */

/* d_H = |E(H)| / |V| - 1 (Section IV), with |E(G)| and |E(H)| (each output
 * nullable). */
dg_status dg_sparsifier_density(dg_ctx* ctx, int32_t graph_id, double* d_h_out, int64_t* m_g_out,
                                int64_t* m_h_out);

#define DG_LAP_G 0
#define DG_LAP_H 1

/* y = L x for the Laplacian L = D - A of G (which = DG_LAP_G) or H
 * (DG_LAP_H), Section II-A.  d_x and d_y are device arrays of n doubles owned
 * by the caller (they may not overlap).  Row x sums its neighbours in
 * ascending neighbour order; the weighted degree is summed the same way.
 * cuda_stream: NULL = the context's stream (the call waits for it). */
dg_status dg_laplacian_apply(dg_ctx* ctx, int32_t graph_id, int32_t which, const double* d_x, double* d_y,
                             void* cuda_stream);

#define DG_PRECOND_NONE 0
#define DG_PRECOND_JACOBI 1     /* M = diag(L_G) */
#define DG_PRECOND_SPARSIFIER 2 /* M = L_H (Section IV, Table IV) */

typedef struct {
    double tol;             /* stop when ||r_k|| / ||b|| < tol (Section IV uses 1e-8) */
    int32_t max_iter;       /* outer iterations (> 0) */
    int32_t precond;        /* DG_PRECOND_* */
    double inner_tol;       /* DG_PRECOND_SPARSIFIER: each L_H solve runs to this relative residual */
    int32_t inner_max_iter; /* ... or this many iterations */
    int32_t reserved;
} dg_pcg_options;           /* 32 bytes */

typedef struct {
    int32_t iters;          /* outer iterations run */
    int32_t converged;      /* 1 when ||r|| / ||b|| < tol was reached */
    double rel_residual;    /* ||b - L_G x|| / ||b|| recomputed from x at the end */
    int64_t inner_iters;    /* inner (L_H) iterations over all outer ones */
    int32_t inner_max;      /* most inner iterations one L_H solve took */
    int32_t inner_unconverged; /* L_H solves that stopped at inner_max_iter */
    double ms;              /* device time of the solve */
} dg_pcg_info;              /* 40 bytes */

/*
 * Preconditioned conjugate gradients on L_G x = b from x = 0 (Section IV):
 * alpha = (r, z) / (p, L_G p); x += alpha p; r -= alpha L_G p; stop when
 * ||r|| / ||b|| < tol; z = M^-1 r; beta = (r_new, z_new) / (r, z);
 * p = z + beta p.  With DG_PRECOND_SPARSIFIER, z = L_H^+ r is computed by an
 * inner conjugate-gradient solve on L_H preconditioned by H's maximum-weight
 * spanning forest F (ties: the smaller edge in lexicographic order), whose
 * Laplacian is solved exactly through an Euler tour of every tree (subtree
 * sums of r give the current through each tree edge, root-path sums of
 * current / weight the potentials), to inner_tol.  b (device, n doubles,
 * caller-owned) must sum to zero over every connected component of G (else
 * the singular system has no solution); x (device, n doubles) receives
 * the solution (defined up to a constant per component).  H must span every
 * component of G (DG_E_STATE otherwise).  hist (nullable, host, max_iter + 1
 * doubles) receives ||r_k|| / ||b|| for k = 0..iters.  info (nullable).
 */
dg_status dg_pcg_solve(dg_ctx* ctx, int32_t graph_id, const double* d_b, double* d_x, const dg_pcg_options* opt,
                       dg_pcg_info* info, double* hist);

typedef struct {
    int32_t max_iter;       /* Lanczos steps (> 0) */
    int32_t check_every;    /* Ritz values are checked every this many steps (> 0) */
    double tol;             /* stop when lambda_max moved by less than tol * lambda_max between checks */
    double inner_tol;       /* each L_H solve runs to this relative residual ... */
    int32_t inner_max_iter; /* ... or this many iterations */
    int32_t reserved;
    const double* d_v0;     /* start vector (device, n doubles; NULL: Philox4x32-10 draws keyed by seed) */
    uint64_t seed;
} dg_kappa_options;         /* 48 bytes */

typedef struct {
    double kappa;           /* lambda_max of the pencil (L_G, L_H) (+inf when H does not span G's components) */
    double lambda_min;      /* smallest Ritz value (approaches 1 from above for a subgraph H) */
    int32_t iters;          /* Lanczos steps taken */
    int32_t converged;
    int64_t inner_iters;    /* inner (L_H) iterations over all steps */
    double ms;
} dg_kappa_info;            /* 40 bytes */

/*
 * kappa(L_G, L_H) (Eqs. 6-10): for H a subgraph of G the smallest eigenvalue
 * of the pencil is 1 (Section III-C), so kappa is its largest, found here by
 * Lanczos in the L_H inner product on L_H^+ L_G: v_1 = v_0 / ||v_0||_H; per
 * step u = L_G v_j, alpha_j = (v_j, u), w = L_H^+ u - alpha_j v_j -
 * beta_{j-1} v_{j-1}, beta_j = ||w||_H, v_{j+1} = w / beta_j.  The largest
 * eigenvalue of the tridiagonal (alpha, beta) is found by multisection on
 * its Sturm counts.  L_H^+ is the inner solve of dg_pcg_solve.  With
 * d_v0 == NULL the start vector is x -> 2 u(x) - 1, u(x) the first Philox
 * word of counter (x, 0, 0, 0) and key (seed low, seed high) scaled by 2^-32.
 */
dg_status dg_condition_number(dg_ctx* ctx, int32_t graph_id, const dg_kappa_options* opt, dg_kappa_info* info);

/* Test hooks of the quality calls.  dg_debug_sparsifier_forest writes the
 * edges (u < v, lexicographic order) of H's maximum-weight spanning forest
 * into host arrays of cap entries, *nf_out = their count (cap too small:
 * DG_E_INVALID).  dg_debug_forest_solve sets d_z = L_F^+ d_r up to a
 * constant per tree (z = 0 at each tree's smallest vertex), F that forest. */
dg_status dg_debug_sparsifier_forest(dg_ctx* ctx, int32_t graph_id, int64_t cap, int32_t* fu, int32_t* fv,
                                     int64_t* nf_out);
dg_status dg_debug_forest_solve(dg_ctx* ctx, int32_t graph_id, const double* d_r, double* d_z);

#ifdef __cplusplus
}
#endif
#endif /* DYGRASS_H */
