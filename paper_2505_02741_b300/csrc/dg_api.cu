// dg_api.cu -- the C ABI (include/dygrass.h): contexts, graphs, batches,
// queries and the serving scheduler (continuous batching over resident graphs).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>

#include "dg_ctx.h"

namespace dg {

static thread_local std::string t_last_error;

void set_last_error(const std::string& msg) { t_last_error = msg; }

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

DGraph& Ctx::graph(int32_t gid) {
    std::lock_guard<std::mutex> lk(mu);
    auto it = graphs.find(gid);
    if (it == graphs.end()) throw Error(DG_E_INVALID, "unknown graph id");
    return *it->second;
}

template <typename F>
static dg_status guarded(dg_ctx* ctx, F&& f) {
    try {
        if (ctx) {
            Ctx* c = reinterpret_cast<Ctx*>(ctx);
            DG_CUDA(cudaSetDevice(c->device));
        }
        f();
        return DG_OK;
    } catch (const Error& e) {
        t_last_error = e.what();
        return e.code;
    } catch (const std::bad_alloc&) {
        t_last_error = "host allocation failed";
        return DG_E_NOMEM;
    } catch (const std::exception& e) {
        t_last_error = e.what();
        return DG_E_CUDA;
    }
}

static Ctx& C(dg_ctx* ctx) {
    if (!ctx) throw Error(DG_E_INVALID, "null context");
    return *reinterpret_cast<Ctx*>(ctx);
}

// working-set estimate of one batch of nu updates (serving admission)
static uint64_t request_bytes(const Config& cfg, uint64_t nu) {
    uint64_t b = 1024;
    while (b < nu) b <<= 1;
    const uint64_t per = 24 + 32 + 64 + 2 * 80 + (uint64_t)cfg.s * 12 + (uint64_t)(cfg.T + 1) * 4 + 8 * 60 + 2 * 16 * 32 * 2;
    return b * per + (8u << 20);
}

// ---------------------------------------------------------------------------
// serving workers
// ---------------------------------------------------------------------------
static void worker_loop(Ctx* c) {
    cudaSetDevice(c->device);
    for (;;) {
        std::shared_ptr<Request> rq;
        DGraph* g = nullptr;
        {
            std::unique_lock<std::mutex> lk(c->smu);
            for (;;) {
                if (c->stopping) return;
                uint64_t resident = 0;
                {
                    std::lock_guard<std::mutex> lg(c->mu);
                    for (auto& kv : c->graphs) resident += kv.second->G.bytes() + kv.second->H.bytes();
                }
                bool refused = false;
                for (auto it = c->queue.begin(); it != c->queue.end(); ++it) {
                    auto& r = *it;
                    if (c->busy[r->gid]) continue;
                    const bool fits = c->cfg.budget == 0 ||
                                      resident + c->in_flight_bytes + r->need_bytes <= c->cfg.budget;
                    if (!fits) {
                        // with nothing in flight it can never be admitted: fail it instead of waiting
                        if (c->in_flight_bytes == 0) {
                            r->status = DG_E_NOMEM;
                            r->error = "request does not fit the HBM budget next to the resident graphs";
                            r->t_done = now_ms();
                            r->done = true;
                            c->queue.erase(it);
                            refused = true;
                            break;
                        }
                        continue;
                    }
                    rq = r;
                    c->queue.erase(it);
                    break;
                }
                if (refused) {
                    c->dcv.notify_all();
                    continue;
                }
                if (rq) break;
                c->scv.wait(lk);
            }
            c->busy[rq->gid] = true;
            rq->t_start = now_ms();
            c->in_flight_bytes += rq->need_bytes;
        }
        dg_status st = DG_OK;
        std::string err;
        try {
            g = &c->graph(rq->gid);
            std::lock_guard<std::mutex> glk(g->mu);
            if (!g->stream) DG_CUDA(cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking));
            graph_apply(*c, *g, (int64_t)rq->ups.size(), rq->ups.data(), rq->res, false, g->stream);
            if (c->cfg.budget) {  // under a budget, give the working set back between requests
                graph_release_ws(*c, *g, g->stream);
                DG_CUDA(cudaStreamSynchronize(g->stream));
            }
        } catch (const Error& e) {
            st = e.code;
            err = e.what();
        } catch (const std::exception& e) {
            st = DG_E_CUDA;
            err = e.what();
        }
        {
            std::lock_guard<std::mutex> lk(c->smu);
            rq->status = st;
            rq->error = err;
            rq->t_done = now_ms();
            rq->done = true;
            c->busy[rq->gid] = false;
            c->in_flight_bytes -= rq->need_bytes;
        }
        c->dcv.notify_all();
        c->scv.notify_all();
    }
}

static void ensure_workers(Ctx& c) {
    std::lock_guard<std::mutex> lk(c.smu);
    if (!c.workers.empty()) return;
    int nw = c.n_workers > 0 ? c.n_workers : 4;
    for (int i = 0; i < nw; ++i) c.workers.emplace_back(worker_loop, &c);
}

}  // namespace dg

using namespace dg;

extern "C" {

void dg_config_default(dg_config* cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->seed = 0;
    cfg->K = 100.0;
    cfg->T = 100;
    cfg->s = 32;
    cfg->ins_early_exit = 1;
    cfg->del_prune = 1;
    cfg->walk_mode = DG_WALK_BATCHED;
    cfg->slack = 1.25;
    cfg->overflow_frac = 0.5;
    cfg->hbm_budget_bytes = 0;
    cfg->autotune = 1;
    cfg->timeout_ms = 60000;
    cfg->use_cuda_graphs = 1;
    cfg->record_walkers = 0;
    cfg->device = 0;
}

const char* dg_status_str(dg_status st) {
    switch (st) {
        case DG_OK: return "ok";
        case DG_E_INVALID: return "invalid argument";
        case DG_E_NOMEM: return "out of device memory";
        case DG_E_CUDA: return "CUDA error";
        case DG_E_TIMEOUT: return "timeout";
        case DG_E_STATE: return "invalid state";
        case DG_E_BUSY: return "busy";
        default: return "unknown status";
    }
}

const char* dg_last_error(void) { return t_last_error.c_str(); }

dg_status dg_create(const dg_config* cfg_in, dg_ctx** out) {
    return guarded(nullptr, [&]() {
        if (!out) throw Error(DG_E_INVALID, "null output pointer");
        dg_config cfg;
        if (cfg_in) cfg = *cfg_in;
        else dg_config_default(&cfg);
        if (cfg.T < 1 || cfg.T > 65535) throw Error(DG_E_INVALID, "T must be in 1..65535");
        if (cfg.s < 1 || cfg.s > 1024) throw Error(DG_E_INVALID, "s must be in 1..1024");
        if (!(cfg.K >= 0.0)) throw Error(DG_E_INVALID, "K must be >= 0");
        if (!(cfg.slack >= 1.0) || !(cfg.overflow_frac >= 0.0)) throw Error(DG_E_INVALID, "bad slack / overflow");
        if (cfg.walk_mode != DG_WALK_BATCHED && cfg.walk_mode != DG_WALK_PER_UPDATE)
            throw Error(DG_E_INVALID, "bad walk_mode");
        if ((cfg.alloc == nullptr) != (cfg.free == nullptr)) throw Error(DG_E_INVALID, "alloc and free go together");
        int ndev = 0;
        DG_CUDA(cudaGetDeviceCount(&ndev));
        if (cfg.device < 0 || cfg.device >= ndev) throw Error(DG_E_INVALID, "bad device ordinal");
        DG_CUDA(cudaSetDevice(cfg.device));
        if (!cfg.alloc) {
            // batch workspaces come and go through the stream-ordered allocator:
            // keep freed blocks in this process's pool instead of returning them
            // to the driver at every synchronization (a later batch would pay
            // for mapping them again)
            cudaMemPool_t pool = nullptr;
            if (cudaDeviceGetDefaultMemPool(&pool, cfg.device) == cudaSuccess && pool) {
                uint64_t keep = ~0ull;
                cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
            }
            cudaGetLastError();
        }
        // optional L2 fetch granularity hint for this process's context (bytes;
        // a walk step reads one 32-byte sector, so larger fetches waste DRAM bandwidth)
        if (const char* f = std::getenv("DG_L2_FETCH")) {
            const long v = std::strtol(f, nullptr, 10);
            if (v == 0 || v == 32 || v == 64 || v == 128) DG_CUDA(cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, (size_t)v));
        }
        // optional persisting-L2 set-aside (MB) for the sparsifier during walks
        if (const char* f = std::getenv("DG_L2_PERSIST_MB")) {
            const long mb = std::strtol(f, nullptr, 10);
            int max_persist = 0, max_win = 0;
            cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, cfg.device);
            cudaDeviceGetAttribute(&max_win, cudaDevAttrMaxAccessPolicyWindowSize, cfg.device);
            size_t want = mb > 0 ? (size_t)mb << 20 : 0;
            if (want > (size_t)max_persist) want = (size_t)max_persist;
            if (want > 0 && max_win > 0) {
                DG_CUDA(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want));
                walk_set_l2_persist(want, (size_t)max_win);
            }
        }
        auto c = std::make_unique<Ctx>();
        c->device = cfg.device;
        c->cfg.seed = cfg.seed;
        c->cfg.K = cfg.K;
        c->cfg.T = cfg.T;
        c->cfg.s = cfg.s;
        c->cfg.early_exit = cfg.ins_early_exit ? 1 : 0;
        c->cfg.del_prune = cfg.del_prune ? 1 : 0;
        c->cfg.walk_mode = cfg.walk_mode;
        c->cfg.slack = cfg.slack;
        c->cfg.overflow = cfg.overflow_frac;
        c->cfg.budget = cfg.hbm_budget_bytes;
        c->cfg.autotune = cfg.autotune;
        c->cfg.timeout_ms = cfg.timeout_ms > 0 ? cfg.timeout_ms : 60000;
        c->cfg.use_graphs = cfg.use_cuda_graphs;
        c->cfg.record = cfg.record_walkers;
        c->alloc.fn_alloc = cfg.alloc;
        c->alloc.fn_free = cfg.free;
        c->alloc.user = cfg.alloc_user;
        DG_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        *out = reinterpret_cast<dg_ctx*>(c.release());
    });
}

dg_status dg_destroy(dg_ctx* ctx) {
    if (!ctx) return DG_OK;
    return guarded(ctx, [&]() {
        Ctx* c = reinterpret_cast<Ctx*>(ctx);
        {
            std::lock_guard<std::mutex> lk(c->smu);
            c->stopping = true;
        }
        c->scv.notify_all();
        for (auto& t : c->workers) t.join();
        c->workers.clear();
        for (auto& kv : c->graphs) graph_release(*c, *kv.second);
        c->graphs.clear();
        cudaStreamSynchronize(c->stream);
        cudaStreamDestroy(c->stream);
        delete c;
    });
}

dg_status dg_load_graph(dg_ctx* ctx, int32_t n, int64_t m, const int32_t* u, const int32_t* v, const double* w,
                        int32_t* graph_id_out) {
    return guarded(ctx, [&]() {
        Ctx& c = C(ctx);
        if (!graph_id_out) throw Error(DG_E_INVALID, "null graph id pointer");
        if (m > 0 && (!u || !v || !w)) throw Error(DG_E_INVALID, "null edge arrays");
        auto g = std::make_unique<DGraph>();
        try {
            graph_load(c, *g, n, m, u, v, w);
        } catch (...) {
            graph_release(c, *g);
            throw;
        }
        std::lock_guard<std::mutex> lk(c.mu);
        g->id = c.next_gid++;
        *graph_id_out = g->id;
        c.graphs[g->id] = std::move(g);
    });
}

dg_status dg_unload_graph(dg_ctx* ctx, int32_t gid) {
    return guarded(ctx, [&]() {
        Ctx& c = C(ctx);
        std::unique_ptr<DGraph> g;
        {
            std::lock_guard<std::mutex> sl(c.smu);  // lock order: smu before mu
            std::lock_guard<std::mutex> lk(c.mu);
            auto it = c.graphs.find(gid);
            if (it == c.graphs.end()) throw Error(DG_E_INVALID, "unknown graph id");
            if (c.busy[gid]) throw Error(DG_E_BUSY, "graph has a request in flight");
            for (auto& r : c.queue)
                if (r->gid == gid) throw Error(DG_E_BUSY, "graph has queued requests");
            g = std::move(it->second);
            c.graphs.erase(it);
        }
        graph_release(c, *g);
    });
}

dg_status dg_init_sparsifier(dg_ctx* ctx, int32_t gid, int64_t mh, const int32_t* u, const int32_t* v) {
    return guarded(ctx, [&]() {
        Ctx& c = C(ctx);
        DGraph& g = c.graph(gid);
        if (mh > 0 && (!u || !v)) throw Error(DG_E_INVALID, "null edge arrays");
        std::lock_guard<std::mutex> lk(g.mu);
        graph_init_h(c, g, mh, u, v);
    });
}

dg_status dg_apply_updates(dg_ctx* ctx, int32_t gid, int64_t nu, const dg_update* ups, dg_update_result* res,
                           void* stream) {
    return guarded(ctx, [&]() {
        Ctx& c = C(ctx);
        DGraph& g = c.graph(gid);
        if (nu > 0 && !ups) throw Error(DG_E_INVALID, "null update array");
        std::lock_guard<std::mutex> lk(g.mu);
        graph_apply(c, g, nu, ups, res, false, stream ? (cudaStream_t)stream : c.stream);
    });
}

dg_status dg_apply_updates_device(dg_ctx* ctx, int32_t gid, int64_t nu, const dg_update* d_ups,
                                  dg_update_result* d_res, void* stream) {
    return guarded(ctx, [&]() {
        Ctx& c = C(ctx);
        DGraph& g = c.graph(gid);
        if (nu > 0 && !d_ups) throw Error(DG_E_INVALID, "null update array");
        std::lock_guard<std::mutex> lk(g.mu);
        graph_apply(c, g, nu, d_ups, d_res, true, stream ? (cudaStream_t)stream : c.stream);
    });
}

dg_status dg_query_sparsifier(dg_ctx* ctx, int32_t gid, int64_t cap, int32_t* u, int32_t* v, double* w,
                              int64_t* count_out) {
    return guarded(ctx, [&]() {
        Ctx& c = C(ctx);
        DGraph& g = c.graph(gid);
        std::lock_guard<std::mutex> lk(g.mu);
        graph_export(c, g, true, cap, u, v, w, count_out, c.stream);
    });
}

dg_status dg_query_graph(dg_ctx* ctx, int32_t gid, int64_t cap, int32_t* u, int32_t* v, double* w,
                         int64_t* count_out) {
    return guarded(ctx, [&]() {
        Ctx& c = C(ctx);
        DGraph& g = c.graph(gid);
        std::lock_guard<std::mutex> lk(g.mu);
        graph_export(c, g, false, cap, u, v, w, count_out, c.stream);
    });
}

dg_status dg_get_batch_stats(dg_ctx* ctx, int32_t gid, dg_batch_stats* out) {
    return guarded(ctx, [&]() {
        Ctx& c = C(ctx);
        if (!out) throw Error(DG_E_INVALID, "null output");
        DGraph& g = c.graph(gid);
        std::lock_guard<std::mutex> lk(g.mu);
        *out = g.stats;
        // counted now (one pass over each graph's degrees): the current G and H,
        // i.e. after the last batch
        out->g_edges = (int64_t)csr_edge_count(g.G, c.alloc, c.stream);
        out->h_edges = g.has_h ? (int64_t)csr_edge_count(g.H, c.alloc, c.stream) : 0;
    });
}

dg_status dg_get_walker_records(dg_ctx* ctx, int32_t gid, int64_t cap, int32_t* reason, int32_t* steps,
                                int32_t* paths) {
    return guarded(ctx, [&]() {
        Ctx& c = C(ctx);
        DGraph& g = c.graph(gid);
        std::lock_guard<std::mutex> lk(g.mu);
        if (!c.cfg.record || !g.ws.dbg_reason.p) throw Error(DG_E_STATE, "record_walkers is off");
        const int64_t nu = g.stats.updates;
        if (cap < nu) throw Error(DG_E_INVALID, "cap smaller than the last batch");
        const size_t rows = (size_t)nu * c.cfg.s;
        const int s = c.cfg.s;
        // walked updates of the batch (task order): rows of the others read 0
        const size_t W = g.hs.counts[0];
        std::vector<uint32_t> idx(W);
        if (W) DG_CUDA(cudaMemcpy(idx.data(), g.ws.t_idx.p, W * 4, cudaMemcpyDeviceToHost));
        std::vector<uint8_t> walked((size_t)nu, 0);
        for (size_t j = 0; j < W; ++j) walked[idx[j]] = 1;
        auto blank_unwalked = [&](int32_t* a) {
            for (int64_t i = 0; i < nu; ++i)
                if (!walked[(size_t)i]) std::fill(a + (size_t)i * s, a + (size_t)(i + 1) * s, 0);
        };
        if (reason) {
            DG_CUDA(cudaMemcpy(reason, g.ws.dbg_reason.p, rows * 4, cudaMemcpyDeviceToHost));
            blank_unwalked(reason);
        }
        if (steps) {
            DG_CUDA(cudaMemcpy(steps, g.ws.dbg_steps.p, rows * 4, cudaMemcpyDeviceToHost));
            blank_unwalked(steps);
        }
        if (paths) {
            if (!g.ws.dbg_paths.p) throw Error(DG_E_STATE, "paths are kept only when T <= 256");
            // paths are stored per walked update (task order); re-order by update index.
            // A walker's row holds the vertices it reached; positions past its
            // reported step count (after an early-exit or pruning cut) read -1.
            const size_t row = (size_t)c.cfg.T + 1;
            std::vector<int32_t> buf(W * s * row);
            if (W) DG_CUDA(cudaMemcpy(buf.data(), g.ws.dbg_paths.p, buf.size() * 4, cudaMemcpyDeviceToHost));
            std::vector<int32_t> wsteps(rows);
            if (rows) DG_CUDA(cudaMemcpy(wsteps.data(), g.ws.dbg_steps.p, rows * 4, cudaMemcpyDeviceToHost));
            std::fill(paths, paths + rows * row, -1);
            for (size_t j = 0; j < W; ++j)
                for (int k = 0; k < s; ++k) {
                    const size_t src = (j * s + k) * row, dst = ((size_t)idx[j] * s + k) * row;
                    const size_t len = std::min<size_t>(row, (size_t)wsteps[(size_t)idx[j] * s + k] + 1);
                    std::copy(buf.begin() + src, buf.begin() + src + len, paths + dst);
                }
        }
    });
}

dg_status dg_compact(dg_ctx* ctx, int32_t gid) {
    return guarded(ctx, [&]() {
        Ctx& c = C(ctx);
        DGraph& g = c.graph(gid);
        std::lock_guard<std::mutex> lk(g.mu);
        graph_compact(c, g, c.stream);
    });
}

dg_status dg_graph_bytes(dg_ctx* ctx, int32_t gid, uint64_t* bytes_out) {
    return guarded(ctx, [&]() {
        Ctx& c = C(ctx);
        if (!bytes_out) throw Error(DG_E_INVALID, "null output");
        DGraph& g = c.graph(gid);
        *bytes_out = g.G.bytes() + g.H.bytes();
    });
}

uint64_t dg_launch_count(dg_ctx* ctx) {
    if (!ctx) return 0;
    return reinterpret_cast<Ctx*>(ctx)->launches.load();
}

dg_status dg_set_next_update_id(dg_ctx* ctx, int32_t gid, uint64_t next_id) {
    return guarded(ctx, [&]() {
        DGraph& g = C(ctx).graph(gid);
        std::lock_guard<std::mutex> lk(g.mu);
        g.next_id = next_id;
    });
}

dg_status dg_get_next_update_id(dg_ctx* ctx, int32_t gid, uint64_t* next_id) {
    return guarded(ctx, [&]() {
        if (!next_id) throw Error(DG_E_INVALID, "null output");
        DGraph& g = C(ctx).graph(gid);
        std::lock_guard<std::mutex> lk(g.mu);
        *next_id = g.next_id;
    });
}

dg_status dg_set_walk_shape(dg_ctx* ctx, int32_t gid, int32_t block, int32_t ilp, int32_t blocks_per_sm) {
    return guarded(ctx, [&]() {
        DGraph& g = C(ctx).graph(gid);
        std::lock_guard<std::mutex> lk(g.mu);
        if (block) {
            if (block % 32 || block < 32 || block > 256) throw Error(DG_E_INVALID, "block must be 32..256, x32");
            g.shape.block = block;
        }
        if (ilp) {
            if (ilp != 1 && ilp != 2 && ilp != 4) throw Error(DG_E_INVALID, "ilp must be 1, 2 or 4");
            g.shape.ilp = ilp;
        }
        if (blocks_per_sm) {
            if (blocks_per_sm < 0 || blocks_per_sm > 64) throw Error(DG_E_INVALID, "bad blocks_per_sm");
            g.shape.blocks_per_sm = blocks_per_sm;
        }
        g.tuned = true;
        ++g.layout_gen;
    });
}

dg_status dg_set_walk_refill(dg_ctx* ctx, int32_t gid, int32_t refill_min) {
    return guarded(ctx, [&]() {
        DGraph& g = C(ctx).graph(gid);
        std::lock_guard<std::mutex> lk(g.mu);
        if (refill_min < 1 || refill_min > 32) throw Error(DG_E_INVALID, "refill_min must be 1..32");
        g.shape.refill = refill_min;
        g.tuned = true;
        ++g.layout_gen;
    });
}

dg_status dg_set_walk_coop(dg_ctx* ctx, int32_t gid, int32_t lanes, int32_t tile) {
    return guarded(ctx, [&]() {
        DGraph& g = C(ctx).graph(gid);
        std::lock_guard<std::mutex> lk(g.mu);
        if (lanes != 1 && lanes != 2 && lanes != 4 && lanes != 8 && lanes != 32)
            throw Error(DG_E_INVALID, "lanes must be 1, 2, 4, 8 or 32");
        if (tile < 0 || tile > 16) throw Error(DG_E_INVALID, "tile must be 0..16");
        g.shape.lanes = lanes;
        g.shape.tile = tile;
        g.tuned = true;
        ++g.layout_gen;
    });
}

dg_status dg_get_tune_log(dg_ctx* ctx, int32_t gid, int64_t cap, int32_t* shapes, float* ms, int64_t* count_out) {
    return guarded(ctx, [&]() {
        DGraph& g = C(ctx).graph(gid);
        std::lock_guard<std::mutex> lk(g.mu);
        const int64_t n = (int64_t)g.tune_log.size();
        if (count_out) *count_out = n;
        if (n > cap || (n && (!shapes || !ms))) throw Error(DG_E_INVALID, "output arrays too small");
        for (int64_t i = 0; i < n; ++i) {
            const WalkShape& sh = g.tune_log[i].first;
            const int32_t v[6] = {sh.block, sh.ilp, sh.refill, sh.lanes, sh.tile, sh.cut};
            for (int q = 0; q < 6; ++q) shapes[6 * i + q] = v[q];
            ms[i] = g.tune_log[i].second;
        }
    });
}

dg_status dg_shard_begin(dg_ctx* ctx, int32_t gid, int64_t nu, const dg_update* ups, int32_t rank, int32_t world,
                         void* stream, uint64_t* nrec_out) {
    return guarded(ctx, [&]() {
        Ctx& c = C(ctx);
        DGraph& g = c.graph(gid);
        std::lock_guard<std::mutex> lk(g.mu);
        graph_shard_begin(c, g, nu, ups, rank, world, stream ? (cudaStream_t)stream : c.stream, nrec_out);
    });
}

dg_status dg_shard_export(dg_ctx* ctx, int32_t gid, void* recs, uint64_t cap, uint64_t* nrec_out) {
    return guarded(ctx, [&]() {
        Ctx& c = C(ctx);
        DGraph& g = c.graph(gid);
        std::lock_guard<std::mutex> lk(g.mu);
        graph_shard_export(c, g, static_cast<ShardRec*>(recs), cap, nrec_out);
    });
}

dg_status dg_shard_commit(dg_ctx* ctx, int32_t gid, uint64_t nrec, const void* recs, dg_update_result* res) {
    return guarded(ctx, [&]() {
        Ctx& c = C(ctx);
        DGraph& g = c.graph(gid);
        std::lock_guard<std::mutex> lk(g.mu);
        graph_shard_commit(c, g, static_cast<const ShardRec*>(recs), nrec, res);
    });
}

dg_status dg_prepare(dg_ctx* ctx, int32_t gid, int64_t max_batch) {
    return guarded(ctx, [&]() {
        Ctx& c = C(ctx);
        DGraph& g = c.graph(gid);
        std::lock_guard<std::mutex> lk(g.mu);
        graph_prepare(c, g, max_batch, c.stream);
    });
}

dg_status dg_debug_set_wait_limit(dg_ctx* ctx, int64_t polls) {
    return guarded(ctx, [&]() {
        Ctx& c = C(ctx);
        std::lock_guard<std::mutex> lk(c.mu);
        c.fin_wait_polls = polls < 0 ? -1 : polls;
        for (auto& kv : c.graphs) {  // captured steps hold the limit: capture them again
            std::lock_guard<std::mutex> gl(kv.second->mu);
            ++kv.second->layout_gen;
        }
    });
}

dg_status dg_submit_updates(dg_ctx* ctx, int32_t gid, int64_t nu, const dg_update* ups, dg_update_result* res,
                            uint64_t* ticket_out) {
    return guarded(ctx, [&]() {
        Ctx& c = C(ctx);
        if (!ticket_out) throw Error(DG_E_INVALID, "null ticket pointer");
        if (nu < 0 || (nu > 0 && !ups)) throw Error(DG_E_INVALID, "bad update array");
        c.graph(gid);  // must exist
        auto rq = std::make_shared<Request>();
        rq->gid = gid;
        rq->ups.assign(ups, ups + nu);
        rq->res = res;
        rq->need_bytes = request_bytes(c.cfg, (uint64_t)nu);
        if (c.cfg.budget) {
            uint64_t resident = 0;
            {
                std::lock_guard<std::mutex> lg(c.mu);
                for (auto& kv : c.graphs) resident += kv.second->G.bytes() + kv.second->H.bytes();
            }
            if (resident + rq->need_bytes > c.cfg.budget)
                throw Error(DG_E_NOMEM, "request can never fit the HBM budget");
        }
        ensure_workers(c);
        {
            std::lock_guard<std::mutex> lk(c.smu);
            rq->ticket = c.next_ticket++;
            rq->t_submit = now_ms();
            c.tickets[rq->ticket] = rq;
            c.queue.push_back(rq);
            *ticket_out = rq->ticket;
        }
        c.scv.notify_all();
    });
}

dg_status dg_wait(dg_ctx* ctx, uint64_t ticket, int32_t timeout_ms, double* latency_ms) {
    return dg_wait_ex(ctx, ticket, timeout_ms, latency_ms, nullptr);
}

dg_status dg_wait_ex(dg_ctx* ctx, uint64_t ticket, int32_t timeout_ms, double* latency_ms, double* queue_ms) {
    dg_status inner = DG_OK;
    dg_status outer = guarded(ctx, [&]() {
        Ctx& c = C(ctx);
        const int tmo = timeout_ms >= 0 ? timeout_ms : c.cfg.timeout_ms;
        std::unique_lock<std::mutex> lk(c.smu);
        auto it = c.tickets.find(ticket);
        if (it == c.tickets.end()) throw Error(DG_E_INVALID, "unknown ticket");
        auto rq = it->second;
        if (!c.dcv.wait_for(lk, std::chrono::milliseconds(tmo), [&] { return rq->done; }))
            throw Error(DG_E_TIMEOUT, "request not finished within timeout");
        if (latency_ms) *latency_ms = rq->t_done - rq->t_submit;
        if (queue_ms) *queue_ms = (rq->t_start > 0.0 ? rq->t_start : rq->t_done) - rq->t_submit;
        inner = rq->status;
        if (inner != DG_OK) t_last_error = rq->error;
        c.tickets.erase(it);
    });
    return outer != DG_OK ? outer : inner;
}

}  // extern "C"
