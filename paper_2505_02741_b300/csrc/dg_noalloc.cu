// dg_noalloc.cu -- dg_walk_estimate_noalloc: the walkers of a set of queries on
// a resident graph, with all scratch in one static device array, so that the
// call itself never allocates device memory.  It exists for callers that
// cannot allocate while they run (stream capture in progress, latency-critical
// threads, embedders whose device memory is already handed out).
//
// The walker step and the per-query reduction state the same rules as the
// batched walk kernels (Section III-B: non-backtracking pick, threshold K,
// step limit T, leaf stop; Eq. 12 minimum; early exit by step index).
#include <cmath>
#include <mutex>

#include "dg_ctx.h"

namespace dg {

namespace {

constexpr uint32_t NA_NONE = 0xFFFFFFFFu;
constexpr uint32_t NA_MAX_Q = DG_NOALLOC_MAX_QUERIES;
constexpr uint32_t NA_MAX_W = DG_NOALLOC_MAX_WALKERS;

// scratch layout: R[NA_MAX_W] f64 | meta[NA_MAX_W] u32 | kstar[NA_MAX_Q] u32 | next u64
constexpr size_t NA_OFF_R = 0;
constexpr size_t NA_OFF_META = NA_OFF_R + sizeof(double) * NA_MAX_W;
constexpr size_t NA_OFF_KSTAR = NA_OFF_META + sizeof(uint32_t) * NA_MAX_W;
constexpr size_t NA_OFF_NEXT = NA_OFF_KSTAR + sizeof(uint32_t) * NA_MAX_Q;
constexpr size_t NA_BYTES = NA_OFF_NEXT + 256;

static_assert(sizeof(dg_walk_query) == 32, "dg_walk_query is 32 bytes");
static_assert(sizeof(dg_walk_estimate) == 32, "dg_walk_estimate is 32 bytes");

}  // namespace

// the scratch every call shares (one per device that loads the library)
static __device__ __align__(256) unsigned char g_dg_noalloc_scratch[NA_BYTES];

// host side: device address of the array, looked up once per device
static std::mutex g_na_mu;
static void* g_na_addr[256] = {nullptr};

static void* noalloc_scratch_address(int device) {
    if (device < 0 || device >= 256) throw Error(DG_E_INVALID, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_dg_noalloc_scratch);
        if (e != cudaSuccess || !p)
            throw Error(DG_E_CUDA, std::string("cudaGetSymbolAddress of the static scratch: ") + cudaGetErrorString(e));
        g_na_addr[device] = p;
    }
    return g_na_addr[device];
}

struct NaArgs {
    CSRView H, G;
    const dg_walk_query* q;
    dg_walk_estimate* out;
    uint32_t nq;
    uint32_t s, T, early_exit;
    double K;
    uint32_t key0, key1;
    double* R;
    uint32_t* meta;
    uint32_t* kstar;
    unsigned long long* next;
};

__device__ __forceinline__ bool na_query_ok(const dg_walk_query& q, uint32_t n, int32_t* status) {
    int32_t st = ST_OK;
    if (q.kind != DG_OP_INSERT && q.kind != DG_OP_DELETE) st = ST_BAD_OP;
    else if (q.u < 0 || q.v < 0 || (uint32_t)q.u >= n || (uint32_t)q.v >= n) st = ST_BAD_VERTEX;
    else if (q.u == q.v) st = ST_SELF_LOOP;
    else if (q.kind == DG_OP_INSERT && !(isfinite(q.w) && q.w > 0.0)) st = ST_BAD_WEIGHT;
    if (status) *status = st;
    return st == ST_OK;
}

__global__ void k_na_init(NaArgs a) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.nq; i += gridDim.x * blockDim.x)
        a.kstar[i] = NA_NONE;
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.next = 0ull;
}

// one walker per thread, walkers handed out in order by a counter
__global__ void __launch_bounds__(256) k_na_walk(NaArgs a) {
    const uint32_t total = a.nq * a.s;
    const uint32_t n = (uint32_t)a.G.n;
    for (;;) {
        const unsigned long long id = atomicAdd(a.next, 1ull);
        if (id >= total) return;
        const uint32_t wid = (uint32_t)id;
        const uint32_t j = wid / a.s, k = wid - j * a.s;
        const dg_walk_query q = a.q[j];
        if (!na_query_ok(q, n, nullptr)) {
            a.meta[wid] = 0u | (4u << 16);
            a.R[wid] = 0.0;
            continue;
        }
        const bool ins = q.kind == DG_OP_INSERT;
        const CSRView& g = ins ? a.H : a.G;
        const uint32_t ulo = (uint32_t)q.id, uhi = (uint32_t)(q.id >> 32);
        uint32_t c = (uint32_t)q.u, off = g.off[c], deg = g.deg[c], prev = NA_NONE, steps = 0, reason = 0;
        bool pid = false;
        double R = 0.0;
        for (;;) {
            const uint32_t neff = deg - (prev != NA_NONE ? 1u : 0u);
            if (neff == 0) { reason = 4; break; }
            if (ins && a.early_exit && __ldcg(&a.kstar[j]) <= steps) { reason = 5; break; }
            const uint32_t x = philox_word0(steps, k, ulo, uhi, a.key0, a.key1);
            uint4 h;
            double2 tl;
            if (nb_step(g, x, c, off, deg, prev, pid, h, tl) <= 0) { reason = 4; break; }
            R = __dadd_rn(R, tl.x);
            steps += 1;
            if (c == (uint32_t)q.v && (!ins || __dmul_rn(q.w, R) <= a.K)) {
                if (ins && a.early_exit) atomicMin(&a.kstar[j], steps);
                reason = 1;
                break;
            }
            if (ins && __dmul_rn(q.w, R) > a.K) { reason = 2; break; }
            if (steps == a.T) { reason = 3; break; }
        }
        a.meta[wid] = steps | (reason << 16);
        a.R[wid] = R;
    }
}

// one warp per query: first hitting step, cut, minimum resistance (lowest walker on ties)
__global__ void k_na_reduce(NaArgs a) {
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t n = (uint32_t)a.G.n;
    for (uint32_t j = warp; j < a.nq; j += nwarps) {
        const dg_walk_query q = a.q[j];
        int32_t status = ST_OK;
        const bool ok = na_query_ok(q, n, &status);
        const bool ee = ok && q.kind == DG_OP_INSERT && a.early_exit;
        uint32_t ks = NA_NONE;
        if (ok)
            for (uint32_t k = lane; k < a.s; k += 32) {
                const uint32_t m = a.meta[(size_t)j * a.s + k];
                if ((m >> 16) == 1u) ks = min(ks, m & 0xFFFFu);
            }
        for (int o = 16; o > 0; o >>= 1) ks = min(ks, __shfl_xor_sync(0xffffffffu, ks, o));
        uint32_t nh = 0, tot = 0;
        double bR = INFINITY;
        int bk = -1;
        if (ok)
            for (uint32_t k = lane; k < a.s; k += 32) {
                const uint32_t m = a.meta[(size_t)j * a.s + k];
                uint32_t st = m & 0xFFFFu, rs = m >> 16;
                if (ee && ks != NA_NONE && st > ks) {
                    st = ks;
                    rs = 5;
                }
                tot += st;
                if (rs == 1u) {
                    ++nh;
                    const double R = a.R[(size_t)j * a.s + k];
                    if (bk < 0 || R < bR) {
                        bR = R;
                        bk = (int)k;
                    }
                }
            }
        for (int o = 16; o > 0; o >>= 1) {
            nh += __shfl_xor_sync(0xffffffffu, nh, o);
            tot += __shfl_xor_sync(0xffffffffu, tot, o);
            const double oR = __shfl_xor_sync(0xffffffffu, bR, o);
            const int ok2 = __shfl_xor_sync(0xffffffffu, bk, o);
            if (ok2 >= 0 && (bk < 0 || oR < bR || (oR == bR && ok2 < bk))) {
                bR = oR;
                bk = ok2;
            }
        }
        if (lane == 0) {
            dg_walk_estimate e;
            e.status = status;
            e.nhits = (int32_t)nh;
            e.best_walker = bk;
            e.steps = (int32_t)tot;
            e.r_est = nh > 0 ? bR : INFINITY;
            e.hit = nh > 0;
            for (int i = 0; i < 7; ++i) e.reserved[i] = 0;
            a.out[j] = e;
        }
    }
}

}  // namespace dg

using namespace dg;

extern "C" dg_status dg_walk_estimate_noalloc(dg_ctx* ctx, int32_t graph_id, int64_t nq,
                                              const dg_walk_query* d_queries, dg_walk_estimate* d_out,
                                              void* cuda_stream) {
    try {
        if (!ctx) throw Error(DG_E_INVALID, "null context");
        Ctx& c = *reinterpret_cast<Ctx*>(ctx);
        if (nq < 0) throw Error(DG_E_INVALID, "negative query count");
        if (nq > (int64_t)NA_MAX_Q)
            throw Error(DG_E_INVALID, "more queries than DG_NOALLOC_MAX_QUERIES (4096)");
        if (nq * (int64_t)c.cfg.s > (int64_t)NA_MAX_W)
            throw Error(DG_E_INVALID, "queries x walkers exceed DG_NOALLOC_MAX_WALKERS (131072)");
        if (nq > 0 && (!d_queries || !d_out)) throw Error(DG_E_INVALID, "null query or output pointer");
        DG_CUDA(cudaSetDevice(c.device));
        DGraph& g = c.graph(graph_id);
        std::lock_guard<std::mutex> lk(g.mu);
        if (!g.has_h) throw Error(DG_E_STATE, "no sparsifier");
        unsigned char* base = static_cast<unsigned char*>(noalloc_scratch_address(c.device));
        if (nq == 0) return DG_OK;
        NaArgs a;
        a.H = g.H.view();
        a.G = g.G.view();
        a.q = d_queries;
        a.out = d_out;
        a.nq = (uint32_t)nq;
        a.s = (uint32_t)c.cfg.s;
        a.T = (uint32_t)c.cfg.T;
        a.early_exit = c.cfg.early_exit ? 1u : 0u;
        a.K = c.cfg.K;
        a.key0 = (uint32_t)c.cfg.seed;
        a.key1 = (uint32_t)(c.cfg.seed >> 32);
        a.R = reinterpret_cast<double*>(base + NA_OFF_R);
        a.meta = reinterpret_cast<uint32_t*>(base + NA_OFF_META);
        a.kstar = reinterpret_cast<uint32_t*>(base + NA_OFF_KSTAR);
        a.next = reinterpret_cast<unsigned long long*>(base + NA_OFF_NEXT);
        cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : c.stream;
        // Outside a stream capture the call orders itself against changes of
        // this graph: its kernels wait for the last change of G or H, and the
        // next change waits for its kernels (events created with the graph).
        // During a capture the caller orders it (no event recorded outside the
        // capture is waited on).
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        DG_CUDA(cudaStreamIsCapturing(st, &cap));
        const bool ordered = cap == cudaStreamCaptureStatusNone;
        if (ordered) DG_CUDA(cudaStreamWaitEvent(st, g.ev_mut, 0));
        const int sms = device_sms();
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_na_walk, 256, 0);
        if (occ < 1) occ = 1;
        uint32_t walk_blocks = (uint32_t)(((uint64_t)a.nq * a.s + 255) / 256);
        if (walk_blocks > (uint32_t)(sms * occ)) walk_blocks = (uint32_t)(sms * occ);
        const uint32_t red_blocks = (a.nq + 7) / 8;
        k_na_init<<<(a.nq + 255) / 256, 256, 0, st>>>(a);
        k_na_walk<<<walk_blocks, 256, 0, st>>>(a);
        k_na_reduce<<<red_blocks, 256, 0, st>>>(a);
        DG_CHECK_LAUNCH();
        if (ordered) DG_CUDA(cudaEventRecord(g.ev_est, st));
        c.launches += 3;
        return DG_OK;
    } catch (const Error& e) {
        set_last_error(e.what());
        return e.code;
    } catch (const std::exception& e) {
        set_last_error(e.what());
        return DG_E_CUDA;
    }
}
