// dg_seq.cu -- sequential semantics on top of the batched step.
//
// Algorithm 1 applies the updates of the stream one at a time: every update
// walks the G and H its predecessors left.  The batched step instead walks one
// snapshot per batch (the deferral of Section III-F).  This file gives the
// one-at-a-time results at batch speed where the updates do not interact: the
// stream is cut into prefixes whose batched execution provably equals the
// one-at-a-time execution, and each prefix runs as an ordinary batch.
//
// Why a prefix P is safe.  A walk reads the adjacency lists of the vertices
// it stands on, and nothing else.  Update x of P changes the lists of a known
// set of vertices: its endpoints in G (insert or delete), its endpoints in H
// (accepted insertion, deleted H edge) and, for a recovered deletion, the
// vertices of the recovered path in H.  If no walk of any update of P stands
// on a vertex that another update of P changes, every walk of the batch sees
// exactly the lists it would see one at a time (the batch's snapshot differs
// from the one-at-a-time state only at vertices other updates change), so
// every decision and every change is the same.
//
// Finding P.  A dry run walks every update of a window on the current state,
// with the same Philox counters and the same neighbour pick as the batched
// walk (a deletion's walk skips its own edge, which the batch has removed),
// records every walker's vertices, decides each update as the batch would
// (hit / accepted; argmin walker of a deletion) and lists each update's
// changed vertices.  With, per vertex, the two smallest update indices that
// change it (in G and in H), each walked vertex v of update j names the first
// other update x changing v; the pair (j, x) cannot both be in P, so
// P ends before max(j, x).  An update's status depends on its own edge only,
// and whether a deletion walks on that edge being in H, which another update
// changes only by recovering a path through both endpoints: a change to the
// H list of j's endpoint by another update x ends P before max(j, x) as
// well.  The prefix is cut further before the second occurrence of a
// repeated edge (whose status depends on the first) and after a deletion
// whose walkers all missed (its fallback edge is not known to the dry run).  A walker counts up to where the batch's walker stops: an
// insertion's walkers at its first hit's step, a deletion's once their
// resistance exceeds the least hit's (the batch reports exactly those counts,
// whatever its schedule).
#include <algorithm>
#include <vector>

#include "dg_ctx.h"

namespace dg {

namespace {

constexpr int ST = 256;
constexpr uint32_t SEQ_NONE = 0xFFFFFFFFu;
constexpr uint32_t SEQ_MAX_WINDOW = 4096;
constexpr uint32_t SEQ_MIN_WINDOW = 64;

int s_grid(uint64_t items) {
    const uint64_t b = (items + ST - 1) / ST;
    const uint64_t cap = (uint64_t)device_sms() * 8;
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(b, cap));
}

struct SeqArgs {
    CSRView G, H;
    const dg_update* ups;  // the window's updates
    uint32_t m;            // window size
    uint32_t s, T;
    double K;
    uint32_t key0, key1;
    uint32_t early_exit, del_prune;  // the batch's cuts (insertions) and pruning (deletions)
    uint64_t id0;          // update id of the window's first update
    uint8_t* kind;         // per update: WALK_NONE / WALK_INS / WALK_DEL
    uint8_t* valid;        // per update: the update changes G
    uint8_t* accepted;     // per walked insertion
    uint32_t* qslot;       // per deletion: position of v in u's G list
    uint32_t* best;        // per walked deletion: the argmin walker (SEQ_NONE: all missed)
    uint64_t* key;         // per update: canonical edge key
    uint32_t* paths;       // per walker: T + 1 vertices
    double* pathR;         // per walker: the resistance after each step
    uint32_t* lim;         // per walked insertion: the first hit's step (the batch cuts every walker there)
    uint32_t* kb;          // per walked update, during the dry run: the least hit step (insertion) or
                           // the high word of the least hit resistance (deletion) found so far
    double* rbar;          // per walked deletion: the least hit resistance (the batch prunes beyond it)
    uint32_t* wsteps;      // per walker
    uint8_t* whit;
    uint8_t* wleaf;        // per walker: it stopped at a vertex with no neighbour to go to
    double* wR;
    uint32_t* g1;          // per vertex: smallest update index changing its G list
    uint32_t* g2;          // ... the second smallest
    uint32_t* h1;          // the same for H
    uint32_t* h2;
    uint32_t* cut;         // the prefix length (atomicMin)
};

// status and walk kind of every update against the current G and H
__global__ void k_seq_classify(SeqArgs a) {
    const uint32_t n = (uint32_t)a.G.n;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < a.m; j += gridDim.x * blockDim.x) {
        const dg_update up = a.ups[j];
        uint8_t kind = WALK_NONE, valid = 0;
        uint32_t qs = SEQ_NONE;
        uint64_t key = ~0ull;
        const bool in_range = up.u >= 0 && up.v >= 0 && (uint32_t)up.u < n && (uint32_t)up.v < n;
        if (in_range && up.u != up.v) {
            const uint32_t u = (uint32_t)up.u, v = (uint32_t)up.v;
            key = ((uint64_t)min(u, v) << 32) | max(u, v);
            const bool in_g = has_edge(a.G, u, v);
            if (up.op == DG_OP_INSERT) {
                if (!in_g && isfinite(up.w) && up.w > 0.0) {
                    valid = 1;
                    kind = WALK_INS;
                }
            } else if (up.op == DG_OP_DELETE) {
                if (in_g) {
                    valid = 1;
                    if (has_edge(a.H, u, v)) {
                        kind = WALK_DEL;
                        qs = find_nbr(a.G, u, v);
                    }
                }
            }
        }
        a.kind[j] = kind;
        a.valid[j] = valid;
        a.qslot[j] = qs;
        a.key[j] = key;
        a.best[j] = SEQ_NONE;
        a.accepted[j] = 0;
        a.kb[j] = SEQ_NONE;
    }
}

// the second occurrence of an edge ends the prefix before it
__global__ void k_seq_repeats(SeqArgs a) {
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < a.m; j += gridDim.x * blockDim.x) {
        const uint64_t k = a.key[j];
        if (k == ~0ull) continue;
        for (uint32_t i = 0; i < j; ++i)
            if (a.key[i] == k) {
                atomicMin(a.cut, j);
                break;
            }
    }
}

// one thread per walker: the walk the batch would run, every vertex recorded.
// A walker may stop as soon as the batch's own cut of its update is certain
// to end it (the same rules as the batched walk): an insertion's walker once a
// walker of its update hit at a step no later than its own, a deletion's once
// its resistance is above a hit of its update.  Every vertex the batch's
// walker reads is recorded all the same (the conflict test stops at the
// update's least hit, which such a bound never undercuts), and the hits
// that decide the update are unchanged.  The Philox word of the next step is
// formed while the entry load is in flight.
__device__ __forceinline__ uint32_t seq_r_key(double R) {
    return (uint32_t)((unsigned long long)__double_as_longlong(R) >> 32);
}

__global__ void k_seq_walk(SeqArgs a) {
    const uint32_t total = a.m * a.s;
    for (uint32_t wid = blockIdx.x * blockDim.x + threadIdx.x; wid < total; wid += gridDim.x * blockDim.x) {
        const uint32_t j = wid / a.s, k = wid - j * a.s;
        const uint8_t kind = a.kind[j];
        uint32_t* path = a.paths + (size_t)wid * (a.T + 1);
        if (kind != WALK_INS && kind != WALK_DEL) {
            a.wsteps[wid] = 0;
            a.whit[wid] = 0;
            a.wleaf[wid] = 0;
            a.wR[wid] = 0.0;
            continue;
        }
        const bool ins = kind == WALK_INS;
        const bool cut = ins ? a.early_exit != 0 : a.del_prune != 0;
        const CSRView& g = ins ? a.H : a.G;
        const dg_update up = a.ups[j];
        const uint32_t u = (uint32_t)up.u, q = (uint32_t)up.v;
        const uint64_t id = a.id0 + j;
        const uint32_t own = ins ? SEQ_NONE : a.qslot[j];
        uint32_t c = u, prev_slot = SEQ_NONE, steps = 0;
        // after arriving at a hub the previous vertex p is known by id only,
        // with a hint of its slot (the reference's, possibly drifted)
        bool pid = false;
        uint32_t p = SEQ_NONE, hint = 0;
        double R = 0.0;
        bool hit = false, leaf = false;
        path[0] = u;
        uint32_t off = g.off[u], deg = g.deg[u];
        uint32_t x = philox_word0(0u, k, (uint32_t)id, (uint32_t)(id >> 32), a.key0, a.key1);
        for (;;) {
            if (pid && c == u && own != SEQ_NONE) {  // two skips, one of them by id: find its slot
                prev_slot = find_nbr(g, c, p);
                pid = false;
            }
            Ent e;
            if (pid) {
                // the jj-th neighbour other than p is L[jj] when L[jj] < p and
                // L[jj + 1] otherwise; the hint picks which to load first
                if (deg <= 1) {
                    leaf = true;
                    break;
                }
                const uint32_t jj = __umulhi(x, deg - 1);
                uint32_t idx = jj + (jj >= hint ? 1u : 0u);
                e = g.pool[off + idx];
                if (idx == jj ? !(e.nbr < p) : !(e.nbr > p)) {
                    idx = idx == jj ? jj + 1u : jj;
                    e = g.pool[off + idx];
                }
            } else {
                // skipped positions: the previous vertex and, at u, a deletion's own edge
                uint32_t e1 = prev_slot, e2 = c == u ? own : SEQ_NONE;
                if (e1 > e2) {
                    const uint32_t t = e1;
                    e1 = e2;
                    e2 = t;
                }
                const uint32_t skip = (e1 != SEQ_NONE) + (e2 != SEQ_NONE);
                if (deg <= skip) {  // a leaf: no neighbour to go to
                    leaf = true;
                    break;
                }
                uint32_t idx = __umulhi(x, deg - skip);  // the idx-th allowed neighbour in list order
                if (idx >= e1) ++idx;
                if (idx >= e2) ++idx;
                e = g.pool[off + idx];
            }
            x = philox_word0(steps + 1u, k, (uint32_t)id, (uint32_t)(id >> 32), a.key0, a.key1);
            const uint32_t nx = e.nbr;
            R = __dadd_rn(R, e.r);
            ++steps;
            path[steps] = nx;
            a.pathR[(size_t)wid * (a.T + 1) + steps] = R;
            if (nx == q && (!ins || __dmul_rn(up.w, R) <= a.K)) {
                hit = true;
                if (cut) atomicMin(&a.kb[j], ins ? steps : seq_r_key(R));
                break;
            }
            if (ins && __dmul_rn(up.w, R) > a.K) break;
            if (steps == a.T) break;
            if (cut) {
                const uint32_t b = __ldcg(&a.kb[j]);
                if (ins ? b <= steps : seq_r_key(R) > b) break;
            }
            // the next list and our slot in it: cached in the entry; a hub's from
            // the vertex arrays, our slot there known by id (and a hint)
            if (e.noff != HUBREF && e.ndeg != 0) {
                off = e.noff;
                deg = e.ndeg;
                prev_slot = e.rev;
                pid = false;
            } else if (e.noff == HUBREF) {
                off = g.off[nx];
                deg = g.deg[nx];
                pid = true;
                p = c;
                hint = e.rev;
            } else {  // an entry whose cache was never filled
                off = g.off[nx];
                deg = g.deg[nx];
                prev_slot = find_nbr(g, nx, c);
                pid = false;
            }
            c = nx;
        }
        a.wsteps[wid] = steps;
        a.whit[wid] = hit;
        a.wleaf[wid] = leaf;
        a.wR[wid] = R;
    }
}

// the batch's decision: an insertion is kept when no walker hit; a deletion
// recovers the path of its hit walker of least resistance (lowest index on
// ties), and one whose walkers all missed ends the prefix after it
__global__ void k_seq_decide(SeqArgs a) {
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < a.m; j += gridDim.x * blockDim.x) {
        const uint8_t kind = a.kind[j];
        if (kind == WALK_INS) {
            uint32_t first = SEQ_NONE;
            for (uint32_t k = 0; k < a.s; ++k)
                if (a.whit[j * a.s + k]) first = min(first, a.wsteps[j * a.s + k]);
            a.accepted[j] = first == SEQ_NONE;
            a.lim[j] = first;
        } else if (kind == WALK_DEL) {
            uint32_t best = SEQ_NONE;
            double bR = 0.0;
            for (uint32_t k = 0; k < a.s; ++k) {
                const uint32_t w = j * a.s + k;
                if (a.whit[w] && (best == SEQ_NONE || a.wR[w] < bR)) {
                    best = k;
                    bR = a.wR[w];
                }
            }
            a.best[j] = best;
            a.rbar[j] = best == SEQ_NONE ? INFINITY : bR;
            if (best == SEQ_NONE) atomicMin(a.cut, j + 1);
        }
    }
}

// the vertices whose lists update j changes; PASS 1 takes the smallest
// index per vertex, PASS 2 the second smallest
template <int PASS>
__device__ __forceinline__ void mark(uint32_t* t1, uint32_t* t2, uint32_t v, uint32_t j) {
    if (PASS == 1) atomicMin(&t1[v], j);
    else if (__ldcg(&t1[v]) != j) atomicMin(&t2[v], j);
}

template <int PASS>
__global__ void k_seq_edits(SeqArgs a) {
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < a.m; j += gridDim.x * blockDim.x) {
        if (!a.valid[j]) continue;
        const dg_update up = a.ups[j];
        const uint32_t u = (uint32_t)up.u, v = (uint32_t)up.v;
        mark<PASS>(a.g1, a.g2, u, j);
        mark<PASS>(a.g1, a.g2, v, j);
        const uint8_t kind = a.kind[j];
        if ((kind == WALK_INS && a.accepted[j]) || kind == WALK_DEL) {
            mark<PASS>(a.h1, a.h2, u, j);
            mark<PASS>(a.h1, a.h2, v, j);
        }
        if (kind == WALK_DEL && a.best[j] != SEQ_NONE) {
            const uint32_t w = j * a.s + a.best[j];
            const uint32_t* path = a.paths + (size_t)w * (a.T + 1);
            for (uint32_t i = 0; i <= a.wsteps[w]; ++i) mark<PASS>(a.h1, a.h2, path[i], j);
        }
    }
}

__device__ __forceinline__ uint32_t other(const uint32_t* t1, const uint32_t* t2, uint32_t v, uint32_t j) {
    const uint32_t x = t1[v];
    return x != j ? x : t2[v];
}

// every vertex a walker of update j stands on, and j's endpoints: the first
// other update changing it ends the prefix before max(j, that update).  A
// warp takes a walker: its lanes look at 32 steps of the path at once.
__global__ void k_seq_conflicts(SeqArgs a) {
    const uint32_t total = a.m * a.s;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; wid < total; wid += nwarps) {
        const uint32_t j = wid / a.s;
        const uint8_t kind = a.kind[j];
        if (kind != WALK_INS && kind != WALK_DEL) continue;
        const uint32_t* path = a.paths + (size_t)wid * (a.T + 1);
        const double* pR = a.pathR + (size_t)wid * (a.T + 1);
        // what the batch's walker reads: an insertion's walkers stop at the
        // first hit's step, a deletion's once their resistance exceeds the
        // least hit's (the vertex reached then is kept, its list unread)
        uint32_t steps = a.wsteps[wid];
        if (kind == WALK_INS && a.early_exit) steps = min(steps, a.lim[j]);
        const double rb = kind == WALK_DEL && a.del_prune ? a.rbar[j] : INFINITY;
        // A deletion walker reads the G list of every vertex it leaves, and of
        // the one it stops on only when it stops there for want of a neighbour:
        // its arrival at the target, its last step, or its arrival above R~
        // reads nothing of the vertex reached (the entry it came by holds it).
        const bool leaf = a.wleaf[wid] != 0 && steps == a.wsteps[wid];
        uint32_t first = SEQ_NONE;
        for (uint32_t base = 0; base <= steps; base += 32u) {
            const uint32_t i = base + lane;
            const bool in = i <= steps;
            const bool over = in && i > 0 && pR[i] > rb;
            const uint32_t om = __ballot_sync(0xffffffffu, over);
            const uint32_t last = om ? base + (uint32_t)(__ffs(om) - 1) : SEQ_NONE;  // included, then stop
            if (in && i <= last) {
                const uint32_t v = path[i];
                uint32_t x = other(a.h1, a.h2, v, j);
                const bool stop_here = om ? i == last : i == steps;
                if (kind == WALK_DEL && (!stop_here || (leaf && !om))) x = min(x, other(a.g1, a.g2, v, j));
                first = min(first, x);
            }
            if (om) break;
        }
        for (int o = 16; o > 0; o >>= 1) first = min(first, __shfl_xor_sync(0xffffffffu, first, o));
        if (lane == 0 && first != SEQ_NONE) atomicMin(a.cut, max(j, first));
    }
    // whether j's edge is in H (which decides whether a deletion walks) can be
    // changed by another update only through the H lists of j's endpoints (a
    // recovered path through them); G lists matter only where j's walks read
    // them, which the walker scan above covers
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < a.m; j += gridDim.x * blockDim.x) {
        if (!a.valid[j]) continue;
        const uint32_t u = (uint32_t)a.ups[j].u, v = (uint32_t)a.ups[j].v;
        const uint32_t x = min(other(a.h1, a.h2, u, j), other(a.h1, a.h2, v, j));
        if (x != SEQ_NONE) atomicMin(a.cut, max(j, x));
    }
}

struct SeqWS {
    uint32_t n = 0, wmax = 0, s = 0, T = 0;
    DBuf<uint8_t> kind, valid, accepted, whit, wleaf;
    DBuf<uint32_t> qslot, best, paths, wsteps, tabs, cut, lim, kb;
    DBuf<uint64_t> key;
    DBuf<double> wR, pathR, rbar;
    DBuf<dg_update> ups;
    DBuf<dg_update_result> res;
    void ensure(DevAlloc& a, uint32_t nv, uint32_t w, uint32_t ss, uint32_t TT, cudaStream_t st) {
        n = nv;
        wmax = w;
        s = ss;
        T = TT;
        const size_t nw = (size_t)w * ss;
        kind.ensure(a, w, st);
        valid.ensure(a, w, st);
        accepted.ensure(a, w, st);
        whit.ensure(a, nw, st);
        wleaf.ensure(a, nw, st);
        qslot.ensure(a, w, st);
        best.ensure(a, w, st);
        key.ensure(a, w, st);
        paths.ensure(a, nw * (TT + 1), st);
        pathR.ensure(a, nw * (TT + 1), st);
        lim.ensure(a, w, st);
        kb.ensure(a, w, st);
        rbar.ensure(a, w, st);
        wsteps.ensure(a, nw, st);
        wR.ensure(a, nw, st);
        tabs.ensure(a, 4ull * nv + 4, st);
        cut.ensure(a, 2, st);
    }
    void release(DevAlloc& a, cudaStream_t st) {
        for (auto* b : {&kind, &valid, &accepted, &whit, &wleaf}) b->release(a, st);
        for (auto* b : {&qslot, &best, &paths, &wsteps, &tabs, &cut, &lim, &kb}) b->release(a, st);
        key.release(a, st);
        for (auto* b : {&wR, &pathR, &rbar}) b->release(a, st);
        ups.release(a, st);
        res.release(a, st);
    }
};

}  // namespace

// the stream's updates one at a time, run as safe prefixes (see the top of the file)
void graph_apply_sequential(Ctx& c, DGraph& g, int64_t nu64, const dg_update* ups_h, dg_update_result* res_h,
                            int64_t* prefixes_out) {
    if (!g.has_h) throw Error(DG_E_STATE, "no sparsifier");
    if (g.shard.active) throw Error(DG_E_STATE, "a sharded batch is in progress on this graph");
    if (nu64 < 0 || nu64 > (1ll << 26)) throw Error(DG_E_INVALID, "stream length out of range");
    if (nu64 > 0 && !ups_h) throw Error(DG_E_INVALID, "null update array");
    if (prefixes_out) *prefixes_out = 0;
    if (nu64 == 0) return;
    const uint32_t nu = (uint32_t)nu64;
    cudaStream_t st = c.stream;
    DevAlloc& al = c.alloc;
    const uint32_t n = (uint32_t)g.n;
    const uint32_t S = (uint32_t)c.cfg.s, T = (uint32_t)c.cfg.T;
    SeqWS w;
    uint32_t a0 = 0;  // updates applied so far
    int64_t prefixes = 0;
    try {
        w.ensure(al, n, SEQ_MAX_WINDOW, S, T, st);
        w.ups.ensure(al, nu, st);
        w.res.ensure(al, nu, st);
        DG_CUDA(cudaMemcpyAsync(w.ups.p, ups_h, sizeof(dg_update) * nu, cudaMemcpyHostToDevice, st));
        uint32_t win = 256;
        while (a0 < nu) {
            const uint32_t m = std::min(win, nu - a0);
            graph_wait_estimates(g, st);
            SeqArgs A;
            A.G = g.G.view();
            A.H = g.H.view();
            A.ups = w.ups.p + a0;
            A.m = m;
            A.s = S;
            A.T = T;
            A.K = c.cfg.K;
            A.key0 = (uint32_t)c.cfg.seed;
            A.key1 = (uint32_t)(c.cfg.seed >> 32);
            A.early_exit = (uint32_t)c.cfg.early_exit;
            A.del_prune = (uint32_t)c.cfg.del_prune;
            A.id0 = g.next_id;
            A.kind = w.kind.p;
            A.valid = w.valid.p;
            A.accepted = w.accepted.p;
            A.qslot = w.qslot.p;
            A.best = w.best.p;
            A.key = w.key.p;
            A.paths = w.paths.p;
            A.pathR = w.pathR.p;
            A.lim = w.lim.p;
            A.kb = w.kb.p;
            A.rbar = w.rbar.p;
            A.wsteps = w.wsteps.p;
            A.whit = w.whit.p;
            A.wleaf = w.wleaf.p;
            A.wR = w.wR.p;
            A.g1 = w.tabs.p;
            A.g2 = w.tabs.p + n;
            A.h1 = w.tabs.p + 2ull * n;
            A.h2 = w.tabs.p + 3ull * n;
            A.cut = w.cut.p;
            DG_CUDA(cudaMemsetAsync(w.tabs.p, 0xFF, 16ull * n, st));
            DG_CUDA(cudaMemcpyAsync(w.cut.p, &m, 4, cudaMemcpyHostToDevice, st));
            k_seq_classify<<<s_grid(m), ST, 0, st>>>(A);
            k_seq_repeats<<<s_grid(m), ST, 0, st>>>(A);
            k_seq_walk<<<s_grid((uint64_t)m * S), ST, 0, st>>>(A);
            k_seq_decide<<<s_grid(m), ST, 0, st>>>(A);
            k_seq_edits<1><<<s_grid(m), ST, 0, st>>>(A);
            k_seq_edits<2><<<s_grid(m), ST, 0, st>>>(A);
            k_seq_conflicts<<<s_grid((uint64_t)m * S * 32), ST, 0, st>>>(A);
            g_launches += 7;
            uint32_t cnt = 0;
            DG_CUDA(cudaMemcpyAsync(&cnt, w.cut.p, 4, cudaMemcpyDeviceToHost, st));
            DG_CUDA(cudaStreamSynchronize(st));
            if (cnt == 0 || cnt > m) throw Error(DG_E_CUDA, "sequential prefix out of range");
            graph_apply(c, g, cnt, w.ups.p + a0, w.res.p + a0, true, st);
            a0 += cnt;
            ++prefixes;
            win = cnt == m ? std::min(SEQ_MAX_WINDOW, win * 2)
                           : std::max(SEQ_MIN_WINDOW, std::min(SEQ_MAX_WINDOW, 2 * cnt));
        }
        if (res_h)
            DG_CUDA(cudaMemcpyAsync(res_h, w.res.p, sizeof(dg_update_result) * nu, cudaMemcpyDeviceToHost, st));
        DG_CUDA(cudaStreamSynchronize(st));
        if (prefixes_out) *prefixes_out = prefixes;
    } catch (...) {
        // the prefixes already run stay applied: hand back their results
        cudaStreamSynchronize(st);
        if (res_h && a0 && w.res.p &&
            cudaMemcpy(res_h, w.res.p, sizeof(dg_update_result) * a0, cudaMemcpyDeviceToHost) != cudaSuccess)
            cudaGetLastError();
        if (prefixes_out) *prefixes_out = prefixes;
        w.release(al, st);
        throw;
    }
    w.release(al, st);
}

}  // namespace dg

using namespace dg;

extern "C" dg_status dg_apply_updates_sequential(dg_ctx* ctx, int32_t graph_id, int64_t nu, const dg_update* ups,
                                                 dg_update_result* res, int64_t* prefixes_out) {
    try {
        if (!ctx) throw Error(DG_E_INVALID, "null context");
        Ctx& c = *reinterpret_cast<Ctx*>(ctx);
        DG_CUDA(cudaSetDevice(c.device));
        DGraph& g = c.graph(graph_id);
        std::lock_guard<std::mutex> lk(g.mu);
        graph_apply_sequential(c, g, nu, ups, res, prefixes_out);
        return DG_OK;
    } catch (const Error& e) {
        set_last_error(e.what());
        return e.code;
    } catch (const std::bad_alloc&) {
        set_last_error("host allocation failed");
        return DG_E_NOMEM;
    } catch (const std::exception& e) {
        set_last_error(e.what());
        return DG_E_CUDA;
    }
}
