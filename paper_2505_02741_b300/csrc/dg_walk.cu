// dg_walk.cu -- NBRW walkers (Section III-B/C), per-update reduction (Eq. 12),
// path replay and fallback edges for deletions (Section III-C).
//
// Walker step (counter-based, so every walker's path is a pure function of
// (seed, update id, walker, graph snapshot)):
//   n_eff = deg(c) - [a previous vertex exists]; n_eff == 0 -> leaf stop
//   x     = Philox4x32-10((step, walker, lo32(id), hi32(id)), seed)[0]
//   j     = floor(x * n_eff / 2^32)                  (j-th allowed neighbour)
//   idx   = j + (j >= pos(prev))                     (skip the previous vertex;
//                                                    lists are sorted by id)
//   R    += r(c, L[idx]); step += 1
//   stop on: reaching v with (deletion or w_pq*R <= K) -> hit;
//            insertion and w_pq*R > K;  step == T.
// Optional cuts that leave every decision unchanged: an insertion's walkers
// stop at the first step index at which one of them hit (early exit); a
// deletion's walker stops once R exceeds the resistance of a hit already
// found for its update (pruning: it can no longer give the minimum of Eq. 12).
// Pruning compares the high 32 bits of the FP64 patterns (non-negative
// doubles order like their bit patterns), so a walker is cut only when its R
// is certainly above that hit's R; the walker at the minimum is never cut.
// The entry read at idx carries the next list's offset/degree and pos(prev)
// for the next step, so each step is one dependent 32-byte load.
#include <algorithm>
#include <cmath>

#include "dg_prims.cuh"
#include "dg_walk.cuh"

namespace dg {

static int g_sms = 0;
int device_sms() {
    if (g_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_sms <= 0) g_sms = 148;
    }
    return g_sms;
}

constexpr uint32_t NONE = 0xFFFFFFFFu;

__device__ __forceinline__ bool walk_aborted(const uint32_t* d_err) { return (*d_err & ABORT_MASK) != 0u; }

// GPU-scope acquire/release operations of the finalize hand-off: a walker's
// record stores are ordered before its count of the update (release), the last
// walker's count sees every other walker's records (acquire), its queue store
// publishes them (release, cumulative) and a worker's queue load acquires them.
__device__ __forceinline__ uint32_t atom_add_acq_rel(uint32_t* p, uint32_t v) {
    uint32_t old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// high 32 bits of a non-negative double (the pruning key)
__device__ __forceinline__ uint32_t r_key(double R) { return (uint32_t)((unsigned long long)__double_as_longlong(R) >> 32); }

struct Walker {
    uint32_t wid;    // absolute walker index j*s + k
    uint32_t j, k;
    uint32_t q;      // target
    uint32_t c, off, deg, prev;
    uint32_t steps;
    uint32_t ulo, uhi;
    double R, wpq;
    bool ins;
    bool active;
    bool pid;  // prev holds the previous vertex's id (arrived at a hub)
};

struct WalkKernelArgs {
    CSRView H, G;
    WalkTasks t;
    WalkParams p;
    WalkRecs r;
    const BatchHdr* hdr;
    unsigned long long* next;
    uint32_t j_lo, j_hi;
    uint32_t refill_min;  // empty slots a warp with walkers left waits for before refilling (1..32)
    uint32_t* d_err;
    FinArgs f;
};

// ---------------------------------------------------------------------------
// per-update finalization: device functions shared by the stand-alone kernels
// and by the finalizing warps of the batched walk.  Walker records written in
// the same launch are read through L2 (__ldcg), never from a stale L1 line.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void emit_edge(Cands& c, uint32_t x, uint32_t y, double w, uint32_t n,
                                          uint32_t* d_err) {
    const uint32_t pos = agg_add(c.count, 2u);
    if (pos + 2 > c.cap) {
        atomicOr(d_err, (uint32_t)ERR_CAP_COMMIT);
        return;
    }
    c.keys[pos] = (uint64_t)x * n + y;
    c.keys[pos + 1] = (uint64_t)y * n + x;
    c.vals[pos] = pos;
    c.vals[pos + 1] = pos + 1;
    c.w[pos] = w;
    c.w[pos + 1] = w;
}

struct UpdTotals {
    unsigned long long steps = 0, walked = 0, hits = 0, acc = 0, rec = 0;
};

__device__ __forceinline__ void add_totals(BatchCounters* ctr, const UpdTotals& u) {
    if (u.walked) {
        atomicAdd(&ctr->steps, u.steps);
        atomicAdd(&ctr->walked, u.walked);
    }
    if (u.hits) atomicAdd(&ctr->hits, u.hits);
    if (u.acc) atomicAdd(&ctr->accepted, u.acc);
    if (u.rec) atomicAdd(&ctr->recovered, u.rec);
}

// First step of deletion walker k of walked update j whose resistance exceeds
// rbar, the update's minimum (the walker's recorded resistance is above it, so
// that step exists): the exact pruned step count, whatever moment the walker
// itself was cut at.  With step records (pr non-null) the walker's own
// partial sums are searched: its last step first (a walker is usually cut at
// the step where it passes rbar), then a binary search (the sums increase).
// Without them the partial sums are formed again from its Philox counters on
// G_b, in walk order with one rounding per addition, as the walker did.  0 and
// ERR_INTERNAL if the sums never pass rbar (records inconsistent with the walk).
__device__ uint32_t del_cross_step(uint32_t j, uint32_t k, uint32_t steps, double rbar, const CSRView& G,
                                   const WalkTasks& t, const WalkParams& p, const double* pr, uint64_t id0,
                                   uint32_t* d_err) {
    if (pr) {
        // pr[base + q * s] = resistance after step q + 1; the one after step `steps` exceeds rbar
        const size_t base = (size_t)j * p.T * p.s + k;
        if (steps == 0 || !(__ldcg(&pr[base + (size_t)(steps - 1) * p.s]) > rbar)) {
            atomicOr(d_err, (uint32_t)ERR_INTERNAL);
            return 0;
        }
        if (steps == 1 || !(__ldcg(&pr[base + (size_t)(steps - 2) * p.s]) > rbar)) return steps;
        uint32_t lo = 0, hi = steps - 2;  // the first q with pr > rbar lies in [lo, hi]
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (__ldcg(&pr[base + (size_t)mid * p.s]) > rbar) hi = mid;
            else lo = mid + 1;
        }
        return lo + 1;
    }
    double R = 0.0;
    const uint64_t id = id0 + t.idx[j];
    const uint32_t ulo = (uint32_t)id, uhi = (uint32_t)(id >> 32);
    const uint32_t u = t.u[j];
    uint32_t cv = u, off = G.off[u], deg = G.deg[u], prev = NONE;
    bool pid = false;
    for (uint32_t s = 0; s < steps; ++s) {
        const uint32_t x = philox_word0(s, k, ulo, uhi, p.key0, p.key1);
        uint4 h;
        double2 tl;
        if (nb_step(G, x, cv, off, deg, prev, pid, h, tl) <= 0) break;
        R = __dadd_rn(R, tl.x);
        if (R > rbar) return s + 1;
    }
    atomicOr(d_err, (uint32_t)ERR_INTERNAL);
    return 0;
}

// Eq. 12 and the cut readings over the s records of walked update j, one
// warp.  Lane 0 writes the update's result and best[j] and adds to tot; every
// lane gets the argmin walker (-1 if none) and the number of hits.
//
// Deletion pruning (del_prune): a walker stops once its resistance is above a
// hit of its update, at a step that depends on when that hit became visible.
// The counts reported are those of the exact rule instead -- every walker
// stops at its first step whose resistance exceeds R~ (del_cross_step) -- so
// steps, nhits (the walkers at R~) and the debug records do not depend on
// scheduling; hit, R~, the argmin walker and the recovered path are the same
// with or without pruning.
__device__ int reduce_update(uint32_t j, int lane, const WalkTasks& t, const WalkParams& p, const WalkRecs& r,
                             dg_update_result* res, int32_t* best, int32_t* dbg_reason, int32_t* dbg_steps,
                             UpdTotals& tot, uint32_t& nh_out, const CSRView& G, const double* pr, uint64_t id0,
                             uint32_t* d_err) {
    const bool ins = t.kind[j] == WALK_INS;
    const bool ee = ins && p.early_exit;
    const uint32_t i = t.idx[j];
    const uint32_t* meta = r.meta + (size_t)j * p.s;
    const double* Rr = r.R + (size_t)j * p.s;
    uint32_t ks = NONE;
    for (uint32_t k = lane; k < p.s; k += 32) {
        const uint32_t m = __ldcg(&meta[k]);
        if ((m >> 16) == R_HIT) ks = min(ks, m & 0xFFFFu);
    }
    for (int o = 16; o > 0; o >>= 1) ks = min(ks, __shfl_xor_sync(0xffffffffu, ks, o));
    uint32_t nh = 0, nmin = 0;  // nmin: hits at the lane's minimum bR
    double bR = INFINITY;
    int bk = -1;
    for (uint32_t k = lane; k < p.s; k += 32) {
        const uint32_t m = __ldcg(&meta[k]);
        uint32_t st = m & 0xFFFFu, rs = m >> 16;
        if (ee && ks != NONE && st > ks) rs = R_CUT;
        if (rs == R_HIT) {
            ++nh;
            const double R = __ldcg(&Rr[k]);
            if (bk < 0 || R < bR) {  // k ascends per lane: first minimum keeps the lower index
                bR = R;
                bk = (int)k;
                nmin = 1;
            } else if (R == bR) {
                ++nmin;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        nh += __shfl_xor_sync(0xffffffffu, nh, o);
        const double oR = __shfl_xor_sync(0xffffffffu, bR, o);
        const int ok = __shfl_xor_sync(0xffffffffu, bk, o);
        const uint32_t on = __shfl_xor_sync(0xffffffffu, nmin, o);
        if (ok >= 0 && (bk < 0 || oR < bR)) {
            bR = oR;
            bk = ok;
            nmin = on;
        } else if (ok >= 0 && oR == bR) {
            bk = min(bk, ok);
            nmin += on;
        }
    }
    // pruned deletions with a hit: walkers whose resistance ends above R~ are
    // counted up to their first step above it (hits above R~ included)
    const bool prune = !ins && p.del_prune && bk >= 0;
    if (prune) nh = nmin;
    uint32_t tsum = 0;
    for (uint32_t k = lane; k < p.s; k += 32) {
        const uint32_t m = __ldcg(&meta[k]);
        uint32_t st = m & 0xFFFFu, rs = m >> 16;
        if (ee && ks != NONE && st > ks) {
            st = ks;
            rs = R_CUT;
        }
        if (prune && __ldcg(&Rr[k]) > bR) {
            st = del_cross_step(j, k, st, bR, G, t, p, pr, id0, d_err);
            rs = R_CUT;
        }
        tsum += st;
        if (dbg_reason) {
            dbg_reason[(size_t)i * p.s + k] = (int32_t)rs;
            dbg_steps[(size_t)i * p.s + k] = (int32_t)st;
        }
    }
    for (int o = 16; o > 0; o >>= 1) tsum += __shfl_xor_sync(0xffffffffu, tsum, o);
    if (lane == 0) {
        dg_update_result& o = res[i];
        o.hit = nh > 0;
        o.nhits = (int32_t)nh;
        o.best_walker = bk;
        o.steps = (int32_t)tsum;
        o.r_est = nh > 0 ? bR : INFINITY;
        o.accepted = ins && nh == 0;
        best[j] = bk;
        tot.steps += tsum;
        tot.walked += 1;
        tot.hits += nh > 0 ? 1 : 0;
        tot.acc += (ins && nh == 0) ? 1 : 0;
    }
    nh_out = nh;
    return bk;
}

// Replays walker b of walked deletion j on G_b (same counters on the same
// snapshot give the same path, Section III-C) and stores its vertices and edge
// weights; false (ERR_INTERNAL) if it does not reach v after the recorded steps.
__device__ bool replay_path(uint32_t j, int32_t b, const CSRView& G, const WalkTasks& t, const WalkParams& p,
                            const WalkRecs& r, uint64_t id0, const PathBufs& pb, uint32_t* d_err) {
    const uint32_t i = t.idx[j];
    const uint32_t u = t.u[j], v = t.v[j], n = (uint32_t)G.n;
    const uint32_t steps = __ldcg(&r.meta[(size_t)j * p.s + b]) & 0xFFFFu;
    if (steps > p.T) {  // records are written by this batch's walk; anything else is an internal error
        atomicOr(d_err, (uint32_t)ERR_INTERNAL);
        pb.len[j] = 0;
        return false;
    }
    const uint64_t id = id0 + i;
    const uint32_t ulo = (uint32_t)id, uhi = (uint32_t)(id >> 32);
    uint32_t* path = pb.v + (size_t)j * (p.T + 1);
    double* pw = pb.w + (size_t)j * p.T;
    uint32_t cv = u, off = G.off[u], deg = G.deg[u], prev = NONE, s = 0;
    bool pid = false;
    path[0] = u;
    for (; s < steps; ++s) {
        const uint32_t x = philox_word0(s, (uint32_t)b, ulo, uhi, p.key0, p.key1);
        uint4 h;
        double2 tl;
        if (nb_step(G, x, cv, off, deg, prev, pid, h, tl) <= 0 || cv >= n) break;
        path[s + 1] = cv;
        pw[s] = tl.y;
    }
    if (s != steps || cv != v) {  // a recorded hit must replay to v
        atomicOr(d_err, (uint32_t)ERR_INTERNAL);
        pb.len[j] = 0;
        return false;
    }
    pb.len[j] = steps;
    return true;
}

// The same replay split over the warp: lane q takes the steps after resume
// point q (q = 0: the start), so the chain of dependent loads is one spacing
// long instead of the whole path.  Returns the success flag (all lanes).
__device__ bool replay_path_warp(uint32_t j, int32_t b, int lane, const CSRView& G, const WalkTasks& t,
                                 const WalkParams& p, const WalkRecs& r, uint64_t id0, const PathBufs& pb,
                                 const FinArgs& f, uint32_t* d_err) {
    const uint32_t i = t.idx[j];
    const uint32_t u = t.u[j], v = t.v[j], n = (uint32_t)G.n;
    const uint32_t steps = __ldcg(&r.meta[(size_t)j * p.s + b]) & 0xFFFFu;
    bool ok = steps <= p.T;
    const uint64_t id = id0 + i;
    const uint32_t ulo = (uint32_t)id, uhi = (uint32_t)(id >> 32);
    uint32_t* path = pb.v + (size_t)j * (p.T + 1);
    double* pw = pb.w + (size_t)j * p.T;
    const uint32_t span = 1u << f.cp_shift;
    const uint32_t nseg = ok ? (steps + span - 1) >> f.cp_shift : 0u;
    if (lane == 0) path[0] = u;
    for (uint32_t q = lane; q < nseg; q += 32) {
        uint32_t cv = u, off = G.off[u], deg = G.deg[u], prev = NONE;
        bool pid = false;
        if (q > 0) {
            const uint4 st = __ldcg(&f.cp[((size_t)j * p.s + b) * f.ncp + q - 1]);
            cv = st.x;
            off = st.y;
            deg = st.z;
            prev = st.w & 0x7FFFFFFFu;
            pid = (st.w >> 31) != 0u;
        }
        const uint32_t s0 = q << f.cp_shift, s1 = min(steps, s0 + span);
        uint32_t s = s0;
        for (; s < s1; ++s) {
            const uint32_t x = philox_word0(s, (uint32_t)b, ulo, uhi, p.key0, p.key1);
            uint4 h;
            double2 tl;
            if (nb_step(G, x, cv, off, deg, prev, pid, h, tl) <= 0 || cv >= n) break;
            path[s + 1] = cv;
            pw[s] = tl.y;
        }
        if (s != s1 || (s1 == steps && cv != v)) ok = false;  // a recorded hit must replay to v
    }
    ok = __all_sync(0xffffffffu, ok);
    if (lane == 0) {
        if (!ok) atomicOr(d_err, (uint32_t)ERR_INTERNAL);
        pb.len[j] = ok ? steps : 0u;
    }
    __syncwarp();
    return ok;
}

// Membership in H of the edges (a[q], b[q]) for the q with on[q], each by
// binary search in the shorter endpoint list; the N searches advance in
// lockstep, so their loads overlap instead of forming N chains.
template <int N>
__device__ __forceinline__ void has_edges(const CSRView& g, const uint32_t* a, const uint32_t* b, const bool* on,
                                          bool* found) {
    uint32_t y[N], lo[N], hi[N], d[N];
    const Ent* L[N];
    uint32_t da[N], db[N];
#pragma unroll
    for (int q = 0; q < N; ++q) {
        da[q] = on[q] ? g.deg[a[q]] : 0u;
        db[q] = on[q] ? g.deg[b[q]] : 0u;
    }
#pragma unroll
    for (int q = 0; q < N; ++q) {
        const bool sw = db[q] < da[q];
        const uint32_t x = sw ? b[q] : a[q];
        y[q] = sw ? a[q] : b[q];
        d[q] = sw ? db[q] : da[q];
        L[q] = g.pool + (on[q] ? g.off[x] : 0u);
        lo[q] = 0;
        hi[q] = on[q] ? d[q] : 0u;
    }
    for (;;) {
        uint32_t v[N];
        bool any = false;
#pragma unroll
        for (int q = 0; q < N; ++q) {
            const bool act = lo[q] < hi[q];
            any |= act;
            v[q] = act ? L[q][(lo[q] + hi[q]) >> 1].nbr : 0u;
        }
        if (!any) break;
#pragma unroll
        for (int q = 0; q < N; ++q) {
            if (lo[q] < hi[q]) {
                const uint32_t mid = (lo[q] + hi[q]) >> 1;
                if (v[q] < y[q]) lo[q] = mid + 1; else hi[q] = mid;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < N; ++q) found[q] = on[q] && lo[q] < d[q] && L[q][lo[q]].nbr == y[q];
}

// The path of walker b of walked deletion j from its step records (vertex
// reached and entry taken at every step), one warp; the same vertices and
// weights a replay would produce, without its chain of dependent loads.
// Returns the success flag (all lanes).
__device__ bool path_from_records(uint32_t j, int32_t b, int lane, const CSRView& G, const WalkTasks& t,
                                  const WalkParams& p, const WalkRecs& r, const PathBufs& pb, const FinArgs& f,
                                  uint32_t* d_err) {
    const uint32_t u = t.u[j], v = t.v[j], n = (uint32_t)G.n;
    const uint32_t steps = __ldcg(&r.meta[(size_t)j * p.s + b]) & 0xFFFFu;
    bool ok = steps <= p.T;
    uint32_t* path = pb.v + (size_t)j * (p.T + 1);
    double* pw = pb.w + (size_t)j * p.T;
    if (lane == 0) path[0] = u;
    for (uint32_t q = lane; ok && q < steps; q += 32) {
        const size_t rec = ((size_t)j * p.T + q) * p.s + (uint32_t)b;
        const uint32_t e = __ldcg(&f.pe[rec]);
        if ((uint64_t)e >= G.pool_cap) {
            ok = false;
            break;
        }
        const uint32_t x = G.pool[e].nbr;
        if (x >= n) {
            ok = false;
            break;
        }
        path[q + 1] = x;
        pw[q] = G.pool[e].w;
        if (q + 1 == steps && x != v) ok = false;  // a recorded hit ends at v
    }
    ok = __all_sync(0xffffffffu, ok);
    if (lane == 0) {
        if (!ok) atomicOr(d_err, (uint32_t)ERR_INTERNAL);
        pb.len[j] = ok ? steps : 0u;
    }
    __syncwarp();
    return ok;
}

// Recovered edges of the replayed path of walked deletion j, one warp: every
// edge of the walk that did not appear earlier in it and is not in H'.  A
// path shorter than EMIT_SMEM is staged in the warp's shared buffer sbuf
// (nullable), so the scan for earlier copies of an edge reads no global
// memory, and a lane looks up EMIT_ILP of its edges in H' together.
// Returns the number emitted (all lanes).
constexpr uint32_t EMIT_SMEM = 256;  // path vertices a warp's shared buffer holds
constexpr int EMIT_ILP = 2;

__device__ uint32_t emit_path_warp(uint32_t j, int lane, const CSRView& H, const WalkParams& p, Cands& c,
                                   const PathBufs& pb, uint32_t* d_err, uint32_t* sbuf) {
    const uint32_t len = pb.len[j];
    const uint32_t* gpath = pb.v + (size_t)j * (p.T + 1);
    const bool staged = sbuf != nullptr && len < EMIT_SMEM;
    if (staged) {
        for (uint32_t s = lane; s <= len; s += 32) sbuf[s] = __ldcg(&gpath[s]);
        __syncwarp();
    }
    const uint32_t* path = staged ? sbuf : gpath;
    uint32_t cnt = 0;
    for (uint32_t s0 = 0; s0 < len; s0 += 32u * EMIT_ILP) {
        uint32_t x[EMIT_ILP], y[EMIT_ILP];
        bool cand[EMIT_ILP], inh[EMIT_ILP];
#pragma unroll
        for (int q = 0; q < EMIT_ILP; ++q) {
            const uint32_t s = s0 + 32u * q + lane;
            cand[q] = s < len;
            x[q] = cand[q] ? path[s] : 0u;
            y[q] = cand[q] ? path[s + 1] : 0u;
            for (uint32_t s2 = 0; s2 < s && cand[q]; ++s2) {
                const uint32_t a0 = path[s2], a1 = path[s2 + 1];
                if ((a0 == x[q] && a1 == y[q]) || (a0 == y[q] && a1 == x[q])) cand[q] = false;
            }
        }
        has_edges<EMIT_ILP>(H, x, y, cand, inh);
#pragma unroll
        for (int q = 0; q < EMIT_ILP; ++q) {
            if (cand[q] && !inh[q]) {
                emit_edge(c, x[q], y[q], pb.w[(size_t)j * p.T + s0 + 32u * q + lane], (uint32_t)H.n, d_err);
                ++cnt;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    return cnt;  // the shuffles above keep the buffer's readers ahead of its next writer
}

__device__ __forceinline__ unsigned long long* fb_nb(const PathBufs& pb) {
    return reinterpret_cast<unsigned long long*>(pb.fb_count + 2);
}

// Queue walked deletion j for k_fallback (one thread).  Each endpoint with more
// than FB_WARP_MAX neighbours is claimed once per batch for the split scan:
// it gets a slot and ceil(deg / FB_CHUNK) chunks from one 64-bit atomic, so
// that the chunk ranges ascend with the slot.
__device__ __forceinline__ void fb_queue(const PathBufs& pb, const CSRView& G, const WalkTasks& t, uint32_t j) {
    pb.fb_list[atomicAdd(pb.fb_count, 1u)] = j;
    for (int e2 = 0; e2 < 2; ++e2) {
        const uint32_t x = e2 ? t.v[j] : t.u[j];
        const uint32_t d = G.deg[x];
        if (d <= FB_WARP_MAX) continue;
        if (atomicCAS(&pb.fb_slot[x], NONE, NONE - 1u) != NONE) continue;  // claimed by another deletion
        const uint32_t P = (d + FB_CHUNK - 1) / FB_CHUNK;
        const unsigned long long old = atomicAdd(fb_nb(pb), (1ull << 32) | (unsigned long long)P);
        const uint32_t sl = (uint32_t)(old >> 32);
        pb.fb_big[sl] = x;
        pb.fb_cbase[sl] = (uint32_t)old;
        pb.fb_slot[x] = sl;
    }
}

// Fallback of walked deletion j (no walker reached v), one warp: for each
// endpoint x the G_b edge of minimum resistance not in H' (ties: smaller
// neighbour id; reading R11).  false when an endpoint list is longer than
// FB_WARP_MAX (left to the block-wide kernel).
__device__ bool fallback_warp(uint32_t j, int lane, const CSRView& H, const CSRView& G, const WalkTasks& t,
                              Cands& c, uint32_t* d_err, uint32_t& emitted) {
    const uint32_t ends[2] = {t.u[j], t.v[j]};
    if (G.deg[ends[0]] > FB_WARP_MAX || G.deg[ends[1]] > FB_WARP_MAX) return false;
    uint32_t py[2];
    double pw[2];
#pragma unroll
    for (int e2 = 0; e2 < 2; ++e2) {
        const uint32_t x = ends[e2];
        const Ent* L = G.pool + G.off[x];
        const uint32_t d = G.deg[x];
        double br = INFINITY, bw = 0.0;
        uint32_t by = NONE;
        for (uint32_t k = lane; k < d; k += 32) {
            const double rr = L[k].r;
            if (!(rr < br)) continue;  // this lane's ids ascend: strict < keeps the smaller id
            const uint32_t y = L[k].nbr;
            if (has_edge(H, x, y)) continue;
            br = rr;
            by = y;
            bw = L[k].w;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double orr = __shfl_xor_sync(0xffffffffu, br, o);
            const uint32_t oy = __shfl_xor_sync(0xffffffffu, by, o);
            const double ow = __shfl_xor_sync(0xffffffffu, bw, o);
            if (orr < br || (orr == br && oy < by)) {
                br = orr;
                by = oy;
                bw = ow;
            }
        }
        py[e2] = by;
        pw[e2] = bw;
    }
    uint32_t e = 0;
    if (lane == 0) {
        for (int e2 = 0; e2 < 2; ++e2) {
            if (py[e2] == NONE) continue;
            // both endpoints picked the edge (u, v) itself (it was re-inserted in the batch)
            if (e2 == 1 && py[0] != NONE && py[0] == ends[1] && py[1] == ends[0]) continue;
            emit_edge(c, ends[e2], py[e2], pw[e2], (uint32_t)G.n, d_err);
            ++e;
        }
    }
    emitted = __shfl_sync(0xffffffffu, e, 0);
    return true;
}

// everything that follows the walks of update j, one warp: result, kept
// insertion, or the recovered (path or fallback) edges of a deletion
__device__ void finalize_update(uint32_t j, int lane, const WalkKernelArgs& a, UpdTotals& tot, uint32_t* sbuf) {
    uint32_t nh = 0;
    const int bk = reduce_update(j, lane, a.t, a.p, a.r, a.f.res, a.f.best, a.f.dbg_reason, a.f.dbg_steps, tot, nh,
                                 a.G, a.f.pr, a.hdr->id0, a.d_err);
    const uint32_t i = a.t.idx[j];
    Cands c = a.f.c;
    if (a.t.kind[j] == WALK_INS) {
        if (lane == 0) {
            a.f.pb.len[j] = 0;
            if (bk < 0 && !isnan(a.f.fin_w[i])) emit_edge(c, a.t.u[j], a.t.v[j], a.f.fin_w[i], (uint32_t)a.G.n, a.d_err);
        }
        return;
    }
    if (bk >= 0) {
        bool ok = false;
        if (a.f.pr) {
            ok = path_from_records(j, bk, lane, a.G, a.t, a.p, a.r, a.f.pb, a.f, a.d_err);
        } else if (a.f.cp) {
            ok = replay_path_warp(j, bk, lane, a.G, a.t, a.p, a.r, a.hdr->id0, a.f.pb, a.f, a.d_err);
        } else {
            if (lane == 0) ok = replay_path(j, bk, a.G, a.t, a.p, a.r, a.hdr->id0, a.f.pb, a.d_err);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            __syncwarp();
        }
        const uint32_t e = ok ? emit_path_warp(j, lane, a.H, a.p, c, a.f.pb, a.d_err, sbuf) : 0u;
        if (lane == 0) {
            a.f.res[i].nrecovered = (int32_t)e;
            tot.rec += e;
        }
    } else {
        if (lane == 0) {
            a.f.pb.len[j] = 0;
            a.f.res[i].fallback = 1;
        }
        uint32_t e = 0;
        if (fallback_warp(j, lane, a.H, a.G, a.t, c, a.d_err, e)) {
            if (lane == 0) {
                a.f.res[i].nrecovered = (int32_t)e;
                tot.rec += e;
            }
        } else if (lane == 0) {
            fb_queue(a.f.pb, a.G, a.t, j);
        }
    }
}


__device__ __forceinline__ void walker_start(Walker& w, const WalkKernelArgs& a, uint32_t wid, uint64_t id0) {
    w.wid = wid;
    w.j = wid / a.p.s;
    w.k = wid - w.j * a.p.s;
    const uint32_t u = a.t.u[w.j];
    w.q = a.t.v[w.j];
    w.ins = a.t.kind[w.j] == WALK_INS;
    w.wpq = a.t.wpq[w.j];
    const uint64_t id = id0 + a.t.idx[w.j];
    w.ulo = (uint32_t)id;
    w.uhi = (uint32_t)(id >> 32);
    const CSRView& g = w.ins ? a.H : a.G;
    w.off = g.off[u];
    w.deg = g.deg[u];
    w.c = u;
    w.prev = NONE;
    w.pid = false;
    w.steps = 0;
    w.R = 0.0;
    w.active = true;
    if (a.r.paths) a.r.paths[(size_t)wid * (a.p.T + 1)] = (int32_t)u;
}

__device__ __forceinline__ void walker_finish(Walker& w, const WalkKernelArgs& a, uint32_t reason) {
    a.r.meta[w.wid] = w.steps | (reason << 16);
    a.r.R[w.wid] = w.R;
    w.active = false;
}

// after nb_step moved the walker along an edge of resistance r: accumulate and
// test the stop rules
__device__ __forceinline__ void walker_advance(Walker& w, const WalkKernelArgs& a, double r) {
    w.R = __dadd_rn(w.R, r);
    w.steps += 1;
    if (a.r.paths) a.r.paths[(size_t)w.wid * (a.p.T + 1) + w.steps] = (int32_t)w.c;
    if (!w.ins && a.p.del_prune && r_key(w.R) > __ldcg(&a.t.kstar[w.j])) {
        walker_finish(w, a, R_CUT);
        return;
    }
    if (w.c == w.q) {
        if (!w.ins || __dmul_rn(w.wpq, w.R) <= a.p.K) {
            if (w.ins && a.p.early_exit) atomicMin(&a.t.kstar[w.j], w.steps);
            if (!w.ins && a.p.del_prune) atomicMin(&a.t.kstar[w.j], r_key(w.R));
            walker_finish(w, a, R_HIT);
            return;
        }
    }
    if (w.ins && __dmul_rn(w.wpq, w.R) > a.p.K) {
        walker_finish(w, a, R_OVER_K);
        return;
    }
    if (w.steps == a.p.T) walker_finish(w, a, R_AT_T);
}

// Walker state of the batched kernel, kept small so more walkers fit per SM.
// The Philox word of the next step is computed while the current step's
// entry load is in flight (it depends only on the counter, not on the load).
struct Lean {
    uint32_t j, k;      // walked-update index, walker index
    uint32_t q;         // target
    uint32_t c, off, deg, prev, steps;
    uint32_t ulo, uhi;  // update id (Philox counter words 2, 3)
    uint32_t x;         // random word of the next step
    uint32_t hint;      // at a hub (pid): the previous vertex's slot in the hub's list as the
                        // reference we arrived by last recorded it (it may have drifted)
    bool ins, active;
    bool pid;           // prev holds the previous vertex's id (we arrived at a hub)
    bool plus;          // the entry in flight was picked as L[jj + 1] on the hint's word
    double R;
    uint64_t rmax;      // insertion: w_pq * R <= K  <=>  bits(R) <= rmax
};

__device__ __forceinline__ void lean_start(Lean& w, const WalkKernelArgs& a, uint32_t wid, uint64_t id0) {
    w.j = wid / a.p.s;
    w.k = wid - w.j * a.p.s;
    const uint32_t u = a.t.u[w.j];
    w.q = a.t.v[w.j];
    w.ins = a.t.kind[w.j] == WALK_INS;
    w.rmax = a.t.rmax[w.j];
    const uint64_t id = id0 + a.t.idx[w.j];
    w.ulo = (uint32_t)id;
    w.uhi = (uint32_t)(id >> 32);
    const CSRView& g = w.ins ? a.H : a.G;
    w.off = g.off[u];
    w.deg = g.deg[u];
    w.c = u;
    w.prev = NONE;
    w.pid = false;
    w.hint = 0;
    w.plus = false;
    w.steps = 0;
    w.R = 0.0;
    w.active = true;
    w.x = philox_word0(0u, w.k, w.ulo, w.uhi, a.p.key0, a.p.key1);
    if (a.r.paths) a.r.paths[(size_t)wid * (a.p.T + 1)] = (int32_t)u;
}

// records the walker's stop (its finalize count follows through the warp's PendList)
__device__ __forceinline__ void lean_finish(Lean& w, const WalkKernelArgs& a, uint32_t reason) {
    const size_t wid = (size_t)w.j * a.p.s + w.k;
    a.r.meta[wid] = w.steps | (reason << 16);
    a.r.R[wid] = w.R;
    w.active = false;
}

// adds cnt stopped walkers to update j; the count that completes it queues j
__device__ __forceinline__ void count_stops(const WalkKernelArgs& a, uint32_t j, uint32_t cnt) {
    if (atom_add_acq_rel(&a.f.fin[j], cnt) + cnt == a.p.s) {
        const uint32_t pos = atomicAdd(&a.f.qctr[1], 1u);
        st_release(&a.f.queue[pos], j);
    }
}

// Finalize counts a warp has not published yet: (update, stopped walkers)
// pairs in shared memory.  Publishing costs a GPU-scope release (the warp
// waits for its record stores to reach L2), so a warp publishes its pending
// counts together -- when the list fills or every PEND_EVERY iterations, and
// when it runs out of walkers -- instead of on every iteration with a stop.
constexpr uint32_t PEND_FLUSH = 48;               // pairs that trigger a publication
constexpr uint32_t PEND_CAP = PEND_FLUSH + 32 * 4;  // room for one more iteration of 32 stops per walker slot
constexpr uint32_t PEND_EVERY = 8;                // iterations between publications
struct PendList {
    uint32_t j[PEND_CAP];
    uint32_t n[PEND_CAP];
    uint32_t cnt;
};

// adds the walkers that stopped in this iteration (one pair per update), the
// whole warp converged
__device__ __forceinline__ void pend_stops(PendList& pl, bool stopped, uint32_t j, int lane) {
    const uint32_t peers = __match_any_sync(0xffffffffu, stopped ? j : NONE);
    const bool lead = stopped && lane == __ffs(peers) - 1;
    const uint32_t lm = __ballot_sync(0xffffffffu, lead);
    const uint32_t base = pl.cnt;
    __syncwarp();
    if (lead) {
        const uint32_t q = base + (uint32_t)__popc(lm & ((1u << lane) - 1u));
        pl.j[q] = j;
        pl.n[q] = (uint32_t)__popc(peers);
    }
    __syncwarp();
    if (lane == 0) pl.cnt = base + (uint32_t)__popc(lm);
    __syncwarp();
}

// Publishes the pending counts, one acquire-release atomic per pair, the
// lanes in parallel: the warp barrier orders every lane's record stores
// before the releases; the count that completes an update queues it.
__device__ __forceinline__ void flush_stops(const WalkKernelArgs& a, PendList& pl, int lane) {
    __syncwarp();
    const uint32_t n = pl.cnt;
    if (n == 0) return;
    for (uint32_t q = (uint32_t)lane; q < n; q += 32) count_stops(a, pl.j[q], pl.n[q]);
    __syncwarp();
    if (lane == 0) pl.cnt = 0;
    __syncwarp();
}

// head (nbr, noff, ndeg, rev) and resistance of the entry at pool index i
__device__ __forceinline__ void load_step(const Ent* pool, uint32_t i, uint4& h, double& r) {
    const uint4* q = reinterpret_cast<const uint4*>(pool + i);
    h = __ldg(q);
    r = __ldg(reinterpret_cast<const double*>(q + 1));
}

// The step when the walker stands on a hub (previous vertex p known by id
// only) or the chosen entry leads to a hub (HUBREF: the list comes from the
// vertex arrays).  At a hub the j-th neighbour other than p is L[jj] when
// L[jj] < p and L[jj + 1] otherwise; the entry in flight was picked by the
// slot hint (plus: L[jj + 1]), and the pick is checked against p: L[jj] is
// right iff its id is below p, L[jj + 1] iff its id is above p.  A wrong
// guess (a hint that drifted past jj) loads the other entry.  Moves the walker
// (r ends as the step's resistance, added by the caller); false on a bad
// offset.
__device__ __forceinline__ bool lean_hub_step(Lean& v, const WalkKernelArgs& a, uint4& h, double& r, uint32_t& at) {
    const CSRView& g = v.ins ? a.H : a.G;
    if (v.pid && (v.plus ? h.x <= v.prev : h.x >= v.prev)) {
        const uint32_t alt = v.plus ? at - 1u : at + 1u;
        if ((uint64_t)alt >= g.pool_cap) {
            atomicOr(a.d_err, (uint32_t)ERR_INTERNAL);
            return false;
        }
        at = alt;
        load_step(g.pool, at, h, r);
    }
    v.steps += 1;
    const uint32_t from = v.c;
    v.c = h.x;
    if (h.y == HUBREF) {
        v.off = g.off[v.c];
        v.deg = g.deg[v.c];
        v.prev = from;
        v.hint = h.w;
        v.pid = true;
    } else {
        v.off = h.y;
        v.deg = h.z;
        v.prev = h.w;
        v.pid = false;
    }
    return true;
}

// Sends out the entry load of the walker's next step (and the early-exit /
// pruning probe of its update); false when there is no next step (n_eff = 0)
// or the offset would leave the pool (a broken mutation, reported).
template <bool HUBS>
__device__ __forceinline__ bool lean_issue(Lean& v, const WalkKernelArgs& a, uint4& h, double& r, uint32_t& ks,
                                           uint32_t& at) {
    const uint32_t neff = v.deg - (v.prev != NONE ? 1u : 0u);
    if (neff == 0) {
        // a hub reference met by the hub-free variant ends here (its cached
        // degree is 1): report it instead of stopping silently
        if (!HUBS && v.off == HUBREF) atomicOr(a.d_err, (uint32_t)ERR_INTERNAL);
        return false;
    }
    const uint32_t jj = __umulhi(v.x, neff);
    // slot of the previous vertex known: skip it by position; after a hub
    // arrival its slot is only hinted: pick by the hint, checked on arrival
    const uint32_t skip = (HUBS && v.pid) ? v.hint : v.prev;
    const uint32_t idx = jj + (jj >= skip ? 1u : 0u);
    v.plus = idx != jj;
    const uint64_t pcap = v.ins ? a.H.pool_cap : a.G.pool_cap;
    if ((uint64_t)v.off + idx >= pcap) {
        atomicOr(a.d_err, (uint32_t)ERR_INTERNAL);
        return false;
    }
    at = v.off + idx;
    load_step(v.ins ? a.H.pool : a.G.pool, at, h, r);
    ks = (v.ins ? a.p.early_exit : a.p.del_prune) ? __ldcg(&a.t.kstar[v.j]) : NONE;
    return true;
}

// Up to 256 threads per block; register caps that keep spills out: 4 blocks
// of 256 per SM for one walker per thread, 3 for two.  HUBS selects the variant that
// handles hub references; both variants are launched and the one that does
// not match the device-side hub counts of G and H returns at once, so graphs
// without hubs (meshes) run a loop with no hub branch and no host round trip
// is needed to choose.
//
// Software pipelining: the address of a walker's next entry depends only on
// the entry just read and on a Philox word computed in advance, so the next
// load is sent out before the stop rules of the current step are evaluated.
// The FP64 accumulation and the resistance tests then overlap that load
// instead of sitting on the chain of dependent loads; a walker that stops
// drops the load it has in flight.
template <int ILP, bool HUBS>
__global__ void __launch_bounds__(256, (ILP == 1 ? 4 : (ILP == 2 ? 3 : 1))) k_walk_batched(WalkKernelArgs a) {
    if (walk_aborted(a.d_err)) return;
    if (((*a.H.nhub | *a.G.nhub) != 0u) != HUBS) return;
    const uint32_t W = min(*a.t.count, a.j_hi);
    if (W <= a.j_lo) return;
    const uint32_t total = (W - a.j_lo) * a.p.s;
    const uint32_t wbase = a.j_lo * a.p.s;
    const uint64_t id0 = a.hdr->id0;
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    Lean w[ILP];
    uint4 h[ILP];
    double r[ILP];
    uint32_t ks[ILP], at[ILP];
    bool fly[ILP];  // an entry load of the walker's next step is in flight
#pragma unroll
    for (int i = 0; i < ILP; ++i) {
        w[i].active = false;
        fly[i] = false;
    }
    bool exhausted = false;
    __shared__ PendList s_pend[8];  // per warp (blocks of at most 256 threads)
    PendList& pend = s_pend[threadIdx.x >> 5];
    if (lane == 0) pend.cnt = 0;
    __syncwarp();
    uint32_t iter = 0;
    bool stop[ILP];
    for (;;) {
#pragma unroll
        for (int i = 0; i < ILP; ++i) stop[i] = false;
        // Refill empty slots, one atomic per warp and slot; a new walker sends
        // out its first load at once.  Starting walkers holds the whole warp
        // up for three dependent reads (id, task fields, start list), so a
        // warp that still has walkers waits until at least refill_min of its
        // slots are empty.  The walkers of one update are handed out together
        // and tend to stop together, so the wait leaves few lanes idle.
#pragma unroll
        for (int i = 0; i < ILP; ++i) {
            const bool idle = !w[i].active && !exhausted;
            const uint32_t im = __ballot_sync(0xffffffffu, idle);
            const uint32_t am = __ballot_sync(0xffffffffu, w[i].active);
            const bool need = idle && ((uint32_t)__popc(im) >= a.refill_min || am == 0u);
            const uint32_t m = __ballot_sync(0xffffffffu, need);
            if (m) {
                const int leader = __ffs(m) - 1;
                unsigned long long b = 0;
                if (lane == leader) b = atomicAdd(a.next, (unsigned long long)__popc(m));
                b = __shfl_sync(0xffffffffu, b, leader);
                if (need) {
                    const unsigned long long id = b + __popc(m & lt);
                    if (id < total) {
                        lean_start(w[i], a, wbase + (uint32_t)id, id0);
                        fly[i] = lean_issue<HUBS>(w[i], a, h[i], r[i], ks[i], at[i]);
                        if (!fly[i]) {
                            lean_finish(w[i], a, R_LEAF);
                            stop[i] = true;  // counted with this iteration's stops
                        } else {
                            w[i].x = philox_word0(1u, w[i].k, w[i].ulo, w[i].uhi, a.p.key0, a.p.key1);
                        }
                    } else {
                        exhausted = true;
                    }
                }
            }
        }
        bool any = false;
#pragma unroll
        for (int i = 0; i < ILP; ++i) any |= w[i].active;
        if (!__any_sync(0xffffffffu, any)) {
            if (a.f.on) {
#pragma unroll
                for (int i = 0; i < ILP; ++i) pend_stops(pend, stop[i], w[i].j, lane);
            }
            break;
        }
#pragma unroll
        for (int i = 0; i < ILP; ++i) {
            if (!fly[i]) continue;
            Lean& v = w[i];
            stop[i] = true;  // cleared below if the walker goes on
            const uint32_t ks_now = ks[i];
            if (v.ins && ks_now <= v.steps) {  // a walker of this update hit at a step <= ours: cut
                lean_finish(v, a, R_CUT);
                fly[i] = false;
                continue;
            }
            if (HUBS && (v.pid || h[i].y == HUBREF)) {  // leaving or entering a hub
                if (!lean_hub_step(v, a, h[i], r[i], at[i])) {
                    lean_finish(v, a, R_LEAF);
                    fly[i] = false;
                    continue;
                }
            } else {
                v.steps += 1;
                v.c = h[i].x;
                v.off = h[i].y;
                v.deg = h[i].z;
                v.prev = h[i].w;
            }
            const double r_step = r[i];
            const uint32_t took = at[i];  // pool index of the entry this step took
            // reaching v ends the walk whatever R is (hit, or over K for an insertion);
            // the next load goes out first, the rest of the step follows it
            const bool at_q = v.c == v.q;
            fly[i] = !at_q && v.steps < a.p.T && lean_issue<HUBS>(v, a, h[i], r[i], ks[i], at[i]);
            v.R = __dadd_rn(v.R, r_step);
            if (a.f.pr && !v.ins) {
                const size_t rec = ((size_t)v.j * a.p.T + v.steps - 1) * a.p.s + v.k;
                a.f.pr[rec] = v.R;
                a.f.pe[rec] = took;
            }
            if (a.r.paths) a.r.paths[((size_t)v.j * a.p.s + v.k) * (a.p.T + 1) + v.steps] = (int32_t)v.c;
            if (a.f.cp && !v.ins && (v.steps & ((1u << a.f.cp_shift) - 1u)) == 0u) {
                const uint32_t q = (v.steps >> a.f.cp_shift) - 1u;
                if (q < a.f.ncp)
                    a.f.cp[((size_t)v.j * a.p.s + v.k) * a.f.ncp + q] =
                        make_uint4(v.c, v.off, v.deg, v.prev | (v.pid ? 0x80000000u : 0u));
            }
            const bool over = (unsigned long long)__double_as_longlong(v.R) > v.rmax;  // insertions: w_pq * R > K
            if (!v.ins && r_key(v.R) > ks_now) {  // above a hit of this deletion: cannot be the minimum
                lean_finish(v, a, R_CUT);
            } else if (at_q && (!v.ins || !over)) {
                if (v.ins ? a.p.early_exit : a.p.del_prune)
                    atomicMin(&a.t.kstar[v.j], v.ins ? v.steps : r_key(v.R));
                lean_finish(v, a, R_HIT);
            } else if (v.ins && over) {
                lean_finish(v, a, R_OVER_K);
            } else if (v.steps == a.p.T) {
                lean_finish(v, a, R_AT_T);
            } else if (!fly[i]) {
                lean_finish(v, a, R_LEAF);
            }
            if (!v.active) {
                fly[i] = false;
            } else {
                stop[i] = false;
                v.x = philox_word0(v.steps + 1, v.k, v.ulo, v.uhi, a.p.key0, a.p.key1);
            }
        }
        if (a.f.on) {
#pragma unroll
            for (int i = 0; i < ILP; ++i) pend_stops(pend, stop[i], w[i].j, lane);
            ++iter;
            static_assert(ILP <= 4, "pending list sized for four walker slots");
            if (pend.cnt >= PEND_FLUSH || (iter % PEND_EVERY) == 0u) flush_stops(a, pend, lane);
        }
    }
    if (!a.f.on) return;
    flush_stops(a, pend, lane);
    __shared__ uint32_t s_emit[8][EMIT_SMEM];  // per warp (blocks of at most 256 threads)
    // No walkers left for this warp: finalize queued updates (in order of
    // completion) until every walked update of the launch is done.  Updates
    // complete because their walkers belong to warps that are running; the
    // wait for the next one is still bounded.
    const uint32_t Wl = W - a.j_lo;
    UpdTotals tot;
    for (;;) {
        uint32_t qi = 0;
        if (lane == 0) qi = atomicAdd(&a.f.qctr[0], 1u);
        qi = __shfl_sync(0xffffffffu, qi, 0);
        if (qi >= Wl) break;
        uint32_t j = NONE;
        if (lane == 0) {
            for (uint32_t spins = 0; spins < a.f.spin_limit; ++spins) {
                j = ld_acquire(&a.f.queue[qi]);
                if (j != NONE) break;
                __nanosleep(128);
            }
        }
        j = __shfl_sync(0xffffffffu, j, 0);
        if (j == NONE) {
            if (lane == 0) atomicOr(a.d_err, (uint32_t)ERR_SPIN);
            break;
        }
        (void)ld_acquire(&a.f.queue[qi]);  // every lane acquires the records it is about to read
        finalize_update(j, lane, a, tot, s_emit[threadIdx.x >> 5]);
    }
    if (lane == 0) add_totals(a.f.ctr, tot);
}

// the paper's scheme: one block per walked update, one thread per walker
__global__ void k_walk_one(WalkKernelArgs a, uint32_t j) {
    if (walk_aborted(a.d_err)) return;
    if (j >= *a.t.count) return;
    __shared__ uint32_t ks;
    if (threadIdx.x == 0) ks = NONE;
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < a.p.s; k += blockDim.x) {
        Walker w;
        walker_start(w, a, j * a.p.s + k, a.hdr->id0);
        while (w.active) {
            const uint32_t neff = w.deg - (w.prev != NONE ? 1u : 0u);
            if (neff == 0) {
                walker_finish(w, a, R_LEAF);
                break;
            }
            if (w.ins && a.p.early_exit && *(volatile uint32_t*)&ks <= w.steps) {
                walker_finish(w, a, R_CUT);
                break;
            }
            const uint32_t x = philox_word0(w.steps, w.k, w.ulo, w.uhi, a.p.key0, a.p.key1);
            uint4 h;
            double2 tl;
            if (nb_step(w.ins ? a.H : a.G, x, w.c, w.off, w.deg, w.prev, w.pid, h, tl) <= 0) {
                atomicOr(a.d_err, (uint32_t)ERR_INTERNAL);  // n_eff > 0 here: only a bad offset stops it
                walker_finish(w, a, R_LEAF);
                break;
            }
            const uint32_t before = w.steps;
            walker_advance(w, a, tl.x);
            if (!w.active && w.ins && a.p.early_exit && (a.r.meta[w.wid] >> 16) == R_HIT)
                atomicMin(&ks, before + 1);
        }
    }
}

static WalkKernelArgs make_args(const CSRView& H, const CSRView& G, const WalkTasks& t, const WalkParams& p,
                                const WalkRecs& r, const BatchHdr* d_hdr, unsigned long long* d_next,
                                uint32_t j_lo, uint32_t j_hi, const uint32_t* d_err) {
    WalkKernelArgs a = {};
    a.H = H;
    a.G = G;
    a.t = t;
    a.p = p;
    a.r = r;
    a.hdr = d_hdr;
    a.next = d_next;
    a.j_lo = j_lo;
    a.j_hi = j_hi;
    a.refill_min = 1;
    a.d_err = const_cast<uint32_t*>(d_err);
    return a;
}

// Optional L2 residency for the sparsifier: the walk launch carries an access
// policy window over H's pool, so H's entries (read by every insertion walk)
// persist in the set-aside part of L2 while deletion walks stream through G.
static size_t g_persist_bytes = 0;  // set-aside L2 bytes of this context (0 = off)
static size_t g_max_window = 0;

void walk_set_l2_persist(size_t persist_bytes, size_t max_window) {
    g_persist_bytes = persist_bytes;
    g_max_window = max_window;
}

template <int ILP, bool HUBS>
static void launch_ilp(const WalkKernelArgs& a, const WalkShape& shape, cudaStream_t st) {
    int bps = shape.blocks_per_sm;
    if (bps <= 0) {
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_walk_batched<ILP, HUBS>, shape.block, 0);
        bps = occ > 0 ? occ : 1;
    }
    const int grid = device_sms() * bps;
    if (g_persist_bytes == 0 || a.H.pool == nullptr) {
        k_walk_batched<ILP, HUBS><<<grid, shape.block, 0, st>>>(a);
        return;
    }
    size_t win = (size_t)a.H.pool_cap * sizeof(Ent);
    if (win > g_max_window) win = g_max_window;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(shape.block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeAccessPolicyWindow;
    attr[0].val.accessPolicyWindow.base_ptr = (void*)a.H.pool;
    attr[0].val.accessPolicyWindow.num_bytes = win;
    attr[0].val.accessPolicyWindow.hitRatio = win > g_persist_bytes ? (float)g_persist_bytes / (float)win : 1.0f;
    attr[0].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    attr[0].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    DG_CUDA(cudaLaunchKernelEx(&cfg, k_walk_batched<ILP, HUBS>, a));
}

// Both variants are launched; the one that does not match the graphs' hub
// counts returns at once.  With a side stream the hub variant runs there,
// beside the hub-free one, so the variant that exits costs the critical path
// nothing.
template <int ILP>
static void launch_both(const WalkKernelArgs& a, const WalkShape& shape, cudaStream_t st, cudaStream_t side,
                        cudaEvent_t fork, cudaEvent_t join) {
    if (side) {
        DG_CUDA(cudaEventRecord(fork, st));
        DG_CUDA(cudaStreamWaitEvent(side, fork, 0));
        launch_ilp<ILP, true>(a, shape, side);
        DG_CUDA(cudaEventRecord(join, side));
        launch_ilp<ILP, false>(a, shape, st);
        DG_CUDA(cudaStreamWaitEvent(st, join, 0));
    } else {
        launch_ilp<ILP, false>(a, shape, st);
        launch_ilp<ILP, true>(a, shape, st);
    }
}

void launch_walk_batched(const CSRView& H, const CSRView& G, const WalkTasks& t, const WalkParams& p,
                         const WalkRecs& r, const BatchHdr* d_hdr, unsigned long long* d_next,
                         uint32_t j_lo, uint32_t j_hi, const WalkShape& shape, const FinArgs& f,
                         const uint32_t* d_err, cudaStream_t st, cudaStream_t side, cudaEvent_t fork,
                         cudaEvent_t join) {
    WalkKernelArgs a = make_args(H, G, t, p, r, d_hdr, d_next, j_lo, j_hi, d_err);
    a.f = f;
    a.refill_min = (uint32_t)std::min(32, std::max(1, shape.refill));
    DG_CUDA(cudaMemsetAsync(d_next, 0, sizeof(unsigned long long), st));
    switch (shape.ilp) {
        case 1: launch_both<1>(a, shape, st, side, fork, join); break;
        case 4: launch_both<4>(a, shape, st, side, fork, join); break;
        default: launch_both<2>(a, shape, st, side, fork, join); break;
    }
    g_launches += 2;
    DG_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// The batching engine's other work shapes, for the autotuner: a block claims
// a tile of `tile` walked updates at a time and stages their task fields in
// shared memory (the frontier tile), and LANES lanes walk one walker
// together -- the group's lanes compute the Philox words of the next LANES
// steps side by side, then every lane of the group takes the same steps (the
// group's loads coincide).  The launch writes the walker records only; the
// per-update reduction and the emission kernels follow it, as after a cut
// launch.  Outputs are the same as with any other shape: every walker draws
// the same words and makes the same picks.
// ---------------------------------------------------------------------------
constexpr uint32_t TILE_MAX = 16;

template <int LANES>
__global__ void __launch_bounds__(256) k_walk_tiled(WalkKernelArgs a, uint32_t tile) {
    if (walk_aborted(a.d_err)) return;
    const uint32_t W = min(*a.t.count, a.j_hi);
    if (W <= a.j_lo) return;
    __shared__ uint32_t s_u[TILE_MAX], s_v[TILE_MAX], s_idx[TILE_MAX];
    __shared__ double s_wpq[TILE_MAX];
    __shared__ uint8_t s_kind[TILE_MAX];
    __shared__ uint32_t s_j0;
    const uint64_t id0 = a.hdr->id0;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t gl = lane & (LANES - 1u);  // lane inside the group
    const uint32_t gmask = LANES == 32 ? 0xffffffffu : (((1u << LANES) - 1u) << (lane & ~(LANES - 1u)));
    const uint32_t group = threadIdx.x / LANES, ngroups = blockDim.x / LANES;
    const uint32_t S = a.p.s;
    for (;;) {
        if (threadIdx.x == 0) s_j0 = a.j_lo + (uint32_t)atomicAdd(a.next, (unsigned long long)tile);
        __syncthreads();
        const uint32_t j0 = s_j0;
        if (j0 >= W) break;
        const uint32_t nt = min(tile, W - j0);
        if (threadIdx.x < nt) {
            const uint32_t j = j0 + threadIdx.x;
            s_u[threadIdx.x] = a.t.u[j];
            s_v[threadIdx.x] = a.t.v[j];
            s_idx[threadIdx.x] = a.t.idx[j];
            s_wpq[threadIdx.x] = a.t.wpq[j];
            s_kind[threadIdx.x] = a.t.kind[j];
        }
        __syncthreads();
        for (uint32_t wl = group; wl < nt * S; wl += ngroups) {
            const uint32_t jj = wl / S, k = wl - jj * S, j = j0 + jj;
            const size_t wid = (size_t)j * S + k;
            const bool ins = s_kind[jj] == WALK_INS;
            const CSRView& g = ins ? a.H : a.G;
            const uint32_t u = s_u[jj], q = s_v[jj];
            const double wpq = s_wpq[jj];
            const uint64_t id = id0 + s_idx[jj];
            uint32_t c = u, off = g.off[u], deg = g.deg[u], prev = NONE, steps = 0, reason = R_LEAF;
            bool pid = false;
            double R = 0.0;
            if (a.r.paths && gl == 0) a.r.paths[wid * (a.p.T + 1)] = (int32_t)u;
            uint32_t wbase = 0;
            uint32_t word = philox_word0(gl, k, (uint32_t)id, (uint32_t)(id >> 32), a.p.key0, a.p.key1);
            for (;;) {
                const uint32_t neff = deg - (prev != NONE ? 1u : 0u);
                if (neff == 0) {
                    reason = R_LEAF;
                    break;
                }
                if (ins && a.p.early_exit && __ldcg(&a.t.kstar[j]) <= steps) {
                    reason = R_CUT;
                    break;
                }
                if (steps - wbase >= LANES) {  // the group draws the words of the next LANES steps
                    wbase = steps;
                    word = philox_word0(wbase + gl, k, (uint32_t)id, (uint32_t)(id >> 32), a.p.key0, a.p.key1);
                }
                const uint32_t x = LANES == 1 ? word : __shfl_sync(gmask, word, (int)(steps - wbase), LANES);
                uint4 h;
                double2 tl;
                if (nb_step(g, x, c, off, deg, prev, pid, h, tl) <= 0) {
                    if (gl == 0) atomicOr(a.d_err, (uint32_t)ERR_INTERNAL);
                    reason = R_LEAF;
                    break;
                }
                R = __dadd_rn(R, tl.x);
                steps += 1;
                if (a.r.paths && gl == 0) a.r.paths[wid * (a.p.T + 1) + steps] = (int32_t)c;
                if (!ins && a.p.del_prune && r_key(R) > __ldcg(&a.t.kstar[j])) {
                    reason = R_CUT;
                    break;
                }
                if (c == q && (!ins || __dmul_rn(wpq, R) <= a.p.K)) {
                    if (gl == 0) {
                        if (ins && a.p.early_exit) atomicMin(&a.t.kstar[j], steps);
                        if (!ins && a.p.del_prune) atomicMin(&a.t.kstar[j], r_key(R));
                    }
                    reason = R_HIT;
                    break;
                }
                if (ins && __dmul_rn(wpq, R) > a.p.K) {
                    reason = R_OVER_K;
                    break;
                }
                if (steps == a.p.T) {
                    reason = R_AT_T;
                    break;
                }
            }
            if (gl == 0) {
                a.r.meta[wid] = steps | (reason << 16);
                a.r.R[wid] = R;
            }
        }
        __syncthreads();  // the tile's staged fields are read until here
    }
}

void launch_walk_tiled(const CSRView& H, const CSRView& G, const WalkTasks& t, const WalkParams& p,
                       const WalkRecs& r, const BatchHdr* d_hdr, unsigned long long* d_next, uint32_t j_lo,
                       uint32_t j_hi, const WalkShape& shape, const uint32_t* d_err, cudaStream_t st) {
    WalkKernelArgs a = make_args(H, G, t, p, r, d_hdr, d_next, j_lo, j_hi, d_err);
    const uint32_t tile = (uint32_t)std::min<int>(TILE_MAX, std::max(1, shape.tile));
    const int block = shape.block;
    DG_CUDA(cudaMemsetAsync(d_next, 0, sizeof(unsigned long long), st));
    auto go = [&](auto kern) {
        int bps = shape.blocks_per_sm;
        if (bps <= 0) {
            int occ = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, block, 0);
            bps = occ > 0 ? occ : 1;
        }
        kern<<<device_sms() * bps, block, 0, st>>>(a, tile);
    };
    switch (shape.lanes) {
        case 2: go(k_walk_tiled<2>); break;
        case 4: go(k_walk_tiled<4>); break;
        case 8: go(k_walk_tiled<8>); break;
        case 32: go(k_walk_tiled<32>); break;
        default: go(k_walk_tiled<1>); break;
    }
    ++g_launches;
    DG_CHECK_LAUNCH();
}

void launch_walk_one(const CSRView& H, const CSRView& G, const WalkTasks& t, const WalkParams& p,
                     const WalkRecs& r, const BatchHdr* d_hdr, uint32_t j, const uint32_t* d_err,
                     cudaStream_t st) {
    WalkKernelArgs a = make_args(H, G, t, p, r, d_hdr, nullptr, 0, 0, d_err);
    int threads = (int)p.s;
    if (threads > 1024) threads = 1024;
    threads = (threads + 31) / 32 * 32;
    k_walk_one<<<1, threads, 0, st>>>(a, j);
    ++g_launches;
}

// ---------------------------------------------------------------------------
// per-update reduction (Eq. 12 and the early-exit reading)
// ---------------------------------------------------------------------------
__global__ void k_walk_reduce(CSRView G, WalkTasks t, WalkParams p, WalkRecs r, const BatchHdr* hdr,
                              dg_update_result* res, int32_t* best, BatchCounters* ctr, int32_t* dbg_reason,
                              int32_t* dbg_steps, uint32_t j_lo, uint32_t j_hi, uint32_t* d_err) {
    if (walk_aborted(d_err)) return;
    const uint32_t W = min(*t.count, j_hi);
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint64_t id0 = hdr->id0;
    UpdTotals tot;  // this warp's totals (lane 0)
    for (uint32_t j = j_lo + warp; j < W; j += nwarps) {
        uint32_t nh;
        reduce_update(j, lane, t, p, r, res, best, dbg_reason, dbg_steps, tot, nh, G, nullptr, id0, d_err);
    }
    if (lane == 0) add_totals(ctr, tot);
}

void launch_walk_reduce(const CSRView& G, const WalkTasks& t, const WalkParams& p, const WalkRecs& r,
                        const BatchHdr* d_hdr, dg_update_result* res, int32_t* best, BatchCounters* ctr,
                        int32_t* dbg_reason, int32_t* dbg_steps, uint32_t j_lo, uint32_t j_hi, uint32_t* d_err,
                        cudaStream_t st) {
    const uint32_t span = j_hi > j_lo ? j_hi - j_lo : 0u;
    uint32_t blocks = (span + 7) / 8;
    const uint32_t cap = (uint32_t)device_sms() * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_walk_reduce<<<blocks, 256, 0, st>>>(G, t, p, r, d_hdr, res, best, ctr, dbg_reason, dbg_steps, j_lo, j_hi,
                                          d_err);
    ++g_launches;
    DG_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// commit candidates: kept insertions, recovered path edges, fallback edges
// ---------------------------------------------------------------------------

// Replay of the argmin walker of every walked deletion that hit: the same
// counters on the same snapshot give the same path.  One thread per deletion
// only follows the path (one dependent load per step) and records it; the
// edges are judged in parallel by k_emit_path.  Kept insertions and the
// fallback of deletions without a hit are emitted here.
__global__ void k_replay(CSRView H, CSRView G, WalkTasks t, WalkParams p, WalkRecs r, const BatchHdr* hdr,
                         const int32_t* best, const double* fin_w, dg_update_result* res, BatchCounters* ctr,
                         Cands c, PathBufs pb, uint32_t w_max, uint32_t* d_err) {
    if (walk_aborted(d_err)) return;
    const uint32_t W = min(*t.count, w_max);
    const uint32_t n = (uint32_t)G.n;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < W; j += gridDim.x * blockDim.x) {
        const uint32_t i = t.idx[j];
        pb.len[j] = 0;
        if (t.kind[j] == WALK_INS) {
            if (best[j] < 0 && !isnan(fin_w[i])) emit_edge(c, t.u[j], t.v[j], fin_w[i], n, d_err);
            continue;
        }
        res[i].nrecovered = 0;
        const int32_t b = best[j];
        if (b >= 0) {
            replay_path(j, b, G, t, p, r, hdr->id0, pb, d_err);
        } else {
            // no walker reached v: the fallback edges are chosen by k_fallback
            res[i].fallback = 1;
            fb_queue(pb, G, t, j);
        }
    }
}

// (r, neighbour) lexicographic minimum over the block; the result is valid in
// thread 0.  br/by/bw: this thread's candidate (INFINITY / NONE when none).
__device__ __forceinline__ void fb_block_min(double& br, uint32_t& by, double& bw, double* s_r, uint32_t* s_y,
                                             double* s_w) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        const double orr = __shfl_xor_sync(0xffffffffu, br, o);
        const uint32_t oy = __shfl_xor_sync(0xffffffffu, by, o);
        const double ow = __shfl_xor_sync(0xffffffffu, bw, o);
        if (orr < br || (orr == br && oy < by)) {
            br = orr;
            by = oy;
            bw = ow;
        }
    }
    if (lane == 0) {
        s_r[warp] = br;
        s_y[warp] = by;
        s_w[warp] = bw;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q)
            if (s_r[q] < br || (s_r[q] == br && s_y[q] < by)) {
                br = s_r[q];
                by = s_y[q];
                bw = s_w[q];
            }
    }
}

// This thread's candidate over entries [k0, k1) of x's G_b list, taken
// k0 + threadIdx.x, + blockDim.x, ... (ascending, so strict < keeps the
// smaller neighbour id): minimum resistance among the edges not in H'.
__device__ __forceinline__ void fb_scan_range(const CSRView& H, const Ent* L, uint32_t x, uint32_t k0, uint32_t k1,
                                              double& br, uint32_t& by, double& bw) {
    // eight resistances per round are loaded together, then taken in order
    constexpr uint32_t U = 8;
    for (uint32_t b0 = k0 + threadIdx.x; b0 < k1; b0 += U * blockDim.x) {
        double rr[U];
#pragma unroll
        for (uint32_t q = 0; q < U; ++q) {
            const uint32_t k = b0 + q * blockDim.x;
            rr[q] = k < k1 ? L[k].r : INFINITY;
        }
#pragma unroll
        for (uint32_t q = 0; q < U; ++q) {
            const uint32_t k = b0 + q * blockDim.x;
            if (!(rr[q] < br)) continue;
            const uint32_t y = L[k].nbr;
            if (has_edge(H, x, y)) continue;
            br = rr[q];
            by = y;
            bw = L[k].w;
        }
    }
}

// First index i in [0, d) of a neighbour-sorted list with L[i].nbr >= key (d
// when none), one warp: 32 probes per round shrink the range 33-fold.
__device__ __forceinline__ uint32_t warp_lower_bound(const Ent* L, uint32_t d, uint32_t key, int lane) {
    uint32_t lo = 0, hi = d;  // entries before lo are < key, entries from hi on are >= key
    while (hi - lo > 32u) {
        const uint64_t span = hi - lo;
        const uint32_t p = lo + (uint32_t)(span * (uint32_t)(lane + 1) / 33u);
        const uint32_t m = __ballot_sync(0xffffffffu, L[p].nbr >= key);
        const int f = m ? __ffs(m) - 1 : 32;  // first probe at or above key
        const uint32_t nlo = f > 0 ? lo + (uint32_t)(span * (uint32_t)f / 33u) + 1u : lo;
        const uint32_t nhi = f < 32 ? lo + (uint32_t)(span * (uint32_t)(f + 1) / 33u) : hi;
        lo = nlo;
        hi = nhi;
    }
    const uint32_t p = lo + (uint32_t)lane;
    const uint32_t m = __ballot_sync(0xffffffffu, p < hi ? L[p].nbr >= key : true);
    return m ? lo + (uint32_t)(__ffs(m) - 1) : hi;
}

constexpr uint32_t FB_HS = 2048;  // H' entries staged in shared memory per scanned range

// fb_scan_range with the H' lookups served from shared memory: x's H' entries
// whose neighbour lies in the range's id span (both lists ascend by
// neighbour) are found by two warp searches and staged in s_h; when more
// than FB_HS of them fall in the span the lookups go to the H' lists.
// Block-wide (every thread calls it with the same arguments).
__device__ void fb_scan_staged(const CSRView& H, const CSRView& G, uint32_t x, uint32_t k0, uint32_t k1,
                               uint32_t* s_h, uint32_t* s_rng, double& br, uint32_t& by, double& bw) {
    if (k1 <= k0) return;
    const Ent* L = G.pool + G.off[x];
    const Ent* HL = H.pool + H.off[x];
    const uint32_t hd = H.deg[x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < 2) {
        const uint32_t key = warp == 0 ? L[k0].nbr : L[k1 - 1].nbr + 1u;
        const uint32_t p = warp_lower_bound(HL, hd, key, lane);
        if (lane == 0) s_rng[warp] = p;
    }
    __syncthreads();
    const uint32_t h0 = s_rng[0], hs = s_rng[1] - s_rng[0];
    if (hs > FB_HS) {
        __syncthreads();
        fb_scan_range(H, L, x, k0, k1, br, by, bw);
        return;
    }
    for (uint32_t i = threadIdx.x; i < hs; i += blockDim.x) s_h[i] = HL[h0 + i].nbr;
    __syncthreads();
    constexpr uint32_t U = 8;
    for (uint32_t b0 = k0 + threadIdx.x; b0 < k1; b0 += U * blockDim.x) {
        double rr[U];
#pragma unroll
        for (uint32_t q = 0; q < U; ++q) {
            const uint32_t k = b0 + q * blockDim.x;
            rr[q] = k < k1 ? L[k].r : INFINITY;
        }
#pragma unroll
        for (uint32_t q = 0; q < U; ++q) {
            const uint32_t k = b0 + q * blockDim.x;
            if (!(rr[q] < br)) continue;
            const uint32_t y = L[k].nbr;
            const uint32_t p = lower_bound_arr(s_h, 0u, hs, y);
            if (p < hs && s_h[p] == y) continue;  // (x, y) is in H'
            br = rr[q];
            by = y;
            bw = L[k].w;
        }
    }
    __syncthreads();  // s_h and s_rng are reused by the next range
}

// First look at every long endpoint list claimed by fb_queue, one warp per
// list: G_b's resistances are bounded below by G.minr, so the first entry (in
// neighbour order) whose resistance equals that bound and whose edge is not in
// H' is the list's minimum of (resistance, neighbour).  When one turns up
// among the first FB_QUICK entries it becomes the result of the list's first
// chunk and the list is marked done (fb_done); otherwise the chunked scan
// decides.  Graphs whose weights tie at their minimum (unit weights) resolve
// here instead of scanning hub lists of 10^5 entries.
constexpr uint32_t FB_QUICK = 256;
__global__ void __launch_bounds__(256) k_fb_quick(CSRView H, CSRView G, PathBufs pb, uint32_t* d_err) {
    if (walk_aborted(d_err)) return;
    const unsigned long long nb = *fb_nb(pb);
    const uint32_t S = (uint32_t)(nb >> 32);
    const unsigned long long lb = *G.minr;
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t sl = warp; sl < S; sl += nwarps) {
        const uint32_t x = pb.fb_big[sl], cb = pb.fb_cbase[sl];
        const uint32_t d = G.deg[x];
        uint32_t done = 0;
        if (cb + (d + FB_CHUNK - 1) / FB_CHUNK <= FB_CHUNK_CAP) {
            const Ent* L = G.pool + G.off[x];
            const uint32_t lim = min(d, FB_QUICK);
            for (uint32_t b0 = 0; b0 < lim && !done; b0 += 32) {
                const uint32_t k = b0 + (uint32_t)lane;
                bool ok = false;
                uint32_t y = NONE;
                double rr = 0.0, ww = 0.0;
                if (k < lim) {
                    rr = L[k].r;
                    y = L[k].nbr;
                    ww = L[k].w;
                    ok = (unsigned long long)__double_as_longlong(rr) == lb && !has_edge(H, x, y);
                }
                const uint32_t m = __ballot_sync(0xffffffffu, ok);
                if (m) {
                    const int f = __ffs(m) - 1;
                    if (lane == f) {
                        pb.fb_pr[cb] = rr;
                        pb.fb_py[cb] = y;
                        pb.fb_pw[cb] = ww;
                    }
                    done = 1;
                }
            }
        }
        if (lane == 0) pb.fb_done[sl] = done;
    }
}

// Split scan of the long endpoint lists claimed by fb_queue: every fallback
// deletion's endpoint slots are looked up (the claims are complete), then one
// block per chunk finds the chunk's minimum (lists k_fb_quick resolved keep
// its result in their first chunk; their other chunks read as empty).
__global__ void __launch_bounds__(256) k_fb_chunks(CSRView H, CSRView G, WalkTasks t, PathBufs pb, uint32_t w_max,
                                                   uint32_t* d_err) {
    if (walk_aborted(d_err)) return;
    __shared__ double s_r[8];
    __shared__ uint32_t s_y[8];
    __shared__ double s_w[8];
    __shared__ uint32_t s_h[FB_HS];
    __shared__ uint32_t s_rng[2];
    const uint32_t F = min(*pb.fb_count, w_max);
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < 2 * F; q += gridDim.x * blockDim.x) {
        const uint32_t j = pb.fb_list[q >> 1];
        const uint32_t x = (q & 1u) ? t.v[j] : t.u[j];
        pb.fb_dslot[q] = G.deg[x] > FB_WARP_MAX ? pb.fb_slot[x] : NONE;
    }
    const unsigned long long nb = *fb_nb(pb);
    const uint32_t S = (uint32_t)(nb >> 32), total = min((uint32_t)nb, FB_CHUNK_CAP);
    for (uint32_t ch = blockIdx.x; ch < total; ch += gridDim.x) {
        // the chunk's slot: the last one whose first chunk is <= ch (slot 0 starts at 0)
        uint32_t lo = 0, hi = S;
        while (hi - lo > 1u) {
            const uint32_t mid = (lo + hi) >> 1;
            if (pb.fb_cbase[mid] <= ch) lo = mid;
            else hi = mid;
        }
        const uint32_t cb = pb.fb_cbase[lo], x = pb.fb_big[lo];
        const uint32_t d = G.deg[x];
        if (cb + (d + FB_CHUNK - 1) / FB_CHUNK > FB_CHUNK_CAP) continue;  // scanned whole by k_fallback
        if (pb.fb_done[lo]) {
            if (ch != cb && threadIdx.x == 0) {
                pb.fb_pr[ch] = INFINITY;
                pb.fb_py[ch] = NONE;
                pb.fb_pw[ch] = 0.0;
            }
            continue;
        }
        const uint32_t k0 = (ch - cb) * FB_CHUNK, k1 = min(k0 + FB_CHUNK, d);
        double br = INFINITY, bw = 0.0;
        uint32_t by = NONE;
        fb_scan_staged(H, G, x, k0, k1, s_h, s_rng, br, by, bw);
        fb_block_min(br, by, bw, s_r, s_y, s_w);
        if (threadIdx.x == 0) {
            pb.fb_pr[ch] = br;
            pb.fb_py[ch] = by;
            pb.fb_pw[ch] = bw;
        }
        __syncthreads();
    }
}

// Fallback of a walked deletion whose walkers all missed: for each endpoint x,
// the G_b edge of minimum resistance not in H' (ties: smaller neighbour id).
// One block per deletion: an endpoint with a slot takes the minimum over its
// chunks' results, any other endpoint list is scanned by the block.  The
// claims of the split scan are cleared here (nothing below reads them).
__global__ void __launch_bounds__(256) k_fallback(CSRView H, CSRView G, WalkTasks t, dg_update_result* res,
                                                  BatchCounters* ctr, Cands c, PathBufs pb, uint32_t w_max,
                                                  uint32_t* d_err) {
    {
        const uint32_t S = (uint32_t)(*fb_nb(pb) >> 32);
        for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < S; q += gridDim.x * blockDim.x)
            pb.fb_slot[pb.fb_big[q]] = NONE;
    }
    if (walk_aborted(d_err)) return;
    __shared__ double s_r[8];
    __shared__ uint32_t s_y[8];
    __shared__ double s_w[8];
    __shared__ uint32_t pick_y[2];
    __shared__ double pick_w[2];
    __shared__ uint32_t s_h[FB_HS];
    __shared__ uint32_t s_rng[2];
    const uint32_t F = min(*pb.fb_count, w_max);
    const uint32_t n = (uint32_t)G.n;
    for (uint32_t f = blockIdx.x; f < F; f += gridDim.x) {
        const uint32_t j = pb.fb_list[f];
        const uint32_t ends[2] = {t.u[j], t.v[j]};
        for (int e2 = 0; e2 < 2; ++e2) {
            const uint32_t x = ends[e2];
            const uint32_t d = G.deg[x];
            const uint32_t sl = pb.fb_dslot[2 * f + e2];
            const uint32_t cb = sl != NONE ? pb.fb_cbase[sl] : 0u;
            const uint32_t P = (d + FB_CHUNK - 1) / FB_CHUNK;
            double br = INFINITY, bw = 0.0;
            uint32_t by = NONE;
            if (sl != NONE && cb + P <= FB_CHUNK_CAP) {
                for (uint32_t q = threadIdx.x; q < P; q += blockDim.x) {
                    const double rr = pb.fb_pr[cb + q];
                    const uint32_t yy = pb.fb_py[cb + q];
                    if (rr < br || (rr == br && yy < by)) {
                        br = rr;
                        by = yy;
                        bw = pb.fb_pw[cb + q];
                    }
                }
            } else {
                fb_scan_staged(H, G, x, 0u, d, s_h, s_rng, br, by, bw);
            }
            fb_block_min(br, by, bw, s_r, s_y, s_w);
            if (threadIdx.x == 0) {
                pick_y[e2] = by;
                pick_w[e2] = bw;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const uint32_t i = t.idx[j];
            uint32_t emitted = 0;
            for (int e2 = 0; e2 < 2; ++e2) {
                if (pick_y[e2] == NONE) continue;
                // both endpoints picked the edge (u, v) itself (it was re-inserted in the batch)
                if (e2 == 1 && pick_y[0] != NONE && pick_y[0] == ends[1] && pick_y[1] == ends[0]) continue;
                emit_edge(c, ends[e2], pick_y[e2], pick_w[e2], n, d_err);
                ++emitted;
            }
            res[i].nrecovered = (int32_t)emitted;
            if (emitted) atomicAdd(&ctr->recovered, (unsigned long long)emitted);
        }
        __syncthreads();
    }
}

// one thread per (deletion, path edge): recover the edge unless it already
// appeared earlier in the same walk or is in H'
__global__ void k_emit_path(CSRView H, WalkTasks t, WalkParams p, dg_update_result* res, BatchCounters* ctr,
                            Cands c, PathBufs pb, uint32_t w_max, uint32_t* d_err) {
    if (walk_aborted(d_err)) return;
    const uint32_t W = min(*t.count, w_max);
    const uint32_t n = (uint32_t)H.n;
    const uint64_t items = (uint64_t)W * p.T;
    for (uint64_t it = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; it < items;
         it += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t j = (uint32_t)(it / p.T), s = (uint32_t)(it - (uint64_t)j * p.T);
        if (s >= pb.len[j]) continue;
        const uint32_t* path = pb.v + (size_t)j * (p.T + 1);
        const uint32_t x = path[s], y = path[s + 1];
        bool dup = false;
        for (uint32_t s2 = 0; s2 < s && !dup; ++s2) {
            const uint32_t a0 = path[s2], a1 = path[s2 + 1];
            dup = (a0 == x && a1 == y) || (a0 == y && a1 == x);
        }
        if (dup || has_edge(H, x, y)) continue;
        emit_edge(c, x, y, pb.w[(size_t)j * p.T + s], n, d_err);
        atomicAdd(&res[t.idx[j]].nrecovered, 1);
        atomicAdd(&ctr->recovered, 1ull);
    }
}

void launch_emit(const CSRView& H, const CSRView& G, const WalkTasks& t, const WalkParams& p,
                 const WalkRecs& r, const BatchHdr* d_hdr, const int32_t* best, const double* fin_w,
                 dg_update_result* res, BatchCounters* ctr, Cands c, PathBufs pb, uint32_t w_max,
                 uint32_t* d_err, cudaStream_t st) {
    uint32_t blocks = (w_max + 127) / 128;
    const uint32_t cap = (uint32_t)device_sms() * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    DG_CUDA(cudaMemsetAsync(pb.fb_count, 0, 16, st));
    k_replay<<<blocks, 128, 0, st>>>(H, G, t, p, r, d_hdr, best, fin_w, res, ctr, c, pb, w_max, d_err);
    k_emit_path<<<(unsigned)device_sms() * 8, 256, 0, st>>>(H, t, p, res, ctr, c, pb, w_max, d_err);
    g_launches += 2;
    DG_CHECK_LAUNCH();
    launch_fallback(H, G, t, res, ctr, c, pb, w_max, d_err, st);
}

void launch_fallback(const CSRView& H, const CSRView& G, const WalkTasks& t, dg_update_result* res,
                     BatchCounters* ctr, Cands c, PathBufs pb, uint32_t w_max, uint32_t* d_err, cudaStream_t st) {
    const unsigned sms = (unsigned)device_sms();
    k_fb_quick<<<sms * 2, 256, 0, st>>>(H, G, pb, d_err);
    k_fb_chunks<<<sms * 4, 256, 0, st>>>(H, G, t, pb, w_max, d_err);
    k_fallback<<<sms * 4, 256, 0, st>>>(H, G, t, res, ctr, c, pb, w_max, d_err);
    g_launches += 3;
    DG_CHECK_LAUNCH();
}

}  // namespace dg
