// dg_batch.cu -- graph load / sparsifier init / the batch step of Algorithm 1.
//
// Batch step (one snapshot per batch, the deferral of Section III-F):
//   pre:    validate updates in order (runs of equal edge keys after a stable
//           sort), net G changes, H removals (Algorithm 1 deletion branch),
//           plan + execute both mutations, walks (Section III-B/C), reduction
//           (Eq. 12, accept rule);
//   commit: kept insertions + recovered / fallback edges (Section III-C) as
//           sorted unique half-edges not already in H', merged into H.
// All kernels read their counts from device memory, so the whole step can be
// captured once per batch-size class and replayed as a CUDA graph.
#include <chrono>
#include <cmath>
#include <cstring>
#include <thread>

#include "dg_ctx.h"

namespace dg {

constexpr int BT = 256;  // threads per block of the small batch kernels

__device__ __forceinline__ bool batch_aborted(const uint32_t* d_err) { return (*d_err & ABORT_MASK) != 0u; }

static cudaError_t record_event(cudaEvent_t ev, cudaStream_t st) { return record_timing_event(ev, st); }

static int grid_for(uint64_t items) {
    uint64_t g = (items + BT - 1) / BT;
    const uint64_t cap = (uint64_t)device_sms() * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

// ---------------------------------------------------------------------------
// load / init kernels
// ---------------------------------------------------------------------------
__global__ void k_load_keys(const int32_t* __restrict__ u, const int32_t* __restrict__ v,
                            const double* __restrict__ w, uint32_t m, uint32_t n, uint64_t* __restrict__ keys,
                            uint32_t* __restrict__ vals, uint32_t* d_err) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const int32_t a = u[i], b = v[i];
        const double ww = w[i];
        const bool ok = a >= 0 && b >= 0 && (uint32_t)a < n && (uint32_t)b < n && a != b && isfinite(ww) && ww > 0.0;
        if (!ok) {
            atomicOr(d_err, (uint32_t)ERR_BAD_INPUT);
            keys[2 * i] = 0;
            keys[2 * i + 1] = 0;
        } else {
            keys[2 * i] = (uint64_t)a * n + (uint32_t)b;
            keys[2 * i + 1] = (uint64_t)b * n + (uint32_t)a;
        }
        vals[2 * i] = i;
        vals[2 * i + 1] = i;
    }
}

// H(0) half-edges with weights looked up in G
__global__ void k_inith_keys(const int32_t* __restrict__ u, const int32_t* __restrict__ v, uint32_t m, CSRView G,
                             uint64_t* __restrict__ keys, uint32_t* __restrict__ vals, double* __restrict__ ws,
                             uint32_t* d_err) {
    const uint32_t n = (uint32_t)G.n;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const int32_t a = u[i], b = v[i];
        double w = 0.0;
        const bool ok = a >= 0 && b >= 0 && (uint32_t)a < n && (uint32_t)b < n && a != b &&
                        has_edge(G, (uint32_t)a, (uint32_t)b, &w);
        if (!ok) {
            atomicOr(d_err, (uint32_t)ERR_NOT_IN_G);
            keys[2 * i] = 0;
            keys[2 * i + 1] = 0;
        } else {
            keys[2 * i] = (uint64_t)a * n + (uint32_t)b;
            keys[2 * i + 1] = (uint64_t)b * n + (uint32_t)a;
        }
        vals[2 * i] = 2 * i;
        vals[2 * i + 1] = 2 * i + 1;
        ws[2 * i] = w;
        ws[2 * i + 1] = w;
    }
}

// keep the first of each run of equal keys
__global__ void k_first_of_run(const uint64_t* __restrict__ keys, const uint32_t* d_n, uint32_t n_max,
                               uint32_t* __restrict__ flag) {
    const uint32_t n = d_n ? min(*d_n, n_max) : n_max;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        flag[c] = (c == 0 || keys[c - 1] != keys[c]) ? 1u : 0u;
}

__global__ void k_compact_kv(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                             const uint32_t* __restrict__ flag, const uint32_t* __restrict__ pos,
                             const uint32_t* d_n, uint32_t n_max, uint64_t* __restrict__ okeys,
                             uint32_t* __restrict__ ovals) {
    const uint32_t n = d_n ? min(*d_n, n_max) : n_max;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        if (flag[c]) {
            okeys[pos[c]] = keys[c];
            ovals[pos[c]] = vals[c];
        }
}

// ---------------------------------------------------------------------------
// batch kernels
// ---------------------------------------------------------------------------
// per update: basic checks (op, range, self-loop, weight); sort key of its edge
// Edge keys of the batch go into an open-addressing table (2^k >= 2 b_max
// slots, all-ones = empty, cleared per batch); *dup is set when a key is seen
// twice.  Without repeated edges every update is its own run and validation
// needs no sort.
__device__ __forceinline__ void note_key(unsigned long long* table, uint32_t mask, uint64_t key, uint32_t* dup) {
    uint32_t h = (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> 32) & mask;
    for (uint32_t probe = 0; probe <= mask; ++probe) {  // at most half full: ends at an empty slot
        const unsigned long long old = atomicCAS(&table[h], ~0ull, (unsigned long long)key);
        if (old == ~0ull) return;
        if (old == key) {
            atomicOr(dup, 1u);
            return;
        }
        h = (h + 1) & mask;
    }
    atomicOr(dup, 1u);  // unreachable at load <= 1/2; sorting is always correct
}

__global__ void k_val_prep(const dg_update* __restrict__ ups, const BatchHdr* hdr, uint32_t n, uint32_t b_max,
                           dg_update_result* __restrict__ res, uint64_t* __restrict__ keys,
                           uint32_t* __restrict__ vals, uint8_t* __restrict__ wkind, double* __restrict__ fin_w,
                           uint32_t* __restrict__ fdel, uint32_t* __restrict__ fins, unsigned long long* table,
                           uint32_t tmask, uint32_t* dup) {
    const uint32_t nu = min(hdr->nu, b_max);
    const uint64_t sent = (uint64_t)n * n;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nu; i += gridDim.x * blockDim.x) {
        const dg_update up = ups[i];
        int32_t st = ST_OK;
        if (up.op != DG_OP_INSERT && up.op != DG_OP_DELETE) st = ST_BAD_OP;
        else if (up.u < 0 || up.v < 0 || (uint32_t)up.u >= n || (uint32_t)up.v >= n) st = ST_BAD_VERTEX;
        else if (up.u == up.v) st = ST_SELF_LOOP;
        else if (up.op == DG_OP_INSERT && !(isfinite(up.w) && up.w > 0.0)) st = ST_BAD_WEIGHT;
        dg_update_result r;
        r.status = st;
        r.walked = r.hit = r.accepted = r.fallback = 0;
        r.nhits = 0;
        r.best_walker = -1;
        r.nrecovered = 0;
        r.steps = 0;
        r.r_est = INFINITY;
        res[i] = r;
        if (st == ST_OK) {
            const uint32_t a = (uint32_t)min(up.u, up.v), b = (uint32_t)max(up.u, up.v);
            keys[i] = (uint64_t)a * n + b;
            note_key(table, tmask, keys[i], dup);
        } else {
            keys[i] = sent;
        }
        vals[i] = i;
        wkind[i] = WALK_NONE;
        fdel[i] = 0;  // walked-deletion / walked-insertion flags, set by k_val_runs
        fins[i] = 0;
        fin_w[i] = __longlong_as_double(0x7ff8000000000000ll);  // NaN: edge absent at batch end
    }
}

struct RunArgs {
    const uint64_t* keys;        // sorted by key (when *dup), else the keys in update order
    const uint32_t* vals;
    const uint64_t* keys_plain;  // update order
    const uint32_t* vals_plain;
    const uint32_t* dup;
    const dg_update* ups;
    const BatchHdr* hdr;
    uint32_t n, b_max;
    CSRView G, H;
    dg_update_result* res;
    uint8_t* wkind;
    uint32_t* fdel;  // walk flags per update (deletions / insertions)
    uint32_t* fins;
    double* fin_w;
    // net G changes (half-edges), appended
    uint64_t* gkeys;
    uint32_t* gvals;
    uint8_t* gkind;
    uint8_t* ghrem;
    double* gw;
    uint32_t* gcount;
    BatchCounters* ctr;
};

// Is {x, y} in G (and with which weight) and in H?  The two lookups run side by
// side (each in the shorter of the two endpoint lists) so their dependent
// loads overlap instead of adding up.
__device__ __forceinline__ void lookup_gh(const CSRView& G, const CSRView& H, uint32_t x, uint32_t y, bool& in_g,
                                          double& w, bool& in_h) {
    const uint32_t gx = G.deg[x], gy = G.deg[y], hx = H.deg[x], hy = H.deg[y];
    const uint32_t ga = gy < gx ? y : x, gb = gy < gx ? x : y, gd = gy < gx ? gy : gx;
    const uint32_t ha = hy < hx ? y : x, hb = hy < hx ? x : y, hd = hy < hx ? hy : hx;
    const Ent* LG = G.pool + G.off[ga];
    const Ent* LH = H.pool + H.off[ha];
    uint32_t glo = 0, ghi = gd, hlo = 0, hhi = hd;
    while (glo < ghi || hlo < hhi) {
        const uint32_t gm = (glo + ghi) >> 1, hm = (hlo + hhi) >> 1;
        const uint32_t gv = glo < ghi ? LG[gm].nbr : 0u;
        const uint32_t hv = hlo < hhi ? LH[hm].nbr : 0u;
        if (glo < ghi) {
            if (gv < gb) glo = gm + 1; else ghi = gm;
        }
        if (hlo < hhi) {
            if (hv < hb) hlo = hm + 1; else hhi = hm;
        }
    }
    in_g = glo < gd && LG[glo].nbr == gb;
    w = in_g ? LG[glo].w : 0.0;
    in_h = hlo < hd && LH[hlo].nbr == hb;
}

// one thread per run of equal edges: replay the run in update order against
// the batch-local view (presence, weight) of that edge
__global__ void k_val_runs(RunArgs a) {
    const uint32_t nu = min(a.hdr->nu, a.b_max);
    const uint64_t sent = (uint64_t)a.n * a.n;
    if (!*a.dup) {  // every edge appears once: the update-order arrays are runs of one
        a.keys = a.keys_plain;
        a.vals = a.vals_plain;
    }
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < nu; c += gridDim.x * blockDim.x) {
        const uint64_t key = a.keys[c];
        if (key == sent) continue;
        if (c > 0 && a.keys[c - 1] == key) continue;
        const uint32_t x = (uint32_t)(key / a.n), y = (uint32_t)(key % a.n);
        double w0 = 0.0;
        bool present0 = false, h0 = false;
        lookup_gh(a.G, a.H, x, y, present0, w0, h0);
        const bool in_h = present0 && h0;
        bool state = present0, any_valid = false, hrem = false;
        double wcur = w0;
        uint32_t valid = 0;
        uint32_t e = c;
        for (; e < nu && a.keys[e] == key; ++e) {
            const uint32_t i = a.vals[e];
            const dg_update up = a.ups[i];
            if (up.op == DG_OP_INSERT) {
                if (state) {
                    a.res[i].status = ST_DUP_INSERT;
                } else {
                    state = true;
                    wcur = up.w;
                    any_valid = true;
                    ++valid;
                    a.wkind[i] = WALK_INS;
                    a.fins[i] = 1;
                    a.res[i].walked = 1;
                }
            } else {
                if (!state) {
                    a.res[i].status = ST_MISSING_DELETE;
                } else {
                    state = false;
                    any_valid = true;
                    ++valid;
                    if (in_h) {
                        hrem = true;
                        a.wkind[i] = WALK_DEL;
                        a.fdel[i] = 1;
                        a.res[i].walked = 1;
                    }
                }
            }
        }
        // final presence / weight of the edge, needed by kept insertions
        if (state)
            for (uint32_t e2 = c; e2 < e; ++e2) {
                const uint32_t i = a.vals[e2];
                if (a.wkind[i] == WALK_INS) a.fin_w[i] = wcur;
            }
        agg_count(&a.ctr->valid, valid);
        uint8_t kind = 255;
        if (present0 && !state) kind = CHG_DEL;
        else if (!present0 && state) kind = CHG_INS;
        else if (present0 && state && any_valid) kind = CHG_SETW;
        if (kind == 255) continue;
        const uint32_t pos = agg_add(a.gcount, 2u);
        a.gkeys[pos] = key;
        a.gkeys[pos + 1] = (uint64_t)y * a.n + x;
        a.gvals[pos] = pos;
        a.gvals[pos + 1] = pos + 1;
        a.gkind[pos] = a.gkind[pos + 1] = kind;
        a.ghrem[pos] = a.ghrem[pos + 1] = hrem ? 1 : 0;
        a.gw[pos] = a.gw[pos + 1] = wcur;
    }
}

// Task list from the walk flags k_val_runs set: walked deletions (no K, the
// longest walks) first, so they start first and the short insertion walks
// fill the tail of the persistent launch.
// Largest R >= 0 (as an FP64 bit pattern) with fl(w_pq * R) <= K.  The
// rounded product is non-decreasing in R and non-negative doubles order like
// their bit patterns, so the insertion threshold test of a walk step becomes
// one integer comparison R_bits <= r_limit, with the same outcome as forming
// the product.  Binary search over the patterns of [0, +inf].
__device__ uint64_t r_limit_bits(double wpq, double K) {
    uint64_t lo = 0ull, hi = 0x7FF0000000000000ull;  // fl(w * 0) = 0 <= K
    if (__dmul_rn(wpq, __longlong_as_double((long long)hi)) <= K) return hi;
    while (hi - lo > 1ull) {
        const uint64_t mid = lo + ((hi - lo) >> 1);
        if (__dmul_rn(wpq, __longlong_as_double((long long)mid)) <= K) lo = mid;
        else hi = mid;
    }
    return lo;
}

__global__ void k_make_tasks(const dg_update* __restrict__ ups, const uint8_t* __restrict__ wkind,
                             const uint32_t* __restrict__ pdel, const uint32_t* __restrict__ pins,
                             const uint32_t* __restrict__ totals, const BatchHdr* hdr, uint32_t b_max, double K,
                             WalkTasks t, uint32_t* __restrict__ fin, uint32_t* __restrict__ queue,
                             uint32_t* __restrict__ qctr) {
    const uint32_t nu = min(hdr->nu, b_max);
    const uint32_t ndel = totals[0];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *t.count = ndel + totals[1];
        qctr[0] = 0;
        qctr[1] = 0;
    }
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nu; i += gridDim.x * blockDim.x) {
        const uint8_t k = wkind[i];
        if (k == WALK_NONE) continue;
        const uint32_t j = k == WALK_DEL ? pdel[i] : ndel + pins[i];
        const dg_update up = ups[i];
        t.u[j] = (uint32_t)up.u;
        t.v[j] = (uint32_t)up.v;
        t.idx[j] = i;
        t.wpq[j] = k == WALK_INS ? up.w : 0.0;
        fin[j] = 0;
        queue[j] = 0xFFFFFFFFu;
        t.rmax[j] = k == WALK_INS ? r_limit_bits(up.w, K) : ~0ull;
        t.kind[j] = k;
    }
}

// commit candidates: first of each equal-key run and not already in H'
__global__ void k_commit_flags(const uint64_t* __restrict__ keys, const uint32_t* d_n, uint32_t n_max, CSRView H,
                               uint32_t* __restrict__ flag, const uint32_t* d_err) {
    if (batch_aborted(d_err)) return;
    const uint32_t n = min(*d_n, n_max);
    const uint32_t nv = (uint32_t)H.n;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const uint64_t k = keys[c];
        bool keep = (c == 0 || keys[c - 1] != k);
        if (keep) keep = find_nbr(H, (uint32_t)(k / nv), (uint32_t)(k % nv)) == 0xFFFFFFFFu;
        flag[c] = keep ? 1u : 0u;
    }
}

// ---------------------------------------------------------------------------
// workspace
// ---------------------------------------------------------------------------
uint64_t BatchWS::bytes() const {
    uint64_t b = 0;
    b += ups.bytes() + res.bytes() + hdr.bytes() + err.bytes() + ctr.bytes() + next.bytes();
    b += vkeys.bytes() + vkeys_alt.bytes() + vvals.bytes() + vvals_alt.bytes() + vhist.bytes() + vscan.bytes();
    b += wkind.bytes() + fin_w.bytes() + wflag.bytes() + wpos.bytes() + wflag2.bytes() + wpos2.bytes();
    b += gkeys.bytes() + gkeys_alt.bytes() + hkeys.bytes() + gvals.bytes() + gvals_alt.bytes() + ghist.bytes();
    b += gscan.bytes() + gcount.bytes() + hpos.bytes() + hvals.bytes() + hcount.bytes();
    b += gkind.bytes() + ghrem.bytes() + kind_del.bytes() + gw.bytes() + vtab.bytes();
    b += t_u.bytes() + t_v.bytes() + t_idx.bytes() + t_kstar.bytes() + t_count.bytes() + meta.bytes();
    b += t_fin.bytes() + t_queue.bytes() + qctr.bytes() + cp.bytes() + step_r.bytes() + step_e.bytes();
    b += t_wpq.bytes() + t_rmax.bytes() + recR.bytes() + t_kind.bytes() + best.bytes();
    b += ckeys.bytes() + ckeys_alt.bytes() + ck2.bytes() + cvals.bytes() + cvals_alt.bytes() + chist.bytes();
    b += cscan.bytes() + ccount.bytes() + cflag.bytes() + cpos.bytes() + cv2.bytes() + ccount2.bytes();
    b += cw.bytes() + kind_ins.bytes() + path_buf.bytes() + path_len.bytes() + path_w.bytes() + fb_list.bytes() +
         fb_count.bytes();
    b += fb_slot.bytes() + fb_big.bytes() + fb_cbase.bytes() + fb_done.bytes() + fb_dslot.bytes() + fb_py.bytes() + fb_pr.bytes() +
         fb_pw.bytes();
    b += dbg_reason.bytes() + dbg_steps.bytes() + dbg_paths.bytes() + shard_recs.bytes();
    b += apG.bytes() + apH.bytes() + apC.bytes();
    return b;
}

static void ensure_cands(Ctx& c, DGraph& g, uint32_t cap, cudaStream_t st) {
    BatchWS& w = g.ws;
    if (cap <= w.cand_cap && w.ckeys.p) return;
    DevAlloc& a = c.alloc;
    w.ckeys.ensure(a, cap, st);
    w.ckeys_alt.ensure(a, cap, st);
    w.ck2.ensure(a, cap, st);
    w.cvals.ensure(a, cap, st);
    w.cvals_alt.ensure(a, cap, st);
    w.cflag.ensure(a, cap, st);
    w.cpos.ensure(a, cap, st);
    w.cv2.ensure(a, cap, st);
    w.cw.ensure(a, cap, st);
    w.kind_ins.ensure(a, cap, st);
    DG_CUDA(cudaMemsetAsync(w.kind_ins.p, CHG_INS, w.kind_ins.bytes(), st));
    w.chist.ensure(a, sort_hist_words(cap), st);
    w.cscan.ensure(a, std::max(sort_scan_tmp_words(cap), scan_tmp_words(cap + 1)), st);
    w.apC.ensure(a, cap, (uint64_t)cap * 8, st);
    w.cand_cap = cap;
    ++g.layout_gen;
}

static void ensure_ws(Ctx& c, DGraph& g, uint32_t b_max, cudaStream_t st) {
    BatchWS& w = g.ws;
    const uint32_t s = (uint32_t)c.cfg.s, T = (uint32_t)c.cfg.T;
    const bool need_dbg = c.cfg.record && !w.dbg_reason.p;
    if (b_max <= w.b_max && !need_dbg) return;
    if (b_max < w.b_max) b_max = w.b_max;
    DevAlloc& a = c.alloc;
    const uint32_t B = b_max, B2 = 2 * b_max;
    w.ups.ensure(a, B, st);
    w.res.ensure(a, B, st);
    w.hdr.ensure(a, 1, st);
    w.err.ensure(a, 4, st);
    w.ctr.ensure(a, 1, st);
    w.next.ensure(a, 1, st);
    w.vkeys.ensure(a, B, st);
    w.vtab_slots = 1024;
    while (w.vtab_slots < 2 * B) w.vtab_slots *= 2;
    w.vtab.ensure(a, (size_t)w.vtab_slots + 1, st);
    w.vkeys_alt.ensure(a, B, st);
    w.vvals.ensure(a, B, st);
    w.vvals_alt.ensure(a, B, st);
    w.vhist.ensure(a, sort_hist_words(B), st);
    w.vscan.ensure(a, std::max(sort_scan_tmp_words(B), scan_tmp_words(B + 1)), st);
    w.wkind.ensure(a, B, st);
    w.fin_w.ensure(a, B, st);
    w.wflag.ensure(a, B, st);
    w.wpos.ensure(a, B, st);
    w.wflag2.ensure(a, B, st);
    w.wpos2.ensure(a, B, st);
    w.gkeys.ensure(a, B2, st);
    w.gkeys_alt.ensure(a, B2, st);
    w.hkeys.ensure(a, B2, st);
    w.gvals.ensure(a, B2, st);
    w.gvals_alt.ensure(a, B2, st);
    w.ghist.ensure(a, sort_hist_words(B2), st);
    w.gscan.ensure(a, std::max(sort_scan_tmp_words(B2), scan_tmp_words(B2 + 1)), st);
    w.gcount.ensure(a, 1, st);
    w.hpos.ensure(a, B2, st);
    w.hvals.ensure(a, B2, st);
    w.hcount.ensure(a, 1, st);
    w.gkind.ensure(a, B2, st);
    w.ghrem.ensure(a, B2, st);
    w.kind_del.ensure(a, B2, st);
    DG_CUDA(cudaMemsetAsync(w.kind_del.p, CHG_DEL, w.kind_del.bytes(), st));
    w.gw.ensure(a, B2, st);
    w.t_u.ensure(a, B, st);
    w.t_v.ensure(a, B, st);
    w.t_idx.ensure(a, B, st);
    w.t_kstar.ensure(a, B, st);
    w.t_fin.ensure(a, B, st);
    w.t_queue.ensure(a, B, st);
    w.qctr.ensure(a, 2, st);
    // Step records of deletion walkers replace the resume points (no replay
    // at finalization) while they fit in STEP_REC_BYTES: 12 bytes per slot of
    // B * T * s.
    constexpr uint64_t STEP_REC_BYTES = 6ull << 30;
    if ((uint64_t)B * T * s * 12 <= STEP_REC_BYTES) {
        w.step_r.ensure(a, (size_t)B * T * s, st);
        w.step_e.ensure(a, (size_t)B * T * s, st);
    } else {  // records of a smaller workspace must not be used at this size
        w.step_r.release(a, st);
        w.step_e.release(a, st);
        if (walk_ncp(T) > 0) w.cp.ensure(a, (size_t)B * s * walk_ncp(T), st);
    }
    w.t_count.ensure(a, 4, st);
    w.t_wpq.ensure(a, B, st);
    w.t_rmax.ensure(a, B, st);
    w.t_kind.ensure(a, B, st);
    w.best.ensure(a, B, st);
    w.meta.ensure(a, (size_t)B * s, st);
    w.recR.ensure(a, (size_t)B * s, st);
    w.ccount.ensure(a, 1, st);
    w.ccount2.ensure(a, 1, st);
    w.path_buf.ensure(a, (size_t)B * (T + 1), st);
    w.path_w.ensure(a, (size_t)B * T, st);
    w.path_len.ensure(a, B, st);
    w.fb_list.ensure(a, B, st);
    w.fb_count.ensure(a, 4, st);
    w.fb_big.ensure(a, (size_t)B * 2, st);
    w.fb_cbase.ensure(a, (size_t)B * 2, st);
    w.fb_done.ensure(a, (size_t)B * 2, st);
    w.fb_dslot.ensure(a, (size_t)B * 2, st);
    w.fb_pr.ensure(a, FB_CHUNK_CAP, st);
    w.fb_pw.ensure(a, FB_CHUNK_CAP, st);
    w.fb_py.ensure(a, FB_CHUNK_CAP, st);
    if (!w.fb_slot.p || w.fb_slot.n < (size_t)g.n) {  // all unclaimed
        w.fb_slot.ensure(a, (size_t)g.n, st);
        DG_CUDA(cudaMemsetAsync(w.fb_slot.p, 0xFF, w.fb_slot.bytes(), st));
    }
    if (c.cfg.record) {
        w.dbg_reason.ensure(a, (size_t)B * s, st);
        w.dbg_steps.ensure(a, (size_t)B * s, st);
        if (T <= 256) w.dbg_paths.ensure(a, (size_t)B * s * (T + 1), st);
    }
    w.apG.ensure(a, B2, (uint64_t)B2 * 16, st);
    w.apH.ensure(a, B2, (uint64_t)B2 * 16, st);
    w.b_max = b_max;
    ensure_cands(c, g, std::max<uint32_t>(B2 * 2, w.cand_cap), st);
    // pinned staging
    if (g.hs.cap < b_max) {
        if (g.hs.ups) {
            cudaFreeHost(g.hs.ups);
            cudaFreeHost(g.hs.res);
        }
        DG_CUDA(cudaMallocHost(&g.hs.ups, sizeof(dg_update) * b_max));
        DG_CUDA(cudaMallocHost(&g.hs.res, sizeof(dg_update_result) * b_max));
        g.hs.cap = b_max;
    }
    if (!g.hs.hdr) {
        DG_CUDA(cudaMallocHost(&g.hs.hdr, sizeof(BatchHdr)));
        DG_CUDA(cudaMallocHost(&g.hs.err, sizeof(uint32_t) * 4));
        DG_CUDA(cudaMallocHost(&g.hs.ctr, sizeof(BatchCounters)));
        DG_CUDA(cudaMallocHost(&g.hs.tops, sizeof(unsigned long long) * 2));
        DG_CUDA(cudaMallocHost(&g.hs.counts, sizeof(uint32_t) * 8));
        DG_CUDA(cudaHostGetDevicePointer((void**)&g.hs.d_err, g.hs.err, 0));
        DG_CUDA(cudaHostGetDevicePointer((void**)&g.hs.d_ctr, g.hs.ctr, 0));
        DG_CUDA(cudaHostGetDevicePointer((void**)&g.hs.d_tops, g.hs.tops, 0));
        DG_CUDA(cudaHostGetDevicePointer((void**)&g.hs.d_counts, g.hs.counts, 0));
    }
    ++g.layout_gen;
}

static uint32_t bucket_of(uint64_t nu) {
    uint32_t b = 1024;
    while (b < nu) b <<= 1;
    return b;
}

// ---------------------------------------------------------------------------
// load / init / export
// ---------------------------------------------------------------------------
// host memory allocated pinned or registered with CUDA (copied without staging)
static bool host_pinned(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeHost;
}

static void wait_stream(Ctx& c, cudaStream_t st) {
    cudaEvent_t ev;
    DG_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    DG_CUDA(cudaEventRecord(ev, st));
    const int tmo = c.cfg.timeout_ms > 0 ? c.cfg.timeout_ms : 60000;
    const double t0 = now_ms();
    for (;;) {
        cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) {
            cudaEventDestroy(ev);
            throw Error(DG_E_CUDA, std::string("device error: ") + cudaGetErrorString(e));
        }
        const double t = now_ms() - t0;
        if (t > tmo) {
            cudaEventDestroy(ev);
            throw Error(DG_E_TIMEOUT, "device work did not finish within timeout_ms");
        }
        // a batch step takes about a millisecond: poll without sleeping at first,
        // so the caller sees the result within microseconds of the device
        if (t > 2.0) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    cudaEventDestroy(ev);
}

void graph_load(Ctx& c, DGraph& g, int32_t n, int64_t m, const int32_t* u, const int32_t* v, const double* w) {
    cudaStream_t st = c.stream;
    DevAlloc& a = c.alloc;
    if (n < 0 || m < 0) throw Error(DG_E_INVALID, "negative size");
    if ((uint64_t)n * (uint64_t)n >= (1ull << 62)) throw Error(DG_E_INVALID, "too many vertices");
    if (2 * (uint64_t)m >= 0xFFFFFFF0ull) throw Error(DG_E_INVALID, "too many edges");
    g.n = n;
    g.G.slack = g.H.slack = (float)c.cfg.slack;
    g.G.overflow = g.H.overflow = c.cfg.overflow;
    csr_alloc_vertices(g.G, a, n, st);
    csr_alloc_vertices(g.H, a, n, st);
    g.touched.ensure(a, (size_t)n + 1, st);
    DG_CUDA(cudaMemsetAsync(g.touched.p, 0, g.touched.bytes(), st));
    g.touched_h.ensure(a, (size_t)n + 1, st);
    DG_CUDA(cudaMemsetAsync(g.touched_h.p, 0, g.touched_h.bytes(), st));
    const uint32_t M = (uint32_t)m, M2 = 2 * (uint32_t)m;
    DBuf<int32_t> du, dv;
    DBuf<double> dw;
    DBuf<uint64_t> k0, k1;
    DBuf<uint32_t> v0, v1, hist, stmp, err;
    du.ensure(a, M + 1, st);
    dv.ensure(a, M + 1, st);
    dw.ensure(a, M + 1, st);
    k0.ensure(a, M2 + 1, st);
    k1.ensure(a, M2 + 1, st);
    v0.ensure(a, M2 + 1, st);
    v1.ensure(a, M2 + 1, st);
    hist.ensure(a, sort_hist_words(M2 + 1), st);
    stmp.ensure(a, sort_scan_tmp_words(M2 + 1), st);
    err.ensure(a, 1, st);
    DG_CUDA(cudaMemsetAsync(err.p, 0, 4, st));
    if (M) {
        DG_CUDA(cudaMemcpyAsync(du.p, u, 4ull * M, cudaMemcpyHostToDevice, st));
        DG_CUDA(cudaMemcpyAsync(dv.p, v, 4ull * M, cudaMemcpyHostToDevice, st));
        DG_CUDA(cudaMemcpyAsync(dw.p, w, 8ull * M, cudaMemcpyHostToDevice, st));
        k_load_keys<<<grid_for(M), BT, 0, st>>>(du.p, dv.p, dw.p, M, (uint32_t)n, k0.p, v0.p, err.p);
        ++g_launches;
    }
    uint32_t herr = 0;
    DG_CUDA(cudaMemcpyAsync(&herr, err.p, 4, cudaMemcpyDeviceToHost, st));
    wait_stream(c, st);
    auto cleanup = [&]() {
        du.release(a, st); dv.release(a, st); k0.release(a, st); k1.release(a, st);
        v0.release(a, st); v1.release(a, st); hist.release(a, st); stmp.release(a, st); err.release(a, st);
        dw.release(a, st);
    };
    if (herr) {
        cleanup();
        throw Error(DG_E_INVALID, "graph edge with a vertex out of range, a self-loop or a weight not finite > 0");
    }
    const uint64_t* keys = k0.p;
    const uint32_t* vals = v0.p;
    if (M2) {
        SortBufs sb{k0.p, v0.p, k1.p, v1.p, hist.p, stmp.p};
        const int nbits = bit_length((uint64_t)n * n - 1);
        if (radix_sort_pairs(sb, nullptr, M2, nbits, st)) {
            keys = k1.p;
            vals = v1.p;
        }
    }
    csr_build(g.G, a, keys, vals, dw.p, M2, err.p, st);
    DG_CUDA(cudaMemcpyAsync(&herr, err.p, 4, cudaMemcpyDeviceToHost, st));
    wait_stream(c, st);
    cleanup();
    if (herr & ERR_DUP_EDGE) throw Error(DG_E_INVALID, "graph lists an edge twice");
    if (herr) throw Error(DG_E_CUDA, "internal error while building the graph");
    csr_build(g.H, a, nullptr, nullptr, nullptr, 0, nullptr, st);
    g.has_h = true;  // empty sparsifier
    g.next_id = 0;
    for (int i = 0; i < 9; ++i) DG_CUDA(cudaEventCreate(&g.ev[i]));
    for (int i = 0; i < 7; ++i) DG_CUDA(cudaEventCreateWithFlags(&g.fk[i], cudaEventDisableTiming));
    DG_CUDA(cudaEventCreateWithFlags(&g.ev_mut, cudaEventDisableTiming));
    DG_CUDA(cudaEventCreateWithFlags(&g.ev_est, cudaEventDisableTiming));
    DG_CUDA(cudaStreamCreateWithFlags(&g.side, cudaStreamNonBlocking));
    wait_stream(c, st);
    graph_mark_mutation(g, st);
}

// Work that changes G or H first waits for the walk estimates already issued
// on this graph (a wait on an event never recorded returns at once).
void graph_wait_estimates(DGraph& g, cudaStream_t st) {
    if (g.ev_est) DG_CUDA(cudaStreamWaitEvent(st, g.ev_est, 0));
}

void graph_mark_mutation(DGraph& g, cudaStream_t st) {
    if (g.ev_mut) DG_CUDA(cudaEventRecord(g.ev_mut, st));
}

void graph_init_h(Ctx& c, DGraph& g, int64_t mh, const int32_t* u, const int32_t* v, bool device_arrays) {
    if (g.shard.active) throw Error(DG_E_STATE, "a sharded batch is in progress on this graph");
    cudaStream_t st = c.stream;
    DevAlloc& a = c.alloc;
    if (mh < 0 || 2 * (uint64_t)mh >= 0xFFFFFFF0ull) throw Error(DG_E_INVALID, "bad sparsifier size");
    const uint32_t M = (uint32_t)mh, M2 = 2 * M;
    DBuf<int32_t> du, dv;
    DBuf<double> dw;
    DBuf<uint64_t> k0, k1, k2;
    DBuf<uint32_t> v0, v1, v2, hist, stmp, err, flag, pos, cnt;
    du.ensure(a, M + 1, st);
    dv.ensure(a, M + 1, st);
    dw.ensure(a, M2 + 1, st);
    k0.ensure(a, M2 + 1, st);
    k1.ensure(a, M2 + 1, st);
    k2.ensure(a, M2 + 1, st);
    v0.ensure(a, M2 + 1, st);
    v1.ensure(a, M2 + 1, st);
    v2.ensure(a, M2 + 1, st);
    flag.ensure(a, M2 + 1, st);
    pos.ensure(a, M2 + 1, st);
    cnt.ensure(a, 2, st);
    hist.ensure(a, sort_hist_words(M2 + 1), st);
    stmp.ensure(a, std::max(sort_scan_tmp_words(M2 + 1), scan_tmp_words(M2 + 1)), st);
    err.ensure(a, 1, st);
    DG_CUDA(cudaMemsetAsync(err.p, 0, 4, st));
    DG_CUDA(cudaMemsetAsync(cnt.p, 0, 8, st));
    if (M) {
        const cudaMemcpyKind kind = device_arrays ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        DG_CUDA(cudaMemcpyAsync(du.p, u, 4ull * M, kind, st));
        DG_CUDA(cudaMemcpyAsync(dv.p, v, 4ull * M, kind, st));
        k_inith_keys<<<grid_for(M), BT, 0, st>>>(du.p, dv.p, M, g.G.view(), k0.p, v0.p, dw.p, err.p);
        ++g_launches;
    }
    uint32_t herr = 0;
    DG_CUDA(cudaMemcpyAsync(&herr, err.p, 4, cudaMemcpyDeviceToHost, st));
    wait_stream(c, st);
    auto cleanup = [&]() {
        DBuf<int32_t>* i32s[] = {&du, &dv};
        for (auto* b : i32s) b->release(a, st);
        DBuf<uint64_t>* u64s[] = {&k0, &k1, &k2};
        for (auto* b : u64s) b->release(a, st);
        DBuf<uint32_t>* u32s[] = {&v0, &v1, &v2, &hist, &stmp, &err, &flag, &pos, &cnt};
        for (auto* b : u32s) b->release(a, st);
        dw.release(a, st);
    };
    if (herr) {
        cleanup();
        throw Error(DG_E_INVALID, "sparsifier edge that is not an edge of G");
    }
    const uint64_t* keys = k0.p;
    const uint32_t* vals = v0.p;
    uint32_t uniq = 0;
    if (M2) {
        SortBufs sb{k0.p, v0.p, k1.p, v1.p, hist.p, stmp.p};
        const int nbits = bit_length((uint64_t)g.n * g.n - 1);
        if (radix_sort_pairs(sb, nullptr, M2, nbits, st)) {
            keys = k1.p;
            vals = v1.p;
        }
        k_first_of_run<<<grid_for(M2), BT, 0, st>>>(keys, nullptr, M2, flag.p);
        ScanJob j;
        j.in[0] = flag.p;
        j.out[0] = pos.p;
        j.total[0] = cnt.p;
        j.k = 1;
        scan_exclusive(j, nullptr, M2, stmp.p, st);
        k_compact_kv<<<grid_for(M2), BT, 0, st>>>(keys, vals, flag.p, pos.p, nullptr, M2, k2.p, v2.p);
        g_launches += 2;
        DG_CUDA(cudaMemcpyAsync(&uniq, cnt.p, 4, cudaMemcpyDeviceToHost, st));
        wait_stream(c, st);
    }
    graph_wait_estimates(g, st);
    csr_release(g.H, a, st);
    g.H.slack = (float)c.cfg.slack;
    g.H.overflow = c.cfg.overflow;
    csr_alloc_vertices(g.H, a, g.n, st);
    csr_build(g.H, a, k2.p, v2.p, dw.p, uniq, err.p, st);
    DG_CUDA(cudaMemcpyAsync(&herr, err.p, 4, cudaMemcpyDeviceToHost, st));
    wait_stream(c, st);
    cleanup();
    if (herr) throw Error(DG_E_CUDA, "internal error while building the sparsifier");
    g.has_h = true;
    ++g.layout_gen;
    graph_mark_mutation(g, st);
}

void graph_export(Ctx& c, DGraph& g, bool which_h, int64_t cap, int32_t* u, int32_t* v, double* w,
                  int64_t* count, cudaStream_t st) {
    CSR& s = which_h ? g.H : g.G;
    DevAlloc& a = c.alloc;
    const uint64_t cnt = csr_edge_count(s, a, st);
    if (count) *count = (int64_t)cnt;
    if (!u && !v && !w) return;  // size query
    if ((int64_t)cnt > cap) throw Error(DG_E_INVALID, "output arrays too small (count_out holds the size)");
    if (cnt == 0) return;
    DBuf<int32_t> da, db;
    DBuf<double> dw;
    da.ensure(a, cnt, st);
    db.ensure(a, cnt, st);
    dw.ensure(a, cnt, st);
    csr_export(s, a, da.p, db.p, dw.p, st);
    if (u) DG_CUDA(cudaMemcpyAsync(u, da.p, 4 * cnt, cudaMemcpyDeviceToHost, st));
    if (v) DG_CUDA(cudaMemcpyAsync(v, db.p, 4 * cnt, cudaMemcpyDeviceToHost, st));
    if (w) DG_CUDA(cudaMemcpyAsync(w, dw.p, 8 * cnt, cudaMemcpyDeviceToHost, st));
    wait_stream(c, st);
    da.release(a, st);
    db.release(a, st);
    dw.release(a, st);
}

void graph_compact(Ctx& c, DGraph& g, cudaStream_t st) {
    if (g.shard.active) throw Error(DG_E_STATE, "a sharded batch is in progress on this graph");
    graph_wait_estimates(g, st);
    csr_compact(g.G, c.alloc, 0, st);
    csr_compact(g.H, c.alloc, 0, st);
    ++g.layout_gen;
    graph_mark_mutation(g, st);
}

void graph_release(Ctx& c, DGraph& g) {
    cudaStream_t st = c.stream;
    if (g.ev_est) cudaEventSynchronize(g.ev_est);
    cudaStreamSynchronize(st);
    if (g.stream) cudaStreamSynchronize(g.stream);
    for (auto& kv : g.steps)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    g.steps.clear();
    csr_release(g.G, c.alloc, st);
    csr_release(g.H, c.alloc, st);
    g.touched.release(c.alloc, st);
    g.touched_h.release(c.alloc, st);
    graph_release_ws(c, g, st);
    if (g.hs.ups) cudaFreeHost(g.hs.ups);
    if (g.hs.res) cudaFreeHost(g.hs.res);
    if (g.hs.hdr) cudaFreeHost(g.hs.hdr);
    if (g.hs.err) cudaFreeHost(g.hs.err);
    if (g.hs.ctr) cudaFreeHost(g.hs.ctr);
    if (g.hs.tops) cudaFreeHost(g.hs.tops);
    if (g.hs.counts) cudaFreeHost(g.hs.counts);
    g.hs = HostStage{};
    for (int i = 0; i < 9; ++i)
        if (g.ev[i]) cudaEventDestroy(g.ev[i]);
    for (int i = 0; i < 7; ++i)
        if (g.fk[i]) cudaEventDestroy(g.fk[i]);
    if (g.ev_mut) cudaEventDestroy(g.ev_mut);
    if (g.ev_est) cudaEventDestroy(g.ev_est);
    g.ev_mut = g.ev_est = nullptr;
    if (g.side) {
        cudaStreamSynchronize(g.side);
        cudaStreamDestroy(g.side);
    }
    g.side = nullptr;
    if (g.stream) cudaStreamDestroy(g.stream);
    g.stream = nullptr;
    cudaStreamSynchronize(st);
}

// give back a graph's batch workspace (it is re-created by the next batch)
void graph_release_ws(Ctx& c, DGraph& g, cudaStream_t st) {
    for (auto& kv : g.steps)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    g.steps.clear();
    BatchWS& w = g.ws;
    w.apG.release(c.alloc, st);
    w.apH.release(c.alloc, st);
    w.apC.release(c.alloc, st);
#define REL(b) w.b.release(c.alloc, st)
    REL(ups); REL(res); REL(hdr); REL(err); REL(ctr); REL(next); REL(vkeys); REL(vtab); REL(vkeys_alt); REL(vvals);
    REL(vvals_alt); REL(vhist); REL(vscan); REL(wkind); REL(fin_w); REL(wflag); REL(wpos); REL(wflag2); REL(wpos2); REL(gkeys);
    REL(gkeys_alt); REL(hkeys); REL(gvals); REL(gvals_alt); REL(ghist); REL(gscan); REL(gcount);
    REL(hpos); REL(hvals); REL(hcount); REL(gkind); REL(ghrem); REL(kind_del); REL(gw); REL(t_u); REL(t_v);
    REL(t_idx); REL(t_kstar); REL(t_fin); REL(t_queue); REL(qctr); REL(cp); REL(step_r); REL(step_e); REL(t_count); REL(meta); REL(t_wpq); REL(t_rmax); REL(recR); REL(t_kind); REL(best);
    REL(ckeys); REL(ckeys_alt); REL(ck2); REL(cvals); REL(cvals_alt); REL(chist); REL(cscan); REL(ccount);
    REL(cflag); REL(cpos); REL(cv2); REL(ccount2); REL(cw); REL(kind_ins); REL(path_buf); REL(path_w); REL(path_len); REL(fb_list); REL(fb_count); REL(fb_slot); REL(fb_big); REL(fb_cbase); REL(fb_done); REL(fb_dslot); REL(fb_py); REL(fb_pr); REL(fb_pw); REL(dbg_reason);
    REL(dbg_steps); REL(dbg_paths); REL(shard_recs);
#undef REL
    w.b_max = 0;
    w.cand_cap = 0;
    ++g.layout_gen;
}

// ---------------------------------------------------------------------------
// the batch step
// ---------------------------------------------------------------------------

static WalkTasks tasks_of(BatchWS& w) {
    WalkTasks t;
    t.u = w.t_u.p;
    t.v = w.t_v.p;
    t.idx = w.t_idx.p;
    t.wpq = w.t_wpq.p;
    t.rmax = w.t_rmax.p;
    t.kind = w.t_kind.p;
    t.kstar = w.t_kstar.p;
    t.count = w.t_count.p;
    return t;
}

static WalkParams params_of(const Config& cfg) {
    WalkParams p;
    p.K = cfg.K;
    p.T = (uint32_t)cfg.T;
    p.s = (uint32_t)cfg.s;
    p.early_exit = cfg.early_exit ? 1u : 0u;
    p.del_prune = cfg.del_prune ? 1u : 0u;
    p.key0 = (uint32_t)cfg.seed;
    p.key1 = (uint32_t)(cfg.seed >> 32);
    return p;
}

static Cands cands_of(BatchWS& w) {
    Cands cd;
    cd.keys = w.ckeys.p;
    cd.vals = w.cvals.p;
    cd.w = w.cw.p;
    cd.count = w.ccount.p;
    cd.cap = w.cand_cap;
    return cd;
}

static PathBufs paths_of(BatchWS& w) {
    return PathBufs{w.path_buf.p, w.path_w.p, w.path_len.p, w.fb_list.p, w.fb_count.p, w.fb_slot.p,
                    w.fb_big.p,   w.fb_cbase.p, w.fb_done.p, w.fb_dslot.p, w.fb_pr.p, w.fb_pw.p, w.fb_py.p};
}

static FinArgs fin_of(Ctx& c, BatchWS& w, bool on) {
    FinArgs f;
    f.res = w.res.p;
    f.best = w.best.p;
    f.ctr = w.ctr.p;
    f.dbg_reason = c.cfg.record ? w.dbg_reason.p : nullptr;
    f.dbg_steps = c.cfg.record ? w.dbg_steps.p : nullptr;
    f.fin = w.t_fin.p;
    f.queue = w.t_queue.p;
    f.qctr = w.qctr.p;
    f.fin_w = w.fin_w.p;
    f.c = cands_of(w);
    f.pb = paths_of(w);
    f.pr = on ? w.step_r.p : nullptr;
    f.pe = on ? w.step_e.p : nullptr;
    f.cp = (on && !f.pr) ? w.cp.p : nullptr;
    f.cp_shift = walk_cp_shift((uint32_t)c.cfg.T);
    f.ncp = walk_ncp((uint32_t)c.cfg.T);
    f.on = on ? 1u : 0u;
    f.spin_limit = c.fin_wait_polls < 0 ? FIN_SPIN_LIMIT : (uint32_t)std::min<int64_t>(c.fin_wait_polls, FIN_SPIN_LIMIT);
    return f;
}

static WalkRecs recs_of(Ctx& c, BatchWS& w) {
    WalkRecs r;
    r.meta = w.meta.p;
    r.R = w.recR.p;
    r.paths = (c.cfg.record && w.dbg_paths.p) ? w.dbg_paths.p : nullptr;
    return r;
}

// scratch regions a batch step needs zero on entry (look-back scan status,
// sort histograms, counters)
struct ClearList {
    static constexpr int MAX = 16;
    uint32_t* p[MAX];
    uint32_t words[MAX];
    int n = 0;
    void add(uint32_t* ptr, size_t w, size_t cap) {
        if (n >= MAX || w > cap || w > 0xFFFFFFFFull) throw Error(DG_E_CUDA, "batch scratch layout");
        p[n] = ptr;
        words[n] = (uint32_t)w;
        ++n;
    }
};

// per-batch state cleared in one launch: error words (4), counters, change
// count, k* bounds (all ones), the edge-key table (all ones) and the
// repeated-edge flag behind it (2 words), and the regions of the clear list
__global__ void k_batch_reset(uint32_t* err, BatchCounters* ctr, uint32_t* gcount, uint32_t* kstar, uint32_t B,
                              unsigned long long* vtab, uint32_t vtab_slots, ClearList cl) {
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t n = B > vtab_slots ? B : vtab_slots;
    for (uint32_t i = gt; i < n; i += stride) {
        if (i < B) kstar[i] = 0xFFFFFFFFu;
        if (i < vtab_slots) vtab[i] = ~0ull;
    }
    for (int e = 0; e < cl.n; ++e) {
        uint32_t* p = cl.p[e];
        const uint32_t w = cl.words[e];
        for (uint32_t i = gt; i < w; i += stride) p[i] = 0u;
    }
    if (blockIdx.x == 0) {
        const uint32_t t = threadIdx.x;
        if (t < 4) err[t] = 0u;
        if (t < sizeof(BatchCounters) / sizeof(unsigned long long))
            reinterpret_cast<unsigned long long*>(ctr)[t] = 0ull;
        if (t == 32) *gcount = 0u;
        if (t == 33) vtab[vtab_slots] = 0ull;  // the repeated-edge flag words
    }
}

// validation and both mutations (G -> G_b, H -> H'); nothing is written to G
// or H unless both plans found enough space
static void enqueue_mutate(Ctx& c, DGraph& g, cudaStream_t st) {
    BatchWS& w = g.ws;
    const uint32_t B = w.b_max, B2 = 2 * w.b_max, n = (uint32_t)g.n, CC = w.cand_cap;
    const int bits_v = bit_length((uint64_t)n * n), bits_g = bit_length((uint64_t)n * n - 1);
    {
        // scratch of this step's scans and sorts (validation, G changes, both
        // plans, commit) and the walk's candidate and fallback counts
        ClearList cl;
        cl.add(w.vhist.p, sort_clear_words(B, bits_v), w.vhist.n);
        cl.add(w.vscan.p, scan_tmp_words(B), w.vscan.n);
        cl.add(w.ghist.p, sort_clear_words(B2, bits_g), w.ghist.n);
        cl.add(w.gscan.p, scan_tmp_words(B2), w.gscan.n);
        cl.add(w.apG.scan_tmp.p, 2 * w.apG.scan_words, w.apG.scan_tmp.n);
        cl.add(w.apH.scan_tmp.p, 2 * w.apH.scan_words, w.apH.scan_tmp.n);
        cl.add(w.chist.p, sort_clear_words(CC, bits_g), w.chist.n);
        cl.add(w.cscan.p, scan_tmp_words(CC), w.cscan.n);
        cl.add(w.apC.scan_tmp.p, 2 * w.apC.scan_words, w.apC.scan_tmp.n);
        cl.add(w.ccount.p, 1, w.ccount.n);
        cl.add(w.fb_count.p, 4, w.fb_count.n);
        const uint64_t items = std::max<uint64_t>(B, w.vtab_slots);
        int blocks = grid_for(items);
        if (blocks < 1) blocks = 1;
        k_batch_reset<<<blocks, BT, 0, st>>>(w.err.p, w.ctr.p, w.gcount.p, w.t_kstar.p, B, w.vtab.p, w.vtab_slots,
                                            cl);
        ++g_launches;
    }
    const uint32_t* d_nu = &w.hdr.p->nu;
    uint32_t* d_dup = reinterpret_cast<uint32_t*>(w.vtab.p + w.vtab_slots);
    k_val_prep<<<grid_for(B), BT, 0, st>>>(w.ups.p, w.hdr.p, n, B, w.res.p, w.vkeys.p, w.vvals.p, w.wkind.p,
                                          w.fin_w.p, w.wflag.p, w.wflag2.p, w.vtab.p, w.vtab_slots - 1u, d_dup);
    ++g_launches;
    // sorted by edge key only when some edge appears twice (the kernels return at once otherwise)
    SortBufs vs{w.vkeys.p, w.vvals.p, w.vkeys_alt.p, w.vvals_alt.p, w.vhist.p, w.vscan.p, w.err.p};
    const bool valt = radix_sort_pairs(vs, d_nu, B, bits_v, st, d_dup, true);
    RunArgs ra;
    ra.keys = valt ? w.vkeys_alt.p : w.vkeys.p;
    ra.vals = valt ? w.vvals_alt.p : w.vvals.p;
    ra.keys_plain = w.vkeys.p;
    ra.vals_plain = w.vvals.p;
    ra.dup = d_dup;
    ra.ups = w.ups.p;
    ra.hdr = w.hdr.p;
    ra.n = n;
    ra.b_max = B;
    ra.G = g.G.view();
    ra.H = g.H.view();
    ra.res = w.res.p;
    ra.wkind = w.wkind.p;
    ra.fin_w = w.fin_w.p;
    ra.gkeys = w.gkeys.p;
    ra.gvals = w.gvals.p;
    ra.gkind = w.gkind.p;
    ra.ghrem = w.ghrem.p;
    ra.gw = w.gw.p;
    ra.gcount = w.gcount.p;
    ra.ctr = w.ctr.p;
    ra.fdel = w.wflag.p;
    ra.fins = w.wflag2.p;
    k_val_runs<<<grid_for(B), BT, 0, st>>>(ra);
    ++g_launches;
    // Two streams from here (captured as parallel branches of the step's graph):
    //   side: walk tasks; H' = H minus the deleted H edges (list, plan, execute)
    //   st:   sort of the net G changes; G_b (plan, execute)
    // Each execution also waits for the other CSR's plan, so an abort raised by
    // either plan still leaves both G and H untouched.
    cudaStream_t sd = g.side;
    DG_CUDA(cudaEventRecord(g.fk[0], st));
    DG_CUDA(cudaStreamWaitEvent(sd, g.fk[0], 0));
    {
        ScanJob j;
        j.in[0] = w.wflag.p;
        j.out[0] = w.wpos.p;
        j.total[0] = w.t_count.p + 2;
        j.in[1] = w.wflag2.p;
        j.out[1] = w.wpos2.p;
        j.total[1] = w.t_count.p + 3;
        j.k = 2;
        j.err = w.err.p;
        scan_exclusive(j, d_nu, B, w.vscan.p, sd, true);
    }
    WalkTasks tasks = tasks_of(w);
    k_make_tasks<<<grid_for(B), BT, 0, sd>>>(w.ups.p, w.wkind.p, w.wpos.p, w.wpos2.p, w.t_count.p + 2, w.hdr.p, B,
                                            c.cfg.K, tasks, w.t_fin.p, w.t_queue.p, w.qctr.p);
    ++g_launches;
    // net G changes, sorted by (vertex, neighbour)
    SortBufs gs{w.gkeys.p, w.gvals.p, w.gkeys_alt.p, w.gvals_alt.p, w.ghist.p, w.gscan.p, w.err.p};
    const bool galt = radix_sort_pairs(gs, w.gcount.p, B2, bits_g, st, nullptr, true);
    const uint64_t* gk = galt ? w.gkeys_alt.p : w.gkeys.p;
    const uint32_t* gv = galt ? w.gvals_alt.p : w.gvals.p;
    DG_CUDA(cudaEventRecord(g.fk[1], st));
    DG_CUDA(cudaStreamWaitEvent(sd, g.fk[1], 0));
    {
        // H's change list: the G changes that remove an H edge, compacted by
        // the scan of their flags (generated from the removal marks)
        ScanJob j;
        j.gen.mode = 2;
        j.gen.bytes = w.ghrem.p;
        j.gen.idx = gv;
        j.out[0] = w.hpos.p;
        j.total[0] = w.hcount.p;
        j.k = 1;
        j.err = w.err.p;
        j.cmp.keys = gk;
        j.cmp.vals = gv;
        j.cmp.okeys = w.hkeys.p;
        j.cmp.ovals = w.hvals.p;
        scan_exclusive(j, w.gcount.p, B2, w.gscan.p, sd, true);
    }
    ChangeList clG;
    clG.keys = gk;
    clG.vals = gv;
    clG.kinds = w.gkind.p;
    clG.ws = w.gw.p;
    clG.d_count = w.gcount.p;
    clG.max_count = B2;
    ChangeList clH;
    clH.keys = w.hkeys.p;
    clH.vals = w.hvals.p;
    clH.kinds = w.kind_del.p;
    clH.ws = w.gw.p;
    clH.d_count = w.hcount.p;
    clH.max_count = B2;
    csr_plan(g.H, clH, w.apH, w.err.p, ERR_POOL_G, ERR_CAP_PRE, sd, true);
    DG_CUDA(cudaEventRecord(g.fk[2], sd));
    csr_plan(g.G, clG, w.apG, w.err.p, ERR_POOL_G, ERR_CAP_PRE, st, true);
    DG_CUDA(cudaEventRecord(g.fk[3], st));
    DG_CUDA(cudaStreamWaitEvent(st, g.fk[2], 0));
    DG_CUDA(cudaStreamWaitEvent(sd, g.fk[3], 0));
    csr_exec(g.G, clG, w.apG, g.touched.p, w.err.p, st, g.ev[7], g.ev[8]);
    csr_exec(g.H, clH, w.apH, g.touched_h.p, w.err.p, sd);
    DG_CUDA(cudaEventRecord(g.fk[4], sd));
    DG_CUDA(cudaStreamWaitEvent(st, g.fk[4], 0));
    DG_CUDA(record_event(g.ev[4], st));
}

// Walks on the snapshot (H' for insertions, G_b for deletions) and the
// per-update reduction; per_update_W >= 0 selects the one-launch-per-update
// form.  A single batched launch also finalizes every update (reduction,
// argmin path, commit candidates) in the walk's tail; returns true then, and
// the commit only adds the fallbacks left to the block-wide kernel.
static bool enqueue_walks(Ctx& c, DGraph& g, cudaStream_t st, int64_t per_update_W) {
    BatchWS& w = g.ws;
    const WalkParams wp = params_of(c.cfg);
    const WalkRecs wr = recs_of(c, w);
    const WalkTasks tasks = tasks_of(w);
    const uint32_t cut = g.shape.cut > 1 ? (uint32_t)g.shape.cut : 1u;
    const bool tiled = g.shape.lanes > 1 || g.shape.tile > 0;
    const bool fused = per_update_W < 0 && cut == 1 && !tiled;
    // (the candidate and fallback counts start at zero: cleared with the step's
    // scratch, and again after the autotuner's trial walks)
    DG_CUDA(record_event(g.ev[0], st));
    if (per_update_W < 0) {
        for (uint32_t c2 = 0; c2 < cut; ++c2) {
            const uint32_t lo = (uint32_t)((uint64_t)w.b_max * c2 / cut);
            const uint32_t hi = (uint32_t)((uint64_t)w.b_max * (c2 + 1) / cut);
            if (tiled)
                launch_walk_tiled(g.H.view(), g.G.view(), tasks, wp, wr, w.hdr.p, w.next.p, lo, hi, g.shape,
                                  w.err.p, st);
            else
                launch_walk_batched(g.H.view(), g.G.view(), tasks, wp, wr, w.hdr.p, w.next.p, lo, hi, g.shape,
                                    fin_of(c, w, fused), w.err.p, st, g.side, g.fk[5], g.fk[6]);
        }
    } else {
        for (int64_t j = 0; j < per_update_W; ++j)
            launch_walk_one(g.H.view(), g.G.view(), tasks, wp, wr, w.hdr.p, (uint32_t)j, w.err.p, st);
    }
    DG_CUDA(record_event(g.ev[1], st));
    if (!fused)
        launch_walk_reduce(g.G.view(), tasks, wp, wr, w.hdr.p, w.res.p, w.best.p, w.ctr.p,
                           c.cfg.record ? w.dbg_reason.p : nullptr, c.cfg.record ? w.dbg_steps.p : nullptr, 0u,
                           w.b_max, w.err.p, st);
    DG_CUDA(record_event(g.ev[5], st));
    return fused;
}

// Autotuner: after the mutation of one large batch, time the walk phase on
// that snapshot under each candidate launch shape (threads per block, walkers
// per thread), then the batch cut for the winner, and keep the fastest.  Every
// trial computes the same walks (outputs never depend on the shape); the
// batch's own walk then runs once more with the chosen shape.
static void autotune_walks(Ctx& c, DGraph& g, cudaStream_t st) {
    BatchWS& w = g.ws;
    const WalkParams wp = params_of(c.cfg);
    const WalkRecs wr = recs_of(c, w);
    const WalkTasks tasks = tasks_of(w);
    cudaEvent_t e0, e1;
    DG_CUDA(cudaEventCreate(&e0));
    DG_CUDA(cudaEventCreate(&e1));
    // each trial starts from a cold L2 (a write larger than L2), as a batch does
    const size_t flush_bytes = 192ull << 20;
    void* flush = c.alloc.get(flush_bytes, st);
    auto trial = [&](const WalkShape& sh) -> float {
        DG_CUDA(cudaMemsetAsync(flush, 0, flush_bytes, st));
        DG_CUDA(cudaMemsetAsync(w.t_kstar.p, 0xFF, 4ull * w.b_max, st));
        DG_CUDA(cudaEventRecord(e0, st));
        for (int cidx = 0; cidx < sh.cut; ++cidx) {
            const uint32_t lo = (uint32_t)((uint64_t)w.b_max * cidx / sh.cut);
            const uint32_t hi = (uint32_t)((uint64_t)w.b_max * (cidx + 1) / sh.cut);
            if (sh.lanes > 1 || sh.tile > 0)
                launch_walk_tiled(g.H.view(), g.G.view(), tasks, wp, wr, w.hdr.p, w.next.p, lo, hi, sh, w.err.p, st);
            else
                launch_walk_batched(g.H.view(), g.G.view(), tasks, wp, wr, w.hdr.p, w.next.p, lo, hi, sh,
                                    fin_of(c, w, false), w.err.p, st);
        }
        DG_CUDA(cudaEventRecord(e1, st));
        wait_stream(c, st);
        float ms = 0.f;
        DG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        return ms;
    };
    // every trial starts from a flushed L2; a candidate's time is the median of
    // three runs, and it replaces the default shape (256 threads x 2 walkers)
    // only when it is at least 3 % faster
    g.tune_log.clear();
    auto median3 = [&](const WalkShape& sh) {
        float a0 = trial(sh), a1 = trial(sh), a2 = trial(sh);
        const float m = std::max(std::min(a0, a1), std::min(std::max(a0, a1), a2));
        g.tune_log.push_back({sh, m});
        return m;
    };
    WalkShape best;
    best.block = 256;
    best.ilp = 2;
    best.blocks_per_sm = 0;
    best.cut = 1;
    trial(best);
    float best_ms = median3(best);
    const int shapes[][2] = {{128, 2}, {64, 2}, {256, 1}, {128, 1}, {256, 4}};
    for (const auto& bi : shapes) {
        WalkShape sh;
        sh.block = bi[0];
        sh.ilp = bi[1];
        sh.blocks_per_sm = 0;
        sh.cut = 1;
        const float ms = median3(sh);
        if (ms < best_ms * 0.97f) {
            best_ms = ms;
            best = sh;
        }
    }
    // then the refill threshold of the winning shape
    const WalkShape base = best;
    for (const int rf : {1, 8, 24, 32}) {
        WalkShape sh = base;
        sh.refill = rf;
        const float ms = median3(sh);
        if (ms < best_ms * 0.97f) {
            best_ms = ms;
            best = sh;
        }
    }
    // then the tiled launch: lanes per walker and updates per block claim
    // (its walks are followed by separate reduction and emission kernels, so
    // it must win by more than the in-kernel finalization it gives up)
    const int coop[][2] = {{1, 1}, {1, 4}, {2, 1}, {4, 1}, {8, 1}, {32, 1}, {32, 4}};
    for (const auto& lt : coop) {
        WalkShape sh;
        sh.block = 256;
        sh.ilp = 1;
        sh.lanes = lt[0];
        sh.tile = lt[1];
        const float ms = median3(sh);
        if (ms < best_ms * 0.85f) {
            best_ms = ms;
            best = sh;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c.alloc.put(flush, flush_bytes, st);
    DG_CUDA(cudaMemsetAsync(w.t_kstar.p, 0xFF, 4ull * w.b_max, st));
    DG_CUDA(cudaMemsetAsync(w.ccount.p, 0, 4, st));
    DG_CUDA(cudaMemsetAsync(w.fb_count.p, 0, 16, st));
    g.shape = best;
    g.tuned = true;
    g.stats.autotuned = 1;
    ++g.layout_gen;
}

// kept insertions, recovered and fallback edges -> H (re-runnable).  After a
// finalizing walk (walk_emitted) the candidates are already there except the
// fallbacks at long lists; otherwise they are generated here from the results.
// scratch_zeroed: the commit's sort, scan and plan scratch were cleared at the
// step start and not used since (false when only the commit re-runs)
static void enqueue_commit(Ctx& c, DGraph& g, cudaStream_t st, bool walk_emitted, bool scratch_zeroed) {
    BatchWS& w = g.ws;
    const uint32_t B = w.b_max, n = (uint32_t)g.n, CC = w.cand_cap;
    const Cands cd = cands_of(w);
    if (walk_emitted) {
        launch_fallback(g.H.view(), g.G.view(), tasks_of(w), w.res.p, w.ctr.p, cd, paths_of(w), B, w.err.p, st);
    } else {
        DG_CUDA(cudaMemsetAsync(w.ccount.p, 0, 4, st));
        launch_emit(g.H.view(), g.G.view(), tasks_of(w), params_of(c.cfg), recs_of(c, w), w.hdr.p, w.best.p,
                    w.fin_w.p, w.res.p, w.ctr.p, cd, paths_of(w), B, w.err.p, st);
    }
    DG_CUDA(record_event(g.ev[6], st));
    SortBufs cs{w.ckeys.p, w.cvals.p, w.ckeys_alt.p, w.cvals_alt.p, w.chist.p, w.cscan.p, w.err.p};
    const bool calt = radix_sort_pairs(cs, w.ccount.p, CC, bit_length((uint64_t)n * n - 1), st, nullptr,
                                       scratch_zeroed);
    const uint64_t* ck = calt ? w.ckeys_alt.p : w.ckeys.p;
    const uint32_t* cv = calt ? w.cvals_alt.p : w.cvals.p;
    k_commit_flags<<<grid_for(CC), BT, 0, st>>>(ck, w.ccount.p, CC, g.H.view(), w.cflag.p, w.err.p);
    ++g_launches;
    {
        ScanJob j;
        j.in[0] = w.cflag.p;
        j.out[0] = w.cpos.p;
        j.total[0] = w.ccount2.p;
        j.k = 1;
        j.err = w.err.p;
        j.cmp.keys = ck;  // the candidates kept, compacted by the same scan
        j.cmp.vals = cv;
        j.cmp.okeys = w.ck2.p;
        j.cmp.ovals = w.cv2.p;
        scan_exclusive(j, w.ccount.p, CC, w.cscan.p, st, scratch_zeroed);
    }
    ChangeList clC;
    clC.keys = w.ck2.p;
    clC.vals = w.cv2.p;
    clC.kinds = w.kind_ins.p;
    clC.ws = w.cw.p;
    clC.d_count = w.ccount2.p;
    clC.max_count = CC;
    csr_plan(g.H, clC, w.apC, w.err.p, ERR_POOL_H, ERR_CAP_COMMIT, st, scratch_zeroed);
    csr_exec(g.H, clC, w.apC, g.touched.p, w.err.p, st);
}

// the batch's status for the host (error words, counters, pool tops, walked
// and candidate counts), written by one kernel straight into pinned host
// memory: one node at the end of the captured step instead of six copies
__global__ void k_readback(const uint32_t* err, const BatchCounters* ctr, const unsigned long long* gtop,
                           const unsigned long long* htop, const uint32_t* t_count, const uint32_t* ccount,
                           const uint32_t* gtot, const uint32_t* gcount, uint32_t* h_err, BatchCounters* h_ctr,
                           unsigned long long* h_tops, uint32_t* h_counts) {
    constexpr unsigned CW = sizeof(BatchCounters) / sizeof(unsigned long long);
    static_assert(CW * sizeof(unsigned long long) == sizeof(BatchCounters) && CW <= 8, "counter words");
    const unsigned t = threadIdx.x;
    if (t < 4) h_err[t] = err[t];
    if (t >= 8 && t < 8 + CW)
        reinterpret_cast<unsigned long long*>(h_ctr)[t - 8] = reinterpret_cast<const unsigned long long*>(ctr)[t - 8];
    if (t == 16) h_tops[0] = *gtop;
    if (t == 17) h_tops[1] = *htop;
    if (t == 18) h_counts[0] = *t_count;
    if (t == 19) h_counts[1] = *ccount;
    // G's list execution: its work items (old entries + changes), net insertions
    // and deletions, and its change count (the size of the merge)
    if (t == 20) h_counts[2] = gtot[TOT_WK];
    if (t == 21) h_counts[3] = gtot[TOT_NI];
    if (t == 22) h_counts[4] = gtot[TOT_ND];
    if (t == 23) h_counts[5] = *gcount;
}

static void enqueue_readback(DGraph& g, cudaStream_t st) {
    BatchWS& w = g.ws;
    k_readback<<<1, 32, 0, st>>>(w.err.p, w.ctr.p, g.G.top.p, g.H.top.p, w.t_count.p, w.ccount.p,
                                 w.apG.totals.p, w.gcount.p, g.hs.d_err, g.hs.d_ctr, g.hs.d_tops, g.hs.d_counts);
    ++g_launches;
    DG_CHECK_LAUNCH();
}

static uint32_t read_total(ApplyScratch& s, int which, cudaStream_t st) {
    uint32_t v = 0;
    DG_CUDA(cudaMemcpyAsync(&v, s.totals.p + which, 4, cudaMemcpyDeviceToHost, st));
    DG_CUDA(cudaStreamSynchronize(st));
    return v;
}

// grow what an abort asked for; returns true when the whole batch must re-run
static bool handle_abort(Ctx& c, DGraph& g, uint32_t err, cudaStream_t st) {
    BatchWS& w = g.ws;
    DevAlloc& a = c.alloc;
    if (err & (ERR_POOL_G | ERR_CAP_PRE)) {
        if (err & ERR_POOL_G) {
            const uint32_t R = read_total(w.apG, TOT_R, st);
            csr_compact(g.G, a, (uint64_t)R * 2 + 4096, st);
        }
        if (err & ERR_CAP_PRE) {
            const uint64_t s1 = read_total(w.apG, TOT_S, st), s2 = read_total(w.apH, TOT_S, st);
            w.apG.ensure(a, w.apG.c_max, std::max<uint64_t>(s1 * 2, w.apG.s_cap), st);
            w.apH.ensure(a, w.apH.c_max, std::max<uint64_t>(s2 * 2, w.apH.s_cap), st);
        }
        ++g.layout_gen;
        return true;
    }
    if (err & ERR_POOL_H) {
        const uint32_t R = read_total(w.apC, TOT_R, st);
        csr_compact(g.H, a, (uint64_t)R * 2 + 4096, st);
    }
    if (err & ERR_CAP_COMMIT) {
        const uint32_t need = g.hs.counts[1];
        if (need > w.cand_cap) ensure_cands(c, g, need * 2, st);
        const uint64_t s3 = read_total(w.apC, TOT_S, st);
        if (s3 > w.apC.s_cap) w.apC.ensure(a, w.apC.c_max, s3 * 2, st);
    }
    ++g.layout_gen;
    return false;
}


// proactive growth so that most batches never abort
static void ensure_headroom(Ctx& c, DGraph& g, uint32_t nu, cudaStream_t st) {
    // a cheap guess of the relocation space one batch needs; a batch that needs
    // more aborts before writing anything, grows the pool and re-runs
    const uint64_t want = (uint64_t)nu * 16 + 4096;
    if (g.G.pool_cap - g.G.host_top < want) {
        csr_compact(g.G, c.alloc, want * 2, st);
        ++g.layout_gen;
    }
    if (g.H.pool_cap - g.H.host_top < want) {
        csr_compact(g.H, c.alloc, want * 2, st);
        ++g.layout_gen;
    }
}

// The whole batch step for batches of size class `bucket`, captured once as a
// CUDA graph (again whenever a buffer it names has moved).  direct: the
// update records reach the workspace outside the graph (device or pinned
// caller buffers); otherwise the graph copies them from the pinned staging.
static CapturedStep& capture_step(Ctx& c, DGraph& g, uint32_t bucket, bool direct, cudaStream_t st) {
    BatchWS& w = g.ws;
    CapturedStep& cs = g.steps[bucket];
    if (cs.exec && cs.layout_gen == g.layout_gen && cs.device_io == direct) return cs;
    if (cs.exec) cudaGraphExecDestroy(cs.exec);
    cs.exec = nullptr;
    cudaGraph_t graph = nullptr;
    const uint64_t k0 = g_launches;
    DG_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    try {
        DG_CUDA(cudaMemcpyAsync(w.hdr.p, g.hs.hdr, sizeof(BatchHdr), cudaMemcpyHostToDevice, st));
        if (!direct)
            DG_CUDA(cudaMemcpyAsync(w.ups.p, g.hs.ups, sizeof(dg_update) * bucket, cudaMemcpyHostToDevice, st));
        enqueue_mutate(c, g, st);
        const bool emitted = enqueue_walks(c, g, st, -1);
        enqueue_commit(c, g, st, emitted, true);
        if (!direct)
            DG_CUDA(cudaMemcpyAsync(g.hs.res, w.res.p, sizeof(dg_update_result) * bucket, cudaMemcpyDeviceToHost,
                                    st));
        enqueue_readback(g, st);
    } catch (...) {
        cudaStreamEndCapture(st, &graph);
        if (graph) cudaGraphDestroy(graph);
        throw;
    }
    DG_CUDA(cudaStreamEndCapture(st, &graph));
    DG_CUDA(cudaGraphInstantiate(&cs.exec, graph, 0));
    cudaGraphDestroy(graph);
    DG_CUDA(cudaGraphUpload(cs.exec, st));  // its first replay then pays no upload
    cs.layout_gen = g.layout_gen;
    cs.device_io = direct;
    cs.kernels = g_launches - k0;
    g_launches = k0;  // counted per replay
    return cs;
}

void graph_prepare(Ctx& c, DGraph& g, int64_t max_batch, cudaStream_t st) {
    if (!g.has_h) throw Error(DG_E_STATE, "no sparsifier");
    if (g.shard.active) throw Error(DG_E_STATE, "a sharded batch is in progress on this graph");
    if (max_batch < 1 || max_batch > (1ll << 26)) throw Error(DG_E_INVALID, "max_batch out of range");
    const uint32_t top = bucket_of((uint64_t)max_batch);
    ensure_ws(c, g, top, st);
    // pool headroom for several batches of the largest size, so that a long
    // stream of requests compacts rarely (a compaction stalls the graph)
    ensure_headroom(c, g, (uint32_t)std::min<int64_t>(8 * max_batch, 1ll << 26), st);
    if (c.cfg.use_graphs && !c.cfg.record && c.cfg.walk_mode == DG_WALK_BATCHED)
        for (uint32_t b = 1024; b <= top; b <<= 1) capture_step(c, g, b, false, st);
    wait_stream(c, st);
}

void graph_apply(Ctx& c, DGraph& g, int64_t nu64, const dg_update* ups, dg_update_result* res, bool device_io,
                 cudaStream_t st) {
    if (!g.has_h) throw Error(DG_E_STATE, "no sparsifier");
    if (g.shard.active) throw Error(DG_E_STATE, "a sharded batch is in progress on this graph");
    if (nu64 < 0 || nu64 > (1ll << 26)) throw Error(DG_E_INVALID, "batch size out of range");
    if (nu64 == 0) return;
    const uint32_t nu = (uint32_t)nu64;
    const uint64_t l0 = g_launches;
    const uint32_t bucket = bucket_of(nu);
    graph_wait_estimates(g, st);
    ensure_ws(c, g, bucket, st);
    ensure_headroom(c, g, nu, st);
    BatchWS& w = g.ws;
    const bool per_update = c.cfg.walk_mode == DG_WALK_PER_UPDATE;
    g.hs.hdr->nu = nu;
    g.hs.hdr->pad = 0;
    g.hs.hdr->id0 = g.next_id;
    // Records travel through the pinned staging buffers, or straight between the
    // caller's buffers and the batch workspace when those are device memory or
    // pinned host memory (then only nu records are copied, outside the graph).
    const bool direct = device_io || (host_pinned(ups) && (!res || host_pinned(res)));
    const cudaMemcpyKind kin = device_io ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind kout = device_io ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (!direct) std::memcpy(g.hs.ups, ups, sizeof(dg_update) * nu);

    auto stage_inputs = [&]() {
        DG_CUDA(cudaMemcpyAsync(w.hdr.p, g.hs.hdr, sizeof(BatchHdr), cudaMemcpyHostToDevice, st));
        if (!direct)
            DG_CUDA(cudaMemcpyAsync(w.ups.p, g.hs.ups, sizeof(dg_update) * nu, cudaMemcpyHostToDevice, st));
        else
            DG_CUDA(cudaMemcpyAsync(w.ups.p, ups, sizeof(dg_update) * nu, kin, st));
    };
    auto copy_results = [&]() {
        if (!direct)
            DG_CUDA(cudaMemcpyAsync(g.hs.res, w.res.p, sizeof(dg_update_result) * nu, cudaMemcpyDeviceToHost, st));
        else if (res)
            DG_CUDA(cudaMemcpyAsync(res, w.res.p, sizeof(dg_update_result) * nu, kout, st));
    };
    bool walk_emitted = false;  // the last walk launch also produced the commit candidates
    // eager form of the pre-commit part (validation, mutation, walks, reduction)
    auto run_pre = [&]() {
        enqueue_mutate(c, g, st);
        int64_t W = -1;
        if (per_update) {  // the per-update form needs the walked count on the host to issue its launches
            DG_CUDA(cudaMemcpyAsync(g.hs.counts, w.t_count.p, 4, cudaMemcpyDeviceToHost, st));
            DG_CUDA(cudaMemcpyAsync(g.hs.err, w.err.p, 4, cudaMemcpyDeviceToHost, st));
            wait_stream(c, st);
            W = (g.hs.err[0] & ABORT_MASK) ? 0 : g.hs.counts[0];
            if (g.hs.counts[0] > w.b_max) W = 0;
        }
        walk_emitted = enqueue_walks(c, g, st, W);
    };
    auto finish_eager = [&](bool scratch_zeroed) {
        enqueue_commit(c, g, st, walk_emitted, scratch_zeroed);
        copy_results();
        enqueue_readback(g, st);
        DG_CUDA(record_event(g.ev[3], st));
        wait_stream(c, st);
    };

    const bool tune_now = c.cfg.autotune && !g.tuned && !per_update && nu >= 4096;
    const bool use_graph = c.cfg.use_graphs && !per_update && !c.cfg.record && !tune_now;
    bool replayed = false;
    g.stats.autotuned = 0;
    DG_CUDA(record_event(g.ev[2], st));
    if (tune_now) {
        stage_inputs();
        enqueue_mutate(c, g, st);
        autotune_walks(c, g, st);
        walk_emitted = enqueue_walks(c, g, st, -1);
        finish_eager(true);
    } else if (use_graph) {
        if (direct) DG_CUDA(cudaMemcpyAsync(w.ups.p, ups, sizeof(dg_update) * nu, kin, st));
        CapturedStep& cs = capture_step(c, g, bucket, direct, st);
        DG_CUDA(cudaGraphLaunch(cs.exec, st));
        g_launches += cs.kernels;
        if (direct && res)
            DG_CUDA(cudaMemcpyAsync(res, w.res.p, sizeof(dg_update_result) * nu, kout, st));
        DG_CUDA(record_event(g.ev[3], st));
        wait_stream(c, st);
        replayed = true;
    } else {
        stage_inputs();
        run_pre();
        finish_eager(true);
    }
    int64_t retries = 0;
    for (;;) {
        const uint32_t err = g.hs.err[0];
        if (err & ERR_INTERNAL) throw Error(DG_E_CUDA, "internal consistency check failed on the device");
        if (err & ERR_SPIN) throw Error(DG_E_TIMEOUT, "a bounded device wait gave up");
        if (!(err & ABORT_MASK)) break;
        if (++retries > 8) throw Error(DG_E_NOMEM, "batch could not get enough device memory");
        const bool whole = handle_abort(c, g, err, st);
        DG_CUDA(record_event(g.ev[2], st));
        if (whole) {
            stage_inputs();
            run_pre();
        } else {  // only the commit re-runs; walks and their results are kept, candidates regenerated
            DG_CUDA(cudaMemsetAsync(w.err.p, 0, 16, st));
            DG_CUDA(cudaMemsetAsync(&w.ctr.p->recovered, 0, sizeof(unsigned long long), st));
            walk_emitted = false;
        }
        finish_eager(whole);
        replayed = false;
    }
    graph_mark_mutation(g, st);
    if (res && !direct) std::memcpy(res, g.hs.res, sizeof(dg_update_result) * nu);
    g.G.host_top = g.hs.tops[0];
    g.H.host_top = g.hs.tops[1];
    g.next_id += nu;
    dg_batch_stats& s = g.stats;
    s.updates = nu;
    s.valid = (int64_t)g.hs.ctr->valid;
    s.walked = (int64_t)g.hs.ctr->walked;
    s.steps = (int64_t)g.hs.ctr->steps;
    s.accepted = (int64_t)g.hs.ctr->accepted;
    s.recovered = (int64_t)g.hs.ctr->recovered;
    float ms = 0.f;
    s.walk_ms = (cudaEventElapsedTime(&ms, g.ev[0], g.ev[1]) == cudaSuccess) ? ms : -1.0;
    s.batch_ms = (cudaEventElapsedTime(&ms, g.ev[2], g.ev[3]) == cudaSuccess) ? ms : -1.0;
    s.mutate_ms = (cudaEventElapsedTime(&ms, g.ev[2], g.ev[4]) == cudaSuccess) ? ms : -1.0;
    s.reduce_ms = (cudaEventElapsedTime(&ms, g.ev[1], g.ev[5]) == cudaSuccess) ? ms : -1.0;
    s.emit_ms = (cudaEventElapsedTime(&ms, g.ev[5], g.ev[6]) == cudaSuccess) ? ms : -1.0;
    s.commit_ms = (cudaEventElapsedTime(&ms, g.ev[6], g.ev[3]) == cudaSuccess) ? ms : -1.0;
    s.merge_ms = (cudaEventElapsedTime(&ms, g.ev[7], g.ev[8]) == cudaSuccess) ? ms : -1.0;
    {
        // old entries read + new entries written: sum(od) = items - changes,
        // sum(nd) = sum(od) + insertions - deletions
        const uint64_t wk = g.hs.counts[2], ni = g.hs.counts[3], nd = g.hs.counts[4], cnt = g.hs.counts[5];
        s.merge_entries = (wk >= cnt && 2 * (wk - cnt) + ni >= nd) ? (int64_t)(2 * (wk - cnt) + ni - nd) : 0;
    }
    cudaGetLastError();
    s.retries = retries;
    s.graph_replayed = replayed ? 1 : 0;
    s.walk_block = g.shape.block;
    s.walk_ilp = g.shape.ilp;
    s.walk_blocks_per_sm = g.shape.blocks_per_sm;
    s.walk_cut = g.shape.cut;
    s.walk_refill = g.shape.refill;
    s.walk_lanes = g.shape.lanes;
    s.walk_tile = g.shape.tile;
    s.walk_launches = per_update ? (int64_t)g.hs.counts[0] : 1;
    const uint64_t dl = g_launches - l0;
    s.launches = (int64_t)dl;
    c.launches += dl;
}


// ---------------------------------------------------------------------------
// sharded batch
// ---------------------------------------------------------------------------

// this replica's walked updates [j_lo, j_hi) as records (argmin walker's step
// count from its record; 0 when there is none)
__global__ void k_shard_pack(WalkTasks t, const dg_update_result* __restrict__ res, const int32_t* __restrict__ best,
                             const uint32_t* __restrict__ meta, uint32_t s, uint32_t j_lo, uint32_t j_hi,
                             ShardRec* __restrict__ out) {
    for (uint32_t j = j_lo + blockIdx.x * blockDim.x + threadIdx.x; j < j_hi; j += gridDim.x * blockDim.x) {
        ShardRec rec;
        rec.j = j;
        rec.best = best[j];
        rec.best_steps = rec.best >= 0 ? (meta[(size_t)j * s + (uint32_t)rec.best] & 0xFFFFu) : 0u;
        rec.reserved = 0;
        rec.r = res[t.idx[j]];
        out[j - j_lo] = rec;
    }
}

// every shard's records back into the batch state: result, argmin walker and,
// for a deletion with a hit, the argmin walker's record (the replayed path's
// length); ERR_INTERNAL on a record outside the task list
__global__ void k_shard_unpack(WalkTasks t, const ShardRec* __restrict__ recs, uint32_t nrec, uint32_t s,
                               dg_update_result* __restrict__ res, int32_t* __restrict__ best,
                               uint32_t* __restrict__ meta, uint32_t* d_err) {
    const uint32_t W = *t.count;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nrec; q += gridDim.x * blockDim.x) {
        const ShardRec rec = recs[q];
        if (rec.j >= W || rec.best >= (int32_t)s) {
            atomicOr(d_err, (uint32_t)ERR_INTERNAL);
            continue;
        }
        res[t.idx[rec.j]] = rec.r;
        best[rec.j] = rec.best;
        if (rec.best >= 0) meta[(size_t)rec.j * s + (uint32_t)rec.best] = rec.best_steps | (R_HIT << 16);
    }
}

void graph_shard_begin(Ctx& c, DGraph& g, int64_t nu64, const dg_update* ups, int32_t rank, int32_t world,
                       cudaStream_t st, uint64_t* nrec_out) {
    if (!g.has_h) throw Error(DG_E_STATE, "no sparsifier");
    if (g.shard.active) throw Error(DG_E_STATE, "a sharded batch is already in progress on this graph");
    if (world < 1 || rank < 0 || rank >= world) throw Error(DG_E_INVALID, "rank must lie in [0, world)");
    if (c.cfg.record) throw Error(DG_E_STATE, "record_walkers is not available for sharded batches");
    if (c.cfg.walk_mode != DG_WALK_BATCHED) throw Error(DG_E_STATE, "sharded batches use the batched walk");
    if (nu64 < 0 || nu64 > (1ll << 26)) throw Error(DG_E_INVALID, "batch size out of range");
    const uint32_t nu = (uint32_t)nu64;
    if (nu > 0 && !ups) throw Error(DG_E_INVALID, "null update array");
    const uint32_t bucket = bucket_of(nu > 0 ? nu : 1);
    graph_wait_estimates(g, st);
    ensure_ws(c, g, bucket, st);
    ensure_headroom(c, g, nu, st);
    BatchWS& w = g.ws;
    w.shard_recs.ensure(c.alloc, w.b_max, st);
    g.hs.hdr->nu = nu;
    g.hs.hdr->pad = 0;
    g.hs.hdr->id0 = g.next_id;
    if (nu) std::memcpy(g.hs.ups, ups, sizeof(dg_update) * nu);
    const uint64_t l0 = g_launches;
    DG_CUDA(record_event(g.ev[2], st));
    for (int retries = 0;; ++retries) {
        DG_CUDA(cudaMemcpyAsync(w.hdr.p, g.hs.hdr, sizeof(BatchHdr), cudaMemcpyHostToDevice, st));
        if (nu) DG_CUDA(cudaMemcpyAsync(w.ups.p, g.hs.ups, sizeof(dg_update) * nu, cudaMemcpyHostToDevice, st));
        enqueue_mutate(c, g, st);
        DG_CUDA(cudaMemcpyAsync(g.hs.err, w.err.p, 4, cudaMemcpyDeviceToHost, st));
        DG_CUDA(cudaMemcpyAsync(g.hs.counts, w.t_count.p, 4, cudaMemcpyDeviceToHost, st));
        wait_stream(c, st);
        const uint32_t err = g.hs.err[0];
        if (err & ERR_INTERNAL) throw Error(DG_E_CUDA, "internal consistency check failed on the device");
        if (err & ERR_SPIN) throw Error(DG_E_TIMEOUT, "a bounded device wait gave up");
        if (!(err & ABORT_MASK)) break;
        if (retries >= 8) throw Error(DG_E_NOMEM, "batch could not get enough device memory");
        handle_abort(c, g, err, st);  // nothing was written: grow and run the mutation again
    }
    const uint32_t W = std::min<uint32_t>(g.hs.counts[0], w.b_max);
    if (c.cfg.autotune && !g.tuned && nu >= 4096) autotune_walks(c, g, st);
    const uint32_t j_lo = (uint32_t)((uint64_t)W * (uint32_t)rank / (uint32_t)world);
    const uint32_t j_hi = (uint32_t)((uint64_t)W * (uint32_t)(rank + 1) / (uint32_t)world);
    DG_CUDA(record_event(g.ev[4], st));
    DG_CUDA(record_event(g.ev[0], st));
    if (j_hi > j_lo) {
        const WalkParams wp = params_of(c.cfg);
        const WalkRecs wr = recs_of(c, w);
        const WalkTasks tasks = tasks_of(w);
        launch_walk_batched(g.H.view(), g.G.view(), tasks, wp, wr, w.hdr.p, w.next.p, j_lo, j_hi, g.shape,
                            fin_of(c, w, false), w.err.p, st, g.side, g.fk[5], g.fk[6]);
        DG_CUDA(record_event(g.ev[1], st));
        launch_walk_reduce(g.G.view(), tasks, wp, wr, w.hdr.p, w.res.p, w.best.p, w.ctr.p, nullptr, nullptr, j_lo,
                           j_hi, w.err.p, st);
        k_shard_pack<<<grid_for(j_hi - j_lo), BT, 0, st>>>(tasks, w.res.p, w.best.p, w.meta.p, (uint32_t)c.cfg.s,
                                                            j_lo, j_hi, w.shard_recs.p);
        ++g_launches;
        DG_CHECK_LAUNCH();
    } else {
        DG_CUDA(record_event(g.ev[1], st));
    }
    DG_CUDA(record_event(g.ev[5], st));
    DG_CUDA(cudaMemcpyAsync(g.hs.err, w.err.p, 4, cudaMemcpyDeviceToHost, st));
    wait_stream(c, st);
    if (g.hs.err[0] & ERR_INTERNAL) throw Error(DG_E_CUDA, "internal consistency check failed on the device");
    g.shard.active = true;
    g.shard.nu = nu;
    g.shard.W = W;
    g.shard.j_lo = j_lo;
    g.shard.j_hi = j_hi;
    g.shard.st = st;
    g.stats.launches = (int64_t)(g_launches - l0);
    if (nrec_out) *nrec_out = j_hi - j_lo;
}

void graph_shard_export(Ctx& c, DGraph& g, ShardRec* host, uint64_t cap, uint64_t* n_out) {
    if (!g.shard.active) throw Error(DG_E_STATE, "no sharded batch in progress");
    const uint64_t n = g.shard.j_hi - g.shard.j_lo;
    if (n_out) *n_out = n;
    if (!host) return;  // size query
    if (cap < n) throw Error(DG_E_INVALID, "export buffer holds fewer records than the shard has");
    if (n) DG_CUDA(cudaMemcpy(host, g.ws.shard_recs.p, n * sizeof(ShardRec), cudaMemcpyDeviceToHost));
}

void graph_shard_commit(Ctx& c, DGraph& g, const ShardRec* recs, uint64_t nrec, dg_update_result* res) {
    if (!g.shard.active) throw Error(DG_E_STATE, "no sharded batch in progress");
    const uint32_t W = g.shard.W, nu = g.shard.nu;
    cudaStream_t st = g.shard.st;
    BatchWS& w = g.ws;
    // every walked update exactly once
    if (nrec != W) throw Error(DG_E_INVALID, "the gathered records do not cover the batch's walked updates once");
    if (W && !recs) throw Error(DG_E_INVALID, "null record array");
    {
        std::vector<uint8_t> seen(W, 0);
        for (uint64_t q = 0; q < nrec; ++q) {
            if (recs[q].j >= W || seen[recs[q].j])
                throw Error(DG_E_INVALID, "the gathered records do not cover the batch's walked updates once");
            seen[recs[q].j] = 1;
        }
    }
    const uint64_t l0 = g_launches;
    if (W) {
        DG_CUDA(cudaMemcpyAsync(w.shard_recs.p, recs, W * sizeof(ShardRec), cudaMemcpyHostToDevice, st));
        k_shard_unpack<<<grid_for(W), BT, 0, st>>>(tasks_of(w), w.shard_recs.p, W, (uint32_t)c.cfg.s, w.res.p,
                                                    w.best.p, w.meta.p, w.err.p);
        ++g_launches;
        DG_CHECK_LAUNCH();
    }
    bool scratch_zeroed = true;
    for (int retries = 0;; ++retries) {
        enqueue_commit(c, g, st, false, scratch_zeroed);
        if (nu) DG_CUDA(cudaMemcpyAsync(g.hs.res, w.res.p, sizeof(dg_update_result) * nu, cudaMemcpyDeviceToHost, st));
        enqueue_readback(g, st);
        DG_CUDA(record_event(g.ev[3], st));
        wait_stream(c, st);
        const uint32_t err = g.hs.err[0];
        if (err & ERR_INTERNAL) throw Error(DG_E_CUDA, "internal consistency check failed on the device");
        if (err & ERR_SPIN) throw Error(DG_E_TIMEOUT, "a bounded device wait gave up");
        if (!(err & ABORT_MASK)) break;
        if (retries >= 8) throw Error(DG_E_NOMEM, "batch could not get enough device memory");
        if (handle_abort(c, g, err, st)) throw Error(DG_E_CUDA, "mutation-stage shortage at a sharded commit");
        DG_CUDA(cudaMemsetAsync(w.err.p, 0, 16, st));
        scratch_zeroed = false;
    }
    graph_mark_mutation(g, st);
    if (res && nu) std::memcpy(res, g.hs.res, sizeof(dg_update_result) * nu);
    g.G.host_top = g.hs.tops[0];
    g.H.host_top = g.hs.tops[1];
    g.next_id += nu;
    // statistics of the whole batch, from the gathered results
    dg_batch_stats& s = g.stats;
    s.updates = nu;
    s.valid = s.walked = s.steps = s.accepted = s.recovered = 0;
    for (uint32_t i = 0; i < nu; ++i) {
        const dg_update_result& r = g.hs.res[i];
        s.valid += r.status == DG_UPD_OK;
        s.walked += r.walked;
        s.steps += r.walked ? r.steps : 0;
        s.accepted += r.accepted;
        s.recovered += r.nrecovered;
    }
    float ms = 0.f;
    s.walk_ms = (cudaEventElapsedTime(&ms, g.ev[0], g.ev[1]) == cudaSuccess) ? ms : -1.0;
    s.batch_ms = (cudaEventElapsedTime(&ms, g.ev[2], g.ev[3]) == cudaSuccess) ? ms : -1.0;
    s.mutate_ms = (cudaEventElapsedTime(&ms, g.ev[2], g.ev[4]) == cudaSuccess) ? ms : -1.0;
    s.reduce_ms = (cudaEventElapsedTime(&ms, g.ev[1], g.ev[5]) == cudaSuccess) ? ms : -1.0;
    s.emit_ms = -1.0;
    s.commit_ms = -1.0;
    s.merge_ms = -1.0;
    s.merge_entries = 0;
    cudaGetLastError();
    s.graph_replayed = 0;
    s.launches += (int64_t)(g_launches - l0);
    c.launches += (uint64_t)s.launches;
    g.shard.active = false;
}

}  // namespace dg
