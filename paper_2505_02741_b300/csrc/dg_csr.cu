// dg_csr.cu -- slack-slot CSR kernels (see dg_csr.cuh).
#include "dg_csr.cuh"

namespace dg {

static int g_num_sms = 0;

int flat_grid() {
    if (g_num_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 148;
    }
    return g_num_sms * 8;
}

constexpr int FLAT_THREADS = 256;

__device__ __forceinline__ bool aborted(const uint32_t* d_err) { return (*d_err & ABORT_MASK) != 0u; }

__device__ __forceinline__ uint32_t count_of(const uint32_t* d_count, uint32_t max_count) {
    return min(*d_count, max_count);
}

__device__ __forceinline__ uint64_t ent_key_u64(uint32_t x, uint32_t y, uint32_t n) {
    return (uint64_t)x * (uint64_t)n + (uint64_t)y;
}

// ---------------------------------------------------------------------------
// scratch management
// ---------------------------------------------------------------------------
void ApplyScratch::ensure(DevAlloc& a, uint32_t changes, uint64_t stage_entries, cudaStream_t st) {
    if (changes > c_max || !p_head.p) {
        uint32_t c = changes < 1024 ? 1024 : changes;
        DBuf<uint32_t>* bufs[] = {&p_head, &p_ins, &p_del, &tv, &tstart, &tend,
                                  &odeg, &ndeg, &ooff, &ncap, &rsz, &work, &r_off, &s_off, &w_off,
                                  &fwork, &f_off, &sdeg, &xm, &tdst};
        for (auto* b : bufs) b->ensure(a, (size_t)c + 1, st);
        scan_words = scan_tmp_words(c + 1);
        scan_tmp.ensure(a, 2 * scan_words, st);
        c_max = c;
    }
    totals.ensure(a, 2 * TOT_WORDS, st);
    if (stage_entries > s_cap || !stage.p) {
        uint64_t e = stage_entries < 4096 ? 4096 : stage_entries;
        stage.ensure(a, e, st);
        s_cap = e;
    }
}

void ApplyScratch::release(DevAlloc& a, cudaStream_t st) {
    DBuf<uint32_t>* bufs[] = {&p_head, &p_ins, &p_del, &tv, &tstart, &tend,
                              &odeg, &ndeg, &ooff, &ncap, &rsz, &work, &r_off, &s_off, &w_off,
                              &fwork, &f_off, &sdeg, &xm, &tdst, &scan_tmp, &totals};
    for (auto* b : bufs) b->release(a, st);
    stage.release(a, st);
    c_max = 0;
    s_cap = 0;
}

uint64_t ApplyScratch::bytes() const {
    return 20ull * (c_max + 1) * 4 + scan_tmp.bytes() + totals.bytes() + stage.bytes();
}

void csr_alloc_vertices(CSR& g, DevAlloc& a, int32_t n, cudaStream_t st) {
    g.n = n;
    g.off.ensure(a, (size_t)n + 1, st);
    g.deg.ensure(a, (size_t)n + 1, st);
    g.cap.ensure(a, (size_t)n + 1, st);
    g.hub.ensure(a, (size_t)n + 1, st);
    DG_CUDA(cudaMemsetAsync(g.hub.p, 0, g.hub.bytes(), st));
    g.nhub.ensure(a, 1, st);
    DG_CUDA(cudaMemsetAsync(g.nhub.p, 0, g.nhub.bytes(), st));
    g.twin.ensure(a, (size_t)n + 1, st);
    DG_CUDA(cudaMemsetAsync(g.twin.p, 0xFF, g.twin.bytes(), st));
    g.top.ensure(a, 1, st);
    g.minr.ensure(a, 1, st);
    DG_CUDA(cudaMemsetAsync(g.minr.p, 0xFF, g.minr.bytes(), st));
    DG_CUDA(cudaMemsetAsync(g.off.p, 0, g.off.bytes(), st));
    DG_CUDA(cudaMemsetAsync(g.deg.p, 0, g.deg.bytes(), st));
    DG_CUDA(cudaMemsetAsync(g.cap.p, 0, g.cap.bytes(), st));
    DG_CUDA(cudaMemsetAsync(g.top.p, 0, g.top.bytes(), st));
}

void csr_release(CSR& g, DevAlloc& a, cudaStream_t st) {
    g.off.release(a, st);
    g.deg.release(a, st);
    g.cap.release(a, st);
    g.hub.release(a, st);
    g.nhub.release(a, st);
    g.twin.release(a, st);
    g.pool.release(a, st);
    g.top.release(a, st);
    g.minr.release(a, st);
    g.pool_cap = 0;
    g.n = 0;
}

// ---------------------------------------------------------------------------
// build from sorted unique half-edges
// ---------------------------------------------------------------------------
__global__ void k_build_deg(const uint64_t* __restrict__ keys, uint32_t count, uint32_t n,
                            uint32_t* __restrict__ deg, uint32_t* d_err) {
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < count; c += gridDim.x * blockDim.x) {
        const uint64_t k = keys[c];
        const uint32_t x = (uint32_t)(k / n);
        if (c > 0 && keys[c - 1] == k) atomicOr(d_err, (uint32_t)ERR_DUP_EDGE);
        if (c == 0 || (uint32_t)(keys[c - 1] / n) != x) {
            const uint32_t e = lower_bound_arr<uint64_t>(keys, c, count, (uint64_t)(x + 1) * n);
            deg[x] = e - c;
        }
    }
}

__global__ void k_caps(const uint32_t* __restrict__ deg, uint32_t n, float slack, uint32_t* __restrict__ cap) {
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x)
        cap[x] = cap_for(deg[x], slack);
}

// Every list gets a twin region of its capacity right after it: off holds the
// prefix sums of the capacities on entry and the list offsets on return.  A
// list execution writes a touched list into its twin and keeps the region it
// leaves as the next twin, so no list is rewritten in place.
__global__ void k_twin_layout(uint32_t* __restrict__ off, const uint32_t* __restrict__ cap, uint32_t n,
                              uint32_t* __restrict__ twin) {
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        const uint32_t o = 2u * off[x];
        off[x] = o;
        twin[x] = o + cap[x];
    }
}

__global__ void k_build_fill(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                             const double* __restrict__ ws, uint32_t count, uint32_t n,
                             const uint32_t* __restrict__ off, Ent* __restrict__ pool) {
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < count; c += gridDim.x * blockDim.x) {
        const uint64_t k = keys[c];
        const uint32_t x = (uint32_t)(k / n), y = (uint32_t)(k % n);
        const uint32_t s0 = lower_bound_arr<uint64_t>(keys, 0, c, (uint64_t)x * n);
        const double w = ws[vals[c]];
        Ent e;
        e.nbr = y;
        e.noff = 0;
        e.ndeg = 0;
        e.rev = 0;
        e.w = w;
        e.r = __ddiv_rn(1.0, w);
        pool[off[x] + (c - s0)] = e;
    }
}

// minimum resistance over the built entries (a lower bound for the lists)
__global__ void k_build_minr(const uint32_t* __restrict__ vals, const double* __restrict__ ws, uint32_t count,
                             unsigned long long* minr) {
    unsigned long long m = ~0ull;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < count; c += gridDim.x * blockDim.x)
        m = min(m, (unsigned long long)__double_as_longlong(__ddiv_rn(1.0, ws[vals[c]])));
    for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m != ~0ull) atomicMin(minr, m);
}

// refresh (noff, ndeg, rev) of every entry listed by the sorted key array
__global__ void k_build_fix(const uint64_t* __restrict__ keys, uint32_t count, uint32_t n, CSRView g,
                            uint32_t* d_err) {
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < count; c += gridDim.x * blockDim.x) {
        const uint64_t k = keys[c];
        const uint32_t x = (uint32_t)(k / n), y = (uint32_t)(k % n);
        const uint32_t s0 = lower_bound_arr<uint64_t>(keys, 0, c, (uint64_t)x * n);
        const uint32_t ly = g.off[y], dy = g.deg[y];
        const uint32_t p = lower_bound_nbr(g.pool + ly, dy, x);
        if (p >= dy || g.pool[ly + p].nbr != x) {
            atomicOr(d_err, (uint32_t)ERR_INTERNAL);
            continue;
        }
        // a hub reference keeps x's slot in the hub's list as a hint (HUBREF)
        const uint4 h = g.hub[y] ? make_uint4(y, HUBREF, 1u, p) : make_uint4(y, ly, dy, p);
        *reinterpret_cast<uint4*>(g.pool + g.off[x] + (c - s0)) = h;
    }
}

__global__ void k_hub_init(const uint32_t* __restrict__ deg, uint32_t n, uint8_t* __restrict__ hub,
                           uint32_t* nhub) {
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        const bool h = deg[x] >= HUB_HI;
        hub[x] = h ? 1 : 0;
        if (h) atomicAdd(nhub, 1u);
    }
}

void csr_build(CSR& g, DevAlloc& a, const uint64_t* keys, const uint32_t* vals, const double* ws,
               uint32_t count, uint32_t* d_err, cudaStream_t st) {
    const uint32_t n = (uint32_t)g.n;
    const int grid = flat_grid();
    DG_CUDA(cudaMemsetAsync(g.deg.p, 0, g.deg.bytes(), st));
    if (count > 0) {
        k_build_deg<<<grid, FLAT_THREADS, 0, st>>>(keys, count, n, g.deg.p, d_err);
        ++g_launches;
    }
    k_caps<<<grid, FLAT_THREADS, 0, st>>>(g.deg.p, n, g.slack, g.cap.p);
    DG_CUDA(cudaMemsetAsync(g.nhub.p, 0, 4, st));
    k_hub_init<<<grid, FLAT_THREADS, 0, st>>>(g.deg.p, n, g.hub.p, g.nhub.p);
    g_launches += 2;
    DBuf<uint32_t> tmp, total;
    tmp.ensure(a, scan_tmp_words(n + 1), st);
    total.ensure(a, 2, st);
    ScanJob job;
    job.in[0] = g.cap.p;
    job.out[0] = g.off.p;
    job.total[0] = total.p;
    job.k = 1;
    scan_exclusive(job, nullptr, n, tmp.p, st);
    k_twin_layout<<<grid, FLAT_THREADS, 0, st>>>(g.off.p, g.cap.p, n, g.twin.p);
    ++g_launches;
    uint32_t h_caps = 0;
    DG_CUDA(cudaMemcpyAsync(&h_caps, total.p, 4, cudaMemcpyDeviceToHost, st));
    DG_CUDA(cudaStreamSynchronize(st));
    tmp.release(a, st);
    total.release(a, st);
    const uint64_t h_total = 2ull * h_caps;  // lists and their twins
    const uint64_t want = h_total + (uint64_t)((double)h_total * g.overflow) + 4096;
    if (want >= 0xFFFFFFF0ull) throw Error(DG_E_NOMEM, "graph too large for 32-bit pool offsets");
    g.pool.release(a, st);
    g.pool.ensure(a, want, st);
    g.pool_cap = want;
    unsigned long long t = h_total;
    DG_CUDA(cudaMemcpyAsync(g.top.p, &t, sizeof(t), cudaMemcpyHostToDevice, st));
    g.host_top = h_total;
    if (count > 0) {
        k_build_fill<<<grid, FLAT_THREADS, 0, st>>>(keys, vals, ws, count, n, g.off.p, g.pool.p);
        k_build_fix<<<grid, FLAT_THREADS, 0, st>>>(keys, count, n, g.view(), d_err);
        DG_CUDA(cudaMemsetAsync(g.minr.p, 0xFF, 8, st));
        k_build_minr<<<grid, FLAT_THREADS, 0, st>>>(vals, ws, count, g.minr.p);
        g_launches += 3;
    }
    DG_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// plan
// ---------------------------------------------------------------------------
struct PlanArgs {
    ChangeList cl;
    CSRView g;
    uint32_t n;
    float slack;
    const uint32_t *p_head, *p_ins, *p_del, *totals;
    uint32_t *tv, *tstart, *tend, *odeg, *ndeg, *ooff, *ncap, *rsz, *work, *fwork;
    uint32_t *sdeg, *xm, *tdst;
};

// Placement of a touched list (xm bits 0-1) and of a hub's twin after the
// execution (xm bits 2-3).  A list that stays where it is goes through the
// staging buffer (its old entries are read while the new ones are written); a
// list written elsewhere -- fresh pool space, or a hub's twin region -- is
// written there directly by the merge.  A hub always moves: into its twin when
// it has one and the list fits, and the region it leaves becomes the twin, so
// rewriting a long hub list costs one pass over it instead of two.
enum : uint32_t { XM_INPLACE = 0, XM_FRESH = 1, XM_TWIN = 2 };
enum : uint32_t { TW_NONE = 0, TW_OLD = 1, TW_FRESH = 2 };  // new twin: none, the old region, fresh space after the list

__device__ __forceinline__ uint32_t pre_at(const uint32_t* p, uint32_t c, uint32_t count, uint32_t total) {
    return c < count ? p[c] : total;
}

__global__ void k_plan_touch(PlanArgs a, const uint32_t* d_err) {
    if (aborted(d_err)) return;
    const uint32_t count = count_of(a.cl.d_count, a.cl.max_count);
    const uint32_t NI = a.totals[TOT_NI], ND = a.totals[TOT_ND];
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < count; c += gridDim.x * blockDim.x) {
        const uint32_t x = (uint32_t)(a.cl.keys[c] / a.n);
        if (!(c == 0 || (uint32_t)(a.cl.keys[c - 1] / a.n) != x)) continue;
        // x's list fields and prefix counts do not depend on the run's end: sent first
        const uint32_t od = a.g.deg[x];
        const uint32_t oc = a.g.cap[x];
        const uint32_t oo = a.g.off[x];
        const bool was_hub = a.g.hub[x] != 0;
        const uint32_t t = a.p_head[c];
        const uint32_t pi = a.p_ins[c], pd = a.p_del[c];
        // end of x's run: galloping from c (runs are short except at hubs)
        const uint64_t kend = (uint64_t)(x + 1) * a.n;
        uint32_t lo = c, hi = c + 1, step = 1;
        while (hi < count && a.cl.keys[hi] < kend) {
            lo = hi;
            hi = (count - hi > step) ? hi + step : count;
            step <<= 1;
        }
        const uint32_t e = lower_bound_arr<uint64_t>(a.cl.keys, lo + 1, hi, kend);
        const uint32_t ins = pre_at(a.p_ins, e, count, NI) - pi;
        const uint32_t del = pre_at(a.p_del, e, count, ND) - pd;
        const uint32_t nd = od + ins - del;
        const bool reloc = nd > oc;
        const uint32_t nc = reloc ? cap_for(nd, a.slack) : oc;
        const bool hub_now = hub_next(was_hub, nd);
        const uint32_t tw = a.g.twin[x];
        uint32_t mode, ntw, rs = 0;
        if (!reloc && tw != 0xFFFFFFFFu) {
            mode = XM_TWIN;          // into the twin; the region it leaves becomes the twin
            ntw = TW_OLD;
        } else if (reloc) {
            mode = XM_FRESH;         // grown list: fresh list and fresh twin
            ntw = TW_FRESH;
            rs = 2 * nc;
        } else if (hub_now) {
            mode = XM_FRESH;         // no twin yet: fresh space, the old region becomes the twin
            ntw = TW_OLD;
            rs = oc;
        } else {
            mode = XM_INPLACE;       // no twin (not laid out by a build or compaction)
            ntw = TW_NONE;
        }
        a.tv[t] = x;
        a.tstart[t] = c;
        a.tend[t] = e;
        a.odeg[t] = od;
        a.ndeg[t] = nd;
        a.ooff[t] = oo;
        a.ncap[t] = nc;
        a.rsz[t] = rs;
        a.sdeg[t] = mode == XM_INPLACE ? nd : 0u;
        a.xm[t] = mode | (ntw << 2);
        a.tdst[t] = tw;
        a.work[t] = od + (e - c);
        // cache refresh work: every entry of the new list, or for a hub that
        // stays a hub only its changes (see k_exec_fix)
        a.fwork[t] = (was_hub && hub_now) ? e - c : nd;
    }
}

void csr_plan(CSR& g, const ChangeList& cl, ApplyScratch& s, uint32_t* d_err, uint32_t pool_bit,
              uint32_t cap_bit, cudaStream_t st, bool tmp_zeroed) {
    const int grid = flat_grid();
    const uint32_t C = cl.max_count;
    uint32_t* tot = s.totals.p;
    // run heads, insertions and deletions of the change list, generated inside
    // the scan (no flag arrays)
    ScanJob j1;
    j1.gen.mode = 1;
    j1.gen.keys = cl.keys;
    j1.gen.n_div = (uint64_t)g.n;
    j1.gen.vals = cl.vals;
    j1.gen.kinds = cl.kinds;
    j1.gen.k_ins = CHG_INS;
    j1.gen.k_del = CHG_DEL;
    j1.out[0] = s.p_head.p; j1.total[0] = tot + TOT_X;
    j1.out[1] = s.p_ins.p;  j1.total[1] = tot + TOT_NI;
    j1.out[2] = s.p_del.p;  j1.total[2] = tot + TOT_ND;
    j1.k = 3;
    j1.err = d_err;
    scan_exclusive(j1, cl.d_count, C, s.scan_tmp.p, st, tmp_zeroed);
    PlanArgs pa;
    pa.cl = cl;
    pa.g = g.view();
    pa.n = (uint32_t)g.n;
    pa.slack = g.slack;
    pa.p_head = s.p_head.p; pa.p_ins = s.p_ins.p; pa.p_del = s.p_del.p; pa.totals = tot;
    pa.tv = s.tv.p; pa.tstart = s.tstart.p; pa.tend = s.tend.p; pa.odeg = s.odeg.p; pa.ndeg = s.ndeg.p;
    pa.ooff = s.ooff.p; pa.ncap = s.ncap.p; pa.rsz = s.rsz.p; pa.work = s.work.p; pa.fwork = s.fwork.p;
    pa.sdeg = s.sdeg.p; pa.xm = s.xm.p; pa.tdst = s.tdst.p;
    k_plan_touch<<<grid, FLAT_THREADS, 0, st>>>(pa, d_err);
    ++g_launches;
    ScanJob j2;
    j2.in[0] = s.rsz.p;  j2.out[0] = s.r_off.p; j2.total[0] = tot + TOT_R;
    j2.in[1] = s.sdeg.p; j2.out[1] = s.s_off.p; j2.total[1] = tot + TOT_S;
    j2.in[2] = s.work.p; j2.out[2] = s.w_off.p; j2.total[2] = tot + TOT_WK;
    j2.in[3] = s.fwork.p; j2.out[3] = s.f_off.p; j2.total[3] = tot + TOT_F;
    j2.k = 4;
    j2.err = d_err;
    // the pool allocation follows the totals in the same launch: base = the
    // pool top; the batch aborts (before any list is written) when the new
    // regions or the staged lists do not fit
    j2.post.top = g.top.p;
    j2.post.pool_cap = g.pool_cap;
    j2.post.stage_cap = s.s_cap;
    j2.post.totals = tot;
    j2.post.r_idx = TOT_R;
    j2.post.s_idx = TOT_S;
    j2.post.base_lo = TOT_BASE_LO;
    j2.post.base_hi = TOT_BASE_HI;
    j2.post.err = d_err;
    j2.post.abort_mask = ABORT_MASK;
    j2.post.pool_bit = pool_bit;
    j2.post.cap_bit = cap_bit;
    scan_exclusive(j2, tot + TOT_X, C, s.scan_tmp.p + s.scan_words, st, tmp_zeroed);
    DG_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// execute
// ---------------------------------------------------------------------------
struct ExecArgs {
    ChangeList cl;
    CSRView g;
    uint32_t n;
    const uint32_t *p_ins, *p_del, *totals;
    const uint32_t *tv, *tstart, *tend, *odeg, *ndeg, *ooff, *ncap, *rsz, *r_off, *s_off, *w_off, *f_off;
    const uint32_t *sdeg, *xm, *tdst;
    Ent* stage;
    uint32_t* touched;  // n + 1 words, see csr_exec
};

__device__ __forceinline__ uint64_t base_of(const uint32_t* totals) {
    return (uint64_t)totals[TOT_BASE_LO] | ((uint64_t)totals[TOT_BASE_HI] << 32);
}

__device__ __forceinline__ uint32_t dst_off(const ExecArgs& a, uint32_t t) {
    const uint32_t mode = a.xm[t] & 3u;
    return mode == XM_FRESH ? (uint32_t)(base_of(a.totals) + a.r_off[t]) : mode == XM_TWIN ? a.tdst[t] : a.ooff[t];
}

// every touched vertex's list fields, hub flag and touched mark
__device__ __forceinline__ void exec_meta(const ExecArgs& a) {
    const uint32_t X = a.totals[TOT_X];
    if (blockIdx.x == 0 && threadIdx.x == 0)
        *a.g.top = (unsigned long long)(base_of(a.totals) + a.totals[TOT_R]);
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < X; t += gridDim.x * blockDim.x) {
        const uint32_t x = a.tv[t];
        a.g.off[x] = dst_off(a, t);
        a.g.deg[x] = a.ndeg[t];
        a.g.cap[x] = a.ncap[t];
        const uint32_t ntw = a.xm[t] >> 2;
        a.g.twin[x] = ntw == TW_OLD ? a.ooff[t]
                    : ntw == TW_FRESH ? (uint32_t)(base_of(a.totals) + a.r_off[t] + a.ncap[t])
                                      : 0xFFFFFFFFu;
        // touched bit 0; bit 1 when x's hub status flips (its back-entries change form)
        const bool was = a.g.hub[x] != 0, now = hub_next(was, a.ndeg[t]);
        a.g.hub[x] = now ? 1 : 0;
        if (was != now) atomicAdd(a.g.nhub, now ? 1u : 0xFFFFFFFFu);
        a.touched[x] = (a.touched[a.n] << 2) | 1u | (was != now ? 2u : 0u);
    }
}

// Largest t in [0, nseg) with seg_off[t] <= key (seg_off non-decreasing,
// seg_off[0] = 0 <= key), found by the whole warp: each round the 32 lanes
// probe 32 spread positions, so a round narrows the range 32-fold and the
// search costs log32(nseg) dependent loads instead of log2(nseg).  All lanes
// call it with the same key and get the result.
__device__ __forceinline__ uint32_t warp_last_leq(const uint32_t* seg_off, uint32_t nseg, uint32_t key) {
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t lo = 0, hi = nseg;  // answer in [lo, hi), seg_off[lo] <= key
    while (hi - lo > 1) {
        const uint32_t p = lo + 1u + (uint32_t)(((uint64_t)(hi - lo - 1) * lane) >> 5);
        const bool ok = seg_off[p] <= key;
        const uint32_t m = __ballot_sync(0xffffffffu, ok);
        const uint32_t pj = __shfl_sync(0xffffffffu, p, m ? 31 - __clz(m) : 0);
        const uint32_t pn = __shfl_sync(0xffffffffu, p, m ? min(32 - __clz(m), 31) : 0);
        if (!m) {
            hi = pj;  // every probe is past key: the answer is lo
        } else {
            lo = pj;
            if (m != 0xffffffffu) hi = pn;  // the next probe is past key
        }
    }
    return lo;
}

// Visit items [0, total) of consecutive segments (seg_off: exclusive start of
// each of nseg segments).  Each warp takes one contiguous range of the items
// (a multiple of 32, sized from the live total so all warps share the work)
// and finds the segment of its start with a warp-wide search; per 32 items the
// lanes load the next 32 segment starts together and each finds its own
// segment among them by register shuffles, falling back to stepping forward
// only when more than 32 segments begin inside the 32 items.
template <int IT, typename F>
__device__ __forceinline__ void for_segment_items(const uint32_t* seg_off, uint32_t nseg, uint32_t total, F&& f) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint64_t per = ((((uint64_t)total + nwarps - 1) / nwarps) + 31u) & ~31ull;
    const uint64_t start = (uint64_t)warp * per;
    if (start >= total) return;
    const uint32_t end = (uint32_t)((start + per < (uint64_t)total) ? start + per : (uint64_t)total);
    uint32_t t = warp_last_leq(seg_off, nseg, (uint32_t)start);  // segment of the first item
    uint32_t t_off = seg_off[t];
    for (uint32_t c0 = (uint32_t)start; c0 < end; c0 += 32u) {
        const uint32_t item = c0 + lane;
        // starts of segments t+1 .. t+32 (non-decreasing; past the end: +inf)
        const uint32_t wi = t + 1u + lane;
        const uint32_t wv = wi < nseg ? seg_off[wi] : 0xFFFFFFFFu;
        // k = number of those starts <= item (binary search over the lanes)
        uint32_t k = 0;
#pragma unroll
        for (uint32_t bstep = 16; bstep > 0; bstep >>= 1) {
            const uint32_t v = __shfl_sync(0xffffffffu, wv, (int)(k + bstep - 1u));
            if (v <= item) k += bstep;
        }
        const uint32_t w31 = __shfl_sync(0xffffffffu, wv, 31);
        if (k == 31u && w31 <= item) k = 32u;
        uint32_t ti = t + k;
        const uint32_t wprev = __shfl_sync(0xffffffffu, wv, (int)(k ? k - 1u : 0u));
        uint32_t to = k ? wprev : t_off;
        if (k == 32u) {  // more than 32 segments start before this item
            while (ti + 1 < nseg && seg_off[ti + 1] <= item) ++ti;
            to = seg_off[ti];
        }
        if (item < end) f(item, ti, item - to);
        // the last item's segment is where the next 32 items start looking
        const uint32_t last = min(31u, end - 1u - c0);
        t = __shfl_sync(0xffffffffu, ti, (int)last);
        t_off = __shfl_sync(0xffffffffu, to, (int)last);
    }
}

// Entries the merge moves are read once and written once: streaming loads and
// stores (evict-first), so moving a long list does not push the data the walk
// reads next out of L2 (R-MAT merge 0.588 -> 0.561 ms, walk 0.621 -> 0.613 ms).
__device__ __forceinline__ Ent ld_stream(const Ent* p) {
    const uint4* q = reinterpret_cast<const uint4*>(p);
    const uint4 h0 = __ldcs(q), h1 = __ldcs(q + 1);
    Ent e;
    memcpy(&e, &h0, 16);
    memcpy(reinterpret_cast<char*>(&e) + 16, &h1, 16);
    return e;
}
__device__ __forceinline__ void st_stream(Ent* p, const Ent& e) {
    uint4 h0, h1;
    memcpy(&h0, &e, 16);
    memcpy(&h1, reinterpret_cast<const char*>(&e) + 16, 16);
    __stcs(reinterpret_cast<uint4*>(p), h0);
    __stcs(reinterpret_cast<uint4*>(p) + 1, h1);
}

// merge: one thread per (old entry | change) of every touched vertex
__global__ void k_exec_merge(ExecArgs a, uint32_t* d_err) {
    if (aborted(d_err)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) ++a.touched[a.n];  // this execution's generation (read from meta on)
    const uint32_t X = a.totals[TOT_X];
    const uint32_t WK = a.totals[TOT_WK];
    const uint32_t count = count_of(a.cl.d_count, a.cl.max_count);
    const uint32_t NI = a.totals[TOT_NI], ND = a.totals[TOT_ND];
    for_segment_items<16>(a.w_off, X, WK, [&](uint32_t item, uint32_t t, uint32_t local) {
        const uint32_t x = a.tv[t];
        const uint32_t s0 = a.tstart[t], s1 = a.tend[t];
        const uint32_t od = a.odeg[t];
        const Ent* L = a.g.pool + a.ooff[t];
        uint32_t outpos;
        Ent out;
        if (local < od) {
            out = ld_stream(L + local);
            const uint64_t key = ent_key_u64(x, out.nbr, a.n);
            const uint32_t c0 = lower_bound_arr<uint64_t>(a.cl.keys, s0, s1, key);
            const bool found = c0 < s1 && a.cl.keys[c0] == key;
            uint8_t kd = 255;
            if (found) kd = a.cl.kinds[a.cl.vals[c0]];
            if (kd == CHG_DEL) return;
            if (kd == CHG_INS) {  // insertion of a present edge: inconsistent input
                atomicOr(d_err, (uint32_t)ERR_INTERNAL);
                return;
            }
            const uint32_t ib = pre_at(a.p_ins, c0, count, NI) - a.p_ins[s0];
            const uint32_t db = pre_at(a.p_del, c0, count, ND) - a.p_del[s0];
            outpos = local + ib - db;
            if (kd == CHG_SETW) {
                const double w = a.cl.ws[a.cl.vals[c0]];
                out.w = w;
                out.r = __ddiv_rn(1.0, w);
                atomicMin(a.g.minr, (unsigned long long)__double_as_longlong(out.r));
            }
        } else {
            const uint32_t c = s0 + (local - od);
            if (a.cl.kinds[a.cl.vals[c]] != CHG_INS) return;
            const uint32_t y = (uint32_t)(a.cl.keys[c] - (uint64_t)x * a.n);
            const uint32_t lb = lower_bound_nbr(L, od, y);
            if (lb < od && L[lb].nbr == y) {
                atomicOr(d_err, (uint32_t)ERR_INTERNAL);
                return;
            }
            const uint32_t ib = a.p_ins[c] - a.p_ins[s0];
            const uint32_t db = a.p_del[c] - a.p_del[s0];
            outpos = lb + ib - db;
            const double w = a.cl.ws[a.cl.vals[c]];
            out.nbr = y;
            out.noff = 0;
            out.ndeg = 0;
            out.rev = 0;
            out.w = w;
            out.r = __ddiv_rn(1.0, w);
            atomicMin(a.g.minr, (unsigned long long)__double_as_longlong(out.r));
        }
        if (outpos >= a.ndeg[t]) {
            atomicOr(d_err, (uint32_t)ERR_INTERNAL);
            return;
        }
        // a list that stays in place goes through the staging buffer; one that
        // moves is written at its destination (nothing reads that space now)
        st_stream(a.sdeg[t] ? a.stage + a.s_off[t] + outpos : a.g.pool + dst_off(a, t) + outpos, out);
    });
}

// meta points every touched vertex at its final slots; place copies the
// staged lists (those without a twin) back.  Neither reads what the other
// writes, so one launch does both.
__global__ void k_exec_meta_place(ExecArgs a, const uint32_t* d_err) {
    if (aborted(d_err)) return;
    exec_meta(a);
    const uint32_t X = a.totals[TOT_X];
    const uint32_t S = a.totals[TOT_S];
    for_segment_items<16>(a.s_off, X, S, [&](uint32_t item, uint32_t t, uint32_t local) {
        a.g.pool[dst_off(a, t) + local] = a.stage[item];
    });
}

// Cache refresh after a list execution.  For every touched vertex x the items
// are the entries of its new list, except for a hub that stays a hub: entries
// pointing at such a hub hold HUBREF, so its moved list is cached nowhere, and
// its own entries need work only where an insertion created them (its items are
// then its changes) or where the neighbour's list changed, which that
// neighbour's pass refreshes from its side.  A hub's list can be long and
// change little, so this keeps the work near the size of the batch.
__global__ void k_exec_fix(ExecArgs a, uint32_t* d_err) {
    if (aborted(d_err)) return;
    const uint32_t X = a.totals[TOT_X];
    const uint32_t F = a.totals[TOT_F];
    const uint32_t gen = a.touched[a.n];  // marks of this execution only (older generations read as untouched)
    const bool hubs = *a.g.nhub != 0u;
    for_segment_items<16>(a.f_off, X, F, [&](uint32_t item, uint32_t t, uint32_t local) {
        (void)item;
        const uint32_t x = a.tv[t];
        const uint32_t lx = a.g.off[x];
        const uint32_t mx = a.touched[x];
        const uint32_t tx = (mx >> 2) == gen ? (mx & 3u) : 0u;
        const bool x_hub = a.g.hub[x] != 0;
        if (x_hub && !(tx & 2u)) {
            // a hub that stays a hub: the entry each of its insertions created
            const uint32_t c = a.tstart[t] + local;
            if (a.cl.kinds[a.cl.vals[c]] != CHG_INS) return;
            const uint32_t y = (uint32_t)(a.cl.keys[c] - (uint64_t)x * a.n);
            const uint32_t dx = a.g.deg[x];
            const uint32_t px = lower_bound_nbr(a.g.pool + lx, dx, y);
            if (y >= a.n || px >= dx || a.g.pool[lx + px].nbr != y) {
                atomicOr(d_err, (uint32_t)ERR_INTERNAL);
                return;
            }
            const uint32_t ly = a.g.off[y], dy = a.g.deg[y];
            const uint32_t p = lower_bound_nbr(a.g.pool + ly, dy, x);
            if (p >= dy || a.g.pool[ly + p].nbr != x) {
                atomicOr(d_err, (uint32_t)ERR_INTERNAL);
                return;
            }
            *reinterpret_cast<uint4*>(a.g.pool + lx + px) =
                a.g.hub[y] != 0 ? make_uint4(y, HUBREF, 1u, p) : make_uint4(y, ly, dy, p);
            return;
        }
        const uint4 e = *reinterpret_cast<const uint4*>(a.g.pool + lx + local);
        const uint32_t y = e.x;
        if (y >= a.n) {
            atomicOr(d_err, (uint32_t)ERR_INTERNAL);
            return;
        }
        const uint32_t my = a.touched[y];
        const uint32_t ty = (my >> 2) == gen ? (my & 3u) : 0u;
        const bool fresh = e.z == 0u;
        // a touched neighbour that stays a hub does not visit its entry pointing
        // back at x, so it is written here
        const bool y_stable_hub = hubs && (ty & 1u) && !(ty & 2u) && a.g.hub[y] != 0;
        const bool need_own = fresh || (ty & 1u);
        const bool need_back = !(ty & 1u) || y_stable_hub;
        if (!need_own && !need_back) return;
        const bool y_hub = a.g.hub[y] != 0;
        const uint32_t ly = a.g.off[y], dy = a.g.deg[y];
        uint32_t p = 0xFFFFFFFFu;      // x's slot in y's list, found when needed
        auto locate = [&]() -> bool {
            if (p != 0xFFFFFFFFu) return true;
            if (!fresh && e.y != HUBREF && !(ty & 1u)) {  // a valid copied entry caches the slot
                p = e.w;
            } else if (!fresh) {  // the slot it cached (or a hub's hint) is near
                p = lower_bound_nbr_near(a.g.pool + ly, dy, x, e.w);
            } else {
                p = lower_bound_nbr(a.g.pool + ly, dy, x);
            }
            if (p >= dy || a.g.pool[ly + p].nbr != x) {
                atomicOr(d_err, (uint32_t)ERR_INTERNAL);
                return false;
            }
            return true;
        };
        // (i) this entry: its cache is still right when it was copied from x's old
        // list and y's list did not change
        if (need_own) {
            if (y_hub) {
                // slot hint: a copied entry keeps its old slot in y's list (y's list
                // changed little); a fresh one looks it up
                uint32_t hint = e.w;
                if (fresh) {
                    if (!locate()) return;
                    hint = p;
                }
                *reinterpret_cast<uint4*>(a.g.pool + lx + local) = make_uint4(y, HUBREF, 1u, hint);
            } else {
                if (!locate()) return;
                *reinterpret_cast<uint4*>(a.g.pool + lx + local) = make_uint4(y, ly, dy, p);
            }
        }
        // (ii) y's entry pointing at x (x's list moved or resized), when y's own
        // pass does not write it.  Entries pointing at x hold HUBREF when x is a
        // hub that stayed a hub (handled above), and no change of x's list can
        // make those stale.
        if (!need_back) return;
        if (!locate()) return;
        const uint4 back = x_hub ? make_uint4(x, HUBREF, 1u, local) : make_uint4(x, lx, a.g.deg[x], local);
        *reinterpret_cast<uint4*>(a.g.pool + ly + p) = back;
    });
}

void csr_exec(CSR& g, const ChangeList& cl, ApplyScratch& s, uint32_t* touched, uint32_t* d_err,
              cudaStream_t st, cudaEvent_t merge_t0, cudaEvent_t merge_t1) {
    const int grid = flat_grid();
    ExecArgs a;
    a.cl = cl;
    a.g = g.view();
    a.n = (uint32_t)g.n;
    a.p_ins = s.p_ins.p; a.p_del = s.p_del.p; a.totals = s.totals.p;
    a.tv = s.tv.p; a.tstart = s.tstart.p; a.tend = s.tend.p; a.odeg = s.odeg.p; a.ndeg = s.ndeg.p;
    a.ooff = s.ooff.p; a.ncap = s.ncap.p; a.rsz = s.rsz.p; a.r_off = s.r_off.p; a.s_off = s.s_off.p;
    a.w_off = s.w_off.p;
    a.f_off = s.f_off.p;
    a.sdeg = s.sdeg.p;
    a.xm = s.xm.p;
    a.tdst = s.tdst.p;
    a.stage = s.stage.p;
    a.touched = touched;
    // merge reads the old lists and writes the new ones (into twins or fresh
    // space; lists without a twin into the staging buffer); meta_place then
    // points every touched vertex at its final slots and copies staged lists
    // back; fix refreshes caches.
    if (merge_t0) DG_CUDA(record_timing_event(merge_t0, st));
    k_exec_merge<<<grid, FLAT_THREADS, 0, st>>>(a, d_err);
    if (merge_t1) DG_CUDA(record_timing_event(merge_t1, st));
    k_exec_meta_place<<<grid, FLAT_THREADS, 0, st>>>(a, d_err);
    k_exec_fix<<<grid, FLAT_THREADS, 0, st>>>(a, d_err);
    g_launches += 3;
    DG_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// compaction
// ---------------------------------------------------------------------------
__global__ void k_compact_copy(CSRView g, const uint32_t* __restrict__ noff, uint32_t total,
                               Ent* __restrict__ np) {
    for (uint32_t item = blockIdx.x * blockDim.x + threadIdx.x; item < total; item += gridDim.x * blockDim.x) {
        const uint32_t x = upper_bound_arr<uint32_t>(noff, 0, (uint32_t)g.n, item) - 1;
        const uint32_t local = item - noff[x];
        if (local >= g.deg[x]) continue;
        Ent e = g.pool[g.off[x] + local];
        if (e.noff != HUBREF) e.noff = noff[e.nbr];
        np[item] = e;
    }
}

void csr_compact(CSR& g, DevAlloc& a, uint64_t min_free, cudaStream_t st) {
    const uint32_t n = (uint32_t)g.n;
    const int grid = flat_grid();
    DBuf<uint32_t> ncap, noff, tmp, total;
    ncap.ensure(a, (size_t)n + 1, st);
    noff.ensure(a, (size_t)n + 1, st);
    tmp.ensure(a, scan_tmp_words(n + 1), st);
    total.ensure(a, 2, st);
    k_caps<<<grid, FLAT_THREADS, 0, st>>>(g.deg.p, n, g.slack, ncap.p);
    ++g_launches;
    ScanJob job;
    job.in[0] = ncap.p;
    job.out[0] = noff.p;
    job.total[0] = total.p;
    job.k = 1;
    scan_exclusive(job, nullptr, n, tmp.p, st);
    k_twin_layout<<<grid, FLAT_THREADS, 0, st>>>(noff.p, ncap.p, n, g.twin.p);
    ++g_launches;
    uint32_t h_caps = 0;
    DG_CUDA(cudaMemcpyAsync(&h_caps, total.p, 4, cudaMemcpyDeviceToHost, st));
    DG_CUDA(cudaStreamSynchronize(st));
    const uint64_t h_total = 2ull * h_caps;  // lists and their twins
    uint64_t want = h_total + (uint64_t)((double)h_total * g.overflow) + 4096;
    if (want < h_total + min_free) want = h_total + min_free;
    if (want >= 0xFFFFFFF0ull) throw Error(DG_E_NOMEM, "graph too large for 32-bit pool offsets");
    DBuf<Ent> np;
    np.ensure(a, want, st);
    if (h_total > 0) {
        k_compact_copy<<<grid, FLAT_THREADS, 0, st>>>(g.view(), noff.p, (uint32_t)h_total, np.p);
        ++g_launches;
    }
    DG_CHECK_LAUNCH();
    g.pool.release(a, st);
    g.pool = np;
    g.pool_cap = want;
    std::swap(g.off, noff);
    std::swap(g.cap, ncap);
    noff.release(a, st);
    ncap.release(a, st);
    tmp.release(a, st);
    total.release(a, st);
    unsigned long long t = h_total;
    DG_CUDA(cudaMemcpyAsync(g.top.p, &t, sizeof(t), cudaMemcpyHostToDevice, st));
    g.host_top = h_total;
    DG_CUDA(cudaStreamSynchronize(st));
}

// ---------------------------------------------------------------------------
// export
// ---------------------------------------------------------------------------
__global__ void k_count_upper(CSRView g, uint32_t* __restrict__ cnt) {
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < (uint32_t)g.n; x += gridDim.x * blockDim.x) {
        const uint32_t d = g.deg[x];
        cnt[x] = d - lower_bound_nbr(g.pool + g.off[x], d, x + 1);
    }
}

__global__ void k_export(CSRView g, const uint32_t* __restrict__ pos, int32_t* __restrict__ A,
                         int32_t* __restrict__ B, double* __restrict__ W) {
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < (uint32_t)g.n; x += gridDim.x * blockDim.x) {
        const uint32_t d = g.deg[x];
        const Ent* L = g.pool + g.off[x];
        uint32_t k = lower_bound_nbr(L, d, x + 1);
        uint32_t p = pos[x];
        for (; k < d; ++k, ++p) {
            A[p] = (int32_t)x;
            B[p] = (int32_t)L[k].nbr;
            if (W) W[p] = L[k].w;
        }
    }
}

static uint32_t export_prepare(CSR& g, DevAlloc& a, DBuf<uint32_t>& cnt, DBuf<uint32_t>& pos, cudaStream_t st) {
    const uint32_t n = (uint32_t)g.n;
    const int grid = flat_grid();
    DBuf<uint32_t> tmp, total;
    cnt.ensure(a, (size_t)n + 1, st);
    pos.ensure(a, (size_t)n + 1, st);
    tmp.ensure(a, scan_tmp_words(n + 1), st);
    total.ensure(a, 2, st);
    k_count_upper<<<grid, FLAT_THREADS, 0, st>>>(g.view(), cnt.p);
    ++g_launches;
    ScanJob job;
    job.in[0] = cnt.p;
    job.out[0] = pos.p;
    job.total[0] = total.p;
    job.k = 1;
    scan_exclusive(job, nullptr, n, tmp.p, st);
    uint32_t h = 0;
    DG_CUDA(cudaMemcpyAsync(&h, total.p, 4, cudaMemcpyDeviceToHost, st));
    DG_CUDA(cudaStreamSynchronize(st));
    tmp.release(a, st);
    total.release(a, st);
    return h;
}

uint64_t csr_edge_count(CSR& g, DevAlloc& a, cudaStream_t st) {
    DBuf<uint32_t> cnt, pos;
    uint32_t h = export_prepare(g, a, cnt, pos, st);
    cnt.release(a, st);
    pos.release(a, st);
    return h;
}

void csr_export(CSR& g, DevAlloc& a, int32_t* d_a, int32_t* d_b, double* d_w, cudaStream_t st) {
    DBuf<uint32_t> cnt, pos;
    export_prepare(g, a, cnt, pos, st);
    k_export<<<flat_grid(), FLAT_THREADS, 0, st>>>(g.view(), pos.p, d_a, d_b, d_w);
    ++g_launches;
    DG_CHECK_LAUNCH();
    cnt.release(a, st);
    pos.release(a, st);
}

}  // namespace dg
