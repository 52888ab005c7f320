// dg_csr.cuh -- slack-slot CSR on the device: build, batched mutation (plan /
// execute), compaction and export.
//
// Mutation follows the dynamic CSR idea of Section III-F (lists that outgrow
// their slots move into spare pool space), made parallel and deterministic: a
// batch's half-edge changes arrive sorted by (vertex, neighbour); every
// touched vertex's new list is the sorted merge of its old list and its
// changes, computed with one thread per output position (load-balanced over
// all touched vertices, so hubs cost no more than their degree).  Each list
// has a twin region of its capacity: the merge writes the new list into the
// twin (or into fresh pool space when it outgrew its capacity), and the region
// it leaves becomes the twin; then the cached (off, deg, rev) fields of the
// entries that point at moved or resized lists are refreshed.  A list without
// a twin is merged through a staging buffer and copied back in place.
#pragma once
#include "dg_common.cuh"
#include "dg_host.h"
#include "dg_prims.cuh"

namespace dg {

struct CSR {
    int32_t n = 0;
    uint64_t pool_cap = 0;  // entries
    float slack = 1.25f;
    double overflow = 0.5;
    DBuf<uint32_t> off, deg, cap;
    DBuf<uint8_t> hub;
    DBuf<uint32_t> nhub;
    DBuf<uint32_t> twin;
    DBuf<Ent> pool;
    DBuf<unsigned long long> top;
    DBuf<unsigned long long> minr;  // resistance lower bound (CSRView::minr)
    uint64_t host_top = 0;  // last value read back

    CSRView view() const {
        CSRView v;
        v.off = off.p;
        v.deg = deg.p;
        v.cap = cap.p;
        v.hub = hub.p;
        v.nhub = nhub.p;
        v.twin = twin.p;
        v.pool = pool.p;
        v.top = top.p;
        v.minr = minr.p;
        v.pool_cap = pool_cap;
        v.n = n;
        return v;
    }
    uint64_t bytes() const {
        return off.bytes() + deg.bytes() + cap.bytes() + hub.bytes() + nhub.bytes() + twin.bytes() + pool.bytes() +
               top.bytes() + minr.bytes();
    }
};

// sorted, unique half-edge changes: keys[c] = x * n + y ascending; vals[c]
// indexes the payload arrays kinds[] (CHG_*) and ws[] (new weight).
struct ChangeList {
    const uint64_t* keys = nullptr;
    const uint32_t* vals = nullptr;
    const uint8_t* kinds = nullptr;
    const double* ws = nullptr;
    const uint32_t* d_count = nullptr;
    uint32_t max_count = 0;
};

enum { TOT_X = 0, TOT_NI, TOT_ND, TOT_R, TOT_S, TOT_WK, TOT_BASE_LO, TOT_BASE_HI, TOT_F, TOT_WORDS = 9 };

struct ApplyScratch {
    uint32_t c_max = 0;
    uint64_t s_cap = 0;  // entries of staging space
    DBuf<uint32_t> p_head, p_ins, p_del;  // exclusive run heads, insertions, deletions (the plan's first scan)
    DBuf<uint32_t> tv, tstart, tend, odeg, ndeg, ooff, ncap, rsz, work, r_off, s_off, w_off, fwork, f_off;
    DBuf<uint32_t> sdeg, xm, tdst;  // staged size, placement mode, twin destination (see k_plan_touch)
    DBuf<uint32_t> scan_tmp, totals;  // scan_tmp: one region of scan_words per scan of the plan (2)
    uint64_t scan_words = 0;
    DBuf<Ent> stage;
    void ensure(DevAlloc& a, uint32_t changes, uint64_t stage_entries, cudaStream_t st);
    void release(DevAlloc& a, cudaStream_t st);
    uint64_t bytes() const;
};

void csr_alloc_vertices(CSR& g, DevAlloc& a, int32_t n, cudaStream_t st);
void csr_release(CSR& g, DevAlloc& a, cudaStream_t st);

// Build g (fresh) from sorted unique half-edge keys with weights ws[vals[c]].
// Sets ERR_DUP_EDGE in *d_err when two keys are equal.  count is host-known.
void csr_build(CSR& g, DevAlloc& a, const uint64_t* keys, const uint32_t* vals, const double* ws,
               uint32_t count, uint32_t* d_err, cudaStream_t st);

// plan: sizes, relocation space and staging checks; raises pool_err_bit or
// cap_err_bit in *d_err instead of writing anything when space is short.
// tmp_zeroed: both scan_tmp regions were cleared by the caller
void csr_plan(CSR& g, const ChangeList& cl, ApplyScratch& s, uint32_t* d_err, uint32_t pool_err_bit,
              uint32_t cap_err_bit, cudaStream_t st, bool tmp_zeroed = false);
// execute: merge, place, refresh cached fields (no-op when *d_err has an abort bit)
// touched: n + 1 words; entry x = (generation << 2) | bits for the vertices an
// execution changed, word n = the array's generation (bumped per execution),
// so marks of earlier executions never match and nothing needs clearing.
// merge_t0 / merge_t1 (nullable): timing events recorded around the merge kernel
void csr_exec(CSR& g, const ChangeList& cl, ApplyScratch& s, uint32_t* touched, uint32_t* d_err,
              cudaStream_t st, cudaEvent_t merge_t0 = nullptr, cudaEvent_t merge_t1 = nullptr);

// rebuild every list with fresh slack into a new pool with at least min_free spare entries
void csr_compact(CSR& g, DevAlloc& a, uint64_t min_free, cudaStream_t st);

// number of undirected edges (host, synchronous)
uint64_t csr_edge_count(CSR& g, DevAlloc& a, cudaStream_t st);
// export edges (x < nbr) in lexicographic order into device arrays of size >= count
void csr_export(CSR& g, DevAlloc& a, int32_t* d_a, int32_t* d_b, double* d_w, cudaStream_t st);

int flat_grid();  // grid size of the grid-stride flattened kernels

}  // namespace dg
