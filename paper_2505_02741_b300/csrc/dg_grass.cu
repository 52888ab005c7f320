// dg_grass.cu -- a GRASS-like initial sparsifier on the device.
//
// Section III-A takes H(0) from GRASS: a spanning tree plus the off-tree edges
// that matter spectrally.  Here the caller gives a spanning forest F of G, and
// every off-tree edge e = (p, q) is ranked by its stretch w_e * R_F(p, q), the
// distortion the insertion test of Section III-B measures (on a tree the walk
// from p to q is the tree path, so R_F is what a walker would accumulate).
// H(0) = F + the n_off off-tree edges of largest stretch (ties: smaller
// canonical edge id).
//
// R_F comes from root distances: every tree is rooted at its smallest vertex,
// D[root] = 0 and D[y] = D[x] + r(x, y) for a child y of x (one rounding per
// addition, in the order of the path from the root, so the value does not
// depend on the order the tree is traversed in); R_F(p, q) =
// (D[p] - D[l]) + (D[q] - D[l]) with l the lowest common ancestor; +inf when
// p and q lie in different trees.
//
// Steps: components by minimum-label propagation over the forest edges (the
// label of a tree is its smallest vertex; n - nt trees exactly, else the
// edges close a cycle and are rejected), the forest's adjacency by counting, level-synchronous traversal
// from the roots (parent, depth, D), ancestor tables by pointer doubling,
// stretch of every edge of G in canonical order, a stable radix sort by
// descending stretch, and the sparsifier build of the selected edges.
#include <algorithm>
#include <cmath>
#include <vector>

#include "dg_ctx.h"

namespace dg {

namespace {

constexpr int GT = 256;

int g_grid(uint64_t items) {
    const uint64_t b = (items + GT - 1) / GT;
    const uint64_t cap = (uint64_t)device_sms() * 8;
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(b, cap));
}

__global__ void k_label_init(uint32_t* label, uint32_t n, uint32_t* deg) {
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        label[x] = x;
        deg[x] = 0;
    }
}

// every forest edge must be a G edge with distinct endpoints; r of the edge from G
__global__ void k_forest_check(const int32_t* __restrict__ tu, const int32_t* __restrict__ tv, uint32_t nt, CSRView G,
                               double* __restrict__ tr, uint32_t* d_err) {
    const uint32_t n = (uint32_t)G.n;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nt; i += gridDim.x * blockDim.x) {
        const int32_t a = tu[i], b = tv[i];
        double w = 0.0;
        if (a < 0 || b < 0 || (uint32_t)a >= n || (uint32_t)b >= n || a == b ||
            !has_edge(G, (uint32_t)a, (uint32_t)b, &w)) {
            atomicOr(d_err, (uint32_t)ERR_NOT_IN_G);
            tr[i] = 0.0;
            continue;
        }
        tr[i] = __ddiv_rn(1.0, w);
    }
}

// Components by minimum-label propagation: every label is a vertex of the
// same tree with an id no larger than the vertex's own, and it only ever
// decreases (atomicMin), so repeating the two passes below until nothing
// changes leaves every vertex labelled with the smallest vertex of its tree.
// Edge pass: both endpoints, and the vertex the larger label names, take the
// smaller label.
__global__ void k_label_edges(const int32_t* __restrict__ tu, const int32_t* __restrict__ tv, uint32_t nt,
                              uint32_t* label, uint32_t* changed) {
    bool ch = false;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nt; i += gridDim.x * blockDim.x) {
        const uint32_t a = (uint32_t)tu[i], b = (uint32_t)tv[i];
        const uint32_t la = __ldcg(&label[a]), lb = __ldcg(&label[b]);
        if (la == lb) continue;
        const uint32_t lo = min(la, lb), hi = max(la, lb);
        ch |= atomicMin(&label[a], lo) > lo;
        ch |= atomicMin(&label[b], lo) > lo;
        ch |= atomicMin(&label[hi], lo) > lo;
    }
    if (__any_sync(0xffffffffu, ch) && (threadIdx.x & 31) == 0) *changed = 1u;
}

// Jump pass: a label takes its label's label (both lie in the same tree).
__global__ void k_label_jump(uint32_t* label, uint32_t n, uint32_t* changed) {
    bool ch = false;
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        const uint32_t l = __ldcg(&label[x]);
        const uint32_t ll = __ldcg(&label[l]);
        if (ll < l) ch |= atomicMin(&label[x], ll) > ll;
    }
    if (__any_sync(0xffffffffu, ch) && (threadIdx.x & 31) == 0) *changed = 1u;
}

// trees of the forest: vertices that label themselves
__global__ void k_label_roots(const uint32_t* __restrict__ label, uint32_t n, uint32_t* nroots) {
    uint32_t c = 0;
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) c += label[x] == x;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(nroots, c);
}

__global__ void k_forest_deg(const int32_t* __restrict__ tu, const int32_t* __restrict__ tv, uint32_t nt,
                             uint32_t* deg) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nt; i += gridDim.x * blockDim.x) {
        atomicAdd(&deg[tu[i]], 1u);
        atomicAdd(&deg[tv[i]], 1u);
    }
}

__global__ void k_forest_fill(const int32_t* __restrict__ tu, const int32_t* __restrict__ tv,
                              const double* __restrict__ tr, uint32_t nt, const uint32_t* __restrict__ start,
                              uint32_t* cursor, uint32_t* __restrict__ nb, double* __restrict__ nr) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nt; i += gridDim.x * blockDim.x) {
        const uint32_t a = (uint32_t)tu[i], b = (uint32_t)tv[i];
        const uint32_t pa = start[a] + atomicAdd(&cursor[a], 1u);
        const uint32_t pb = start[b] + atomicAdd(&cursor[b], 1u);
        nb[pa] = b;
        nr[pa] = tr[i];
        nb[pb] = a;
        nr[pb] = tr[i];
    }
}

// level 0: the roots (a root is its own parent)
__global__ void k_roots(const uint32_t* __restrict__ comp, uint32_t n, uint32_t* parent, uint32_t* depth, double* D,
                        uint32_t* frontier, uint32_t* count0) {
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        if (comp[x] != x) continue;
        parent[x] = x;
        depth[x] = 0;
        D[x] = 0.0;
        frontier[atomicAdd(count0, 1u)] = x;
    }
}

// one level of the traversal: the children of the frontier's vertices
__global__ void k_level(const uint32_t* __restrict__ start, const uint32_t* __restrict__ nb,
                        const double* __restrict__ nr, uint32_t* parent, uint32_t* depth, double* D,
                        const uint32_t* __restrict__ cur, const uint32_t* cur_count, uint32_t* next,
                        uint32_t* next_count) {
    const uint32_t F = *cur_count;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < F; q += gridDim.x * blockDim.x) {
        const uint32_t x = cur[q];
        const uint32_t px = parent[x], dx = depth[x];
        const double Dx = D[x];
        for (uint32_t k = start[x]; k < start[x + 1]; ++k) {
            const uint32_t y = nb[k];
            if (y == px) continue;  // the edge up to x's parent (a root is its own parent)
            parent[y] = x;
            depth[y] = dx + 1;
            D[y] = __dadd_rn(Dx, nr[k]);
            next[atomicAdd(next_count, 1u)] = y;
        }
    }
}

__global__ void k_lift(const uint32_t* __restrict__ prev, uint32_t* __restrict__ out, uint32_t n) {
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) out[x] = prev[prev[x]];
}

// stretch of every canonical edge i (0 for forest edges, +inf across trees),
// and the sort key: descending stretch for off-tree edges, forest edges last
__global__ void k_stretch(const int32_t* __restrict__ ea, const int32_t* __restrict__ eb,
                          const double* __restrict__ ew, uint32_t m, const uint32_t* __restrict__ comp,
                          const uint32_t* __restrict__ parent, const uint32_t* __restrict__ depth,
                          const double* __restrict__ D, const uint32_t* __restrict__ up, uint32_t n, int levels,
                          double* __restrict__ stretch, uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const uint32_t p = (uint32_t)ea[i], q = (uint32_t)eb[i];
        vals[i] = i;
        if (parent[p] == q || parent[q] == p) {  // a forest edge (G is simple)
            stretch[i] = 0.0;
            keys[i] = ~0ull;
            continue;
        }
        double st;
        if (comp[p] != comp[q]) {
            st = INFINITY;
        } else {
            uint32_t x = p, y = q;
            if (depth[x] < depth[y]) {
                const uint32_t t = x;
                x = y;
                y = t;
            }
            uint32_t diff = depth[x] - depth[y];
            for (int k = 0; diff; ++k, diff >>= 1)
                if (diff & 1u) x = up[(size_t)k * n + x];
            if (x != y) {
                for (int k = levels - 1; k >= 0; --k) {
                    const uint32_t ax = up[(size_t)k * n + x], ay = up[(size_t)k * n + y];
                    if (ax != ay) {
                        x = ax;
                        y = ay;
                    }
                }
                x = parent[x];
            }
            const double R = __dadd_rn(__dsub_rn(D[p], D[x]), __dsub_rn(D[q], D[x]));
            st = __dmul_rn(ew[i], R);
        }
        stretch[i] = st;
        keys[i] = ~(uint64_t)__double_as_longlong(st);  // non-negative doubles order like their bits
    }
}

// H(0) edge list: the forest edges followed by the first n_off sorted ids
__global__ void k_grass_pick(const int32_t* __restrict__ tu, const int32_t* __restrict__ tv, uint32_t nt,
                             const uint32_t* __restrict__ ids, uint32_t n_off, const int32_t* __restrict__ ea,
                             const int32_t* __restrict__ eb, int32_t* __restrict__ hu, int32_t* __restrict__ hv) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nt + n_off; i += gridDim.x * blockDim.x) {
        if (i < nt) {
            hu[i] = tu[i];
            hv[i] = tv[i];
        } else {
            const uint32_t e = ids[i - nt];
            hu[i] = ea[e];
            hv[i] = eb[e];
        }
    }
}

}  // namespace

void graph_init_grass(Ctx& c, DGraph& g, int64_t nt64, const int32_t* tu_h, const int32_t* tv_h, int64_t n_off64,
                      double* stretch_out) {
    if (g.shard.active) throw Error(DG_E_STATE, "a sharded batch is in progress on this graph");
    cudaStream_t st = c.stream;
    DevAlloc& a = c.alloc;
    const uint32_t n = (uint32_t)g.n;
    if (nt64 < 0 || nt64 >= (int64_t)n + (n == 0) || (nt64 > 0 && (!tu_h || !tv_h)))
        throw Error(DG_E_INVALID, "a forest has at most n - 1 edges");
    if (n_off64 < 0) throw Error(DG_E_INVALID, "negative off-tree edge count");
    const uint32_t nt = (uint32_t)nt64;
    graph_wait_estimates(g, st);
    const uint64_t m64 = csr_edge_count(g.G, a, st);
    if (m64 >= 0x7FFFFFF0ull) throw Error(DG_E_INVALID, "graph too large");
    const uint32_t m = (uint32_t)m64;
    const uint32_t n_off = (uint32_t)std::min<int64_t>(n_off64, (int64_t)m - (int64_t)nt);

    DBuf<int32_t> tu, tv, ea, eb, hu, hv;
    DBuf<double> tr, nr, D, ew, stretch;
    DBuf<uint32_t> comp, deg, start, cursor, nb, parent, depth, fr0, fr1, counts, up, err, vals, vals_alt, hist,
        stmp, tot;
    DBuf<uint64_t> keys, keys_alt;
    auto release_all = [&]() {
        for (auto* b : {&tu, &tv, &ea, &eb, &hu, &hv}) b->release(a, st);
        for (auto* b : {&tr, &nr, &D, &ew, &stretch}) b->release(a, st);
        for (auto* b : {&comp, &deg, &start, &cursor, &nb, &parent, &depth, &fr0, &fr1, &counts, &up, &err, &vals,
                        &vals_alt, &hist, &stmp, &tot})
            b->release(a, st);
        keys.release(a, st);
        keys_alt.release(a, st);
    };
    try {
        tu.ensure(a, nt + 1, st);
        tv.ensure(a, nt + 1, st);
        tr.ensure(a, nt + 1, st);
        comp.ensure(a, n + 1, st);
        deg.ensure(a, n + 1, st);
        start.ensure(a, n + 2, st);
        cursor.ensure(a, n + 1, st);
        nb.ensure(a, 2ull * nt + 1, st);
        nr.ensure(a, 2ull * nt + 1, st);
        parent.ensure(a, n + 1, st);
        depth.ensure(a, n + 1, st);
        D.ensure(a, n + 1, st);
        fr0.ensure(a, n + 1, st);
        fr1.ensure(a, n + 1, st);
        counts.ensure(a, (size_t)n + 2, st);
        err.ensure(a, 1, st);
        tot.ensure(a, 2, st);
        stmp.ensure(a, scan_tmp_words(n + 1), st);
        DG_CUDA(cudaMemsetAsync(err.p, 0, 4, st));
        DG_CUDA(cudaMemsetAsync(counts.p, 0, counts.bytes(), st));
        DG_CUDA(cudaMemsetAsync(cursor.p, 0, cursor.bytes(), st));
        if (nt) {
            DG_CUDA(cudaMemcpyAsync(tu.p, tu_h, 4ull * nt, cudaMemcpyHostToDevice, st));
            DG_CUDA(cudaMemcpyAsync(tv.p, tv_h, 4ull * nt, cudaMemcpyHostToDevice, st));
        }
        // components of the forest (cycle check), adjacency
        k_label_init<<<g_grid(n), GT, 0, st>>>(comp.p, n, deg.p);
        ++g_launches;
        uint32_t herr = 0;
        if (nt) {
            k_forest_check<<<g_grid(nt), GT, 0, st>>>(tu.p, tv.p, nt, g.G.view(), tr.p, err.p);
            ++g_launches;
            DG_CUDA(cudaMemcpyAsync(&herr, err.p, 4, cudaMemcpyDeviceToHost, st));
            DG_CUDA(cudaStreamSynchronize(st));
            if (herr) throw Error(DG_E_INVALID, "a forest edge is not an edge of G");
            for (int round = 0;; ++round) {
                if (round == 64 * 32) throw Error(DG_E_TIMEOUT, "the forest's labels did not settle");
                DG_CUDA(cudaMemsetAsync(tot.p, 0, 4, st));
                k_label_edges<<<g_grid(nt), GT, 0, st>>>(tu.p, tv.p, nt, comp.p, tot.p);
                k_label_jump<<<g_grid(n), GT, 0, st>>>(comp.p, n, tot.p);
                g_launches += 2;
                uint32_t changed = 0;
                DG_CUDA(cudaMemcpyAsync(&changed, tot.p, 4, cudaMemcpyDeviceToHost, st));
                DG_CUDA(cudaStreamSynchronize(st));
                if (!changed) break;
            }
        }
        {
            DG_CUDA(cudaMemsetAsync(tot.p, 0, 4, st));
            k_label_roots<<<g_grid(n), GT, 0, st>>>(comp.p, n, tot.p);
            ++g_launches;
            uint32_t nroots = 0;
            DG_CUDA(cudaMemcpyAsync(&nroots, tot.p, 4, cudaMemcpyDeviceToHost, st));
            DG_CUDA(cudaStreamSynchronize(st));
            if ((uint64_t)nroots + nt != n)  // each forest edge joins two trees
                throw Error(DG_E_INVALID, "the forest edges contain a cycle or a repeated edge");
        }
        if (nt) {
            k_forest_deg<<<g_grid(nt), GT, 0, st>>>(tu.p, tv.p, nt, deg.p);
            ++g_launches;
        }
        {
            ScanJob j;
            j.in[0] = deg.p;
            j.out[0] = start.p;
            j.total[0] = start.p + n;
            j.k = 1;
            scan_exclusive(j, nullptr, n, stmp.p, st);
        }
        if (nt) {
            k_forest_fill<<<g_grid(nt), GT, 0, st>>>(tu.p, tv.p, tr.p, nt, start.p, cursor.p, nb.p, nr.p);
            ++g_launches;
        }
        // level-synchronous traversal from the roots; counts[L] = size of level L
        k_roots<<<g_grid(n), GT, 0, st>>>(comp.p, n, parent.p, depth.p, D.p, fr0.p, counts.p);
        ++g_launches;
        uint32_t levels = 1;
        uint32_t* fr[2] = {fr0.p, fr1.p};
        for (uint32_t L = 0;; L += 64) {
            const uint32_t hi = std::min<uint32_t>(L + 64, n);
            for (uint32_t l = L; l < hi; ++l) {
                k_level<<<g_grid(n), GT, 0, st>>>(start.p, nb.p, nr.p, parent.p, depth.p, D.p, fr[l & 1],
                                                   counts.p + l, fr[(l + 1) & 1], counts.p + l + 1);
                ++g_launches;
            }
            uint32_t c_hi = 0;
            DG_CUDA(cudaMemcpyAsync(&c_hi, counts.p + hi, 4, cudaMemcpyDeviceToHost, st));
            DG_CUDA(cudaStreamSynchronize(st));
            if (c_hi == 0 || hi >= n) {
                std::vector<uint32_t> hc(hi - L + 1);
                DG_CUDA(cudaMemcpy(hc.data(), counts.p + L, 4ull * hc.size(), cudaMemcpyDeviceToHost));
                levels = L;
                for (uint32_t l = 0; l < hc.size() && hc[l]; ++l) levels = L + l + 1;
                break;
            }
        }
        // ancestor tables: up[k][x] = the 2^k-th ancestor (a root maps to itself)
        const uint32_t max_depth = levels > 0 ? levels - 1 : 0;
        const int lv = std::max(1, bit_length((uint64_t)max_depth));
        up.ensure(a, (size_t)lv * n + 1, st);
        DG_CUDA(cudaMemcpyAsync(up.p, parent.p, 4ull * n, cudaMemcpyDeviceToDevice, st));
        for (int k = 1; k < lv; ++k) {
            k_lift<<<g_grid(n), GT, 0, st>>>(up.p + (size_t)(k - 1) * n, up.p + (size_t)k * n, n);
            ++g_launches;
        }
        // every edge of G in canonical order, its stretch and sort key
        ea.ensure(a, m + 1, st);
        eb.ensure(a, m + 1, st);
        ew.ensure(a, m + 1, st);
        stretch.ensure(a, m + 1, st);
        keys.ensure(a, m + 1, st);
        keys_alt.ensure(a, m + 1, st);
        vals.ensure(a, m + 1, st);
        vals_alt.ensure(a, m + 1, st);
        if (m) csr_export(g.G, a, ea.p, eb.p, ew.p, st);
        if (m) {
            k_stretch<<<g_grid(m), GT, 0, st>>>(ea.p, eb.p, ew.p, m, comp.p, parent.p, depth.p, D.p, up.p, n, lv,
                                                 stretch.p, keys.p, vals.p);
            ++g_launches;
        }
        // stable sort by descending stretch: equal stretches keep the edge order
        const uint32_t* ids = vals.p;
        if (n_off && m) {
            hist.ensure(a, sort_hist_words(m), st);
            DBuf<uint32_t> stmp2;
            stmp2.ensure(a, sort_scan_tmp_words(m), st);
            SortBufs sb{keys.p, vals.p, keys_alt.p, vals_alt.p, hist.p, stmp2.p, err.p};
            DG_CUDA(cudaMemcpyAsync(tot.p, &m, 4, cudaMemcpyHostToDevice, st));
            if (radix_sort_pairs(sb, tot.p, m, 64, st)) ids = vals_alt.p;
            DG_CUDA(cudaStreamSynchronize(st));
            stmp2.release(a, st);
        }
        hu.ensure(a, (size_t)nt + n_off + 1, st);
        hv.ensure(a, (size_t)nt + n_off + 1, st);
        if (nt + n_off) {
            k_grass_pick<<<g_grid(nt + n_off), GT, 0, st>>>(tu.p, tv.p, nt, ids, n_off, ea.p, eb.p, hu.p, hv.p);
            ++g_launches;
        }
        if (stretch_out && m)
            DG_CUDA(cudaMemcpyAsync(stretch_out, stretch.p, 8ull * m, cudaMemcpyDeviceToHost, st));
        DG_CUDA(cudaStreamSynchronize(st));
        graph_init_h(c, g, (int64_t)nt + n_off, hu.p, hv.p, true);
    } catch (...) {
        cudaStreamSynchronize(st);
        release_all();
        throw;
    }
    release_all();
}

}  // namespace dg

using namespace dg;

extern "C" dg_status dg_init_sparsifier_grass(dg_ctx* ctx, int32_t graph_id, int64_t nt, const int32_t* tu,
                                              const int32_t* tv, int64_t n_off, double* stretch_out) {
    try {
        if (!ctx) throw Error(DG_E_INVALID, "null context");
        Ctx& c = *reinterpret_cast<Ctx*>(ctx);
        DG_CUDA(cudaSetDevice(c.device));
        DGraph& g = c.graph(graph_id);
        std::lock_guard<std::mutex> lk(g.mu);
        graph_init_grass(c, g, nt, tu, tv, n_off, stretch_out);
        return DG_OK;
    } catch (const Error& e) {
        set_last_error(e.what());
        return e.code;
    } catch (const std::exception& e) {
        set_last_error(e.what());
        return DG_E_CUDA;
    }
}
