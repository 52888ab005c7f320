// dg_quality.cu -- how good the sparsifier is, measured on the device the way
// Section IV measures it: the off-tree density d_H = |E_H| / |V| - 1, the
// relative condition number kappa(L_G, L_H) (Eqs. 6-10), and the iterations
// of PCG on L_G x = b with L_H as the preconditioner (Table IV).
//
// Layout.  Each call copies G and H out of their slack-slot pools into plain
// CSR arrays (column id 4 B + weight 8 B per stored entry, rows in ascending
// neighbour order) so that the many Laplacian products of an iterative solve
// read 12 B per entry instead of the 32-byte walk entry.
//
// L_H^+ is applied by conjugate gradients on L_H preconditioned with H's
// maximum-weight spanning forest F.  F's Laplacian is solved exactly: for a
// tree rooted at r, the current through the edge (parent(y), y) is the sum of
// the right-hand side over y's subtree, and the potential of y is the sum of
// current / weight over the edges of its root path (z_r = 0).  Both sums are
// prefix sums over the Euler tour of the tree: a subtree is a contiguous range
// of the tour, and a root path is what stays open at y's entry.  The tour is
// ranked once per call by pointer jumping; every solve is then two prefix sums
// of 128-bit fixed-point images of the doubles: integer sums are exact in any
// order, so each current and each potential is the exact sum rounded once,
// even where a subtree's sum is small next to the running prefix (and the
// sums cost integer adds, not the FP64 operations a compensated sum needs).
//
// F comes from Boruvka's algorithm with the strict order (weight descending,
// then (min, max) endpoint pair ascending): every component takes its best
// leaving edge (integer atomics on the weight's bits, then on the pair), a
// pair of components that chose the same edge keeps the smaller as root, and
// labels are flattened by pointer jumping.  Under a strict order the result
// is the unique maximum spanning forest, the one Kruskal's scan finds.
//
// Every reduction is deterministic: dot products sum fixed grid-stride slices
// in order, then fixed trees.  The host only launches and reads back the stop
// flags.
#include <algorithm>
#include <cmath>
#include <vector>

#include "dg_ctx.h"

namespace dg {

namespace {

constexpr int QT = 256;        // threads per block of the flat kernels
constexpr uint32_t BIG_ROW = 32;  // rows with more entries get a warp in the Laplacian product
constexpr uint32_t NONE = 0xFFFFFFFFu;

int q_grid(uint64_t items) {
    const uint64_t b = (items + QT - 1) / QT;
    const uint64_t cap = (uint64_t)device_sms() * 8;
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(b, cap));
}
int dot_blocks() { return device_sms() * 2; }

#define QLAUNCH(k, g, b, st, ...)                   \
    do {                                            \
        k<<<(g), (b), 0, (st)>>>(__VA_ARGS__);      \
        ++g_launches;                               \
    } while (0)

// ---------------------------------------------------------------------------
// exact sums of doubles in 128-bit fixed point.  A vector is scaled by 2^s,
// s chosen from its largest exponent so that the sum of all its entries fits
// in 125 bits; each entry becomes an integer (exact unless its lowest bits lie
// 2^100 below the largest entry, where it is rounded), every prefix sum is
// then an exact integer sum in any order, and a difference of two prefixes
// turns back into a double with one rounding.
// ---------------------------------------------------------------------------
typedef __int128 i128;
typedef unsigned __int128 u128;

__device__ __forceinline__ uint32_t biased_exp(double v) {
    return (uint32_t)((__double_as_longlong(v) >> 52) & 0x7FF);
}

// the scale 2^s for a vector whose largest biased exponent is e_max (|v| <
// 2^(e_max - 1022)), summed over at most 2^nbits entries
__device__ __forceinline__ int fixed_scale(uint32_t e_max, int nbits) {
    return e_max == 0 ? 0 : 125 - nbits - ((int)e_max - 1022);
}

__device__ __forceinline__ i128 to_fixed(double v, int s) {
    const long long bits = __double_as_longlong(v);
    const int be = (int)((bits >> 52) & 0x7FF);
    if (be == 0) return 0;  // zero (and subnormals, far below every scale used)
    const long long man = (bits & 0xFFFFFFFFFFFFFll) | (1ll << 52);  // v = man * 2^(be - 1075)
    const int sh = be - 1075 + s;
    i128 q;
    if (sh >= 0) q = (i128)man << sh;
    else if (sh > -62) q = (i128)((man + (1ll << (-sh - 1))) >> (-sh));  // nearest, ties away from zero
    else q = 0;
    return bits < 0 ? -q : q;
}

// v * 2^-s, rounded once to nearest even
__device__ __forceinline__ double from_fixed(i128 v, int s) {
    const bool neg = v < 0;
    const u128 m = neg ? (u128)(-v) : (u128)v;
    const unsigned long long hi = (unsigned long long)(m >> 64);
    double d;
    int up = 0;
    if (hi == 0) {
        d = __ull2double_rn((unsigned long long)m);
    } else {
        const int sh = 64 - __clzll(hi);  // keep the top 64 bits, fold the rest into a sticky bit
        unsigned long long t = (unsigned long long)(m >> sh);
        if ((m & (((u128)1 << sh) - 1)) != 0) t |= 1ull;
        d = __ull2double_rn(t);
        up = sh;
    }
    d = ldexp(d, up - s);
    return neg ? -d : d;
}

__device__ __forceinline__ i128 shfl_up_i128(i128 v, int d) {
    const unsigned long long lo = __shfl_up_sync(0xffffffffu, (unsigned long long)v, d);
    const long long hi = __shfl_up_sync(0xffffffffu, (long long)(v >> 64), d);
    return ((i128)hi << 64) | (i128)lo;
}

// the largest biased exponent of v[0..n) into *e (atomicMax; *e zeroed before)
__global__ void k_max_exp(const double* __restrict__ v, uint32_t n, uint32_t* e, const uint32_t* skip) {
    if (skip && *skip) return;
    uint32_t m = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        m = max(m, biased_exp(v[i]));
    for (int k = 16; k > 0; k >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, k));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(e, m);
}

__global__ void k_zero_words(uint32_t* w, int k, const uint32_t* skip) {
    if (skip && *skip) return;
    if (threadIdx.x < (unsigned)k) w[threadIdx.x] = 0;
}

// block-wide sum of one double per thread in a fixed tree
__device__ double block_sum(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] = __dadd_rn(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------
// compact Laplacians
// ---------------------------------------------------------------------------
struct Lap {
    uint32_t n = 0;
    uint32_t nnz = 0;
    uint32_t nbig = 0;
    DBuf<uint32_t> ptr, col, big, tmp;
    DBuf<double> val, diag;
    void release(DevAlloc& a, cudaStream_t st) {
        ptr.release(a, st);
        col.release(a, st);
        big.release(a, st);
        tmp.release(a, st);
        val.release(a, st);
        diag.release(a, st);
    }
};

__global__ void k_lap_deg(CSRView g, uint32_t* __restrict__ deg) {
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < (uint32_t)g.n; x += gridDim.x * blockDim.x)
        deg[x] = g.deg[x];
}

// one warp per vertex: copy the list (ascending neighbour order), sum the
// weighted degree (lane-strided partial sums, then a fixed shuffle tree), and
// list the rows the product gives a whole warp
__global__ void k_lap_fill(CSRView g, const uint32_t* __restrict__ ptr, uint32_t* __restrict__ col,
                           double* __restrict__ val, double* __restrict__ diag, uint32_t* __restrict__ big,
                           uint32_t* nbig) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t x = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < (uint32_t)g.n; x += warps) {
        const uint32_t d = g.deg[x], o = g.off[x], p = ptr[x];
        double s = 0.0;
        for (uint32_t j = lane; j < d; j += 32) {
            const Ent& e = g.pool[o + j];
            col[p + j] = e.nbr;
            val[p + j] = e.w;
            s = __dadd_rn(s, e.w);
        }
        for (int k = 16; k > 0; k >>= 1) s = __dadd_rn(s, __shfl_xor_sync(0xffffffffu, s, k));
        if (lane == 0) {
            diag[x] = s;
            if (d > BIG_ROW) big[atomicAdd(nbig, 1u)] = x;
        }
    }
}

// y = L x, one thread per row of at most BIG_ROW entries
__global__ void k_spmv_small(uint32_t n, const uint32_t* __restrict__ ptr, const uint32_t* __restrict__ col,
                             const double* __restrict__ val, const double* __restrict__ diag,
                             const double* __restrict__ xv, double* __restrict__ y, const uint32_t* skip) {
    if (skip && *skip) return;
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        const uint32_t a = ptr[x], b = ptr[x + 1];
        if (b - a > BIG_ROW) continue;
        double s = 0.0;
        for (uint32_t j = a; j < b; ++j) s = fma(val[j], xv[col[j]], s);
        y[x] = fma(diag[x], xv[x], -s);
    }
}

// y = L x, one warp per row of more than BIG_ROW entries
__global__ void k_spmv_big(const uint32_t* __restrict__ big, const uint32_t* nbig, const uint32_t* __restrict__ ptr,
                           const uint32_t* __restrict__ col, const double* __restrict__ val,
                           const double* __restrict__ diag, const double* __restrict__ xv, double* __restrict__ y,
                           const uint32_t* skip) {
    if (skip && *skip) return;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t nb = *nbig;
    for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nb; i += warps) {
        const uint32_t x = big[i];
        const uint32_t a = ptr[x], b = ptr[x + 1];
        double s = 0.0;
        for (uint32_t j = a + lane; j < b; j += 32) s = fma(val[j], xv[col[j]], s);
        for (int k = 16; k > 0; k >>= 1) s = __dadd_rn(s, __shfl_xor_sync(0xffffffffu, s, k));
        if (lane == 0) y[x] = fma(diag[x], xv[x], -s);
    }
}

void lap_build(Lap& L, const CSR& c, DevAlloc& a, cudaStream_t st) {
    const uint32_t n = (uint32_t)c.n;
    L.n = n;
    L.ptr.ensure(a, (size_t)n + 1, st);
    L.tmp.ensure(a, std::max<size_t>(scan_tmp_words(n + 1), 2), st);
    L.diag.ensure(a, (size_t)n + 1, st);
    L.big.ensure(a, (size_t)n + 1, st);
    DBuf<uint32_t> deg;
    deg.ensure(a, (size_t)n + 1, st);
    if (n) QLAUNCH(k_lap_deg, q_grid(n), QT, st, c.view(), deg.p);
    ScanJob j;
    j.in[0] = deg.p;
    j.out[0] = L.ptr.p;
    j.total[0] = L.ptr.p + n;
    j.k = 1;
    DG_CUDA(cudaMemsetAsync(L.tmp.p, 0, 4ull * L.tmp.n, st));
    if (n) scan_exclusive(j, nullptr, n, L.tmp.p, st, true);
    else DG_CUDA(cudaMemsetAsync(L.ptr.p, 0, 4, st));
    uint32_t nnz = 0;
    DG_CUDA(cudaMemcpyAsync(&nnz, L.ptr.p + n, 4, cudaMemcpyDeviceToHost, st));
    DG_CUDA(cudaStreamSynchronize(st));
    deg.release(a, st);
    L.nnz = nnz;
    L.col.ensure(a, (size_t)nnz + 1, st);
    L.val.ensure(a, (size_t)nnz + 1, st);
    DG_CUDA(cudaMemsetAsync(L.tmp.p, 0, 4, st));  // word 0: rows with a warp
    if (n) {
        const uint64_t warps = (uint64_t)n;
        QLAUNCH(k_lap_fill, q_grid(warps * 32), QT, st, c.view(), L.ptr.p, L.col.p, L.val.p, L.diag.p, L.big.p,
                L.tmp.p);
    }
    DG_CUDA(cudaMemcpyAsync(&L.nbig, L.tmp.p, 4, cudaMemcpyDeviceToHost, st));
    DG_CUDA(cudaStreamSynchronize(st));
}

// the count of big rows lives in tmp[0] after lap_build
void lap_apply(const Lap& L, const double* x, double* y, cudaStream_t st, const uint32_t* skip = nullptr) {
    if (!L.n) return;
    QLAUNCH(k_spmv_small, q_grid(L.n), QT, st, L.n, L.ptr.p, L.col.p, L.val.p, L.diag.p, x, y, skip);
    if (L.nbig)
        QLAUNCH(k_spmv_big, q_grid((uint64_t)L.nbig * 32), QT, st, L.big.p, L.tmp.p, L.ptr.p, L.col.p, L.val.p,
                L.diag.p, x, y, skip);
}

// ---------------------------------------------------------------------------
// components by minimum-label propagation over a compact CSR (the label of a
// component is its smallest vertex)
// ---------------------------------------------------------------------------
__global__ void k_iota(uint32_t* v, uint32_t n) {
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) v[x] = x;
}

__global__ void k_label_rows(uint32_t n, const uint32_t* __restrict__ ptr, const uint32_t* __restrict__ col,
                             uint32_t* label, uint32_t* changed) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    bool ch = false;
    for (uint32_t x = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n; x += warps) {
        const uint32_t lx = __ldcg(&label[x]);
        uint32_t lo = lx;
        for (uint32_t j = ptr[x] + lane; j < ptr[x + 1]; j += 32) lo = min(lo, __ldcg(&label[col[j]]));
        for (int k = 16; k > 0; k >>= 1) lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, k));
        if (lane == 0 && lo < lx) {
            atomicMin(&label[x], lo);
            atomicMin(&label[lx], lo);  // the vertex the larger label names joins too
            ch = true;
        }
    }
    if (__any_sync(0xffffffffu, ch) && lane == 0) *changed = 1u;
}

__global__ void k_label_flatten(uint32_t* label, uint32_t n, uint32_t* changed) {
    bool ch = false;
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        const uint32_t l = __ldcg(&label[x]);
        const uint32_t ll = __ldcg(&label[l]);
        if (ll < l) ch |= atomicMin(&label[x], ll) > ll;
    }
    if (__any_sync(0xffffffffu, ch) && (threadIdx.x & 31) == 0) *changed = 1u;
}

__global__ void k_count_roots(const uint32_t* __restrict__ label, uint32_t n, uint32_t* cnt) {
    uint32_t c = 0;
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) c += label[x] == x;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, c);
}

// number of connected components of the graph whose Laplacian is L
uint32_t lap_components(const Lap& L, DevAlloc& a, cudaStream_t st) {
    const uint32_t n = L.n;
    if (!n) return 0;
    DBuf<uint32_t> label, flag;
    label.ensure(a, n, st);
    flag.ensure(a, 2, st);
    QLAUNCH(k_iota, q_grid(n), QT, st, label.p, n);
    for (int round = 0;; ++round) {
        if (round == 4096) {
            label.release(a, st);
            flag.release(a, st);
            throw Error(DG_E_TIMEOUT, "component labels did not settle");
        }
        DG_CUDA(cudaMemsetAsync(flag.p, 0, 4, st));
        QLAUNCH(k_label_rows, q_grid((uint64_t)n * 32), QT, st, n, L.ptr.p, L.col.p, label.p, flag.p);
        QLAUNCH(k_label_flatten, q_grid(n), QT, st, label.p, n, flag.p);
        uint32_t ch = 0;
        DG_CUDA(cudaMemcpyAsync(&ch, flag.p, 4, cudaMemcpyDeviceToHost, st));
        DG_CUDA(cudaStreamSynchronize(st));
        if (!ch) break;
    }
    DG_CUDA(cudaMemsetAsync(flag.p, 0, 4, st));
    QLAUNCH(k_count_roots, q_grid(n), QT, st, label.p, n, flag.p);
    uint32_t nc = 0;
    DG_CUDA(cudaMemcpyAsync(&nc, flag.p, 4, cudaMemcpyDeviceToHost, st));
    DG_CUDA(cudaStreamSynchronize(st));
    label.release(a, st);
    flag.release(a, st);
    return nc;
}

// ---------------------------------------------------------------------------
// maximum-weight spanning forest of H (Boruvka)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long pair_key(uint32_t x, uint32_t y) {
    return ((unsigned long long)min(x, y) << 32) | max(x, y);
}

__global__ void k_bv_reset(uint32_t n, unsigned long long* bw, unsigned long long* bid) {
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        bw[x] = 0ull;
        bid[x] = ~0ull;
    }
}

// pass 1: the heaviest edge leaving each component (weights are positive:
// their bits order like the values); pass 2: among those, the smallest pair
template <int PASS>
__global__ void k_bv_best(uint32_t n, const uint32_t* __restrict__ ptr, const uint32_t* __restrict__ col,
                          const double* __restrict__ val, const uint32_t* __restrict__ comp, unsigned long long* bw,
                          unsigned long long* bid) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t x = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n; x += warps) {
        const uint32_t cx = comp[x];
        unsigned long long best = PASS == 1 ? 0ull : ~0ull;
        const unsigned long long want = PASS == 2 ? __ldcg(&bw[cx]) : 0ull;
        for (uint32_t j = ptr[x] + lane; j < ptr[x + 1]; j += 32) {
            const uint32_t y = col[j];
            if (comp[y] == cx) continue;
            const unsigned long long wb = (unsigned long long)__double_as_longlong(val[j]);
            if (PASS == 1) {
                best = max(best, wb);
            } else if (wb == want) {
                best = min(best, pair_key(x, y));
            }
        }
        for (int k = 16; k > 0; k >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, best, k);
            best = PASS == 1 ? max(best, o) : min(best, o);
        }
        if (lane == 0) {
            if (PASS == 1 && best) atomicMax(&bw[cx], best);
            if (PASS == 2 && best != ~0ull) atomicMin(&bid[cx], best);
        }
    }
}

// each root component hooks onto the component across its best edge
__global__ void k_bv_hook(uint32_t n, const uint32_t* __restrict__ comp, const unsigned long long* __restrict__ bid,
                          uint32_t* __restrict__ hook) {
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        if (comp[c] != c || bid[c] == ~0ull) {
            hook[c] = c;
            continue;
        }
        const uint32_t u = (uint32_t)(bid[c] >> 32), v = (uint32_t)bid[c];
        hook[c] = comp[u] == c ? comp[v] : comp[u];
    }
}

// a pair that chose the same edge keeps the smaller component as root; every
// component that hooks adds its edge to the forest
__global__ void k_bv_commit(uint32_t n, const uint32_t* __restrict__ comp, const uint32_t* __restrict__ hook,
                            const unsigned long long* __restrict__ bid, uint32_t* __restrict__ lab,
                            unsigned long long* __restrict__ forest, uint32_t* nf) {
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        if (comp[c] != c) {
            lab[c] = c;  // unused
            continue;
        }
        const uint32_t h = hook[c];
        const bool root = h == c || (hook[h] == c && c < h);
        lab[c] = root ? c : h;
        if (!root) forest[atomicAdd(nf, 1u)] = bid[c];
    }
}

__global__ void k_jump(uint32_t* lab, uint32_t n, uint32_t* changed) {
    bool ch = false;
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        const uint32_t l = lab[x];
        const uint32_t ll = __ldcg(&lab[l]);
        if (ll != l) {
            lab[x] = ll;
            ch = true;
        }
    }
    if (__any_sync(0xffffffffu, ch) && (threadIdx.x & 31) == 0) *changed = 1u;
}

__global__ void k_bv_relabel(uint32_t n, uint32_t* comp, const uint32_t* __restrict__ lab) {
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x)
        comp[x] = lab[comp[x]];
}

// ---------------------------------------------------------------------------
// Euler tours of the forest
// ---------------------------------------------------------------------------
__global__ void k_half_edges(const unsigned long long* __restrict__ forest, uint32_t nf,
                             unsigned long long* __restrict__ keys, uint32_t* __restrict__ vals) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += gridDim.x * blockDim.x) {
        const unsigned long long k = forest[i];
        const uint32_t u = (uint32_t)(k >> 32), v = (uint32_t)k;
        keys[2 * i] = ((unsigned long long)u << 32) | v;
        keys[2 * i + 1] = ((unsigned long long)v << 32) | u;
        vals[2 * i] = 2 * i;
        vals[2 * i + 1] = 2 * i + 1;
    }
}

__global__ void k_tour_deg(const unsigned long long* __restrict__ hk, uint32_t nh, uint32_t* deg) {
    for (uint32_t h = blockIdx.x * blockDim.x + threadIdx.x; h < nh; h += gridDim.x * blockDim.x)
        atomicAdd(&deg[(uint32_t)(hk[h] >> 32)], 1u);
}

// weight of every half-edge (from H's compact rows) and its twin's index
__global__ void k_tour_twin(const unsigned long long* __restrict__ hk, uint32_t nh,
                            const uint32_t* __restrict__ tstart, const uint32_t* __restrict__ hptr,
                            const uint32_t* __restrict__ hcol, const double* __restrict__ hval,
                            uint32_t* __restrict__ twin, double* __restrict__ hw, uint32_t* err) {
    for (uint32_t h = blockIdx.x * blockDim.x + threadIdx.x; h < nh; h += gridDim.x * blockDim.x) {
        const uint32_t x = (uint32_t)(hk[h] >> 32), y = (uint32_t)hk[h];
        const unsigned long long want = ((unsigned long long)y << 32) | x;
        uint32_t lo = tstart[y], hi = tstart[y + 1];
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (hk[mid] < want) lo = mid + 1;
            else hi = mid;
        }
        if (lo >= tstart[y + 1] || hk[lo] != want) atomicOr(err, 1u);
        twin[h] = lo;
        uint32_t a = hptr[x], b = hptr[x + 1];
        while (a < b) {
            const uint32_t mid = (a + b) >> 1;
            if (hcol[mid] < y) a = mid + 1;
            else b = mid;
        }
        if (a >= hptr[x + 1] || hcol[a] != y) atomicOr(err, 2u);
        hw[h] = a < hptr[x + 1] ? hval[a] : 1.0;
    }
}

// root of every vertex's tree: its smallest vertex
__global__ void k_tree_min(uint32_t n, const uint32_t* __restrict__ comp, uint32_t* __restrict__ mn,
                           uint32_t* __restrict__ size) {
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        atomicMin(&mn[comp[x]], x);
        atomicAdd(&size[comp[x]], 1u);
    }
}

__global__ void k_tree_root(uint32_t n, const uint32_t* __restrict__ comp, const uint32_t* __restrict__ mn,
                            const uint32_t* __restrict__ size, uint32_t* __restrict__ root,
                            uint32_t* __restrict__ tlen, uint32_t* __restrict__ tsz) {
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        const uint32_t c = comp[x];
        root[x] = mn[c];
        tlen[x] = mn[c] == x ? 2u * (size[c] - 1u) : 0u;  // the tour of x's tree starts at x
        tsz[x] = mn[c] == x ? size[c] : 0u;
    }
}

// successor on the tour: after (x -> y) comes y's next neighbour after x
// (circularly); the edge that would return to the root's first neighbour ends
// the tour
__global__ void k_tour_succ(const unsigned long long* __restrict__ hk, uint32_t nh,
                            const uint32_t* __restrict__ tstart, const uint32_t* __restrict__ twin,
                            const uint32_t* __restrict__ root, uint32_t* __restrict__ nxt, uint32_t* __restrict__ rank) {
    for (uint32_t h = blockIdx.x * blockDim.x + threadIdx.x; h < nh; h += gridDim.x * blockDim.x) {
        const uint32_t y = (uint32_t)hk[h];
        const uint32_t s = tstart[y], d = tstart[y + 1] - s;
        const uint32_t k = (twin[h] - s + 1) % d;
        const bool end = k == 0 && root[y] == y;
        nxt[h] = end ? NONE : s + k;
        rank[h] = end ? 0u : 1u;
    }
}

// one round of list ranking: rank += rank of the successor, successor skips ahead
__global__ void k_rank_jump(uint32_t nh, const uint32_t* __restrict__ nxt, const uint32_t* __restrict__ rank,
                            uint32_t* __restrict__ nxt2, uint32_t* __restrict__ rank2) {
    for (uint32_t h = blockIdx.x * blockDim.x + threadIdx.x; h < nh; h += gridDim.x * blockDim.x) {
        const uint32_t s = nxt[h];
        if (s == NONE) {
            nxt2[h] = NONE;
            rank2[h] = rank[h];
        } else {
            nxt2[h] = nxt[s];
            rank2[h] = rank[h] + rank[s];
        }
    }
}

// position on the tour, then entry and exit positions and the parent-edge weight of every non-root vertex
__global__ void k_tour_pos(const unsigned long long* __restrict__ hk, uint32_t nh, const uint32_t* __restrict__ rank,
                           const uint32_t* __restrict__ root, const uint32_t* __restrict__ toff,
                           const uint32_t* __restrict__ tlen, uint32_t* __restrict__ pos) {
    for (uint32_t h = blockIdx.x * blockDim.x + threadIdx.x; h < nh; h += gridDim.x * blockDim.x) {
        const uint32_t x = (uint32_t)(hk[h] >> 32);
        const uint32_t r = root[x];
        pos[h] = toff[r] + (tlen[r] - 1u - rank[h]);
    }
}

__global__ void k_tour_inout(const unsigned long long* __restrict__ hk, uint32_t nh, const uint32_t* __restrict__ pos,
                             const uint32_t* __restrict__ twin, const double* __restrict__ hw,
                             uint32_t* __restrict__ tin, uint32_t* __restrict__ tout, double* __restrict__ tw,
                             uint32_t* cnt) {
    for (uint32_t h = blockIdx.x * blockDim.x + threadIdx.x; h < nh; h += gridDim.x * blockDim.x) {
        const uint32_t t = twin[h];
        if (pos[h] < pos[t]) {  // the tour goes down (x -> y) before it comes back up
            const uint32_t y = (uint32_t)hk[h];
            tin[y] = pos[h];
            tout[y] = pos[t];
            tw[y] = hw[h];
            atomicAdd(cnt, 1u);
        }
    }
}

__global__ void k_fill_u32(uint32_t* p, uint32_t n, uint32_t v) {
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) p[x] = v;
}

// ---------------------------------------------------------------------------
// exclusive prefix sums of 128-bit integers (exact, so any grouping gives the
// same result)
// ---------------------------------------------------------------------------
constexpr int IS_ITEMS = 8;
constexpr int IS_TILE = QT * IS_ITEMS;

// exclusive prefix over the block by warp shuffles, then the warp totals;
// total (nullable) = the block's sum
__device__ i128 block_i128_scan(i128 v, i128* sh, i128* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    i128 incl = v;
    for (int d = 1; d < 32; d <<= 1) {
        const i128 t = shfl_up_i128(incl, d);
        if (lane >= d) incl += t;
    }
    if (lane == 31) sh[wid] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        i128 run = 0;
        for (int w = 0; w < nw; ++w) {
            const i128 t = sh[w];
            sh[w] = run;
            run += t;
        }
        sh[nw] = run;
    }
    __syncthreads();
    const i128 excl = sh[wid] + incl - v;
    if (total) *total = sh[nw];
    __syncthreads();
    return excl;
}

// Tile totals.  The sum of a tile is exact whatever the order, so the loads
// are coalesced (item i * QT + thread of the tile) rather than in runs.
__global__ void __launch_bounds__(QT) k_is_tile_sums(const i128* __restrict__ in, uint32_t n, i128* __restrict__ tsum,
                                                     const uint32_t* skip) {
    __shared__ i128 sh[QT / 32 + 1];
    if (skip && *skip) return;
    const uint64_t base = (uint64_t)blockIdx.x * IS_TILE + threadIdx.x;
    i128 s = 0;
#pragma unroll
    for (int i = 0; i < IS_ITEMS; ++i)
        if (base + (uint64_t)i * QT < n) s += in[base + (uint64_t)i * QT];
    i128 tot;
    block_i128_scan(s, sh, &tot);
    if (threadIdx.x == 0) tsum[blockIdx.x] = tot;
}

// exclusive scan of the tile sums by one block (each thread a fixed run of tiles)
__global__ void __launch_bounds__(1024) k_is_scan_tiles(i128* tsum, uint32_t tiles, const uint32_t* skip) {
    __shared__ i128 sh[1024 / 32 + 1];
    if (skip && *skip) return;
    const uint32_t per = (tiles + blockDim.x - 1) / blockDim.x;
    const uint32_t lo = threadIdx.x * per, hi = min(tiles, lo + per);
    i128 s = 0;
    for (uint32_t t = lo; t < hi; ++t) s += tsum[t];
    i128 run = block_i128_scan(s, sh, nullptr);
    for (uint32_t t = lo; t < hi; ++t) {
        const i128 v = tsum[t];
        tsum[t] = run;
        run += v;
    }
}

// slot of tile item p in the staging array: one pad slot per IS_ITEMS items, so
// a thread's run of IS_ITEMS items and the coalesced pattern are both free of
// shared-memory bank conflicts
__device__ __forceinline__ uint32_t is_slot(uint32_t p) { return p + p / IS_ITEMS; }

// Exclusive scan of one tile with the tile's prefix: coalesced loads staged in
// shared memory, each thread scans a run of IS_ITEMS consecutive items, and the
// results leave through the same staging array as coalesced stores.
__global__ void __launch_bounds__(QT) k_is_tile_scan(const i128* __restrict__ in, uint32_t n,
                                                     const i128* __restrict__ tpre, i128* __restrict__ out,
                                                     const uint32_t* skip) {
    __shared__ i128 sh[QT / 32 + 1];
    __shared__ i128 stage[IS_TILE + IS_TILE / IS_ITEMS];
    if (skip && *skip) return;
    const uint64_t tbase = (uint64_t)blockIdx.x * IS_TILE;
#pragma unroll
    for (int i = 0; i < IS_ITEMS; ++i) {
        const uint32_t p = (uint32_t)i * QT + threadIdx.x;
        stage[is_slot(p)] = tbase + p < n ? in[tbase + p] : (i128)0;
    }
    __syncthreads();
    i128 loc[IS_ITEMS];
    i128 s = 0;
#pragma unroll
    for (int i = 0; i < IS_ITEMS; ++i) {
        loc[i] = stage[is_slot(threadIdx.x * IS_ITEMS + i)];
        s += loc[i];
    }
    i128 run = tpre[blockIdx.x] + block_i128_scan(s, sh, nullptr);  // (its barriers order the reads above)
#pragma unroll
    for (int i = 0; i < IS_ITEMS; ++i) {
        stage[is_slot(threadIdx.x * IS_ITEMS + i)] = run;
        run += loc[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < IS_ITEMS; ++i) {
        const uint32_t p = (uint32_t)i * QT + threadIdx.x;
        if (tbase + p < n) out[tbase + p] = stage[is_slot(p)];
    }
}

void i128_scan_exclusive(const i128* in, i128* out, uint32_t n, i128* tsum, cudaStream_t st, const uint32_t* skip) {
    if (!n) return;
    const uint32_t tiles = (n + IS_TILE - 1) / IS_TILE;
    QLAUNCH(k_is_tile_sums, tiles, QT, st, in, n, tsum, skip);
    QLAUNCH(k_is_scan_tiles, 1, 1024, st, tsum, tiles, skip);
    QLAUNCH(k_is_tile_scan, tiles, QT, st, in, n, tsum, out, skip);
}

// ---------------------------------------------------------------------------
// the forest solve z = L_F^+ r (z = 0 at every root)
// ---------------------------------------------------------------------------
struct Forest {
    uint32_t n = 0, nf = 0, nh = 0, ntrees = 0;
    int nbits = 1;  // a tour prefix sum has at most 2^nbits terms
    DBuf<uint32_t> tin, tout, root, toff, tlen, tsz;  // tlen, tsz: tour length and size at each root
    DBuf<uint32_t> ex;                                // largest exponents of the vectors being summed
    DBuf<double> tw, mean, av;
    DBuf<i128> A, P, tsum;
    std::vector<unsigned long long> host_edges;  // filled on request (test hook)
    void release(DevAlloc& a, cudaStream_t st) {
        for (auto* b : {&tin, &tout, &root, &toff, &tlen, &tsz, &ex}) b->release(a, st);
        tw.release(a, st);
        mean.release(a, st);
        av.release(a, st);
        A.release(a, st);
        P.release(a, st);
        tsum.release(a, st);
    }
};

// A[tin_y] = r_y, A[tout_y] = 0 for every non-root y, in fixed point
__global__ void k_fs_scatter(uint32_t n, const uint32_t* __restrict__ tin, const uint32_t* __restrict__ tout,
                             const double* __restrict__ r, const uint32_t* ex, int nbits, i128* __restrict__ A,
                             const uint32_t* skip) {
    if (skip && *skip) return;
    const int s = fixed_scale(ex[0], nbits);
    for (uint32_t y = blockIdx.x * blockDim.x + threadIdx.x; y < n; y += gridDim.x * blockDim.x) {
        const uint32_t i = tin[y];
        if (i == NONE) continue;
        A[i] = to_fixed(r[y], s);
        A[tout[y]] = 0;
    }
}

// current through y's parent edge = subtree sum (exact, rounded once); a_y = I / w
__global__ void k_fs_flow(uint32_t n, const uint32_t* __restrict__ tin, const uint32_t* __restrict__ tout,
                          const double* __restrict__ tw, const i128* __restrict__ P, uint32_t* ex, int nbits,
                          double* __restrict__ av, const uint32_t* skip) {
    if (skip && *skip) return;
    const int s = fixed_scale(ex[0], nbits);
    uint32_t m = 0;
    for (uint32_t y = blockIdx.x * blockDim.x + threadIdx.x; y < n; y += gridDim.x * blockDim.x) {
        const uint32_t i = tin[y];
        if (i == NONE) continue;
        const double I = from_fixed(P[tout[y]] - P[i], s);
        const double a = __ddiv_rn(I, tw[y]);
        av[y] = a;
        m = max(m, biased_exp(a));
    }
    for (int k = 16; k > 0; k >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, k));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(&ex[1], m);
}

// B[tin] = +a, B[tout] = -a in fixed point
__global__ void k_fs_scatter_a(uint32_t n, const uint32_t* __restrict__ tin, const uint32_t* __restrict__ tout,
                               const double* __restrict__ av, const uint32_t* ex, int nbits, i128* __restrict__ B,
                               const uint32_t* skip) {
    if (skip && *skip) return;
    const int s = fixed_scale(ex[1], nbits);
    for (uint32_t y = blockIdx.x * blockDim.x + threadIdx.x; y < n; y += gridDim.x * blockDim.x) {
        const uint32_t i = tin[y];
        if (i == NONE) continue;
        const i128 q = to_fixed(av[y], s);
        B[i] = q;
        B[tout[y]] = -q;
    }
}

// potential: the open edges at y's entry, i.e. the prefix through tin_y minus
// the prefix at the start of y's tour (exact, rounded once).  With part, also
// the block's partial sum of dot_r . z (one per block, fixed slices)
__global__ void __launch_bounds__(QT) k_fs_potential(uint32_t n, const uint32_t* __restrict__ tin,
                                                     const uint32_t* __restrict__ root,
                                                     const uint32_t* __restrict__ toff, const i128* __restrict__ B,
                                                     const i128* __restrict__ Q, const uint32_t* ex, int nbits,
                                                     double* __restrict__ z, const uint32_t* skip,
                                                     const double* __restrict__ dot_r, double* __restrict__ part) {
    __shared__ double sh[QT];
    if (skip && *skip) return;
    const int s = fixed_scale(ex[1], nbits);
    double acc = 0.0;
    for (uint32_t y = blockIdx.x * blockDim.x + threadIdx.x; y < n; y += gridDim.x * blockDim.x) {
        const uint32_t i = tin[y];
        const double zy = i == NONE ? 0.0 : from_fixed(Q[i] + B[i] - Q[toff[root[y]]], s);
        z[y] = zy;
        if (part) acc = fma(dot_r[y], zy, acc);
    }
    if (part) {
        acc = block_sum(acc, sh);
        if (threadIdx.x == 0) part[blockIdx.x] = acc;
    }
}

// z = L_F^+ r; with part, also the partial sums of r . z (q_grid(n) of them)
void forest_solve(Forest& F, const double* r, double* z, cudaStream_t st, const uint32_t* skip = nullptr,
                  double* part = nullptr) {
    const uint32_t n = F.n;
    if (!n) return;
    if (F.nh) {
        QLAUNCH(k_zero_words, 1, 32, st, F.ex.p, 2, skip);
        QLAUNCH(k_max_exp, q_grid(n), QT, st, r, n, F.ex.p, skip);
        QLAUNCH(k_fs_scatter, q_grid(n), QT, st, n, F.tin.p, F.tout.p, r, F.ex.p, F.nbits, F.A.p, skip);
        i128_scan_exclusive(F.A.p, F.P.p, F.nh, F.tsum.p, st, skip);
        QLAUNCH(k_fs_flow, q_grid(n), QT, st, n, F.tin.p, F.tout.p, F.tw.p, F.P.p, F.ex.p, F.nbits, F.av.p, skip);
        QLAUNCH(k_fs_scatter_a, q_grid(n), QT, st, n, F.tin.p, F.tout.p, F.av.p, F.ex.p, F.nbits, F.A.p, skip);
        i128_scan_exclusive(F.A.p, F.P.p, F.nh, F.tsum.p, st, skip);
    }
    QLAUNCH(k_fs_potential, q_grid(n), QT, st, n, F.tin.p, F.root.p, F.toff.p, F.A.p, F.P.p, F.ex.p, F.nbits, z,
            skip, r, part);
}

// mean of v over every tree (at the root): the tour prefix at the tree's end
// minus the prefix at its start covers every vertex but the root (exact sums,
// rounded once)
__global__ void k_tree_mean(uint32_t n, const uint32_t* __restrict__ root, const uint32_t* __restrict__ toff,
                            const uint32_t* __restrict__ tlen, const uint32_t* __restrict__ tsz,
                            const i128* __restrict__ P, const double* __restrict__ v, const uint32_t* ex, int nbits,
                            double* __restrict__ mean, const uint32_t* skip) {
    if (skip && *skip) return;
    const int s = fixed_scale(ex[0], nbits);
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        if (root[x] != x) continue;
        if (tlen[x] == 0) {
            mean[x] = v[x];
            continue;
        }
        const uint32_t o = toff[x];
        mean[x] = from_fixed(P[o + tlen[x]] - P[o] + to_fixed(v[x], s), s) / (double)tsz[x];
    }
}

__global__ void k_tree_sub(uint32_t n, const uint32_t* __restrict__ root, const double* __restrict__ mean,
                           double* __restrict__ v, const uint32_t* skip) {
    if (skip && *skip) return;
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x)
        v[x] -= mean[root[x]];
}

// v -= its mean over every tree of the forest (every component of H): the
// part of v that L_H^+ maps to zero
void forest_center(Forest& F, double* v, cudaStream_t st, const uint32_t* skip = nullptr) {
    const uint32_t n = F.n;
    if (!n) return;
    QLAUNCH(k_zero_words, 1, 32, st, F.ex.p, 2, skip);
    QLAUNCH(k_max_exp, q_grid(n), QT, st, v, n, F.ex.p, skip);
    if (F.nh) {
        QLAUNCH(k_fs_scatter, q_grid(n), QT, st, n, F.tin.p, F.tout.p, v, F.ex.p, F.nbits, F.A.p, skip);
        i128_scan_exclusive(F.A.p, F.P.p, F.nh + 1, F.tsum.p, st, skip);
    }
    QLAUNCH(k_tree_mean, q_grid(n), QT, st, n, F.root.p, F.toff.p, F.tlen.p, F.tsz.p, F.P.p, v, F.ex.p, F.nbits,
            F.mean.p, skip);
    QLAUNCH(k_tree_sub, q_grid(n), QT, st, n, F.root.p, F.mean.p, v, skip);
}

// H's maximum-weight spanning forest and its Euler tours
void forest_build(Forest& F, const Lap& H, DevAlloc& a, cudaStream_t st, bool keep_edges) {
    const uint32_t n = H.n;
    F.n = n;
    DBuf<uint32_t> comp, hook, lab, flag, nfc;
    DBuf<unsigned long long> bw, bid, forest;
    auto rel = [&]() {
        for (auto* b : {&comp, &hook, &lab, &flag, &nfc}) b->release(a, st);
        bw.release(a, st);
        bid.release(a, st);
        forest.release(a, st);
    };
    try {
        comp.ensure(a, (size_t)n + 1, st);
        hook.ensure(a, (size_t)n + 1, st);
        lab.ensure(a, (size_t)n + 1, st);
        flag.ensure(a, 2, st);
        nfc.ensure(a, 2, st);
        bw.ensure(a, (size_t)n + 1, st);
        bid.ensure(a, (size_t)n + 1, st);
        forest.ensure(a, (size_t)n + 1, st);
        DG_CUDA(cudaMemsetAsync(nfc.p, 0, 4, st));
        if (n) QLAUNCH(k_iota, q_grid(n), QT, st, comp.p, n);
        uint32_t nf = 0;
        for (int round = 0; n; ++round) {
            if (round == 64) throw Error(DG_E_TIMEOUT, "spanning forest rounds did not end");
            QLAUNCH(k_bv_reset, q_grid(n), QT, st, n, bw.p, bid.p);
            QLAUNCH(k_bv_best<1>, q_grid((uint64_t)n * 32), QT, st, n, H.ptr.p, H.col.p, H.val.p, comp.p, bw.p,
                    bid.p);
            QLAUNCH(k_bv_best<2>, q_grid((uint64_t)n * 32), QT, st, n, H.ptr.p, H.col.p, H.val.p, comp.p, bw.p,
                    bid.p);
            QLAUNCH(k_bv_hook, q_grid(n), QT, st, n, comp.p, bid.p, hook.p);
            QLAUNCH(k_bv_commit, q_grid(n), QT, st, n, comp.p, hook.p, bid.p, lab.p, forest.p, nfc.p);
            for (int j = 0;; ++j) {
                if (j == 64) throw Error(DG_E_TIMEOUT, "forest labels did not settle");
                DG_CUDA(cudaMemsetAsync(flag.p, 0, 4, st));
                QLAUNCH(k_jump, q_grid(n), QT, st, lab.p, n, flag.p);
                uint32_t ch = 0;
                DG_CUDA(cudaMemcpyAsync(&ch, flag.p, 4, cudaMemcpyDeviceToHost, st));
                DG_CUDA(cudaStreamSynchronize(st));
                if (!ch) break;
            }
            QLAUNCH(k_bv_relabel, q_grid(n), QT, st, n, comp.p, lab.p);
            uint32_t nf2 = 0;
            DG_CUDA(cudaMemcpyAsync(&nf2, nfc.p, 4, cudaMemcpyDeviceToHost, st));
            DG_CUDA(cudaStreamSynchronize(st));
            if (nf2 == nf) break;
            nf = nf2;
        }
        F.nf = nf;
        F.nh = 2 * nf;
        F.ntrees = n - nf;
        if (keep_edges) {
            F.host_edges.resize(nf);
            if (nf) DG_CUDA(cudaMemcpy(F.host_edges.data(), forest.p, 8ull * nf, cudaMemcpyDeviceToHost));
            std::sort(F.host_edges.begin(), F.host_edges.end());
        }
        // half-edges sorted by (x, y)
        const uint32_t nh = F.nh;
        DBuf<unsigned long long> hk, hk_alt;
        DBuf<uint32_t> hv, hv_alt, hist, tstart, tdeg, twin, nxt, rank, nxt2, rank2, pos, mn, size, stmp, err;
        DBuf<double> hw;
        auto rel2 = [&]() {
            hk.release(a, st);
            hk_alt.release(a, st);
            for (auto* b : {&hv, &hv_alt, &hist, &tstart, &tdeg, &twin, &nxt, &rank, &nxt2, &rank2, &pos, &mn, &size,
                            &stmp, &err})
                b->release(a, st);
            hw.release(a, st);
        };
        try {
            F.tin.ensure(a, (size_t)n + 1, st);
            F.tout.ensure(a, (size_t)n + 1, st);
            F.root.ensure(a, (size_t)n + 1, st);
            F.toff.ensure(a, (size_t)n + 1, st);
            F.tw.ensure(a, (size_t)n + 1, st);
            F.A.ensure(a, (size_t)nh + 1, st);
            F.P.ensure(a, (size_t)nh + 1, st);
            DG_CUDA(cudaMemsetAsync(F.A.p + nh, 0, sizeof(i128), st));  // A[nh] = 0: P[nh] is the total
            F.av.ensure(a, (size_t)n + 1, st);
            F.ex.ensure(a, 4, st);
            F.nbits = std::max(1, bit_length((uint64_t)nh + 1));
            F.tsum.ensure(a, ((size_t)nh + 1) / IS_TILE + 2, st);
            err.ensure(a, 2, st);
            mn.ensure(a, (size_t)n + 1, st);
            size.ensure(a, (size_t)n + 1, st);
            F.tlen.ensure(a, (size_t)n + 1, st);
            F.tsz.ensure(a, (size_t)n + 1, st);
            F.mean.ensure(a, (size_t)n + 1, st);
            tstart.ensure(a, (size_t)n + 2, st);
            tdeg.ensure(a, (size_t)n + 1, st);
            stmp.ensure(a, scan_tmp_words(n + 1), st);
            DG_CUDA(cudaMemsetAsync(err.p, 0, 8, st));
            // roots (smallest vertex of each tree), tree sizes, tour offsets
            if (n) {
                QLAUNCH(k_fill_u32, q_grid(n), QT, st, mn.p, n, NONE);
                DG_CUDA(cudaMemsetAsync(size.p, 0, 4ull * n, st));
                QLAUNCH(k_tree_min, q_grid(n), QT, st, n, comp.p, mn.p, size.p);
                QLAUNCH(k_tree_root, q_grid(n), QT, st, n, comp.p, mn.p, size.p, F.root.p, F.tlen.p, F.tsz.p);
                ScanJob j;
                j.in[0] = F.tlen.p;
                j.out[0] = F.toff.p;
                j.k = 1;
                scan_exclusive(j, nullptr, n, stmp.p, st);
                QLAUNCH(k_fill_u32, q_grid(n), QT, st, F.tin.p, n, NONE);
                QLAUNCH(k_fill_u32, q_grid(n), QT, st, F.tout.p, n, NONE);
            }
            if (nh) {
                hk.ensure(a, nh, st);
                hk_alt.ensure(a, nh, st);
                hv.ensure(a, nh, st);
                hv_alt.ensure(a, nh, st);
                hist.ensure(a, sort_hist_words(nh), st);
                QLAUNCH(k_half_edges, q_grid(nf), QT, st, forest.p, nf, hk.p, hv.p);
                SortBufs sb{reinterpret_cast<uint64_t*>(hk.p), hv.p, reinterpret_cast<uint64_t*>(hk_alt.p), hv_alt.p,
                            hist.p, nullptr, err.p};
                DG_CUDA(cudaMemcpyAsync(err.p + 1, &nh, 4, cudaMemcpyHostToDevice, st));
                const int bits = 64;  // keys are (x << 32) | y
                DG_CUDA(cudaMemsetAsync(hist.p, 0, 4ull * sort_clear_words(nh, bits), st));
                const bool alt = radix_sort_pairs(sb, err.p + 1, nh, bits, st, nullptr, true);
                const unsigned long long* K = alt ? hk_alt.p : hk.p;
                DG_CUDA(cudaMemsetAsync(tdeg.p, 0, 4ull * n, st));
                QLAUNCH(k_tour_deg, q_grid(nh), QT, st, K, nh, tdeg.p);
                ScanJob j;
                j.in[0] = tdeg.p;
                j.out[0] = tstart.p;
                j.total[0] = tstart.p + n;
                j.k = 1;
                scan_exclusive(j, nullptr, n, stmp.p, st);
                twin.ensure(a, nh, st);
                hw.ensure(a, nh, st);
                QLAUNCH(k_tour_twin, q_grid(nh), QT, st, K, nh, tstart.p, H.ptr.p, H.col.p, H.val.p, twin.p, hw.p,
                        err.p);
                nxt.ensure(a, nh, st);
                rank.ensure(a, nh, st);
                nxt2.ensure(a, nh, st);
                rank2.ensure(a, nh, st);
                QLAUNCH(k_tour_succ, q_grid(nh), QT, st, K, nh, tstart.p, twin.p, F.root.p, nxt.p, rank.p);
                const int rounds = bit_length((uint64_t)nh) + 1;
                uint32_t *pn = nxt.p, *pr = rank.p, *qn = nxt2.p, *qr = rank2.p;
                for (int r = 0; r < rounds; ++r) {
                    QLAUNCH(k_rank_jump, q_grid(nh), QT, st, nh, pn, pr, qn, qr);
                    std::swap(pn, qn);
                    std::swap(pr, qr);
                }
                pos.ensure(a, nh, st);
                QLAUNCH(k_tour_pos, q_grid(nh), QT, st, K, nh, pr, F.root.p, F.toff.p, F.tlen.p, pos.p);
                DG_CUDA(cudaMemsetAsync(err.p + 1, 0, 4, st));
                QLAUNCH(k_tour_inout, q_grid(nh), QT, st, K, nh, pos.p, twin.p, hw.p, F.tin.p, F.tout.p, F.tw.p,
                        err.p + 1);
                uint32_t he[2] = {0, 0};
                DG_CUDA(cudaMemcpyAsync(he, err.p, 8, cudaMemcpyDeviceToHost, st));
                DG_CUDA(cudaStreamSynchronize(st));
                if ((he[0] & ~PRIM_ERR_SPIN) || he[1] != nf)
                    throw Error(DG_E_CUDA, "spanning forest tour inconsistent");
                if (he[0] & PRIM_ERR_SPIN) throw Error(DG_E_TIMEOUT, "sort look-back wait gave up");
            }
            DG_CUDA(cudaStreamSynchronize(st));
        } catch (...) {
            cudaStreamSynchronize(st);
            rel2();
            throw;
        }
        rel2();
    } catch (...) {
        cudaStreamSynchronize(st);
        rel();
        throw;
    }
    rel();
}

// ---------------------------------------------------------------------------
// deterministic dot products and the CG step kernels
// ---------------------------------------------------------------------------
struct CgScal {
    double rz, alpha, beta, rr, bb, tol2;
    double pad[2];
    uint32_t done, iters, max_iter, fail;
};

__global__ void __launch_bounds__(QT) k_dot_part(const double* __restrict__ a, const double* __restrict__ b, uint32_t n,
                                                 double* __restrict__ part, const uint32_t* skip) {
    __shared__ double sh[QT];
    if (skip && *skip) return;
    double s = 0.0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        s = fma(a[i], b[i], s);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__device__ double sum_parts(const double* part, int np, double* sh) {
    double s = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) s = __dadd_rn(s, part[i]);
    return block_sum(s, sh);
}

// CG start: x = 0, r = b, p = 0, partial sums of b.b
__global__ void __launch_bounds__(QT) k_cg_start(const double* __restrict__ b, double* __restrict__ x,
                                                 double* __restrict__ r, double* __restrict__ p, uint32_t n,
                                                 double* __restrict__ part) {
    __shared__ double sh[QT];
    double s = 0.0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double v = b[i];
        x[i] = 0.0;
        r[i] = v;
        p[i] = 0.0;
        s = fma(v, v, s);
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(QT) k_cg_start_fin(CgScal* s, const double* part, int np, double tol,
                                                     uint32_t max_iter, double* hist) {
    __shared__ double sh[QT];
    const double bb = sum_parts(part, np, sh);
    if (threadIdx.x == 0) {
        s->bb = bb;
        s->rr = bb;
        s->tol2 = tol * tol * bb;
        s->iters = 0;
        s->max_iter = max_iter;
        s->done = (bb == 0.0 || max_iter == 0) ? 1u : 0u;
        s->fail = 0;
        s->beta = 0.0;
        s->rz = 0.0;
        if (hist) hist[0] = bb == 0.0 ? 0.0 : 1.0;
    }
}

// rz = (r, z); beta = rz / rz_old (0 at the start)
__global__ void __launch_bounds__(QT) k_cg_beta(CgScal* s, const double* part, int np) {
    __shared__ double sh[QT];
    if (s->done) return;
    const double rz = sum_parts(part, np, sh);
    if (threadIdx.x == 0) {
        s->beta = s->iters == 0 ? 0.0 : rz / s->rz;
        s->rz = rz;
        // (r, M^-1 r) > 0 for every r the preconditioner does not map to zero:
        // nothing is left to reduce at this precision
        if (!(rz > 0.0)) s->done = 1;
    }
}

__global__ void k_cg_p(const double* __restrict__ z, double* __restrict__ p, uint32_t n, const CgScal* s) {
    if (s->done) return;
    const double beta = s->beta;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        p[i] = fma(beta, p[i], z[i]);
}

// alpha = rz / (p, q)
__global__ void __launch_bounds__(QT) k_cg_alpha(CgScal* s, const double* part, int np) {
    __shared__ double sh[QT];
    if (s->done) return;
    const double pq = sum_parts(part, np, sh);
    if (threadIdx.x == 0) {
        if (!(pq > 0.0)) {  // breakdown: nothing left to reduce (or a non-definite operator)
            s->done = 1;
            s->fail = 1;
        } else {
            s->alpha = s->rz / pq;
        }
    }
}

__global__ void __launch_bounds__(QT) k_cg_xr(double* __restrict__ x, double* __restrict__ r,
                                              const double* __restrict__ p, const double* __restrict__ q, uint32_t n,
                                              const CgScal* s, double* __restrict__ part) {
    __shared__ double sh[QT];
    if (s->done) return;
    const double al = s->alpha;
    double acc = 0.0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        x[i] = fma(al, p[i], x[i]);
        const double ri = fma(-al, q[i], r[i]);
        r[i] = ri;
        acc = fma(ri, ri, acc);
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(QT) k_cg_check(CgScal* s, const double* part, int np, double* hist) {
    __shared__ double sh[QT];
    if (s->done) return;
    const double rr = sum_parts(part, np, sh);
    if (threadIdx.x == 0) {
        s->rr = rr;
        const uint32_t it = ++s->iters;
        if (hist) hist[it] = sqrt(rr / s->bb);
        if (rr < s->tol2 || it >= s->max_iter) s->done = 1;
    }
}

__global__ void k_jacobi(const double* __restrict__ r, const double* __restrict__ d, double* __restrict__ z, uint32_t n,
                         const uint32_t* skip) {
    if (skip && *skip) return;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        z[i] = d[i] > 0.0 ? r[i] / d[i] : r[i];
}

__global__ void k_copy(const double* __restrict__ a, double* __restrict__ b, uint32_t n, const uint32_t* skip) {
    if (skip && *skip) return;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b[i] = a[i];
}

// partial sums of (b - t)^2 and b^2
__global__ void __launch_bounds__(QT) k_resid_part(const double* __restrict__ b, const double* __restrict__ t,
                                                   uint32_t n, double* __restrict__ pn, double* __restrict__ pd) {
    __shared__ double sh[QT];
    double num = 0.0, den = 0.0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double d = b[i] - t[i];
        num = fma(d, d, num);
        den = fma(b[i], b[i], den);
    }
    num = block_sum(num, sh);
    den = block_sum(den, sh);
    if (threadIdx.x == 0) {
        pn[blockIdx.x] = num;
        pd[blockIdx.x] = den;
    }
}

__global__ void __launch_bounds__(QT) k_resid_fin(const double* pn, const double* pd, int np, double* out) {
    __shared__ double sh[QT];
    const double num = sum_parts(pn, np, sh);
    const double den = sum_parts(pd, np, sh);
    if (threadIdx.x == 0) *out = den > 0.0 ? sqrt(num / den) : 0.0;
}

// ---------------------------------------------------------------------------
// CG driver: A x = b with a preconditioner (none, Jacobi, forest, or an inner
// CG on L_H); the host launches the steps and reads the stop flag
// ---------------------------------------------------------------------------
struct Vecs {
    DBuf<double> r, z, p, q;
    void ensure(DevAlloc& a, uint32_t n, cudaStream_t st) {
        r.ensure(a, (size_t)n + 1, st);
        z.ensure(a, (size_t)n + 1, st);
        p.ensure(a, (size_t)n + 1, st);
        q.ensure(a, (size_t)n + 1, st);
    }
    void release(DevAlloc& a, cudaStream_t st) {
        r.release(a, st);
        z.release(a, st);
        p.release(a, st);
        q.release(a, st);
    }
};

enum class Pre { None, Jacobi, Forest, Inner };

struct Solver {
    DevAlloc* a = nullptr;
    cudaStream_t st = nullptr;
    const Lap* G = nullptr;
    const Lap* H = nullptr;
    Forest* F = nullptr;
    Vecs outer, inner;
    DBuf<double> part, part2, rin;
    DBuf<CgScal> sc;  // [0] outer, [1] inner
    CgScal* host_sc = nullptr;  // pinned
    double inner_tol = 1e-12;
    uint32_t inner_max = 1000;
    int np = 0;
    uint32_t hint = 8;
    int64_t inner_total = 0;
    int32_t inner_most = 0;
    int32_t inner_unconv = 0;

    void init(DevAlloc& al, cudaStream_t s, uint32_t n) {
        a = &al;
        st = s;
        np = dot_blocks();
        // the forest solve leaves one partial (r, z) per block of its grid
        part.ensure(al, (size_t)std::max(np, q_grid(n)) + 1, st);
        part2.ensure(al, (size_t)np + 1, st);
        sc.ensure(al, 2, st);
        DG_CUDA(cudaMallocHost(&host_sc, 2 * sizeof(CgScal)));
        outer.ensure(al, n, st);
    }
    void release() {
        outer.release(*a, st);
        inner.release(*a, st);
        part.release(*a, st);
        part2.release(*a, st);
        rin.release(*a, st);
        sc.release(*a, st);
        if (host_sc) cudaFreeHost(host_sc);
        host_sc = nullptr;
    }
    void read_scal(int k) {
        DG_CUDA(cudaMemcpyAsync(host_sc + k, sc.p + k, sizeof(CgScal), cudaMemcpyDeviceToHost, st));
        DG_CUDA(cudaStreamSynchronize(st));
    }

    // z = M^-1 r and the partial sums of (r, z) into part; returns how many
    int precond(Pre pre, const double* r, double* z, uint32_t n, const uint32_t* skip) {
        switch (pre) {
            case Pre::None: QLAUNCH(k_copy, q_grid(n), QT, st, r, z, n, skip); break;
            case Pre::Jacobi: QLAUNCH(k_jacobi, q_grid(n), QT, st, r, G->diag.p, z, n, skip); break;
            case Pre::Forest:
                forest_solve(*F, r, z, st, skip, part.p);  // (r, z) in the same pass
                return q_grid(n);
            case Pre::Inner:
                // the inner solve runs only when the outer iteration goes on
                // (the caller checked the flag on the host)
                hsolve(r, z, n);
                break;
        }
        QLAUNCH(k_dot_part, np, QT, st, r, z, n, part.p, skip);
        return np;
    }

    // z = L_H^+ r: the part of r in the range of L_H (r minus its mean over
    // every component of H) solved by CG on L_H with the forest as
    // preconditioner, and the result's own part in that range
    void hsolve(const double* r, double* z, uint32_t n) {
        rin.ensure(*a, (size_t)n + 1, st);
        QLAUNCH(k_copy, q_grid(n), QT, st, r, rin.p, n, nullptr);
        forest_center(*F, rin.p, st);
        const uint32_t it = cg(*H, Pre::Forest, rin.p, z, n, inner_tol, inner_max, 1, nullptr);
        forest_center(*F, z, st);
        inner_total += it;
        inner_most = std::max<int32_t>(inner_most, (int32_t)it);
        if (!(host_sc[1].rr < host_sc[1].tol2) && host_sc[1].bb > 0.0) ++inner_unconv;
    }

    // CG on A (= *Lp) with preconditioner pre; scalars slot k; returns iterations
    uint32_t cg(const Lap& A, Pre pre, const double* b, double* x, uint32_t n, double tol, uint32_t max_iter, int k,
                double* hist_dev) {
        Vecs& v = k == 0 ? outer : inner;
        if (k == 1) v.ensure(*a, n, st);
        CgScal* s = sc.p + k;
        const uint32_t* done = &s->done;
        QLAUNCH(k_cg_start, np, QT, st, b, x, v.r.p, v.p.p, n, part.p);
        QLAUNCH(k_cg_start_fin, 1, QT, st, s, part.p, np, tol, max_iter, hist_dev);
        // z = M^-1 r, (r, z), p = z + beta p; false when the outer solve already stopped
        auto zstep = [&]() {
            if (pre == Pre::Inner) {
                read_scal(k);
                if (host_sc[k].done) return false;
            }
            const int nz = precond(pre, v.r.p, v.z.p, n, done);
            QLAUNCH(k_cg_beta, 1, QT, st, s, part.p, nz);
            QLAUNCH(k_cg_p, q_grid(n), QT, st, v.z.p, v.p.p, n, s);
            return true;
        };
        auto qstep = [&]() {
            lap_apply(A, v.p.p, v.q.p, st, done);
            QLAUNCH(k_dot_part, np, QT, st, v.p.p, v.q.p, n, part.p, done);
            QLAUNCH(k_cg_alpha, 1, QT, st, s, part.p, np);
            QLAUNCH(k_cg_xr, np, QT, st, x, v.r.p, v.p.p, v.q.p, n, s, part.p);
            QLAUNCH(k_cg_check, 1, QT, st, s, part.p, np, hist_dev);
        };
        zstep();
        uint32_t launched = 0;
        uint32_t chunk = pre == Pre::Inner ? 1 : std::max<uint32_t>(1, k == 1 ? hint : 8);
        while (launched < max_iter) {
            const uint32_t c = std::min(chunk, max_iter - launched);
            for (uint32_t i = 0; i < c; ++i) {
                qstep();
                if (!zstep()) break;
            }
            launched += c;
            read_scal(k);
            if (host_sc[k].done) break;
            chunk = pre == Pre::Inner ? 1 : (k == 1 ? 4 : 32);
        }
        read_scal(k);
        const uint32_t it = host_sc[k].iters;
        if (k == 1) hint = std::max<uint32_t>(1, it);
        return it;
    }
};

// ---------------------------------------------------------------------------
// Lanczos on the pencil (L_G, L_H)
// ---------------------------------------------------------------------------
__global__ void k_philox_vec(double* v, uint32_t n, uint32_t k0, uint32_t k1) {
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        const uint32_t u = philox_word0(x, 0u, 0u, 0u, k0, k1);
        v[x] = 2.0 * ((double)u * 0x1p-32) - 1.0;
    }
}

struct LzScal {
    double nrm;       // current ||w||_H
    uint32_t fail;
    uint32_t pad;
};

// alpha_j = (v, u)
__global__ void __launch_bounds__(QT) k_lz_alpha(const double* part, int np, double* alpha, int j) {
    __shared__ double sh[QT];
    const double s = sum_parts(part, np, sh);
    if (threadIdx.x == 0) alpha[j] = s;
}

// w = w - alpha_j v - beta_{j-1} v_prev
__global__ void k_lz_orth(double* __restrict__ w, const double* __restrict__ v, const double* __restrict__ vp,
                          uint32_t n, const double* alpha, const double* beta, int j) {
    const double al = alpha[j];
    const double be = j > 0 ? beta[j - 1] : 0.0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double t = fma(-al, v[i], w[i]);
        if (j > 0) t = fma(-be, vp[i], t);
        w[i] = t;
    }
}

// beta_j = sqrt((w, H w))
__global__ void __launch_bounds__(QT) k_lz_norm(const double* part, int np, double* out, LzScal* s) {
    __shared__ double sh[QT];
    const double q = sum_parts(part, np, sh);
    if (threadIdx.x == 0) {
        const double b = q > 0.0 ? sqrt(q) : 0.0;
        *out = b;
        s->nrm = b;
        s->fail = q > 0.0 ? 0u : 1u;
    }
}

__global__ void k_lz_scale(const double* __restrict__ w, double* __restrict__ v, uint32_t n, const double* nrm) {
    const double b = *nrm;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        v[i] = b > 0.0 ? w[i] / b : 0.0;
}

// Sturm count: eigenvalues of the k x k tridiagonal (alpha, beta) below x
__device__ int sturm_count(const double* al, const double* be, int k, double x) {
    int c = 0;
    double d = 1.0;
    for (int i = 0; i < k; ++i) {
        const double b2 = i ? be[i - 1] * be[i - 1] : 0.0;
        d = (al[i] - x) - (i ? b2 / d : 0.0);
        if (d == 0.0) d = -1e-300;
        c += d < 0.0;
    }
    return c;
}

// extreme eigenvalues of the tridiagonal by multisection: every round the
// block evaluates QT points of the current bracket and keeps the sub-bracket
// where the count steps across the wanted index
__global__ void __launch_bounds__(QT) k_tri_extremes(const double* __restrict__ al, const double* __restrict__ be,
                                                      int k, double* out) {
    __shared__ int cnt[QT + 1];
    __shared__ double lohi[2];
    double glo = 1e300, ghi = -1e300;
    for (int i = 0; i < k; ++i) {
        const double r = (i ? fabs(be[i - 1]) : 0.0) + (i + 1 < k ? fabs(be[i]) : 0.0);
        glo = fmin(glo, al[i] - r);
        ghi = fmax(ghi, al[i] + r);
    }
    for (int want = 0; want < 2; ++want) {  // 0: smallest (count steps 0 -> 1), 1: largest (k-1 -> k)
        double lo = glo - 1e-12 * fabs(glo) - 1e-300, hi = ghi + 1e-12 * fabs(ghi) + 1e-300;
        for (int round = 0; round < 12; ++round) {
            const double x = lo + (hi - lo) * (double)(threadIdx.x + 1) / (double)(QT + 1);
            cnt[threadIdx.x] = sturm_count(al, be, k, x);
            __syncthreads();
            if (threadIdx.x == 0) {
                const int target = want == 0 ? 1 : k;
                // first point whose count reaches target: the eigenvalue lies below it
                int t = 0;
                while (t < QT && cnt[t] < target) ++t;
                const double nlo = t == 0 ? lo : lo + (hi - lo) * (double)t / (double)(QT + 1);
                const double nhi = t == QT ? hi : lo + (hi - lo) * (double)(t + 1) / (double)(QT + 1);
                lohi[0] = nlo;
                lohi[1] = nhi;
            }
            __syncthreads();
            lo = lohi[0];
            hi = lohi[1];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[want] = 0.5 * (lo + hi);
    }
}

}  // namespace

// ===========================================================================
// host entry points
// ===========================================================================
namespace {

struct QualityCall {
    Ctx& c;
    DGraph& g;
    cudaStream_t st;
    DevAlloc& a;
    Lap G, H;
    Forest F;
    QualityCall(Ctx& cc, DGraph& gg) : c(cc), g(gg), st(cc.stream), a(cc.alloc) {}
    ~QualityCall() {
        cudaStreamSynchronize(st);
        G.release(a, st);
        H.release(a, st);
        F.release(a, st);
    }
    void build(bool g_lap, bool h_lap, bool forest, bool keep_edges = false) {
        graph_wait_estimates(g, st);
        // the compact rows index entries with 32-bit offsets
        if (g_lap && csr_edge_count(g.G, a, st) >= 0x7FFFFFF0ull)
            throw Error(DG_E_INVALID, "graph too large for the quality calls");
        if (g_lap) lap_build(G, g.G, a, st);
        if (h_lap) lap_build(H, g.H, a, st);
        if (forest) forest_build(F, H, a, st, keep_edges);
    }
    // H must span every component of G (it is a subgraph of G)
    bool spans() { return lap_components(G, a, st) == F.ntrees; }
};

float elapsed(cudaEvent_t e0, cudaEvent_t e1) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms;
}

}  // namespace

}  // namespace dg

using namespace dg;

template <class F>
static dg_status q_guard(dg_ctx* ctx, F&& f) {
    try {
        if (!ctx) throw Error(DG_E_INVALID, "null context");
        Ctx& c = *reinterpret_cast<Ctx*>(ctx);
        DG_CUDA(cudaSetDevice(c.device));
        f(c);
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

extern "C" dg_status dg_sparsifier_density(dg_ctx* ctx, int32_t graph_id, double* d_h_out, int64_t* m_g_out,
                                           int64_t* m_h_out) {
    return q_guard(ctx, [&](Ctx& c) {
        DGraph& g = c.graph(graph_id);
        std::lock_guard<std::mutex> lk(g.mu);
        if (!g.has_h) throw Error(DG_E_STATE, "no sparsifier yet");
        graph_wait_estimates(g, c.stream);
        const uint64_t mg = csr_edge_count(g.G, c.alloc, c.stream);
        const uint64_t mh = csr_edge_count(g.H, c.alloc, c.stream);
        if (m_g_out) *m_g_out = (int64_t)mg;
        if (m_h_out) *m_h_out = (int64_t)mh;
        if (d_h_out) *d_h_out = g.n ? (double)mh / (double)g.n - 1.0 : 0.0;
    });
}

extern "C" dg_status dg_laplacian_apply(dg_ctx* ctx, int32_t graph_id, int32_t which, const double* d_x, double* d_y,
                                        void* cuda_stream) {
    return q_guard(ctx, [&](Ctx& c) {
        if (which != DG_LAP_G && which != DG_LAP_H) throw Error(DG_E_INVALID, "which must be DG_LAP_G or DG_LAP_H");
        if ((!d_x || !d_y) && c.graph(graph_id).n) throw Error(DG_E_INVALID, "null vector");
        DGraph& g = c.graph(graph_id);
        std::lock_guard<std::mutex> lk(g.mu);
        if (which == DG_LAP_H && !g.has_h) throw Error(DG_E_STATE, "no sparsifier yet");
        QualityCall q(c, g);
        cudaStream_t ust = cuda_stream ? (cudaStream_t)cuda_stream : c.stream;
        graph_wait_estimates(g, c.stream);
        Lap& L = which == DG_LAP_G ? q.G : q.H;
        lap_build(L, which == DG_LAP_G ? g.G : g.H, c.alloc, c.stream);
        DG_CUDA(cudaStreamSynchronize(ust));
        lap_apply(L, d_x, d_y, c.stream);
        DG_CUDA(cudaStreamSynchronize(c.stream));
    });
}

extern "C" dg_status dg_pcg_solve(dg_ctx* ctx, int32_t graph_id, const double* d_b, double* d_x,
                                  const dg_pcg_options* opt, dg_pcg_info* info, double* hist) {
    return q_guard(ctx, [&](Ctx& c) {
        if (!opt) throw Error(DG_E_INVALID, "null options");
        if (!(opt->tol > 0.0) || opt->max_iter <= 0) throw Error(DG_E_INVALID, "tol must be > 0, max_iter > 0");
        if (opt->precond < DG_PRECOND_NONE || opt->precond > DG_PRECOND_SPARSIFIER)
            throw Error(DG_E_INVALID, "unknown preconditioner");
        if (opt->precond == DG_PRECOND_SPARSIFIER && (!(opt->inner_tol > 0.0) || opt->inner_max_iter <= 0))
            throw Error(DG_E_INVALID, "inner_tol must be > 0, inner_max_iter > 0");
        DGraph& g = c.graph(graph_id);
        std::lock_guard<std::mutex> lk(g.mu);
        const uint32_t n = (uint32_t)g.n;
        if (n && (!d_b || !d_x)) throw Error(DG_E_INVALID, "null vector");
        const bool sp = opt->precond == DG_PRECOND_SPARSIFIER;
        if (sp) {
            if (!g.has_h) throw Error(DG_E_STATE, "no sparsifier yet");
        }
        QualityCall q(c, g);
        q.build(true, sp, sp);
        if (sp && !q.spans()) throw Error(DG_E_STATE, "H does not span every component of G");
        Solver S;
        S.G = &q.G;
        S.H = &q.H;
        S.F = &q.F;
        S.inner_tol = opt->inner_tol;
        S.inner_max = (uint32_t)opt->inner_max_iter;
        DBuf<double> hd;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        try {
            S.init(c.alloc, c.stream, n);
            if (hist) hd.ensure(c.alloc, (size_t)opt->max_iter + 2, c.stream);
            DG_CUDA(cudaEventCreate(&e0));
            DG_CUDA(cudaEventCreate(&e1));
            DG_CUDA(cudaEventRecord(e0, c.stream));
            const Pre pre = opt->precond == DG_PRECOND_NONE ? Pre::None
                            : opt->precond == DG_PRECOND_JACOBI ? Pre::Jacobi : Pre::Inner;
            const uint32_t it = S.cg(q.G, pre, d_b, d_x, n, opt->tol, (uint32_t)opt->max_iter, 0,
                                     hist ? hd.p : nullptr);
            DG_CUDA(cudaEventRecord(e1, c.stream));
            // the true residual of the result: ||b - L_G x|| / ||b||
            DBuf<double> t, rs;
            t.ensure(c.alloc, (size_t)n + 1, c.stream);
            rs.ensure(c.alloc, 2, c.stream);
            lap_apply(q.G, d_x, t.p, c.stream);
            QLAUNCH(k_resid_part, S.np, QT, c.stream, d_b, t.p, n, S.part.p, S.part2.p);
            QLAUNCH(k_resid_fin, 1, QT, c.stream, S.part.p, S.part2.p, S.np, rs.p);
            double rel = 0.0;
            DG_CUDA(cudaMemcpyAsync(&rel, rs.p, 8, cudaMemcpyDeviceToHost, c.stream));
            DG_CUDA(cudaStreamSynchronize(c.stream));
            t.release(c.alloc, c.stream);
            rs.release(c.alloc, c.stream);
            S.read_scal(0);
            if (info) {
                info->iters = (int32_t)it;
                info->converged = S.host_sc[0].rr < S.host_sc[0].tol2 || S.host_sc[0].bb == 0.0;
                info->rel_residual = rel;
                info->inner_iters = S.inner_total;
                info->inner_max = S.inner_most;
                info->inner_unconverged = S.inner_unconv;
                info->ms = elapsed(e0, e1);
            }
            if (hist) {
                DG_CUDA(cudaMemcpyAsync(hist, hd.p, 8ull * (it + 1), cudaMemcpyDeviceToHost, c.stream));
                DG_CUDA(cudaStreamSynchronize(c.stream));
            }
        } catch (...) {
            cudaStreamSynchronize(c.stream);
            S.release();
            hd.release(c.alloc, c.stream);
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
            throw;
        }
        S.release();
        hd.release(c.alloc, c.stream);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    });
}

extern "C" dg_status dg_condition_number(dg_ctx* ctx, int32_t graph_id, const dg_kappa_options* opt,
                                         dg_kappa_info* info) {
    return q_guard(ctx, [&](Ctx& c) {
        if (!opt || !info) throw Error(DG_E_INVALID, "null options or info");
        if (opt->max_iter <= 0 || opt->check_every <= 0 || !(opt->tol >= 0.0) || !(opt->inner_tol > 0.0) ||
            opt->inner_max_iter <= 0)
            throw Error(DG_E_INVALID, "bad Lanczos options");
        DGraph& g = c.graph(graph_id);
        std::lock_guard<std::mutex> lk(g.mu);
        if (!g.has_h) throw Error(DG_E_STATE, "no sparsifier yet");
        const uint32_t n = (uint32_t)g.n;
        QualityCall q(c, g);
        q.build(true, true, true);
        *info = dg_kappa_info{};
        if (!q.spans()) {
            info->kappa = INFINITY;
            info->lambda_min = 1.0;
            info->converged = 1;
            return;
        }
        if (n < 2 || q.F.nf == 0) {
            info->kappa = 1.0;
            info->lambda_min = 1.0;
            info->converged = 1;
            return;
        }
        cudaStream_t st = c.stream;
        DevAlloc& a = c.alloc;
        Solver S;
        S.G = &q.G;
        S.H = &q.H;
        S.F = &q.F;
        S.inner_tol = opt->inner_tol;
        S.inner_max = (uint32_t)opt->inner_max_iter;
        const int K = opt->max_iter;
        DBuf<double> v, vp, u, w, t, al, be, ext, part;
        DBuf<LzScal> ls;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        auto rel = [&]() {
            for (auto* b : {&v, &vp, &u, &w, &t, &al, &be, &ext, &part}) b->release(a, st);
            ls.release(a, st);
            S.release();
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
        };
        try {
            S.init(a, st, n);
            const int np = S.np;
            for (auto* b : {&v, &vp, &u, &w, &t}) b->ensure(a, (size_t)n + 1, st);
            al.ensure(a, (size_t)K + 1, st);
            be.ensure(a, (size_t)K + 1, st);
            ext.ensure(a, 2, st);
            part.ensure(a, (size_t)np + 1, st);
            ls.ensure(a, 1, st);
            DG_CUDA(cudaEventCreate(&e0));
            DG_CUDA(cudaEventCreate(&e1));
            DG_CUDA(cudaEventRecord(e0, st));
            if (opt->d_v0) {
                DG_CUDA(cudaMemcpyAsync(w.p, opt->d_v0, 8ull * n, cudaMemcpyDeviceToDevice, st));
            } else {
                QLAUNCH(k_philox_vec, q_grid(n), QT, st, w.p, n, (uint32_t)opt->seed, (uint32_t)(opt->seed >> 32));
            }
            // v_1 = v_0 / ||v_0||_H
            lap_apply(q.H, w.p, t.p, st);
            QLAUNCH(k_dot_part, np, QT, st, w.p, t.p, n, part.p, nullptr);
            QLAUNCH(k_lz_norm, 1, QT, st, part.p, np, ext.p, ls.p);
            QLAUNCH(k_lz_scale, q_grid(n), QT, st, w.p, v.p, n, ext.p);
            LzScal hs{};
            DG_CUDA(cudaMemcpyAsync(&hs, ls.p, sizeof(LzScal), cudaMemcpyDeviceToHost, st));
            DG_CUDA(cudaStreamSynchronize(st));
            if (hs.fail) throw Error(DG_E_INVALID, "the start vector is constant on every component of H");
            double prev = 0.0, ritz[2] = {0.0, 0.0};
            int j = 0;
            bool conv = false;
            for (; j < K; ++j) {
                lap_apply(q.G, v.p, u.p, st);                                   // u = L_G v_j
                QLAUNCH(k_dot_part, np, QT, st, v.p, u.p, n, part.p, nullptr);  // alpha_j = (v_j, u)
                QLAUNCH(k_lz_alpha, 1, QT, st, part.p, np, al.p, j);
                S.hsolve(u.p, w.p, n);                                          // w = L_H^+ u
                QLAUNCH(k_lz_orth, q_grid(n), QT, st, w.p, v.p, vp.p, n, al.p, be.p, j);
                lap_apply(q.H, w.p, t.p, st);                                   // beta_j = ||w||_H
                QLAUNCH(k_dot_part, np, QT, st, w.p, t.p, n, part.p, nullptr);
                QLAUNCH(k_lz_norm, 1, QT, st, part.p, np, be.p + j, ls.p);
                std::swap(v.p, vp.p);                                           // v_prev = v_j
                QLAUNCH(k_lz_scale, q_grid(n), QT, st, w.p, v.p, n, be.p + j);  // v_{j+1} = w / beta_j
                const bool last = j + 1 == K;
                if ((j + 1) % opt->check_every == 0 || last) {
                    QLAUNCH(k_tri_extremes, 1, QT, st, al.p, be.p, j + 1, ext.p);
                    DG_CUDA(cudaMemcpyAsync(ritz, ext.p, 16, cudaMemcpyDeviceToHost, st));
                    DG_CUDA(cudaMemcpyAsync(&hs, ls.p, sizeof(LzScal), cudaMemcpyDeviceToHost, st));
                    DG_CUDA(cudaStreamSynchronize(st));
                    if (hs.fail || std::fabs(ritz[1] - prev) <= opt->tol * ritz[1]) {
                        conv = true;
                        ++j;
                        break;
                    }
                    prev = ritz[1];
                } else {
                    DG_CUDA(cudaMemcpyAsync(&hs, ls.p, sizeof(LzScal), cudaMemcpyDeviceToHost, st));
                    DG_CUDA(cudaStreamSynchronize(st));
                    if (hs.fail) {  // an invariant subspace: the Ritz values are exact
                        QLAUNCH(k_tri_extremes, 1, QT, st, al.p, be.p, j + 1, ext.p);
                        DG_CUDA(cudaMemcpyAsync(ritz, ext.p, 16, cudaMemcpyDeviceToHost, st));
                        DG_CUDA(cudaStreamSynchronize(st));
                        conv = true;
                        ++j;
                        break;
                    }
                }
            }
            DG_CUDA(cudaEventRecord(e1, st));
            DG_CUDA(cudaStreamSynchronize(st));
            info->kappa = ritz[1];
            info->lambda_min = ritz[0];
            info->iters = j;
            info->converged = conv;
            info->inner_iters = S.inner_total;
            info->ms = elapsed(e0, e1);
        } catch (...) {
            cudaStreamSynchronize(st);
            rel();
            throw;
        }
        rel();
    });
}

extern "C" dg_status dg_debug_sparsifier_forest(dg_ctx* ctx, int32_t graph_id, int64_t cap, int32_t* fu, int32_t* fv,
                                                int64_t* nf_out) {
    return q_guard(ctx, [&](Ctx& c) {
        DGraph& g = c.graph(graph_id);
        std::lock_guard<std::mutex> lk(g.mu);
        if (!g.has_h) throw Error(DG_E_STATE, "no sparsifier yet");
        QualityCall q(c, g);
        q.build(false, true, true, true);
        const int64_t nf = (int64_t)q.F.host_edges.size();
        if (nf_out) *nf_out = nf;
        if (cap < nf || (nf && (!fu || !fv))) throw Error(DG_E_INVALID, "output arrays too small");
        for (int64_t i = 0; i < nf; ++i) {
            fu[i] = (int32_t)(q.F.host_edges[i] >> 32);
            fv[i] = (int32_t)(q.F.host_edges[i] & 0xFFFFFFFFu);
        }
    });
}

extern "C" dg_status dg_debug_forest_solve(dg_ctx* ctx, int32_t graph_id, const double* d_r, double* d_z) {
    return q_guard(ctx, [&](Ctx& c) {
        DGraph& g = c.graph(graph_id);
        std::lock_guard<std::mutex> lk(g.mu);
        if (!g.has_h) throw Error(DG_E_STATE, "no sparsifier yet");
        if (g.n && (!d_r || !d_z)) throw Error(DG_E_INVALID, "null vector");
        QualityCall q(c, g);
        q.build(false, true, true);
        forest_solve(q.F, d_r, d_z, c.stream);
        DG_CUDA(cudaStreamSynchronize(c.stream));
    });
}
