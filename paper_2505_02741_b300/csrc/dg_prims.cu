// dg_prims.cu -- exclusive scan and stable LSD radix sort with device-side
// element counts.
//
// Both large-array paths are single-pass with decoupled look-back: a block
// takes the next tile index from an atomic counter (so every tile it waits on
// belongs to a block that is already running), publishes its tile aggregate,
// then walks back over its predecessors until it meets an inclusive prefix.
// Every wait is bounded: after SPIN_LIMIT polls the block records
// PRIM_ERR_SPIN and stops waiting, so no kernel here can hang.
#include "dg_prims.cuh"

namespace dg {

thread_local uint64_t g_launches = 0;

int bit_length(uint64_t x) {
    int b = 0;
    while (x) {
        ++b;
        x >>= 1;
    }
    return b;
}

constexpr uint32_t SPIN_LIMIT = 1u << 20;

__device__ __forceinline__ uint32_t load_n(const uint32_t* d_n, uint32_t n_max) {
    return d_n ? min(*d_n, n_max) : n_max;
}

__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t* p) { return *(const volatile uint32_t*)p; }
__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p) {
    return *(const volatile unsigned long long*)p;
}

// ---------------------------------------------------------------------------
// scan
// ---------------------------------------------------------------------------
struct ScanArgs {
    const uint32_t* in[4];
    uint32_t* out[4];
    uint32_t* total[4];
    int k;
    uint32_t* err;
    ScanGen gen;
    ScanCompact cmp;
    ScanAlloc post;
};

// element c of input array j (read, or generated: see ScanGen)
__device__ __forceinline__ uint32_t scan_in(const ScanArgs& a, int j, uint32_t c) {
    if (a.gen.mode == 1) {
        if (j == 0) {  // sorted keys: c starts a run iff its predecessor lies below the run's first key
            if (c == 0) return 1u;
            const uint64_t k = a.gen.keys[c];
            return a.gen.keys[c - 1] < k - k % a.gen.n_div ? 1u : 0u;
        }
        const uint8_t kd = a.gen.kinds[a.gen.vals[c]];
        return (j == 1 ? kd == a.gen.k_ins : kd == a.gen.k_del) ? 1u : 0u;
    }
    if (a.gen.mode == 2) return a.gen.bytes[a.gen.idx[c]];
    return a.in[j][c];
}

// the exclusive prefix of item c of array j is pos: store it, and compact
__device__ __forceinline__ void scan_out(const ScanArgs& a, int j, uint32_t c, uint32_t pos, uint32_t v) {
    a.out[j][c] = pos;
    if (j == 0 && a.cmp.keys && v) {
        a.cmp.okeys[pos] = a.cmp.keys[c];
        a.cmp.ovals[pos] = a.cmp.vals[c];
    }
}

// the optional step after the totals (see ScanAlloc); one thread
__device__ __forceinline__ void scan_post(const ScanAlloc& p) {
    if (!p.top) return;
    if (*p.err & p.abort_mask) return;
    const unsigned long long base = *p.top;
    p.totals[p.base_lo] = (uint32_t)base;
    p.totals[p.base_hi] = (uint32_t)(base >> 32);
    if (base + p.totals[p.r_idx] > p.pool_cap) atomicOr(p.err, p.pool_bit);
    else if ((uint64_t)p.totals[p.s_idx] > p.stage_cap) atomicOr(p.err, p.cap_bit);
}

constexpr uint32_t SMALL_SCAN_MAX = 16384;
constexpr int LB_THREADS = 256;
constexpr int LB_ITEMS = 8;
constexpr uint32_t LB_TILE = LB_THREADS * LB_ITEMS;

static inline uint32_t lb_tiles(uint32_t n_max) { return (n_max + LB_TILE - 1) / LB_TILE; }

// layout of tmp: [counter (2 words, 8-byte aligned) | status u64 x 4 arrays x tiles]
size_t scan_tmp_words(uint32_t n_max) { return 4 + 2ull * 4 * (lb_tiles(n_max) + 1); }

// one CTA walks the arrays in chunks of 1024 x 8 with running carries, all
// k arrays of the job in the same chunk loop
__global__ void __launch_bounds__(1024) k_scan_single(ScanArgs a, const uint32_t* d_n, uint32_t n_max) {
    __shared__ uint32_t sh[4][32];
    __shared__ uint32_t carry_sh[4];
    const uint32_t n = load_n(d_n, n_max);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int nw = (int)(blockDim.x >> 5);
    const int K = a.k;
    constexpr int IT = 8;
    if (threadIdx.x < 4) carry_sh[threadIdx.x] = 0;
    __syncthreads();
    for (uint32_t c0 = 0; c0 < n; c0 += blockDim.x * IT) {
        const uint32_t mine = c0 + threadIdx.x * IT;
        uint32_t v[4][IT], s4[4], x4[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            s4[j] = 0;
            if (j < K) {
#pragma unroll
                for (int i = 0; i < IT; ++i) {
                    v[j][i] = (mine + i < n) ? scan_in(a, j, mine + i) : 0u;
                    s4[j] += v[j][i];
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint32_t x = s4[j];
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (l >= o) x += y;
            }
            x4[j] = x;
            if (l == 31) sh[j][w] = x;
        }
        __syncthreads();
        if (w < K) {  // warp j scans the warp totals of array j
            uint32_t tt = (l < nw) ? sh[w][l] : 0u;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, tt, o);
                if (l >= o) tt += y;
            }
            sh[w][l] = tt;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (j >= K) break;
            uint32_t run = carry_sh[j] + ((w > 0) ? sh[j][w - 1] : 0u) + x4[j] - s4[j];
#pragma unroll
            for (int i = 0; i < IT; ++i) {
                if (mine + i < n) scan_out(a, j, mine + i, run, v[j][i]);
                run += v[j][i];
            }
        }
        __syncthreads();
        if (threadIdx.x < (unsigned)K) carry_sh[threadIdx.x] += sh[threadIdx.x][31];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (K > 0 && a.total[0]) *a.total[0] = carry_sh[0];
        if (K > 1 && a.total[1]) *a.total[1] = carry_sh[1];
        if (K > 2 && a.total[2]) *a.total[2] = carry_sh[2];
        if (K > 3 && a.total[3]) *a.total[3] = carry_sh[3];
        scan_post(a.post);
    }
}

// status word: high 32 bits flag (0 empty, 1 aggregate, 2 inclusive), low 32 bits value
constexpr unsigned long long LB_AGG = 1ull << 32, LB_INC = 2ull << 32;

// All k arrays of a job go through one pass together: their tile inputs are
// loaded at once, block-scanned side by side, and warp j looks back for array
// j, so a tile costs the round trips of one array rather than k.
__global__ void __launch_bounds__(LB_THREADS) k_scan_lookback(ScanArgs a, const uint32_t* d_n, uint32_t n_max,
                                                             uint32_t* tmp, uint32_t tiles) {
    constexpr int NW = LB_THREADS / 32;
    __shared__ uint32_t sh[4][NW];
    __shared__ uint32_t s_tile, s_prefix[4];
    unsigned long long* status = reinterpret_cast<unsigned long long*>(tmp + 4);
    const uint32_t n = load_n(d_n, n_max);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (threadIdx.x == 0) s_tile = atomicAdd(tmp, 1u);
    __syncthreads();
    const uint32_t t = s_tile;
    const uint32_t base = t * LB_TILE;
    const uint32_t nt = (n + LB_TILE - 1) / LB_TILE;  // tiles holding data
    if (t >= tiles) return;
    const int K = a.k;
    const uint32_t mine = base + threadIdx.x * LB_ITEMS;
    uint32_t v[4][LB_ITEMS], s4[4], x4[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        s4[j] = 0;
        if (j < K) {
#pragma unroll
            for (int i = 0; i < LB_ITEMS; ++i) {
                v[j][i] = (mine + i < n) ? scan_in(a, j, mine + i) : 0u;
                s4[j] += v[j][i];
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        uint32_t x = s4[j];
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (l >= o) x += y;
        }
        x4[j] = x;
        if (l == 31) sh[j][w] = x;
    }
    __syncthreads();
    if (w < K) {  // warp j: scan of the warp totals of array j, then its look-back
        const int j = w;
        uint32_t tt = (l < NW) ? sh[j][l] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, tt, o);
            if (l >= o) tt += y;
        }
        const uint32_t agg = __shfl_sync(0xffffffffu, tt, NW - 1);
        unsigned long long* st = status + (size_t)j * (tiles + 1);
        uint32_t excl = 0;
        if (t == 0) {
            if (l == 0) atomicExch(&st[t], LB_INC | agg);
        } else {
            if (l == 0) atomicExch(&st[t], LB_AGG | agg);
            int top = (int)t - 1;  // newest predecessor not yet summed
            bool done = false;
            while (!done && top >= 0) {
                const int p = top - l;
                unsigned long long sv = LB_INC;  // lanes before tile 0 act as an inclusive zero
                if (p >= 0) {
                    uint32_t spins = 0;
                    while (((sv = ld_volatile_u64(&st[p])) >> 32) == 0ull && ++spins < SPIN_LIMIT) __nanosleep(32);
                }
                const bool empty = (sv >> 32) == 0ull;
                if (__any_sync(0xffffffffu, empty)) {
                    if (l == 0 && a.err) atomicOr(a.err, PRIM_ERR_SPIN);
                    break;
                }
                const uint32_t inc_mask = __ballot_sync(0xffffffffu, (sv >> 32) == 2ull);
                // sum lanes up to and including the nearest inclusive prefix
                const int stop = inc_mask ? __ffs(inc_mask) - 1 : 31;
                uint32_t part = (l <= stop) ? (uint32_t)sv : 0u;
                for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                excl += part;
                done = inc_mask != 0u;
                top -= 32;
            }
            // the status word carries its own value: no fence orders it
            if (l == 0) atomicExch(&st[t], LB_INC | (unsigned long long)(excl + agg));
        }
        if (l < NW) sh[j][l] = tt;  // inclusive warp totals
        if (l == 0) {
            s_prefix[j] = excl;
            uint32_t* total = j == 0 ? a.total[0] : j == 1 ? a.total[1] : j == 2 ? a.total[2] : a.total[3];
            if (t + 1 == nt && total) *total = excl + agg;
            if (nt == 0 && t == 0 && total) *total = 0;
        }
    }
    __syncthreads();
    // the block that wrote the totals (the barrier orders them before this)
    if (threadIdx.x == 0 && (t + 1 == nt || (nt == 0 && t == 0))) scan_post(a.post);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (j >= K) break;
        uint32_t run = s_prefix[j] + ((w > 0) ? sh[j][w - 1] : 0u) + x4[j] - s4[j];
#pragma unroll
        for (int i = 0; i < LB_ITEMS; ++i) {
            if (mine + i < n) scan_out(a, j, mine + i, run, v[j][i]);
            run += v[j][i];
        }
    }
}

void scan_exclusive(const ScanJob& job, const uint32_t* d_n, uint32_t n_max, uint32_t* tmp,
                    cudaStream_t st, bool tmp_zeroed) {
    ScanArgs a;
    for (int j = 0; j < 4; ++j) {
        a.in[j] = job.in[j];
        a.out[j] = job.out[j];
        a.total[j] = job.total[j];
    }
    a.k = job.k;
    a.err = job.err;
    a.gen = job.gen;
    a.cmp = job.cmp;
    a.post = job.post;
    if (n_max <= SMALL_SCAN_MAX) {
        k_scan_single<<<1, 1024, 0, st>>>(a, d_n, n_max);
        ++g_launches;
        return;
    }
    const uint32_t tiles = lb_tiles(n_max);
    if (!tmp_zeroed) cudaMemsetAsync(tmp, 0, scan_tmp_words(n_max) * 4, st);
    k_scan_lookback<<<tiles, LB_THREADS, 0, st>>>(a, d_n, n_max, tmp, tiles);
    ++g_launches;
}

// ---------------------------------------------------------------------------
// one-sweep radix sort
// ---------------------------------------------------------------------------
constexpr int OS_THREADS = 512;
constexpr int OS_WARPS = OS_THREADS / 32;
constexpr int OS_ITEMS = 4;
constexpr uint32_t OS_TILE = OS_THREADS * OS_ITEMS;  // 2048 keys, a warp holds 128 consecutive ones
constexpr int OS_MAX_PASSES = 8;
constexpr uint32_t OS_AGG = 1u << 30, OS_INC = 2u << 30, OS_VAL = (1u << 30) - 1u;

static inline uint32_t os_tiles(uint32_t n_max) {
    uint32_t t = (n_max + OS_TILE - 1) / OS_TILE;
    return t < 1 ? 1 : t;
}

// hist layout: [digit totals OS_MAX_PASSES x 256 | tile counters 32 | status tiles x 256]
constexpr size_t OS_GHIST = 0;
constexpr size_t OS_CTR = OS_MAX_PASSES * 256;
constexpr size_t OS_STATUS = OS_CTR + 32;

// small sorts keep one status area per pass (cleared by a single memset);
// large ones reuse one area and clear it before every pass
constexpr uint32_t OS_SEPARATE_MAX_TILES = 1024;

__host__ __device__ inline bool os_separate(uint32_t tiles) { return tiles <= OS_SEPARATE_MAX_TILES; }

size_t sort_hist_words(uint32_t n_max) {
    const uint32_t tiles = os_tiles(n_max);
    return OS_STATUS + 256ull * tiles * (os_separate(tiles) ? OS_MAX_PASSES : 1) + 64;
}
size_t sort_scan_tmp_words(uint32_t n_max) { return scan_tmp_words(n_max + 1); }

// digit totals of every pass in one read of the keys (warp-aggregated atomics)
__global__ void __launch_bounds__(256) k_os_hist(const uint64_t* __restrict__ keys, const uint32_t* d_n,
                                                 uint32_t n_max, int passes, uint32_t* __restrict__ ghist,
                                                 const uint32_t* run_if) {
    if (run_if && *run_if == 0u) return;
    __shared__ uint32_t h[OS_MAX_PASSES][256];
    for (int i = threadIdx.x; i < OS_MAX_PASSES * 256; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    const uint32_t n = load_n(d_n, n_max);
    const int l = threadIdx.x & 31;
    const uint32_t lt = (1u << l) - 1u;
    (void)lt;
    const uint32_t stride = gridDim.x * blockDim.x;
    // whole warps iterate together so the match below always sees a full warp
    for (uint32_t i0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); i0 < n; i0 += stride) {
        const uint32_t i = i0 + l;
        const bool valid = i < n;
        const uint64_t k = valid ? keys[i] : 0ull;
        for (int p = 0; p < passes; ++p) {
            const uint32_t d = valid ? (uint32_t)(k >> (8 * p)) & 255u : 256u;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            if (valid && l == __ffs(peers) - 1) atomicAdd(&h[p][d], (uint32_t)__popc(peers));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * 256; i += blockDim.x) {
        const uint32_t c = (&h[0][0])[i];
        if (c) atomicAdd(&ghist[i], c);
    }
}

__global__ void __launch_bounds__(OS_THREADS) k_os_pass(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                        uint64_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                        const uint32_t* d_n, uint32_t n_max, int pass,
                                                        uint32_t* hist, uint32_t tiles, uint32_t* err,
                                                        const uint32_t* run_if) {
    if (run_if && *run_if == 0u) return;
    __shared__ uint32_t s_warp[OS_WARPS][256];
    __shared__ uint32_t s_base[256];
    __shared__ uint32_t s_tile;
    const uint32_t n = load_n(d_n, n_max);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const uint32_t lt = (1u << l) - 1u;
    const int shift = 8 * pass;
    uint32_t* ctr = hist + OS_CTR + pass;
    uint32_t* status = hist + OS_STATUS + (os_separate(tiles) ? (size_t)pass * tiles * 256 : 0);
    const uint32_t* gh = hist + OS_GHIST + 256 * pass;
    if (threadIdx.x == 0) s_tile = atomicAdd(ctr, 1u);
    for (int i = threadIdx.x; i < OS_WARPS * 256; i += OS_THREADS) (&s_warp[0][0])[i] = 0;
    __syncthreads();
    const uint32_t t = s_tile;
    const uint32_t base = t * OS_TILE;
    if (t >= tiles || base >= n) return;
    // the pass's digit totals (warp 0, 8 per lane), read alongside the keys
    uint32_t gv[8];
    if (w == 0) {
#pragma unroll
        for (int q = 0; q < 8; ++q) gv[q] = gh[l * 8 + q];
    }
    // load: warp w holds keys [base + 128 w, base + 128 w + 128), four chunks of 32
    uint64_t k[OS_ITEMS];
    uint32_t v[OS_ITEMS], d[OS_ITEMS], rk[OS_ITEMS];
#pragma unroll
    for (int c = 0; c < OS_ITEMS; ++c) {
        const uint32_t idx = base + w * (32 * OS_ITEMS) + c * 32 + l;
        const bool valid = idx < n;
        k[c] = valid ? kin[idx] : 0ull;
        v[c] = valid ? vin[idx] : 0u;
        d[c] = valid ? ((uint32_t)(k[c] >> shift) & 255u) : 256u;
    }
    // ranks inside the warp, in index order
#pragma unroll
    for (int c = 0; c < OS_ITEMS; ++c) {
        const uint32_t peers = __match_any_sync(0xffffffffu, d[c]);
        rk[c] = (d[c] < 256u) ? s_warp[w][d[c]] + __popc(peers & lt) : 0u;
        __syncwarp();
        if (d[c] < 256u && l == __ffs(peers) - 1) s_warp[w][d[c]] += __popc(peers);
        __syncwarp();
    }
    // global start of every digit: exclusive scan of the digit totals (warp 0, 8 per lane)
    if (w == 0) {
        uint32_t s8 = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) s8 += gv[q];
        uint32_t x = s8;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (l >= o) x += y;
        }
        uint32_t run = x - s8;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            s_base[l * 8 + q] = run;
            run += gv[q];
        }
    }
    __syncthreads();
    if (threadIdx.x < 256) {
        const int dg = threadIdx.x;
        uint32_t run = 0;
#pragma unroll
        for (int ww = 0; ww < OS_WARPS; ++ww) {
            const uint32_t x = s_warp[ww][dg];
            s_warp[ww][dg] = run;
            run += x;
        }
        const uint32_t gstart = s_base[dg];
        // tiles before this one, by decoupled look-back (8 predecessors in flight)
        uint32_t excl = 0;
        if (t == 0) {
            atomicExch(&status[dg], OS_INC | run);
        } else {
            atomicExch(&status[(size_t)t * 256 + dg], OS_AGG | run);
            int top = (int)t - 1;
            bool done = false;
            constexpr int WIN = 8;
            while (!done && top >= 0) {
                uint32_t sv[WIN];
#pragma unroll
                for (int q = 0; q < WIN; ++q)
                    sv[q] = (top - q >= 0) ? ld_volatile_u32(&status[(size_t)(top - q) * 256 + dg]) : OS_INC;
#pragma unroll
                for (int q = 0; q < WIN; ++q) {
                    if (done) break;
                    uint32_t spins = 0;
                    while ((sv[q] >> 30) == 0u && ++spins < SPIN_LIMIT) {
                        __nanosleep(32);
                        sv[q] = ld_volatile_u32(&status[(size_t)(top - q) * 256 + dg]);
                    }
                    if ((sv[q] >> 30) == 0u) {
                        if (err) atomicOr(err, PRIM_ERR_SPIN);
                        done = true;
                        break;
                    }
                    excl += sv[q] & OS_VAL;
                    if ((sv[q] >> 30) == 2u) done = true;
                }
                top -= WIN;
            }
            atomicExch(&status[(size_t)t * 256 + dg], OS_INC | ((excl + run) & OS_VAL));
        }
        s_base[dg] = gstart + excl;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < OS_ITEMS; ++c) {
        if (d[c] >= 256u) continue;
        const uint32_t pos = s_base[d[c]] + s_warp[w][d[c]] + rk[c];
        kout[pos] = k[c];
        vout[pos] = v[c];
    }
}

size_t sort_clear_words(uint32_t n_max, int nbits) {
    if (n_max == 0 || nbits <= 0) return 0;
    const uint32_t tiles = os_tiles(n_max);
    return OS_STATUS + (os_separate(tiles) ? 256ull * tiles * (uint64_t)((nbits + 7) / 8) : 0);
}

bool radix_sort_pairs(const SortBufs& b, const uint32_t* d_n, uint32_t n_max, int nbits,
                      cudaStream_t st, const uint32_t* run_if, bool hist_zeroed) {
    if (n_max == 0 || nbits <= 0) return false;
    const int passes = (nbits + 7) / 8;
    const uint32_t tiles = os_tiles(n_max);
    // digit totals and tile counters, then per pass a cleared status area
    const bool separate = os_separate(tiles);
    if (!hist_zeroed) cudaMemsetAsync(b.hist, 0, sort_clear_words(n_max, nbits) * 4, st);
    uint32_t hblocks = (n_max + 255) / 256;
    if (hblocks > 148u * 8u) hblocks = 148u * 8u;
    k_os_hist<<<hblocks, 256, 0, st>>>(b.keys, d_n, n_max, passes, b.hist + OS_GHIST, run_if);
    ++g_launches;
    const uint64_t* src_k = b.keys;
    const uint32_t* src_v = b.vals;
    uint64_t* dst_k = b.keys_alt;
    uint32_t* dst_v = b.vals_alt;
    bool in_alt = false;
    for (int p = 0; p < passes; ++p) {
        if (!separate) cudaMemsetAsync(b.hist + OS_STATUS, 0, 256ull * tiles * 4, st);
        k_os_pass<<<tiles, OS_THREADS, 0, st>>>(src_k, src_v, dst_k, dst_v, d_n, n_max, p, b.hist, tiles, b.err,
                                                run_if);
        ++g_launches;
        in_alt = !in_alt;
        const uint64_t* tk = dst_k;
        const uint32_t* tv = dst_v;
        dst_k = const_cast<uint64_t*>(src_k);
        dst_v = const_cast<uint32_t*>(src_v);
        src_k = tk;
        src_v = tv;
    }
    return in_alt;
}

}  // namespace dg
