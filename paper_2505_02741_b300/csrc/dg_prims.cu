// dg_prims.cu -- exclusive scan and stable LSD radix sort (warp-tiled,
// __match_any_sync ranking) with device-side element counts.
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

// ---------------------------------------------------------------------------
// scan
// ---------------------------------------------------------------------------
static inline uint32_t scan_blocks(uint32_t n_max) { return (n_max + SCAN_TILE - 1) / SCAN_TILE; }

size_t scan_tmp_words(uint32_t n_max) { return 3u * (size_t)(scan_blocks(n_max) + 1); }

__device__ __forceinline__ uint32_t load_n(const uint32_t* d_n, uint32_t n_max) {
    return d_n ? min(*d_n, n_max) : n_max;
}

struct ScanArgs {
    const uint32_t* in[3];
    uint32_t* out[3];
    uint32_t* total[3];
    int k;
};

__device__ __forceinline__ uint32_t block_sum(uint32_t v, uint32_t* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    uint32_t t = 0;
    if (threadIdx.x < 32) {
        t = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0u;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;  // valid in thread 0
}

__global__ void k_scan_reduce(ScanArgs a, const uint32_t* d_n, uint32_t n_max, uint32_t* tmp,
                              uint32_t nb_max) {
    __shared__ uint32_t sh[32];
    const uint32_t n = load_n(d_n, n_max);
    const uint32_t base = blockIdx.x * SCAN_TILE;
    for (int j = 0; j < a.k; ++j) {
        uint32_t s = 0;
        if (base < n) {
#pragma unroll
            for (int i = 0; i < SCAN_ITEMS; ++i) {
                uint32_t idx = base + i * SCAN_THREADS + threadIdx.x;
                if (idx < n) s += a.in[j][idx];
            }
        }
        uint32_t t = block_sum(s, sh);
        if (threadIdx.x == 0) tmp[j * (nb_max + 1) + blockIdx.x] = t;
    }
}

// one CTA: exclusive scan of the block sums, chunk by chunk with a carry
__global__ void k_scan_mid(ScanArgs a, const uint32_t* d_n, uint32_t n_max, uint32_t* tmp,
                           uint32_t nb_max) {
    __shared__ uint32_t sh[32];
    __shared__ uint32_t carry_sh;
    const uint32_t n = load_n(d_n, n_max);
    const uint32_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int j = 0; j < a.k; ++j) {
        uint32_t* t = tmp + j * (nb_max + 1);
        if (threadIdx.x == 0) carry_sh = 0;
        __syncthreads();
        for (uint32_t c0 = 0; c0 < nb; c0 += blockDim.x) {
            uint32_t idx = c0 + threadIdx.x;
            uint32_t v = idx < nb ? t[idx] : 0u;
            uint32_t x = v;
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (l >= o) x += y;
            }
            if (l == 31) sh[w] = x;
            __syncthreads();
            if (threadIdx.x < 32) {
                uint32_t s = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0u;
                for (int o = 1; o < 32; o <<= 1) {
                    uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
                    if (l >= o) s += y;
                }
                sh[l] = s;  // inclusive per-warp prefix
            }
            __syncthreads();
            const uint32_t warp_prefix = (w > 0) ? sh[w - 1] : 0u;
            const uint32_t carry = carry_sh;
            if (idx < nb) t[idx] = carry + warp_prefix + x - v;
            __syncthreads();
            if (threadIdx.x == blockDim.x - 1) carry_sh = carry + warp_prefix + x;
            __syncthreads();
        }
        if (threadIdx.x == 0 && a.total[j]) *a.total[j] = carry_sh;
        __syncthreads();
    }
}

__global__ void k_scan_apply(ScanArgs a, const uint32_t* d_n, uint32_t n_max, const uint32_t* tmp,
                             uint32_t nb_max) {
    __shared__ uint32_t sh[32];
    const uint32_t n = load_n(d_n, n_max);
    const uint32_t base = blockIdx.x * SCAN_TILE;
    if (base >= n) return;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int j = 0; j < a.k; ++j) {
        uint32_t v[SCAN_ITEMS];
        uint32_t s = 0;
        const uint32_t mine = base + threadIdx.x * SCAN_ITEMS;
#pragma unroll
        for (int i = 0; i < SCAN_ITEMS; ++i) {
            v[i] = (mine + i < n) ? a.in[j][mine + i] : 0u;
            s += v[i];
        }
        uint32_t x = s;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (l >= o) x += y;
        }
        __syncthreads();
        if (l == 31) sh[w] = x;
        __syncthreads();
        if (threadIdx.x < 32) {
            uint32_t t = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0u;
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
                if (l >= o) t += y;
            }
            sh[l] = t;
        }
        __syncthreads();
        uint32_t run = tmp[j * (nb_max + 1) + blockIdx.x] + ((w > 0) ? sh[w - 1] : 0u) + x - s;
#pragma unroll
        for (int i = 0; i < SCAN_ITEMS; ++i) {
            if (mine + i < n) a.out[j][mine + i] = run;
            run += v[i];
        }
    }
}

void scan_exclusive(const ScanJob& job, const uint32_t* d_n, uint32_t n_max, uint32_t* tmp,
                    cudaStream_t st) {
    ScanArgs a;
    for (int j = 0; j < 3; ++j) {
        a.in[j] = job.in[j];
        a.out[j] = job.out[j];
        a.total[j] = job.total[j];
    }
    a.k = job.k;
    const uint32_t nb = scan_blocks(n_max);
    if (nb > 0) {
        k_scan_reduce<<<nb, SCAN_THREADS, 0, st>>>(a, d_n, n_max, tmp, nb);
        ++g_launches;
    }
    k_scan_mid<<<1, 1024, 0, st>>>(a, d_n, n_max, tmp, nb);
    ++g_launches;
    if (nb > 0) {
        k_scan_apply<<<nb, SCAN_THREADS, 0, st>>>(a, d_n, n_max, tmp, nb);
        ++g_launches;
    }
}

// ---------------------------------------------------------------------------
// radix sort: warp tiles of 32 * chunks elements, 8-bit digits
// ---------------------------------------------------------------------------
constexpr int SORT_WARPS = 8;

static inline uint32_t sort_chunks(uint32_t n_max) {
    // enough tiles to occupy the GPU, at most 64 chunks (2048 keys) per warp
    uint32_t c = n_max / (148u * 8u * 32u);
    if (c < 1) c = 1;
    if (c > 64) c = 64;
    return c;
}
static inline uint32_t sort_tiles(uint32_t n_max) {
    const uint32_t tile = 32u * sort_chunks(n_max);
    uint32_t t = (n_max + tile - 1) / tile;
    return t < 1 ? 1 : t;
}

size_t sort_hist_words(uint32_t n_max) { return 256u * (size_t)sort_tiles(n_max) + 1; }
size_t sort_scan_tmp_words(uint32_t n_max) {
    return scan_tmp_words((uint32_t)(256u * (size_t)sort_tiles(n_max)));
}

__global__ void k_radix_hist(const uint64_t* __restrict__ keys, const uint32_t* d_n, uint32_t n_max,
                             int shift, uint32_t chunks, uint32_t ntiles, uint32_t* __restrict__ hist) {
    __shared__ uint32_t cnt[SORT_WARPS][256];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const uint32_t t = blockIdx.x * SORT_WARPS + w;
    for (int d = l; d < 256; d += 32) cnt[w][d] = 0;
    __syncwarp();
    if (t >= ntiles) return;
    const uint32_t n = load_n(d_n, n_max);
    const uint32_t base = t * 32u * chunks;
#pragma unroll 4
    for (uint32_t c = 0; c < chunks; ++c) {
        const uint32_t idx = base + c * 32u + l;
        if (idx < n) atomicAdd(&cnt[w][(uint32_t)(keys[idx] >> shift) & 255u], 1u);
    }
    __syncwarp();
    for (int d = l; d < 256; d += 32) hist[(size_t)d * ntiles + t] = cnt[w][d];
}

__global__ void k_radix_scatter(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                                uint64_t* __restrict__ okeys, uint32_t* __restrict__ ovals,
                                const uint32_t* d_n, uint32_t n_max, int shift, uint32_t chunks,
                                uint32_t ntiles, const uint32_t* __restrict__ hist) {
    __shared__ uint32_t cnt[SORT_WARPS][256];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const uint32_t t = blockIdx.x * SORT_WARPS + w;
    if (t >= ntiles) return;
    for (int d = l; d < 256; d += 32) cnt[w][d] = hist[(size_t)d * ntiles + t];
    __syncwarp();
    const uint32_t n = load_n(d_n, n_max);
    const uint32_t base = t * 32u * chunks;
    const uint32_t lt = (1u << l) - 1u;
    for (uint32_t c = 0; c < chunks; ++c) {
        const uint32_t idx = base + c * 32u + l;
        const bool valid = idx < n;
        uint64_t k = 0;
        uint32_t v = 0, d = 256;
        if (valid) {
            k = keys[idx];
            v = vals[idx];
            d = (uint32_t)(k >> shift) & 255u;
        }
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t pos = 0;
        if (valid) pos = cnt[w][d] + __popc(peers & lt);
        __syncwarp();
        if (valid && l == __ffs(peers) - 1) cnt[w][d] += __popc(peers);
        __syncwarp();
        if (valid) {
            okeys[pos] = k;
            ovals[pos] = v;
        }
    }
}

bool radix_sort_pairs(const SortBufs& b, const uint32_t* d_n, uint32_t n_max, int nbits,
                      cudaStream_t st) {
    if (n_max == 0 || nbits <= 0) return false;
    const uint32_t chunks = sort_chunks(n_max);
    const uint32_t ntiles = sort_tiles(n_max);
    const uint32_t grid = (ntiles + SORT_WARPS - 1) / SORT_WARPS;
    const uint64_t* src_k = b.keys;
    const uint32_t* src_v = b.vals;
    uint64_t* dst_k = b.keys_alt;
    uint32_t* dst_v = b.vals_alt;
    bool in_alt = false;
    for (int shift = 0; shift < nbits; shift += 8) {
        k_radix_hist<<<grid, 32 * SORT_WARPS, 0, st>>>(src_k, d_n, n_max, shift, chunks, ntiles, b.hist);
        ++g_launches;
        ScanJob job;
        job.in[0] = b.hist;
        job.out[0] = b.hist;  // in-place is safe: apply reads its own items before writing them
        job.k = 1;
        scan_exclusive(job, nullptr, 256u * ntiles, b.scan_tmp, st);
        k_radix_scatter<<<grid, 32 * SORT_WARPS, 0, st>>>(src_k, src_v, dst_k, dst_v, d_n, n_max, shift,
                                                          chunks, ntiles, b.hist);
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
