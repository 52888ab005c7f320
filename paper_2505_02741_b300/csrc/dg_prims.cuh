// dg_prims.cuh -- scan and radix-sort primitives used by the slack-CSR mutation
// and batch-validation steps.  Every primitive reads its element count from
// device memory (with a host-side upper bound that fixes grid sizes), so the
// launches can be captured once into a CUDA graph and replayed for any count.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace dg {

// error bit a primitive raises when a look-back wait gives up (bounded spin)
constexpr uint32_t PRIM_ERR_SPIN = 1u << 8;

// Optional last step of a scan, run once by the thread that wrote the totals,
// right after them: the pool allocation of a list-execution plan.  base = *top
// goes to totals[base_lo], totals[base_hi]; err gets pool_bit when base +
// totals[r_idx] exceeds pool_cap, else cap_bit when totals[s_idx] exceeds
// stage_cap.  Nothing happens when *err already has a bit of abort_mask.
struct ScanAlloc {
    const unsigned long long* top = nullptr;  // null: no such step
    uint64_t pool_cap = 0, stage_cap = 0;
    uint32_t* totals = nullptr;
    uint32_t r_idx = 0, s_idx = 0, base_lo = 0, base_hi = 0;
    uint32_t* err = nullptr;
    uint32_t abort_mask = 0, pool_bit = 0, cap_bit = 0;
};

// Optional inputs generated inside the scan instead of read from in[]:
//   mode 1, a change list sorted by key = vertex * n_div + neighbour: array 0 is
//     1 where a vertex's run of changes begins, array 1 is 1 where
//     kinds[vals[c]] == k_ins, array 2 is 1 where kinds[vals[c]] == k_del;
//   mode 2: array 0 is bytes[idx[c]].
struct ScanGen {
    int mode = 0;  // 0: read in[]
    const uint64_t* keys = nullptr;
    uint64_t n_div = 1;
    const uint32_t* vals = nullptr;
    const uint8_t* kinds = nullptr;
    uint8_t k_ins = 0, k_del = 0;
    const uint8_t* bytes = nullptr;
    const uint32_t* idx = nullptr;
};

// Optional compaction by array 0: every item c whose array-0 value is 1 has
// its (keys[c], vals[c]) written at its exclusive prefix in okeys / ovals
// (array 0 must hold 0 / 1 values).
struct ScanCompact {
    const uint64_t* keys = nullptr;  // null: no compaction
    const uint32_t* vals = nullptr;
    uint64_t* okeys = nullptr;
    uint32_t* ovals = nullptr;
};

// Exclusive prefix sums of up to four uint32 arrays of the same length n.
// n = *d_n (or n_max when d_n is null).  total[a] (nullable) receives the sum.
struct ScanJob {
    const uint32_t* in[4] = {nullptr, nullptr, nullptr, nullptr};
    uint32_t* out[4] = {nullptr, nullptr, nullptr, nullptr};
    uint32_t* total[4] = {nullptr, nullptr, nullptr, nullptr};
    int k = 0;
    uint32_t* err = nullptr;  // optional: PRIM_ERR_SPIN is or-ed in here
    ScanGen gen;              // optional generated inputs
    ScanCompact cmp;          // optional compaction by array 0
    ScanAlloc post;           // optional step after the totals
};
size_t scan_tmp_words(uint32_t n_max);  // uint32 words of scratch for one ScanJob
// tmp_zeroed: the caller has cleared scan_tmp_words(n_max) words of tmp (no memset here)
void scan_exclusive(const ScanJob& job, const uint32_t* d_n, uint32_t n_max, uint32_t* tmp,
                    cudaStream_t st, bool tmp_zeroed = false);

// Stable LSD radix sort of (uint64 key, uint32 value) pairs on the low nbits of
// the key (8-bit digits, one-sweep: one histogram kernel, then one kernel per
// digit that ranks a 2048-key tile and finds its offsets by decoupled look-back).
// The count is *d_n <= n_max.  Returns true when the sorted data ends in the
// *_alt buffers.
struct SortBufs {
    uint64_t* keys;
    uint32_t* vals;
    uint64_t* keys_alt;
    uint32_t* vals_alt;
    uint32_t* hist;      // sort_hist_words(n_max): digit totals, tile counters, look-back status
    uint32_t* scan_tmp;  // unused (kept for layout compatibility), may be null
    uint32_t* err = nullptr;
};
size_t sort_hist_words(uint32_t n_max);
size_t sort_scan_tmp_words(uint32_t n_max);
// run_if (nullable device word): when it reads 0 the sort's kernels return at
// once and the data stays where it was (callers then use the unsorted input).
// hist_zeroed: the caller has cleared sort_clear_words(n_max, nbits) words of
// hist (no memset here)
bool radix_sort_pairs(const SortBufs& b, const uint32_t* d_n, uint32_t n_max, int nbits,
                      cudaStream_t st, const uint32_t* run_if = nullptr, bool hist_zeroed = false);
size_t sort_clear_words(uint32_t n_max, int nbits);  // words of hist a sort needs zero on entry

int bit_length(uint64_t x);

// kernel launches issued by this thread (the benchmark's launch tally)
extern thread_local uint64_t g_launches;

}  // namespace dg
