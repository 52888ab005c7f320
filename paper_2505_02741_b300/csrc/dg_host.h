// dg_host.h -- host-side helpers: error propagation, device memory, buffers.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstring>
#include <stdexcept>
#include <string>

#include "../../include/dygrass.h"

namespace dg {

struct Error : std::runtime_error {
    dg_status code;
    Error(dg_status c, const std::string& what) : std::runtime_error(what), code(c) {}
};

#define DG_CUDA(call)                                                                        \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            throw ::dg::Error(e_ == cudaErrorMemoryAllocation ? DG_E_NOMEM : DG_E_CUDA,      \
                              std::string(#call) + ": " + cudaGetErrorString(e_));           \
    } while (0)

#define DG_CHECK_LAUNCH() DG_CUDA(cudaGetLastError())

// timing event: an external event node while the stream is being captured
inline cudaError_t record_timing_event(cudaEvent_t ev, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    if (cs == cudaStreamCaptureStatusActive) return cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
    return cudaEventRecord(ev, st);
}

// Device memory through the caller's allocator (or cudaMallocAsync/cudaFreeAsync).
struct DevAlloc {
    void* (*fn_alloc)(size_t, void*, void*) = nullptr;
    void (*fn_free)(void*, size_t, void*, void*) = nullptr;
    void* user = nullptr;
    std::atomic<uint64_t> live_bytes{0};

    void* get(size_t bytes, cudaStream_t st) {
        if (bytes == 0) bytes = 256;
        bytes = (bytes + 255) & ~size_t(255);
        void* p = nullptr;
        if (fn_alloc) {
            p = fn_alloc(bytes, (void*)st, user);
            if (!p) throw Error(DG_E_NOMEM, "device allocation failed (caller allocator)");
        } else {
            cudaError_t e = cudaMallocAsync(&p, bytes, st);
            if (e != cudaSuccess) {
                cudaGetLastError();
                throw Error(DG_E_NOMEM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
            }
        }
        live_bytes += bytes;
        return p;
    }
    void put(void* p, size_t bytes, cudaStream_t st) {
        if (!p) return;
        if (bytes == 0) bytes = 256;
        bytes = (bytes + 255) & ~size_t(255);
        if (fn_free) fn_free(p, bytes, (void*)st, user);
        else cudaFreeAsync(p, st);
        live_bytes -= bytes;
    }
};

// A typed device buffer that grows on demand (contents not preserved).
template <typename T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;  // elements
    void ensure(DevAlloc& a, size_t want, cudaStream_t st) {
        if (want <= n && p) return;
        size_t nn = want < 16 ? 16 : want;
        if (p) a.put(p, n * sizeof(T), st);
        p = static_cast<T*>(a.get(nn * sizeof(T), st));
        n = nn;
    }
    void release(DevAlloc& a, cudaStream_t st) {
        if (p) a.put(p, n * sizeof(T), st);
        p = nullptr;
        n = 0;
    }
    size_t bytes() const { return n * sizeof(T); }
};

}  // namespace dg
