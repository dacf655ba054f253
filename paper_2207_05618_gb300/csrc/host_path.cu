// htex_lookup_host: filtered lookups on host buffers.  When both buffers
// are page-locked and mapped into the device's address space (and aligned
// as the kernels need), the lookup kernels read the queries and write the
// results across the CPU-GPU link directly: the filter is bound by its
// texel gathers, so reading the queries from host memory costs almost
// nothing and no staging copy is needed.  Otherwise the queries are copied
// in and the results out in chunks, each chunk on one of three
// library-owned streams in turn, so that the host-to-device copy of one
// chunk, the lookup kernel of another and the device-to-host copy of a
// third run at the same time.  The caller's stream orders the whole call:
// the internal streams wait for it on entry and it waits for them on exit.
#include <algorithm>
#include <mutex>

#include <cuda_runtime.h>

#include "htex_internal.h"

namespace {

constexpr int kStages = 3;
constexpr int64_t kChunk = int64_t(1) << 21;   // queries per chunk

// Device address of a page-locked, mapped host buffer (null for any other
// memory, which the kernels must not touch).
const void* mapped_address(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

}  // namespace

struct HostPath {
    std::mutex mu;
    cudaStream_t stream[kStages] = {};
    cudaEvent_t done[kStages] = {};
    cudaEvent_t entry = nullptr;
    void* dq[kStages] = {};
    void* dout[kStages] = {};
};

void htex_host_path_destroy(HostPath* hp) {
    if (!hp) return;
    for (int s = 0; s < kStages; ++s) {
        if (hp->stream[s]) cudaStreamSynchronize(hp->stream[s]);
        cudaFree(hp->dq[s]);
        cudaFree(hp->dout[s]);
        if (hp->done[s]) cudaEventDestroy(hp->done[s]);
        if (hp->stream[s]) cudaStreamDestroy(hp->stream[s]);
    }
    if (hp->entry) cudaEventDestroy(hp->entry);
    delete hp;
}

namespace {

htex_status make_host_path(const htex_textures* t, HostPath** out) {
    HostPath* hp = new (std::nothrow) HostPath;
    if (!hp) return HTEX_ERR_OUT_OF_MEMORY;
    bool ok = cudaEventCreateWithFlags(&hp->entry, cudaEventDisableTiming) == cudaSuccess;
    for (int s = 0; ok && s < kStages; ++s) {
        ok = cudaStreamCreateWithFlags(&hp->stream[s], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&hp->done[s], cudaEventDisableTiming) == cudaSuccess &&
             cudaMalloc(&hp->dq[s], size_t(kChunk) * sizeof(htex_query)) == cudaSuccess &&
             cudaMalloc(&hp->dout[s], size_t(kChunk) * sizeof(float) * size_t(t->C)) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        htex_host_path_destroy(hp);
        return HTEX_ERR_OUT_OF_MEMORY;
    }
    *out = hp;
    return HTEX_OK;
}

}  // namespace

extern "C" htex_status htex_lookup_host(const htex_textures* t, const htex_query* q, int64_t n, float* out,
                                        uint32_t flags, htex_stream stream, int32_t* d_status) {
    if (!t || n < 0) return HTEX_ERR_INVALID_ARG;
    if (flags & ~uint32_t(HTEX_LOOKUP_BIN | HTEX_LOOKUP_GLOBAL)) return HTEX_ERR_INVALID_ARG;
    if (n == 0) return HTEX_OK;
    if (!q || !out) return HTEX_ERR_INVALID_ARG;
    int device = -1;
    if (cudaGetDevice(&device) != cudaSuccess) return HTEX_ERR_CUDA;
    if (device != t->device) return HTEX_ERR_INVALID_ARG;
    {
        const void* mq = mapped_address(q);
        const void* mo = mapped_address(out);
        const uintptr_t out_align = t->C == 4 ? 16u : (t->C == 2 ? 8u : 4u);
        if (mq && mo && (reinterpret_cast<uintptr_t>(mq) & 15u) == 0 &&
            (reinterpret_cast<uintptr_t>(mo) & (out_align - 1)) == 0)
            // one pass in place: sorting would read the queries across the link twice more
            return htex_launch_lookup(t, static_cast<const htex_query*>(mq), n,
                                      static_cast<float*>(const_cast<void*>(mo)), flags & ~uint32_t(HTEX_LOOKUP_BIN),
                                      stream, d_status);
    }
    htex_textures* tm = const_cast<htex_textures*>(t);
    static std::mutex create_mu;
    {
        std::lock_guard<std::mutex> g(create_mu);
        if (!tm->host_path) {
            htex_status st = make_host_path(t, &tm->host_path);
            if (st != HTEX_OK) return st;
        }
    }
    HostPath* hp = tm->host_path;
    std::lock_guard<std::mutex> g(hp->mu);
    cudaStream_t caller = reinterpret_cast<cudaStream_t>(stream);
    if (cudaEventRecord(hp->entry, caller) != cudaSuccess) return HTEX_ERR_CUDA;
    for (int s = 0; s < kStages; ++s)
        if (cudaStreamWaitEvent(hp->stream[s], hp->entry, 0) != cudaSuccess) return HTEX_ERR_CUDA;
    const size_t row = sizeof(float) * size_t(t->C);
    htex_status st = HTEX_OK;
    for (int64_t k = 0, at = 0; at < n && st == HTEX_OK; ++k, at += kChunk) {
        const int s = int(k % kStages);
        const int64_t cnt = std::min<int64_t>(kChunk, n - at);
        cudaStream_t cs = hp->stream[s];
        if (cudaMemcpyAsync(hp->dq[s], q + at, size_t(cnt) * sizeof(htex_query), cudaMemcpyHostToDevice, cs) != cudaSuccess) {
            st = HTEX_ERR_CUDA;
            break;
        }
        st = htex_launch_lookup(t, static_cast<const htex_query*>(hp->dq[s]), cnt, static_cast<float*>(hp->dout[s]),
                                flags, reinterpret_cast<htex_stream>(cs), d_status);
        if (st == HTEX_OK &&
            cudaMemcpyAsync(out + at * t->C, hp->dout[s], size_t(cnt) * row, cudaMemcpyDeviceToHost, cs) != cudaSuccess)
            st = HTEX_ERR_CUDA;
    }
    for (int s = 0; s < kStages; ++s) {
        if (cudaEventRecord(hp->done[s], hp->stream[s]) != cudaSuccess ||
            cudaStreamWaitEvent(caller, hp->done[s], 0) != cudaSuccess)
            st = HTEX_ERR_CUDA;
    }
    return st;
}
