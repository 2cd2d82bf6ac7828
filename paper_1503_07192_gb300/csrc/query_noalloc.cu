// spq_query_noalloc: distance queries that allocate no memory.
//
// spq_query sorts each large batch of pairs by component pair in scratch memory that it
// allocates from the CUDA stream-ordered pool for the duration of the call.  Some
// callers cannot let a library allocate device memory on their request path: a
// serving process that has handed all free device memory to its own pool, or one that
// runs under a fixed memory budget where an allocation could fail or stall at a bad
// moment.  This entry point answers the same queries with the same kernels, but its
// scratch is one file-scope __device__ array of fixed size, created with the module on
// every GPU that loads the library and held until the process exits.
//
//   - At most SPQ_NOALLOC_MAX_PAIRS pairs per call (larger batches: call repeatedly);
//     a larger q is rejected with SPQ_EINVAL before any work is queued.
//   - pairs and dist_out must be device memory (host buffers would need device staging).
//   - The first call on a device looks up the array's device address with
//     cudaGetSymbolAddress (once per device, with that device current); make that first
//     call before any stream capture.
//   - Every call uses the same array, so calls whose work overlaps on the GPU (for
//     instance on two streams without ordering between them) race: order them on one
//     stream or with events.  Nothing in the array needs to start at zero: each call
//     writes every word it later reads (sort keys, values and histograms).
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"

namespace spq {
namespace {

constexpr int64_t kMaxPairs = SPQ_NOALLOC_MAX_PAIRS;
// 4 words per pair (keys, values and their sort copies) + one radix histogram of 256
// words per 4,096-pair tile + 4 spare words, then the grouped kernel's records (18 words
// per pair: table rows, starting values, item records, fallback list; + 8):
// query_scratch_words(kMaxPairs), about 23.1 MB.
constexpr int64_t kWords = 4 * kMaxPairs + (256 * ((kMaxPairs + 4095) / 4096) + 256) + 4 + 18 * kMaxPairs + 8;

static __device__ __align__(256) uint32_t g_noalloc_scratch[kWords];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
uint32_t* g_scratch_addr[kMaxDevices] = {};

bool device_pointer(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t scratch_address(uint32_t** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<uint32_t*>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace spq

extern "C" spq_status spq_query_noalloc(spq_handle* h, const int32_t* pairs, int64_t q, void* dist_out, void* stream) {
    using namespace spq;
    if (!h || q < 0) return SPQ_EINVAL;
    if (q == 0) return SPQ_OK;
    if (!pairs || !dist_out || q > kMaxPairs) return SPQ_EINVAL;
    // the handle's tables and this device's copy of the scratch array must be on the
    // current device
    if (!on_handle_device(h)) return SPQ_EINVAL;
    if (query_scratch_words(q) > kWords) return SPQ_EINVAL;
    if (!device_pointer(pairs) || !device_pointer(dist_out)) return SPQ_EINVAL;
    if (((uintptr_t)pairs & 7u) || ((uintptr_t)dist_out & 3u)) return SPQ_EINVAL;
    uint32_t* scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e == cudaSuccess) {
        QueryCtx<int32_t> ci;
        QueryCtx<float> cf;
        bool f32store = false, out_f32 = false;
        int32_t k = 0;
        handle_query_view(h, &ci, &cf, &f32store, &out_f32, &k);
        cudaStream_t st = (cudaStream_t)stream;
        e = f32store ? launch_query<float>(cf, pairs, q, dist_out, out_f32, (uint32_t)k, scratch, st)
                     : launch_query<int32_t>(ci, pairs, q, dist_out, out_f32, (uint32_t)k, scratch, st);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SPQ_ECUDA;
    }
    return SPQ_OK;
}
