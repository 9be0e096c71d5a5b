// search_noalloc.cu -- a search entry point that allocates no memory.
//
// Some callers cannot allocate device memory at the moment they search:
// code that runs where the device allocator is off limits (a host
// application that has reserved all GPU memory up front for its own pool,
// a latency-critical thread that must not take the allocator's locks or
// risk an out-of-memory error mid-request, a plugin whose host forbids
// allocations after start-up).  sqg_search_noalloc serves them: its scratch
// is one fixed, file-scope device array, so the call itself performs no
// cudaMalloc, cudaFree or stream-ordered allocation.
//
// When the array's memory is committed: the library is built without
// relocatable device code and CUDA loads a module's device code lazily, so
// the 32 MiB are committed on a device when this file's module is first
// loaded there -- by the set-up inside the first sqg_search_noalloc call on
// that device (cudaGetSymbolAddress), not when the library is opened.  A
// caller that means to reserve the rest of the GPU for its own pool makes
// that first call beforehand (a call with nq = 0 does the set-up and
// nothing else), and before any stream capture.  The address found there
// is cached per device ordinal for the life of the process; after a
// cudaDeviceReset of that device it no longer points at the array and the
// entry point must not be called again in that process.
//
// The array is shared by every call in the process on a given GPU and
// keeps whatever the previous call left in it; the search clears what must
// start at zero (the work-queue head, the visited tables before they are
// used) and overwrites the rest before reading it.  Two calls whose work
// overlaps on the same GPU would use the same array at once and race:
// serialize them (one stream, or events).
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/sqg.h"

namespace {

constexpr size_t kScratchBytes = (size_t)32 << 20;  // 32 MiB on every GPU that loads the library
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char sqg_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void *g_scratch[kMaxDevices] = {};

// The device address of the array on `device` (looked up once per device,
// with that device current).
int scratch_on(int device, void **out) {
    if (device < 0 || device >= kMaxDevices) return SQG_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch[device]) {
        int prev = -1;
        if (cudaGetDevice(&prev) != cudaSuccess) return SQG_ERR_CUDA;
        if (prev != device && cudaSetDevice(device) != cudaSuccess) return SQG_ERR_CUDA;
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, sqg_noalloc_scratch);
        if (prev != device) cudaSetDevice(prev);
        if (e != cudaSuccess || !p) return SQG_ERR_CUDA;
        g_scratch[device] = p;
    }
    *out = g_scratch[device];
    return SQG_OK;
}

}  // namespace

extern "C" size_t sqg_noalloc_scratch_bytes(void) { return kScratchBytes; }

extern "C" int sqg_search_noalloc(const sqg_index *ix, const float *queries, int nq, const int32_t *k,
                                  const int32_t *ef, int max_k, int max_ef, uint32_t *out_ids, float *out_dists,
                                  sqg_stream_t stream) {
    if (!ix || nq < 0 || max_k < 1 || max_k > SQG_MAX_K || max_ef < max_k || max_ef > SQG_MAX_EF)
        return SQG_ERR_INVALID_ARG;
    sqg_info info;
    if (sqg_index_info(ix, &info) != SQG_OK) return SQG_ERR_INVALID_ARG;
    const size_t need = sqg_workspace_size(ix, nq, max_k, max_ef);
    if (need == 0) return SQG_ERR_INVALID_ARG;
    if (need > kScratchBytes) return SQG_ERR_CAPACITY;  // batch too large for the fixed scratch
    void *scratch = nullptr;
    const int rc = scratch_on(info.device, &scratch);  // the set-up, also for nq = 0
    if (rc != SQG_OK || nq == 0) return rc;
    sqg_search_params p;
    std::memset(&p, 0, sizeof(p));
    p.multi_estimate = 1;
    p.stop_every = 1;
    p.max_k = max_k;
    p.max_ef = max_ef;
    return sqg_search_ex(ix, queries, nq, k, ef, out_ids, out_dists, &p, scratch, kScratchBytes, nullptr, stream);
}
