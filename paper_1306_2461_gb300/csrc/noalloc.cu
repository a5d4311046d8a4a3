// of_compute_noalloc: the flow computation of of_compute with its workspace in a
// fixed-size static device array instead of memory from cudaMalloc.
//
// Some callers cannot allocate device memory once they are running: a real-time
// acquisition loop, where cudaMalloc/cudaFree can synchronise the whole device and
// stall the camera pipeline for milliseconds, or a host application that owns all
// device memory through its own allocator and forbids any other allocation. For them
// this entry point takes the same plan and caller buffers as of_create + of_compute,
// but runs the kernels on scratch that the library reserved when it was loaded.
//
// The scratch is one file-scope array, OF_NOALLOC_MAX_BYTES long, in device memory of
// every GPU on which the library's code is loaded, held until the process exits. All
// calls share it and it keeps whatever the last call left there; every call fully
// rewrites the pyramids and flow buffers it reads, and clears the status word.
//
// The iteration tiles run in their gathered form (OF_FLAG_GATHER): the staged form waits,
// with a time limit, for its TMA copies and reports a wait that ran out through the
// handle's status word, which a caller without a handle could not read. The gathered
// kernels wait for nothing and give the same fields.
#include <string.h>

#include <mutex>

#include "of_engine.h"
#include "of_internal.cuh"

namespace {

static __device__ __align__(256) char g_noalloc_scratch[OF_NOALLOC_MAX_BYTES];

constexpr int kMaxDevices = 256;
std::mutex g_mu;
char *g_scratch_ptr[kMaxDevices];   // device address of g_noalloc_scratch, per device

// Once per device, with that device current: the device address of the static array
// (the host-side symbol is only a stand-in and must not be passed to a kernel), and
// the kernels' shared-memory limits.
int scratch_on_current_device(char **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return OF_ECUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return OF_ECUDA;
        }
        if (of::configure_lk_kernels() != cudaSuccess) return OF_ECUDA;
        g_scratch_ptr[dev] = static_cast<char *>(ptr);
    }
    *out = g_scratch_ptr[dev];
    return OF_OK;
}

}  // namespace

extern "C" int of_compute_noalloc(const of_plan *p, const void *I1, const void *I2, float *u, float *v,
                                  of_stream_t stream)
{
    if (of_plan_validate(p) != OF_OK || !I1 || !I2 || !u || !v) return OF_EINVAL;
    of::Layout lay;
    of::layout_plan(*p, lay);
    if (lay.total > (size_t)OF_NOALLOC_MAX_BYTES) return OF_ENOMEM;
    char *ws = nullptr;
    int rc = scratch_on_current_device(&ws);
    if (rc) return rc;
    // A handle on the stack that points into the static scratch, laid out exactly as
    // of_create lays out its own workspace.
    of_ctx h;
    h.plan = *p;
    h.plan.flags |= OF_FLAG_GATHER;   // no device-side waits, so nothing to report
    h.lay = lay;
    cudaGetDevice(&h.device);
    of::assign_workspace(&h, ws);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(h.status, 0, sizeof(int), st) != cudaSuccess) return OF_ECUDA;
    return of::enqueue_pair(&h, I1, I2, u, v, 0, 1, st) == cudaSuccess ? OF_OK : OF_ECUDA;
}
