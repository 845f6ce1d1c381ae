// A reduction entry point for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at all: plug-ins whose host application
// owns every device allocation, processes whose device memory is budgeted by
// an allocator they must not bypass, and latency-critical loops that cannot
// afford cudaMalloc/cudaFree (which may synchronize the device) on their
// path.  gdag_vec_reduce_diff_noalloc() serves them:
// the caller passes only inputs and the output, and the kernel's scratch (the
// per-block partial sums and the arrival counter of the last-block-done
// combine) lives in one file-scope __device__ array that every GPU loading
// this library holds until the process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "gdag.h"
#include "kcommon.cuh"

namespace gdag {

// The existing reduction kernel (k_vec.cu), launched unchanged.
__global__ void vec_reduce_diff_kernel(const float *__restrict__ x, const float *__restrict__ y,
                                       float *__restrict__ z, double *scratch, int64_t n);

namespace {

constexpr size_t kNoallocBytes = GDAG_NOALLOC_SCRATCH_BYTES;
static_assert(kNoallocBytes >= reduce_scratch_bytes<1>(), "static scratch too small for the reduction");

// One copy per device.  In host code this name is only a host-side stand-in:
// the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices];  // device address of g_noalloc_scratch, per device

// Set-up, once per device, with that device current: look up the array's
// device address.  Nothing is written to the array here: the partial sums are
// written by every launch before they are read, and the arrival counter is
// cleared on the caller's stream by every call, so no work is issued outside
// the caller's stream (a memset on the legacy default stream would not be
// ordered before a non-blocking caller stream).
int scratch_for_current_device(double **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GDAG_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return GDAG_ERR_CUDA;
        }
        g_addr[dev] = p;
    }
    *out = static_cast<double *>(g_addr[dev]);
    return GDAG_OK;
}

}  // namespace
}  // namespace gdag

extern "C" int gdag_vec_reduce_diff_noalloc(const void *dev_x, const void *dev_y, void *dev_z, int64_t n,
                                            void *stream)
{
    using namespace gdag;
    if (n < 0 || (n > 0 && (!dev_x || !dev_y)) || !dev_z) return GDAG_ERR_INVALID;
    // reduce_grid() caps the grid at kReduceMaxBlocks, and the static_assert
    // above makes the array hold that many partial sums plus the counter, so
    // no n can need more scratch than the array has.
    const unsigned grid = reduce_grid(n >> 2);
    double *scratch = nullptr;
    int r = scratch_for_current_device(&scratch);
    if (r) return r;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the arrival counter must start at zero on every call
    unsigned *counter = reinterpret_cast<unsigned *>(scratch + kReduceMaxBlocks);
    if (cudaMemsetAsync(counter, 0, sizeof(unsigned), s) != cudaSuccess) {
        (void)cudaGetLastError();
        return GDAG_ERR_CUDA;
    }
    vec_reduce_diff_kernel<<<grid, kThreads, 0, s>>>(static_cast<const float *>(dev_x),
                                                     static_cast<const float *>(dev_y), static_cast<float *>(dev_z),
                                                     scratch, n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return GDAG_ERR_CUDA;
    return GDAG_OK;
}
