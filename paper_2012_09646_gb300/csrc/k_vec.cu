// VEC nodes (Section IV-B, VEC): in-place square and the reduction of the
// difference of the two squared vectors.
#include <vector>

#include "catalog.h"
#include "kcommon.cuh"

namespace gdag {

// x := x * x.  HBM-bound: 8 bytes per element.  128-bit loads/stores when x is
// 16-byte aligned, kUnroll float4 in flight per thread.
__global__ void __launch_bounds__(1024) vec_square_kernel(float *__restrict__ x, int64_t n)
{
    if ((reinterpret_cast<uintptr_t>(x) & 15) == 0) {
        float4 *x4 = reinterpret_cast<float4 *>(x);
        const int64_t n4 = n >> 2;
        const int64_t bd = blockDim.x;
        const int64_t tile = bd * kUnroll;
        for (int64_t base = (int64_t)blockIdx.x * tile; base < n4; base += (int64_t)gridDim.x * tile) {
            float4 v[kUnroll];
#pragma unroll
            for (int k = 0; k < kUnroll; ++k) {
                int64_t i = base + threadIdx.x + k * bd;
                if (i < n4) v[k] = x4[i];
            }
#pragma unroll
            for (int k = 0; k < kUnroll; ++k) {
                int64_t i = base + threadIdx.x + k * bd;
                if (i < n4) {
                    v[k].x *= v[k].x;
                    v[k].y *= v[k].y;
                    v[k].z *= v[k].z;
                    v[k].w *= v[k].w;
                    x4[i] = v[k];
                }
            }
        }
        if (blockIdx.x == 0 && threadIdx.x < (n & 3)) {
            int64_t i = (n4 << 2) + threadIdx.x;
            x[i] = x[i] * x[i];
        }
    } else {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
            x[i] = x[i] * x[i];
    }
}

// z[0] = sum_i (x_i - y_i).  Per thread: Kahan-compensated fp32; per block:
// fp64 tree; blocks combined in block order by the last block to arrive.
// scratch: kReduceMaxBlocks doubles + arrival counter (zero on entry, reset
// to zero on exit).
__global__ void __launch_bounds__(kThreads) vec_reduce_diff_kernel(const float *__restrict__ x,
                                                                    const float *__restrict__ y,
                                                                    float *__restrict__ z, double *scratch,
                                                                    int64_t n)
{
    __shared__ double sh[kThreads / 32];
    Kahan acc;
    const bool aligned = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15) == 0;
    if (aligned) {
        const float4 *x4 = reinterpret_cast<const float4 *>(x);
        const float4 *y4 = reinterpret_cast<const float4 *>(y);
        const int64_t n4 = n >> 2;
        const int64_t tile = (int64_t)kThreads * kUnroll;
        for (int64_t base = (int64_t)blockIdx.x * tile; base < n4; base += (int64_t)gridDim.x * tile) {
            float4 a[kUnroll], b[kUnroll];
#pragma unroll
            for (int k = 0; k < kUnroll; ++k) {
                int64_t i = base + threadIdx.x + (int64_t)k * kThreads;
                if (i < n4) {
                    a[k] = x4[i];
                    b[k] = y4[i];
                }
            }
#pragma unroll
            for (int k = 0; k < kUnroll; ++k) {
                int64_t i = base + threadIdx.x + (int64_t)k * kThreads;
                if (i < n4) {
                    acc.add(a[k].x - b[k].x);
                    acc.add(a[k].y - b[k].y);
                    acc.add(a[k].z - b[k].z);
                    acc.add(a[k].w - b[k].w);
                }
            }
        }
        if (blockIdx.x == 0 && threadIdx.x < (n & 3)) {
            int64_t i = (n4 << 2) + threadIdx.x;
            acc.add(x[i] - y[i]);
        }
    } else {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
            acc.add(x[i] - y[i]);
    }
    double bs = block_sum(acc.value(), sh);
    if (threadIdx.x == 0) scratch[blockIdx.x] = bs;
    unsigned *counter = reinterpret_cast<unsigned *>(scratch + kReduceMaxBlocks);
    if (!arrive_last(counter)) return;
    double t = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += kThreads) t += ((volatile double *)scratch)[b];
    t = block_sum(t, sh);
    if (threadIdx.x == 0) {
        z[0] = (float)t;
        *counter = 0u;
    }
}

namespace {

const char *validate_square(const LaunchArgs &a)
{
    int64_t n = a.i64(1);
    if (n < 0) return "n < 0";
    if (a.bytes[0] / 4 < (size_t)n) return "x smaller than n floats";
    return nullptr;
}

int launch_square(const LaunchArgs &a, void *s)
{
    int64_t n = a.i64(1);
    if (n == 0) return cudaSuccess;
    unsigned g = a.auto_cfg ? stream_grid(n >> 2) : a.grid[0];
    unsigned b = a.auto_cfg ? kThreads : a.block[0];
    vec_square_kernel<<<g, b, 0, (cudaStream_t)s>>>(a.p<float>(0), n);
    return cudaGetLastError();
}

const char *validate_reduce_diff(const LaunchArgs &a)
{
    int64_t n = a.i64(4);
    if (n < 0) return "n < 0";
    if (a.bytes[0] / 4 < (size_t)n || a.bytes[1] / 4 < (size_t)n) return "x or y smaller than n floats";
    if (a.bytes[2] < 4) return "z smaller than one float";
    if (a.bytes[3] < reduce_scratch_bytes<1>()) return "scratch smaller than gdag_scratch_bytes()";
    if (!a.auto_cfg && (a.grid[0] > (unsigned)kReduceMaxBlocks || a.block[0] != kThreads))
        return "explicit grid must be <= 1024 blocks of 256 threads";
    return nullptr;
}

int launch_reduce_diff(const LaunchArgs &a, void *s)
{
    int64_t n = a.i64(4);
    unsigned g = a.auto_cfg ? reduce_grid(n >> 2) : a.grid[0];
    vec_reduce_diff_kernel<<<g, kThreads, 0, (cudaStream_t)s>>>(a.p<float>(0), a.p<float>(1), a.p<float>(2),
                                                                 a.p<double>(3), n);
    return cudaGetLastError();
}

}  // namespace

void append_vec_kernels(std::vector<KernelEntry> &v)
{
    KernelEntry e;
    e.name = "vec_square";
    e.fn = (const void *)vec_square_kernel;
    e.nargs = 2;
    e.spec[0] = arr(GDAG_MODE_INOUT);
    e.spec[1] = scal(8);
    e.validate = validate_square;
    e.launcher = launch_square;
    v.push_back(e);

    KernelEntry r;
    r.name = "vec_reduce_diff";
    r.fn = (const void *)vec_reduce_diff_kernel;
    r.nargs = 5;
    r.spec[0] = arr(GDAG_MODE_IN);
    r.spec[1] = arr(GDAG_MODE_IN);
    r.spec[2] = arr(GDAG_MODE_OUT);
    r.spec[3] = arr(GDAG_MODE_INOUT);
    r.spec[4] = scal(8);
    r.validate = validate_reduce_diff;
    r.launcher = launch_reduce_diff;
    v.push_back(r);
}

}  // namespace gdag
