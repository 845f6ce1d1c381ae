// VEC nodes (Section IV-B, VEC): in-place square and the reduction of the
// difference of the two squared vectors.
#include <vector>

#include "catalog.h"
#include "kcommon.cuh"

namespace gdag {

// x := x * x.  HBM-bound: 8 bytes per element.  128-bit loads/stores when x is
// 16-byte aligned, kUnroll float4 in flight per thread.
// One tile: float4s [base, base + kThreads*kUnroll) of x4 below n4
// (blockDim.x == kThreads for the fused form; the plain kernel passes its
// own block size).
__device__ __forceinline__ void square_tile(float4 *x4, int64_t n4, int64_t base, int64_t bd)
{
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

__global__ void __launch_bounds__(1024) vec_square_kernel(float *__restrict__ x, int64_t n)
{
    if ((reinterpret_cast<uintptr_t>(x) & 15) == 0) {
        float4 *x4 = reinterpret_cast<float4 *>(x);
        const int64_t n4 = n >> 2;
        const int64_t bd = blockDim.x;
        const int64_t tile = bd * kUnroll;
        for (int64_t base = (int64_t)blockIdx.x * tile; base < n4; base += (int64_t)gridDim.x * tile)
            square_tile(x4, n4, base, bd);
        if (blockIdx.x == 0 && threadIdx.x < (n & 3)) {
            int64_t i = (n4 << 2) + threadIdx.x;
            x[i] = x[i] * x[i];
        }
    } else {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
            x[i] = x[i] * x[i];
    }
}

// Fused form: the work items are tiles of kThreads*kUnroll float4s
// (kFuseElems floats); member m owns tiles [start[m], start[m+1]), its last
// tile also squaring the n & 3 scalar tail.  One persistent grid walks all
// tiles of all members.
constexpr int64_t kFuseElems = (int64_t)kThreads * kUnroll * 4;

template <int CAP> struct SquareFused {
    int count;
    int64_t start[CAP + 1];
    float *x[CAP];
    int64_t n[CAP];
};

template <int CAP>
__global__ void __launch_bounds__(kThreads) vec_square_fused_kernel(const __grid_constant__ SquareFused<CAP> t)
{
    // one contiguous range of tiles per block; one member search per block
    const int64_t total = t.start[t.count];
    const int64_t per = (total + gridDim.x - 1) / gridDim.x;
    const int64_t it0 = (int64_t)blockIdx.x * per;
    const int64_t it1 = it0 + per < total ? it0 + per : total;
    if (it0 >= it1) return;
    int m = fused_member(t.start, t.count, it0);
    int64_t first = t.start[m], next = t.start[m + 1];
    for (int64_t it = it0; it < it1; ++it) {
        while (it >= next) {
            ++m;
            first = next;
            next = t.start[m + 1];
        }
        const int64_t local = it - first;
        const bool last = it == next - 1;
        float *x = t.x[m];
        const int64_t n = t.n[m];
        if ((reinterpret_cast<uintptr_t>(x) & 15) == 0) {
            const int64_t n4 = n >> 2;
            square_tile(reinterpret_cast<float4 *>(x), n4, local * (kThreads * kUnroll), kThreads);
            if (last && threadIdx.x < (n & 3)) {
                int64_t i = (n4 << 2) + threadIdx.x;
                x[i] = x[i] * x[i];
            }
        } else {
            const int64_t hi = (local + 1) * kFuseElems < n ? (local + 1) * kFuseElems : n;
            for (int64_t i = local * kFuseElems + threadIdx.x; i < hi; i += kThreads) x[i] = x[i] * x[i];
        }
    }
}

// z[0] = sum_i (x_i - y_i).  Per thread: Kahan-compensated fp32; per block:
// fp64 tree; blocks combined in block order by the last block to arrive.
// scratch: kReduceMaxBlocks doubles + arrival counter (zero on entry, reset
// to zero on exit).
// Block `vb` of a launch of `G` blocks of kThreads threads; the plain kernel
// passes (blockIdx.x, gridDim.x), the fused one a member's virtual block, so
// both sum the same elements in the same order.
__device__ __forceinline__ void reduce_diff_block(const float *__restrict__ x, const float *__restrict__ y,
                                                  float *__restrict__ z, double *scratch, int64_t n, int64_t vb,
                                                  int64_t G, double *sh)
{
    Kahan acc;
    const bool aligned = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15) == 0;
    if (aligned) {
        const float4 *x4 = reinterpret_cast<const float4 *>(x);
        const float4 *y4 = reinterpret_cast<const float4 *>(y);
        const int64_t n4 = n >> 2;
        const int64_t tile = (int64_t)kThreads * kUnroll;
        for (int64_t base = vb * tile; base < n4; base += G * tile) {
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
        if (vb == 0 && threadIdx.x < (n & 3)) {
            int64_t i = (n4 << 2) + threadIdx.x;
            acc.add(x[i] - y[i]);
        }
    } else {
        for (int64_t i = vb * kThreads + threadIdx.x; i < n; i += G * kThreads) acc.add(x[i] - y[i]);
    }
    double bs = block_sum(acc.value(), sh);
    if (threadIdx.x == 0) scratch[vb] = bs;
    unsigned *counter = reinterpret_cast<unsigned *>(scratch + kReduceMaxBlocks);
    if (!arrive_last(counter, (unsigned)G)) return;
    double t = 0.0;
    for (int64_t b = threadIdx.x; b < G; b += kThreads) t += ((volatile double *)scratch)[b];
    t = block_sum(t, sh);
    if (threadIdx.x == 0) {
        z[0] = (float)t;
        *counter = 0u;
    }
}

__global__ void __launch_bounds__(kThreads) vec_reduce_diff_kernel(const float *__restrict__ x,
                                                                    const float *__restrict__ y,
                                                                    float *__restrict__ z, double *scratch,
                                                                    int64_t n)
{
    __shared__ double sh[kThreads / 32];
    reduce_diff_block(x, y, z, scratch, n, blockIdx.x, gridDim.x, sh);
}

// Fused form: member m runs its own reduce_grid(n >> 2) virtual blocks
// [start[m], start[m+1]) (the grid its plain launch would use), so its sum
// is bit-identical to the plain launch's; a persistent grid walks them all.
// No block waits for another (the last arrival of a member combines), so
// any physical grid size is safe.
template <int CAP> struct ReduceDiffFused {
    int count;
    int64_t start[CAP + 1];
    const float *x[CAP];
    const float *y[CAP];
    float *z[CAP];
    double *scratch[CAP];
    int64_t n[CAP];
};

template <int CAP>
__global__ void __launch_bounds__(kThreads) vec_reduce_diff_fused_kernel(const __grid_constant__ ReduceDiffFused<CAP> t)
{
    __shared__ double sh[kThreads / 32];
    // one contiguous range of virtual blocks per block; one member search
    const int64_t total = t.start[t.count];
    const int64_t per = (total + gridDim.x - 1) / gridDim.x;
    const int64_t it0 = (int64_t)blockIdx.x * per;
    const int64_t it1 = it0 + per < total ? it0 + per : total;
    if (it0 >= it1) return;
    int m = fused_member(t.start, t.count, it0);
    int64_t first = t.start[m], next = t.start[m + 1];
    for (int64_t it = it0; it < it1; ++it) {
        while (it >= next) {
            ++m;
            first = next;
            next = t.start[m + 1];
        }
        reduce_diff_block(t.x[m], t.y[m], t.z[m], t.scratch[m], t.n[m], it - first, next - first, sh);
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

template <int CAP> int fused_square_cap(const LaunchArgs *a, int count, void *s)
{
    for (int off = 0; off < count; off += CAP) {
        SquareFused<CAP> t;
        t.count = count - off < CAP ? count - off : CAP;
        t.start[0] = 0;
        for (int m = 0; m < t.count; ++m) {
            const LaunchArgs &la = a[off + m];
            t.x[m] = la.p<float>(0);
            t.n[m] = la.i64(1);
            t.start[m + 1] = t.start[m] + ceil_div(t.n[m], kFuseElems);
        }
        const int64_t total = t.start[t.count];
        if (total == 0) continue;
        static int per_sm = 0;
        const unsigned g = fused_grid((const void *)vec_square_fused_kernel<CAP>, kThreads, total, per_sm);
        vec_square_fused_kernel<CAP><<<g, kThreads, 0, (cudaStream_t)s>>>(t);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int fused_square(const LaunchArgs *a, int count, void *s)
{
    return count <= kFuseSmall ? fused_square_cap<kFuseSmall>(a, count, s) : fused_square_cap<kFuseTable>(a, count, s);
}

template <int CAP> int fused_reduce_diff_cap(const LaunchArgs *a, int count, void *s)
{
    for (int off = 0; off < count; off += CAP) {
        ReduceDiffFused<CAP> t;
        t.count = count - off < CAP ? count - off : CAP;
        t.start[0] = 0;
        for (int m = 0; m < t.count; ++m) {
            const LaunchArgs &la = a[off + m];
            t.x[m] = la.p<float>(0);
            t.y[m] = la.p<float>(1);
            t.z[m] = la.p<float>(2);
            t.scratch[m] = la.p<double>(3);
            t.n[m] = la.i64(4);
            t.start[m + 1] = t.start[m] + reduce_grid(t.n[m] >> 2);  // n = 0 still writes z = 0
        }
        const int64_t total = t.start[t.count];
        static int per_sm = 0;
        const unsigned g = fused_grid((const void *)vec_reduce_diff_fused_kernel<CAP>, kThreads, total, per_sm);
        vec_reduce_diff_fused_kernel<CAP><<<g, kThreads, 0, (cudaStream_t)s>>>(t);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int fused_reduce_diff(const LaunchArgs *a, int count, void *s)
{
    return count <= kFuseSmall ? fused_reduce_diff_cap<kFuseSmall>(a, count, s)
                               : fused_reduce_diff_cap<kFuseTable>(a, count, s);
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
    e.fused = fused_square;
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
    r.fused = fused_reduce_diff;
    v.push_back(r);
}

}  // namespace gdag
