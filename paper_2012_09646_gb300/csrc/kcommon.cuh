// Helpers shared by the built-in kernels: launch sizing for 152-SM GB300,
// deterministic block reductions, the last-block-done combine.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "gdag.h"

namespace gdag {

// Multiprocessor count of the current device (queried once per process).
inline int sm_count()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
    }
    return n;
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Members per fused launch (the kernel-parameter table's capacity), and the
// smaller table used for groups that fit it (a smaller parameter block).
constexpr int kFuseTable = GDAG_FUSED_TABLE;
constexpr int kFuseSmall = 32;

// Persistent grid for a fused launch of `threads`-thread blocks: resident
// blocks of kernel `fn` per SM (queried once, into `per_sm`) x SMs, at most
// `items`.
inline unsigned fused_grid(const void *fn, int threads, int64_t items, int &per_sm)
{
    if (per_sm < 1 && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, 0) != cudaSuccess ||
                       per_sm < 1))
        per_sm = 1;
    const int64_t wave = (int64_t)sm_count() * per_sm;
    return (unsigned)(items < wave ? items : wave);
}

// Streaming kernels: each block handles tiles of kThreads x kUnroll float4
// and grid-strides over tiles.  The grid is capped at kBlocksPerSm blocks per
// SM, so for most sizes a block handles about one tile and the hardware's
// block scheduler balances the tail.
constexpr int kThreads = 256;
constexpr int kUnroll = 4;
constexpr int kBlocksPerSm = 32;

inline unsigned stream_grid(int64_t n_vec4)
{
    int64_t tiles = ceil_div(n_vec4 > 0 ? n_vec4 : 1, (int64_t)kThreads * kUnroll);
    int64_t cap = (int64_t)sm_count() * kBlocksPerSm;
    return (unsigned)(tiles < cap ? tiles : cap);
}

// Reductions: a fixed grid that depends only on n and the SM count, so the
// summation order (and the result) is the same on every run.
constexpr int kReduceMaxBlocks = 1024;

inline unsigned reduce_grid(int64_t n_vec4)
{
    int64_t tiles = ceil_div(n_vec4 > 0 ? n_vec4 : 1, (int64_t)kThreads * kUnroll);
    int64_t cap = (int64_t)sm_count() * 6;  // enough bytes in flight per SM
    if (cap > kReduceMaxBlocks) cap = kReduceMaxBlocks;
    return (unsigned)(tiles < cap ? tiles : cap);
}

// Scratch of one reduction: kReduceMaxBlocks partials of `Width` doubles,
// then a 32-bit arrival counter (zero between launches).
template <int Width> constexpr size_t reduce_scratch_bytes()
{
    return sizeof(double) * Width * kReduceMaxBlocks + 16;
}

#ifdef __CUDACC__
// One block of `threads` threads of `kernel` on stream s, launched as a
// programmatic dependent of the kernel before it on s: it may become
// resident while that kernel runs (once every block of it has executed
// griddepcontrol.launch_dependents) and must execute griddepcontrol.wait,
// which returns when that kernel has completed and its writes are visible,
// before it reads anything that kernel wrote.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_dependent(void (*kernel)(KArgs...), int threads, cudaStream_t s, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_min(float v)
{
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Sum of v over the block (blockDim.x == kThreads), fixed order; valid in
// thread 0.  `sh` holds kThreads/32 doubles.
__device__ __forceinline__ double block_sum(double v, double *sh)
{
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = (lane < kThreads / 32) ? sh[lane] : 0.0;
        s = warp_sum(s);
    }
    __syncthreads();
    return s;
}

// Last-block-done: each block publishes its partial(s), then one arrival
// counter tells the last block to combine all partials in block order.
// Returns true in the block that arrived last (all threads).
// `blocks` is the number of (virtual) blocks that publish partials.
__device__ __forceinline__ bool arrive_last(unsigned *counter, unsigned blocks)
{
    __shared__ bool last;
    __threadfence();  // partials visible device-wide before arrival
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned prev = atomicAdd(counter, 1u);
        last = (prev == blocks - 1);
    }
    __syncthreads();
    if (last) __threadfence();  // see every other block's partials
    return last;
}
__device__ __forceinline__ bool arrive_last(unsigned *counter) { return arrive_last(counter, gridDim.x); }

// Fused launches: member m of a table owns the work items
// [start[m], start[m+1]); returns the member of item `it` (the largest m with
// start[m] <= it).  Uniform across a block, so the loads are broadcasts.
__device__ __forceinline__ int fused_member(const int64_t *start, int count, int64_t it)
{
    int lo = 0, hi = count;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (start[mid] <= it) lo = mid;
        else hi = mid;
    }
    return lo;
}

// x / d rounded to nearest, given r = RN(1/d): Markstein's correction
// (P. Markstein, "Computation of elementary functions on the IBM RISC
// System/6000 processor", IBM J. Res. Dev. 34(1), 1990): q = RN(x r) is
// within an ulp of x/d, the residual x - q d is exact under FMA, and one step
// q + (x - q d) r rounds to the correctly rounded quotient for normal
// operands and results.  Three instructions per element instead of a full
// division; r comes from (float)(1.0 / (double)d), which is RN(1/d) because
// rounding the correctly rounded double quotient to float cannot double-round
// (53 >= 2 * 24 + 2).
__device__ __forceinline__ float div_by(float x, float d, float r)
{
    const float q = x * r;
    const float e = fmaf(-q, d, x);
    return fmaf(e, r, q);
}

// Kahan-compensated fp32 accumulation: per-thread sums stay accurate to a
// few ulp however many elements a thread visits.
struct Kahan {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v)
    {
        float y = v - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};
#endif

}  // namespace gdag
