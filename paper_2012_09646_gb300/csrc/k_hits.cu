// HITS nodes (Section IV-B, HITS: hubs and authorities by repeated sparse
// matrix-vector products with a matrix and its transpose).
//   spmv_partition  split points of the merge path of a CSR matrix
//   spmv_csr        y = A x for CSR A (the transpose is passed as its own CSR)
//   l2norm          norm[0] = ||x||_2
//   scale           x := x / norm[0]  (unchanged if norm is 0)
//
// spmv_csr balances power-law rows (one row may hold ~1e6 nonzeros) with
// the merge-path decomposition of Merrill and Garland ("Merge-based parallel
// sparse matrix-vector multiplication", SC 2016), restated here: the
// sequence that merges the n row ends with the nnz nonzeros is cut into
// tiles of equal length (kSpmvTile items), so every block does the same work
// whatever the row lengths.  A block stages its tile's products
// val[j] * x[col[j]] and row ends in shared memory; each thread walks
// kSpmvIpt items, finishing rows and carrying a partial sum; a block-wide
// segmented scan (fixed tree order) hands each thread the partial of the row
// it starts in; rows that cross tiles get the tiles' carries added by a
// second kernel, one warp per row, in tile order.  No atomics: the result is
// the same on every run.  Bytes per product: 4 (col) + 4 (val) + 4 (x
// gather), plus 4 per row for rowptr and 4 for y.
#include <climits>
#include <initializer_list>
#include <vector>

#include "catalog.h"
#include "kcommon.cuh"

namespace gdag {

constexpr int kSpmvThreads = 256;
constexpr int kSpmvIpt = 7;
constexpr int kSpmvTile = kSpmvThreads * kSpmvIpt;

inline int64_t spmv_tiles(int64_t nrows, int64_t nnz) { return ceil_div(nrows + nnz > 0 ? nrows + nnz : 1, kSpmvTile); }

// part[b] = (rows, nonzeros) consumed before merge-path diagonal b * tile:
// the first i with rowptr[i+1] > d - i - 1, i.e. row end i is not yet
// consumed while nonzero d - i is.
__global__ void spmv_partition_kernel(const int *__restrict__ rowptr, int2 *__restrict__ part, int nrows, int nnz,
                                      int tiles)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > tiles) return;
    const int64_t total = (int64_t)nrows + nnz;
    int64_t d = (int64_t)b * kSpmvTile;
    if (d > total) d = total;
    int64_t lo = d - nnz > 0 ? d - nnz : 0, hi = d < nrows ? d : nrows;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((int64_t)rowptr[mid + 1] <= d - mid - 1)
            lo = mid + 1;
        else
            hi = mid;
    }
    part[b] = make_int2((int)lo, (int)(d - lo));
}

struct KeyVal {
    int k;
    float v;
};

// op((ka, va), (kb, vb)) = (kb, ka == kb ? va + vb : vb): sums within runs
// of equal keys; associative, so a scan tree of any shape is exact in keys
// and fixed in summation order.
__device__ __forceinline__ KeyVal kv_op(KeyVal a, KeyVal b) { return KeyVal{b.k, a.k == b.k ? a.v + b.v : b.v}; }

__global__ void __launch_bounds__(kSpmvThreads) spmv_merge_kernel(const int *__restrict__ rowptr,
                                                                  const int *__restrict__ col,
                                                                  const float *__restrict__ val,
                                                                  const float *__restrict__ x,
                                                                  const int2 *__restrict__ part, float *__restrict__ y,
                                                                  float *__restrict__ carry, int nrows)
{
    __shared__ int s_end[kSpmvTile + 1];
    __shared__ float s_prod[kSpmvTile];
    __shared__ KeyVal s_warp[kSpmvThreads / 32];
    const int b = blockIdx.x;
    const int2 p0 = part[b], p1 = part[b + 1];
    const int i0 = p0.x, j0 = p0.y;
    const int tile_rows = p1.x - i0, tile_nnz = p1.y - j0;
    for (int t = threadIdx.x; t <= tile_rows; t += kSpmvThreads) {
        const int r = i0 + t;
        s_end[t] = r < nrows ? __ldcs(rowptr + r + 1) - j0 : INT_MAX;
    }
    // col and val are streamed once (evict-first), x is gathered through L2
    for (int t = threadIdx.x; t < tile_nnz; t += kSpmvThreads) {
        const int j = j0 + t;
        s_prod[t] = __ldcs(val + j) * __ldg(x + __ldcs(col + j));
    }
    __syncthreads();

    // this thread's start on the tile's merge path
    const int tile_len = tile_rows + tile_nnz;
    const int d = min((int)threadIdx.x * kSpmvIpt, tile_len);
    int lo = max(0, d - tile_nnz), hi = min(d, tile_rows);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (s_end[mid] <= d - mid - 1)
            lo = mid + 1;
        else
            hi = mid;
    }
    int i = lo, j = d - lo;
    const int steps = min(kSpmvIpt, tile_len - d);
    float running = 0.f;
    int first_row = -1;  // the first row this thread finishes takes the carry-in
    float first_val = 0.f;
#pragma unroll
    for (int s = 0; s < kSpmvIpt; ++s) {
        if (s < steps) {
            if (j < s_end[i]) {
                running += s_prod[j];
                ++j;
            } else {
                if (first_row < 0) {
                    first_row = i;
                    first_val = running;
                } else {
                    y[i0 + i] = running;
                }
                running = 0.f;
                ++i;
            }
        }
    }

    // block-wide inclusive segmented scan of (row at the thread's end,
    // partial sum of that row)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    KeyVal kv{i, running};
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        KeyVal up{__shfl_up_sync(0xffffffffu, kv.k, o), __shfl_up_sync(0xffffffffu, kv.v, o)};
        if (lane >= o) kv = kv_op(up, kv);
    }
    if (lane == 31) s_warp[warp] = kv;
    __syncthreads();
    if (warp == 0) {
        KeyVal w = lane < kSpmvThreads / 32 ? s_warp[lane] : KeyVal{INT_MAX, 0.f};
#pragma unroll
        for (int o = 1; o < kSpmvThreads / 32; o <<= 1) {
            KeyVal up{__shfl_up_sync(0xffffffffu, w.k, o), __shfl_up_sync(0xffffffffu, w.v, o)};
            if (lane >= o) w = kv_op(up, w);
        }
        if (lane < kSpmvThreads / 32) s_warp[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    if (warp > 0) kv = kv_op(s_warp[warp - 1], kv);
    // exclusive value for this thread: the previous thread's inclusive
    KeyVal ex{__shfl_up_sync(0xffffffffu, kv.k, 1), __shfl_up_sync(0xffffffffu, kv.v, 1)};
    if (lane == 0) ex = warp > 0 ? s_warp[warp - 1] : KeyVal{-1, 0.f};
    const float carry_in = (ex.k == lo) ? ex.v : 0.f;
    if (first_row >= 0) y[i0 + first_row] = first_val + carry_in;
    if (threadIdx.x == kSpmvThreads - 1) carry[b] = kv.v;  // partial of the row crossing into tile b + 1
}

// Rows crossing tiles: tile b carries row part[b+1].x into tile b + 1.  The
// warp of the first tile carrying a row adds all its carries, in tile order,
// to the value the finishing tile wrote.
__global__ void spmv_fixup_kernel(const int2 *__restrict__ part, const float *__restrict__ carry,
                                  float *__restrict__ y, int nrows, int tiles)
{
    const int lane = threadIdx.x & 31;
    const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (b >= tiles) return;
    const int r = part[b + 1].x;
    if (r >= nrows) return;
    if (b > 0 && part[b].x == r) return;  // an earlier tile starts this row's group
    float sum = 0.f;
    for (int base = b;; base += 32) {
        const int bb = base + lane;
        const bool in = bb < tiles && part[bb + 1].x == r;
        const unsigned m = __ballot_sync(0xffffffffu, in);
        if (in) sum += carry[bb];
        if (m != 0xffffffffu) break;
    }
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) y[r] = sum + y[r];
}

// norm[0] = sqrt(sum x_i^2): per thread Kahan fp32, per block fp64 tree,
// blocks combined in order by the last one to arrive.
__global__ void __launch_bounds__(kThreads) l2norm_kernel(const float *__restrict__ x, float *__restrict__ norm,
                                                          double *scratch, int64_t n)
{
    __shared__ double sh[kThreads / 32];
    Kahan acc;
    if ((reinterpret_cast<uintptr_t>(x) & 15) == 0) {
        const float4 *x4 = reinterpret_cast<const float4 *>(x);
        const int64_t n4 = n >> 2, tile = (int64_t)kThreads * kUnroll;
        for (int64_t base = (int64_t)blockIdx.x * tile; base < n4; base += (int64_t)gridDim.x * tile) {
            float4 v[kUnroll];
#pragma unroll
            for (int k = 0; k < kUnroll; ++k) {
                int64_t i = base + threadIdx.x + (int64_t)k * kThreads;
                if (i < n4) v[k] = x4[i];
            }
#pragma unroll
            for (int k = 0; k < kUnroll; ++k) {
                int64_t i = base + threadIdx.x + (int64_t)k * kThreads;
                if (i < n4) {
                    acc.add(v[k].x * v[k].x);
                    acc.add(v[k].y * v[k].y);
                    acc.add(v[k].z * v[k].z);
                    acc.add(v[k].w * v[k].w);
                }
            }
        }
        if (blockIdx.x == 0 && threadIdx.x < (n & 3)) {
            const float t = x[(n4 << 2) + threadIdx.x];
            acc.add(t * t);
        }
    } else {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
            acc.add(x[i] * x[i]);
    }
    const double bs = block_sum(acc.value(), sh);
    if (threadIdx.x == 0) scratch[blockIdx.x] = bs;
    unsigned *counter = reinterpret_cast<unsigned *>(scratch + kReduceMaxBlocks);
    if (!arrive_last(counter)) return;
    double t = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += kThreads) t += ((volatile double *)scratch)[b];
    t = block_sum(t, sh);
    if (threadIdx.x == 0) {
        norm[0] = (float)sqrt(t);
        *counter = 0u;
    }
}

// x := x / norm[0], correctly rounded; a zero norm leaves x unchanged.
__global__ void __launch_bounds__(1024) scale_kernel(float *__restrict__ x, const float *__restrict__ norm, int64_t n)
{
    const float nr = norm[0];
    if (!(nr > 0.f)) return;
    if ((reinterpret_cast<uintptr_t>(x) & 15) == 0) {
        float4 *x4 = reinterpret_cast<float4 *>(x);
        const int64_t n4 = n >> 2, bd = blockDim.x, tile = bd * kUnroll;
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
                if (i < n4)
                    x4[i] = make_float4(__fdiv_rn(v[k].x, nr), __fdiv_rn(v[k].y, nr), __fdiv_rn(v[k].z, nr),
                                        __fdiv_rn(v[k].w, nr));
            }
        }
        if (blockIdx.x == 0 && threadIdx.x < (n & 3)) {
            int64_t i = (n4 << 2) + threadIdx.x;
            x[i] = __fdiv_rn(x[i], nr);
        }
    } else {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
            x[i] = __fdiv_rn(x[i], nr);
    }
}

namespace {

const char *validate_partition(const LaunchArgs &a)
{
    const int nrows = a.i32(2), nnz = a.i32(3);
    if (nrows < 0 || nnz < 0) return "nrows and nnz must be >= 0";
    if ((int64_t)nrows + nnz > INT_MAX - kSpmvTile) return "nrows + nnz too large for int32 indexing";
    if (a.bytes[0] / 4 < (size_t)nrows + 1) return "rowptr smaller than nrows + 1 int32";
    if (a.bytes[1] < (size_t)(spmv_tiles(nrows, nnz) + 1) * 8) return "part smaller than gdag_scratch_bytes()";
    return nullptr;
}

int launch_partition(const LaunchArgs &a, void *s)
{
    const int nrows = a.i32(2), nnz = a.i32(3);
    const int tiles = (int)spmv_tiles(nrows, nnz);
    spmv_partition_kernel<<<(unsigned)ceil_div(tiles + 1, 256), 256, 0, (cudaStream_t)s>>>(
        a.p<int>(0), a.p<int2>(1), nrows, nnz, tiles);
    return cudaGetLastError();
}

const char *validate_spmv(const LaunchArgs &a)
{
    const int nrows = a.i32(7), nnz = a.i32(8);
    if (nrows < 0 || nnz < 0) return "nrows and nnz must be >= 0";
    if ((int64_t)nrows + nnz > INT_MAX - kSpmvTile) return "nrows + nnz too large for int32 indexing";
    const int64_t tiles = spmv_tiles(nrows, nnz);
    if (a.bytes[0] / 4 < (size_t)nrows + 1) return "rowptr smaller than nrows + 1 int32";
    if (a.bytes[1] / 4 < (size_t)nnz || a.bytes[2] / 4 < (size_t)nnz) return "col or val smaller than nnz";
    if (a.bytes[4] < (size_t)(tiles + 1) * 8) return "part smaller than gdag_scratch_bytes(\"spmv_partition\")";
    if (a.bytes[5] / 4 < (size_t)nrows) return "y smaller than nrows floats";
    if (a.bytes[3] / 4 < (size_t)nrows) return "x smaller than nrows floats (square matrices)";
    if (a.bytes[6] < (size_t)tiles * 4) return "carry smaller than gdag_scratch_bytes(\"spmv_csr\")";
    return nullptr;
}

int launch_spmv(const LaunchArgs &a, void *sv)
{
    cudaStream_t s = (cudaStream_t)sv;
    const int nrows = a.i32(7), nnz = a.i32(8);
    if (nrows == 0) return cudaSuccess;
    const int tiles = (int)spmv_tiles(nrows, nnz);
    spmv_merge_kernel<<<tiles, kSpmvThreads, 0, s>>>(a.p<int>(0), a.p<int>(1), a.p<float>(2), a.p<float>(3),
                                                     a.p<int2>(4), a.p<float>(5), a.p<float>(6), nrows);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    spmv_fixup_kernel<<<(unsigned)ceil_div((int64_t)tiles * 32, 256), 256, 0, s>>>(a.p<int2>(4), a.p<float>(6),
                                                                                   a.p<float>(5), nrows, tiles);
    return cudaGetLastError();
}

const char *validate_l2norm(const LaunchArgs &a)
{
    const int64_t n = a.i64(3);
    if (n < 0) return "n < 0";
    if (a.bytes[0] / 4 < (size_t)n) return "x smaller than n floats";
    if (a.bytes[1] < 4) return "norm smaller than one float";
    if (a.bytes[2] < reduce_scratch_bytes<1>()) return "scratch smaller than gdag_scratch_bytes()";
    return nullptr;
}

int launch_l2norm(const LaunchArgs &a, void *s)
{
    const int64_t n = a.i64(3);
    l2norm_kernel<<<reduce_grid(n >> 2), kThreads, 0, (cudaStream_t)s>>>(a.p<float>(0), a.p<float>(1),
                                                                         a.p<double>(2), n);
    return cudaGetLastError();
}

const char *validate_scale(const LaunchArgs &a)
{
    const int64_t n = a.i64(2);
    if (n < 0) return "n < 0";
    if (a.bytes[0] / 4 < (size_t)n) return "x smaller than n floats";
    if (a.bytes[1] < 4) return "norm smaller than one float";
    return nullptr;
}

int launch_scale(const LaunchArgs &a, void *s)
{
    const int64_t n = a.i64(2);
    if (n == 0) return cudaSuccess;
    scale_kernel<<<stream_grid(n >> 2), kThreads, 0, (cudaStream_t)s>>>(a.p<float>(0), a.p<float>(1), n);
    return cudaGetLastError();
}

KernelEntry entry(const char *name, const void *fn, std::initializer_list<gdag_argspec> spec, ValidateFn v,
                  LauncherFn l)
{
    KernelEntry e;
    e.name = name;
    e.fn = fn;
    e.nargs = (int)spec.size();
    int i = 0;
    for (const auto &sp : spec) e.spec[i++] = sp;
    e.validate = v;
    e.launcher = l;
    return e;
}

}  // namespace

size_t spmv_part_bytes(int64_t rows_plus_nnz) { return (size_t)(ceil_div(rows_plus_nnz > 0 ? rows_plus_nnz : 1, kSpmvTile) + 1) * 8; }
size_t spmv_carry_bytes(int64_t rows_plus_nnz) { return (size_t)ceil_div(rows_plus_nnz > 0 ? rows_plus_nnz : 1, kSpmvTile) * 4 + 16; }

void append_hits_kernels(std::vector<KernelEntry> &v)
{
    v.push_back(entry("spmv_partition", (const void *)spmv_partition_kernel,
                      {arr(GDAG_MODE_IN), arr(GDAG_MODE_OUT), scal(4), scal(4)}, validate_partition,
                      launch_partition));
    v.push_back(entry("spmv_csr", (const void *)spmv_merge_kernel,
                      {arr(GDAG_MODE_IN), arr(GDAG_MODE_IN), arr(GDAG_MODE_IN), arr(GDAG_MODE_IN), arr(GDAG_MODE_IN),
                       arr(GDAG_MODE_OUT), arr(GDAG_MODE_INOUT), scal(4), scal(4)},
                      validate_spmv, launch_spmv));
    v.push_back(entry("l2norm", (const void *)l2norm_kernel,
                      {arr(GDAG_MODE_IN), arr(GDAG_MODE_OUT), arr(GDAG_MODE_INOUT), scal(8)}, validate_l2norm,
                      launch_l2norm));
    v.push_back(entry("scale", (const void *)scale_kernel, {arr(GDAG_MODE_INOUT), arr(GDAG_MODE_IN), scal(8)},
                      validate_scale, launch_scale));
}

}  // namespace gdag
