// HITS nodes (Section IV-B, HITS: hubs and authorities by repeated sparse
// matrix-vector products with a matrix and its transpose).
//   spmv_partition  split points of the merge path of a CSR matrix
//   spmv_csr        y = A x for CSR A (the transpose is passed as its own CSR)
//   l2norm          norm[0] = ||x||_2
//   scale           x := x / norm[0]  (unchanged if norm is 0)
//   seg_l2norm      norms[g] = ||x[seg[g] .. seg[g+1])||_2 for G segments
//   seg_scale       x[seg[g] .. seg[g+1]) := ... / norms[g]  (unchanged if 0)
// The seg_ kernels serve a batch of independent graphs stored
// block-diagonally (one CSR whose diagonal blocks are the graphs): the SpMV
// needs nothing new, and the per-graph norms and scaling are one launch each
// for the whole batch instead of one per graph.
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

constexpr int kSpmvThreads = 128;  // measured 7% faster than 256 (more, smaller tiles in flight)
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
    // col and val are streamed once (evict-first); x is gathered through L1
    // and L2: in the transpose of a power-law graph the high-degree vertices
    // recur, and L1-cached gathers measured 18% faster than L2-only ones on
    // the benchmark graph (L2-only was 5% faster only on uniformly random
    // columns).  Issuing all of a thread's loads before any product measured
    // slower (more gathers in flight than the memory pipeline serves well),
    // so the loop stays.
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
// first tile carrying a row (its chain head) adds all the chain's carries to
// the value the finishing tile wrote.  One thread per tile: a head whose
// chain has at most kFixShort tiles sums it alone, in tile order (almost
// every chain: a row rarely spans more than a few 896-item tiles).  Longer
// chains, the power-law rows that span hundreds of tiles, are walked by the
// head's whole warp, 128 tiles per round trip (four per lane, row ends and
// carries loaded together), each lane summing its tiles in increasing order
// and a fixed shuffle tree combining the lanes.  Either way every run gives
// the same sum.
constexpr int kFixShort = 4;

__global__ void __launch_bounds__(256) spmv_fixup_kernel(const int2 *__restrict__ part,
                                                         const float *__restrict__ carry, float *__restrict__ y,
                                                         int nrows, int tiles)
{
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    int r = -1;
    bool head = false;
    if (b < tiles) {
        r = part[b + 1].x;
        head = r < nrows && (b == 0 || part[b].x != r);
    }
    bool longc = false;
    if (head) {
        int pr[kFixShort];
        float cv[kFixShort];
#pragma unroll
        for (int k = 0; k < kFixShort; ++k) {
            const int bb = b + k;
            pr[k] = bb < tiles ? part[bb + 1].x : -1;
            cv[k] = bb < tiles ? carry[bb] : 0.f;
        }
        float sum = 0.f;
        bool in = true;
#pragma unroll
        for (int k = 0; k < kFixShort; ++k) {
            in = in && pr[k] == r;
            if (in) sum += cv[k];
        }
        longc = in;  // all kFixShort tiles carry r: the chain may go on
        if (!longc) y[r] = sum + y[r];
    }
    // every lane reaches the ballot (no early exit above)
    unsigned lm = __ballot_sync(0xffffffffu, longc);
    while (lm) {
        const int src = __ffs(lm) - 1;
        lm &= lm - 1;
        const int hb = __shfl_sync(0xffffffffu, b, src), hr = __shfl_sync(0xffffffffu, r, src);
        float sum = 0.f;
        for (int base = hb;; base += 128) {
            int pr[4];
            float cv[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int bb = base + 32 * k + lane;
                pr[k] = bb < tiles ? part[bb + 1].x : -1;
                cv[k] = bb < tiles ? carry[bb] : 0.f;
            }
            bool all_in = true;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const bool in = pr[k] == hr;
                if (in) sum += cv[k];
                all_in = all_in && in;
            }
            if (!__all_sync(0xffffffffu, all_in)) break;
        }
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == src) y[hr] = sum + y[hr];
    }
}

// norm[0] = sqrt(sum x_i^2), as two kernels on the node's stream.  The first:
// each 128-thread block takes chunks of 2048 float4 (32 KB) and issues all
// sixteen 128-bit loads of a thread at once, so a vector of a few tens of MB
// is requested in about one memory latency (blocks that walked a grid-stride
// loop waited for several rounds); a thread sums its 64 squares as a fixed
// pairwise tree in fp32 (error a few ulp of the chunk's sum, and no
// dependent chain as in compensated summation) and its chunks in fp64; each
// block sums its threads in an fp64 tree and writes its partial.  The
// second, one block, adds the partials in a fixed order and writes the norm.
// It is launched as a programmatic dependent of the first: it becomes
// resident while the first runs and waits (griddepcontrol.wait) for the
// first grid to complete and its writes to be visible, so no block of the
// first takes an arrival atomic and the combine starts as the last partial
// lands.  The grid depends only on n: the same sum on every run.
constexpr int kL2Threads = 128;
constexpr int kL2V = 16;                               // float4 per thread per chunk
constexpr int kL2Chunk4 = kL2Threads * kL2V;           // 2048 float4
constexpr int kL2MaxBlocks = 4096;
constexpr int kL2CombineThreads = 256;
// scratch: the block partials (doubles)
constexpr size_t kL2ScratchBytes = (size_t)kL2MaxBlocks * 8 + 16;

inline unsigned l2norm_grid(int64_t n)
{
    const int64_t chunks = ceil_div(n >> 2, kL2Chunk4);
    return (unsigned)(chunks < 1 ? 1 : (chunks < kL2MaxBlocks ? chunks : kL2MaxBlocks));
}

__global__ void __launch_bounds__(kL2Threads) l2norm_kernel(const float *__restrict__ x, double *__restrict__ part,
                                                            int64_t n)
{
    // the combine kernel may start now: it waits for this grid to finish
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    __shared__ double sh[kL2Threads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float4 *x4 = reinterpret_cast<const float4 *>(x);
    const int64_t n4 = n >> 2, chunks = (n4 + kL2Chunk4 - 1) / kL2Chunk4;
    double acc = 0.0;
    if ((reinterpret_cast<uintptr_t>(x) & 15) == 0) {
        for (int64_t c = blockIdx.x; c < chunks; c += gridDim.x) {
            float4 v[kL2V];
#pragma unroll
            for (int u = 0; u < kL2V; ++u) {
                const int64_t i = c * kL2Chunk4 + threadIdx.x + (int64_t)u * kL2Threads;
                v[u] = i < n4 ? __ldcs(x4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            float q[kL2V];
#pragma unroll
            for (int u = 0; u < kL2V; ++u) q[u] = (v[u].x * v[u].x + v[u].y * v[u].y) + (v[u].z * v[u].z + v[u].w * v[u].w);
#pragma unroll
            for (int w = kL2V / 2; w > 0; w >>= 1)
#pragma unroll
                for (int u = 0; u < w; ++u) q[u] += q[u + w];
            acc += (double)q[0];
        }
        if (blockIdx.x == 0 && threadIdx.x < (n & 3)) {
            const float t = x[(n4 << 2) + threadIdx.x];
            acc += (double)(t * t);
        }
    } else {
        for (int64_t i = (int64_t)blockIdx.x * kL2Threads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kL2Threads)
            acc += (double)(x[i] * x[i]);
    }
    acc = warp_sum(acc);
    if (lane == 0) sh[warp] = acc;
    __syncthreads();
    if (warp == 0) {
        double b = lane < kL2Threads / 32 ? sh[lane] : 0.0;
        b = warp_sum(b);
        if (lane == 0) part[blockIdx.x] = b;
    }
}

__global__ void __launch_bounds__(kL2CombineThreads) l2norm_combine_kernel(const double *__restrict__ part,
                                                                           float *__restrict__ norm, int blocks)
{
    __shared__ double sh[kL2CombineThreads / 32];
    // the partial-sum grid has completed and its writes are visible
    asm volatile("griddepcontrol.wait;" ::: "memory");
    double t = 0.0;
    for (int b = threadIdx.x; b < blocks; b += kL2CombineThreads) t += part[b];
    t = warp_sum(t);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x < 32) {
        double q = threadIdx.x < kL2CombineThreads / 32 ? sh[threadIdx.x] : 0.0;
        q = warp_sum(q);
        if (threadIdx.x == 0) norm[0] = (float)sqrt(q);
    }
}

size_t l2norm_scratch_bytes() { return kL2ScratchBytes; }

// x := x / norm[0], correctly rounded (div_by); a zero norm leaves x
// unchanged.
__global__ void __launch_bounds__(1024) scale_kernel(float *__restrict__ x, const float *__restrict__ norm, int64_t n)
{
    const float nr = norm[0];
    if (!(nr > 0.f)) return;
    const float rr = (float)(1.0 / (double)nr);
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
                    x4[i] = make_float4(div_by(v[k].x, nr, rr), div_by(v[k].y, nr, rr), div_by(v[k].z, nr, rr),
                                        div_by(v[k].w, nr, rr));
            }
        }
        if (blockIdx.x == 0 && threadIdx.x < (n & 3)) {
            int64_t i = (n4 << 2) + threadIdx.x;
            x[i] = div_by(x[i], nr, rr);
        }
    } else {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
            x[i] = div_by(x[i], nr, rr);
    }
}

size_t seg_norm_scratch_bytes(int64_t G);

// Segments are cut into kSegSlices equal slices; block (slice, g) handles
// one slice of segment g.  Segment bounds are clamped to [0, n], so a
// malformed seg array cannot index outside x.
constexpr int kSegSlices = 32;

__device__ __forceinline__ void seg_slice(const int *__restrict__ seg, int g, int sl, int n, int &lo, int &hi)
{
    int b = seg[g], e = seg[g + 1];
    b = b < 0 ? 0 : (b > n ? n : b);
    e = e < b ? b : (e > n ? n : e);
    const int64_t len = e - b;
    lo = b + (int)(len * sl / kSegSlices);
    hi = b + (int)(len * (sl + 1) / kSegSlices);
}

// norms[g] = sqrt(sum of x_i^2 over segment g): per thread, rounds of eight
// 128-bit loads in flight, each round's 32 squares summed as a fixed fp32
// pairwise tree and the rounds in fp64; fp64 block tree per slice; the last
// slice of a segment to arrive adds the slices' partials in slice order (the
// result does not depend on timing) and resets the segment's arrival
// counter.
constexpr int kSegV = 8;  // float4 in flight per thread

__global__ void __launch_bounds__(kThreads) seg_l2norm_kernel(const float *__restrict__ x, const int *__restrict__ seg,
                                                              float *__restrict__ norms, double *scratch, int G, int n)
{
    __shared__ double sh[kThreads / 32];
    __shared__ bool last;
    const int g = blockIdx.y, sl = blockIdx.x;
    int lo, hi;
    seg_slice(seg, g, sl, n, lo, hi);
    double acc = 0.0;
    // scalar head up to a 16-byte boundary, float4 body, scalar tail (x
    // itself is 16-byte aligned: checked on the host)
    const int a0 = min(hi, (lo + 3) & ~3), a1 = max(a0, hi & ~3);
    for (int i = lo + threadIdx.x; i < a0; i += kThreads) acc += (double)(x[i] * x[i]);
    const float4 *x4 = reinterpret_cast<const float4 *>(x);
    for (int j = (a0 >> 2) + threadIdx.x; j < (a1 >> 2); j += kSegV * kThreads) {
        float4 v[kSegV];
#pragma unroll
        for (int u = 0; u < kSegV; ++u) {
            const int q = j + u * kThreads;
            v[u] = q < (a1 >> 2) ? x4[q] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float qs[kSegV];
#pragma unroll
        for (int u = 0; u < kSegV; ++u) qs[u] = (v[u].x * v[u].x + v[u].y * v[u].y) + (v[u].z * v[u].z + v[u].w * v[u].w);
#pragma unroll
        for (int w = kSegV / 2; w > 0; w >>= 1)
#pragma unroll
            for (int u = 0; u < w; ++u) qs[u] += qs[u + w];
        acc += (double)qs[0];
    }
    for (int i = a1 + threadIdx.x; i < hi; i += kThreads) acc += (double)(x[i] * x[i]);
    const double bs = block_sum(acc, sh);
    double *part = scratch + (size_t)g * kSegSlices;
    unsigned *counter = reinterpret_cast<unsigned *>(scratch + (size_t)G * kSegSlices) + g;
    if (threadIdx.x == 0) part[sl] = bs;
    __threadfence();  // the partial visible device-wide before the arrival
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == (unsigned)(kSegSlices - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();  // every slice's partial visible
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kSegSlices; ++k) t += ((volatile double *)part)[k];
        norms[g] = (float)sqrt(t);
        *counter = 0u;
    }
}

// x := x / norms[g] over segment g, correctly rounded (div_by); a zero norm
// leaves the segment unchanged.
__global__ void __launch_bounds__(kThreads) seg_scale_kernel(float *__restrict__ x, const int *__restrict__ seg,
                                                             const float *__restrict__ norms, int n)
{
    const int g = blockIdx.y, sl = blockIdx.x;
    const float nr = norms[g];
    if (!(nr > 0.f)) return;
    const float rr = (float)(1.0 / (double)nr);
    int lo, hi;
    seg_slice(seg, g, sl, n, lo, hi);
    const int a0 = min(hi, (lo + 3) & ~3), a1 = max(a0, hi & ~3);
    for (int i = lo + threadIdx.x; i < a0; i += kThreads) x[i] = div_by(x[i], nr, rr);
    float4 *x4 = reinterpret_cast<float4 *>(x);
    for (int j = (a0 >> 2) + threadIdx.x; j < (a1 >> 2); j += kThreads) {
        const float4 u = x4[j];
        x4[j] = make_float4(div_by(u.x, nr, rr), div_by(u.y, nr, rr), div_by(u.z, nr, rr), div_by(u.w, nr, rr));
    }
    for (int i = a1 + threadIdx.x; i < hi; i += kThreads) x[i] = div_by(x[i], nr, rr);
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
    spmv_fixup_kernel<<<(unsigned)ceil_div(tiles, 256), 256, 0, s>>>(a.p<int2>(4), a.p<float>(6), a.p<float>(5),
                                                                      nrows, tiles);
    return cudaGetLastError();
}

const char *validate_l2norm(const LaunchArgs &a)
{
    const int64_t n = a.i64(3);
    if (n < 0) return "n < 0";
    if (a.bytes[0] / 4 < (size_t)n) return "x smaller than n floats";
    if (a.bytes[1] < 4) return "norm smaller than one float";
    if (a.bytes[2] < kL2ScratchBytes) return "scratch smaller than gdag_scratch_bytes()";
    return nullptr;
}

int launch_l2norm(const LaunchArgs &a, void *s)
{
    const int64_t n = a.i64(3);
    const unsigned g = l2norm_grid(n);
    double *part = a.p<double>(2);
    l2norm_kernel<<<g, kL2Threads, 0, (cudaStream_t)s>>>(a.p<float>(0), part, n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the combine as a programmatic dependent of the partial sums
    return launch_dependent(l2norm_combine_kernel, kL2CombineThreads, (cudaStream_t)s, (const double *)part,
                            a.p<float>(1), (int)g);
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

const char *validate_seg_common(const LaunchArgs &a, int gi, int ni)
{
    const int G = a.i32(gi), n = a.i32(ni);
    if (G < 0 || n < 0) return "G and n must be >= 0";
    if (G > 65535) return "at most 65535 segments";
    if (a.bytes[0] / 4 < (size_t)n) return "x smaller than n floats";
    if (a.bytes[1] / 4 < (size_t)G + 1) return "seg smaller than G + 1 int32";
    if (a.bytes[2] / 4 < (size_t)G) return "norms smaller than G floats";
    if ((reinterpret_cast<uintptr_t>(a.ptr[0]) & 15) != 0) return "x must be 16-byte aligned";
    return nullptr;
}

const char *validate_seg_l2norm(const LaunchArgs &a)
{
    if (const char *m = validate_seg_common(a, 4, 5)) return m;
    if (a.bytes[3] < seg_norm_scratch_bytes(a.i32(4))) return "scratch smaller than gdag_scratch_bytes(\"seg_l2norm\", G)";
    return nullptr;
}

int launch_seg_l2norm(const LaunchArgs &a, void *s)
{
    const int G = a.i32(4);
    if (G == 0) return cudaSuccess;
    seg_l2norm_kernel<<<dim3(kSegSlices, G), kThreads, 0, (cudaStream_t)s>>>(a.p<float>(0), a.p<int>(1), a.p<float>(2),
                                                                           a.p<double>(3), G, a.i32(5));
    return cudaGetLastError();
}

const char *validate_seg_scale(const LaunchArgs &a) { return validate_seg_common(a, 3, 4); }

int launch_seg_scale(const LaunchArgs &a, void *s)
{
    const int G = a.i32(3);
    if (G == 0) return cudaSuccess;
    seg_scale_kernel<<<dim3(kSegSlices, G), kThreads, 0, (cudaStream_t)s>>>(a.p<float>(0), a.p<int>(1), a.p<float>(2),
                                                                          a.i32(4));
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

size_t seg_norm_scratch_bytes(int64_t G) { return (size_t)(G > 0 ? G : 0) * (kSegSlices * 8 + 4) + 16; }
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
    v.push_back(entry("seg_l2norm", (const void *)seg_l2norm_kernel,
                      {arr(GDAG_MODE_IN), arr(GDAG_MODE_IN), arr(GDAG_MODE_OUT), arr(GDAG_MODE_INOUT), scal(4), scal(4)},
                      validate_seg_l2norm, launch_seg_l2norm));
    v.push_back(entry("seg_scale", (const void *)seg_scale_kernel,
                      {arr(GDAG_MODE_INOUT), arr(GDAG_MODE_IN), arr(GDAG_MODE_IN), scal(4), scal(4)}, validate_seg_scale,
                      launch_seg_scale));
}

}  // namespace gdag
