// IMG nodes (Section IV-B, IMG): a sharpened picture combined with copies of
// the image blurred at two frequencies, weighted by edge masks.
//   gauss_blur  separable Gaussian, clamp-to-edge (5x5 and 9x9 nodes)
//   sobel       3x3 Sobel gradient magnitude, clamp-to-edge
//   minmax      global (min, max) of an image
//   extend      x := (x - min) / (max - min), 0 for a flat image
//   unsharp     s = img + alpha (img - blur)
//   combine     out = e5 s + (1 - e5) (e9 b5 + (1 - e9) b9)
// Images are row-major float32, rows x cols.  Every kernel is HBM-bound: the
// stencils stage a tile plus its halo in shared memory so that each input
// pixel is read from DRAM about once.
#include <initializer_list>
#include <vector>

#include "catalog.h"
#include "kcommon.cuh"

namespace gdag {

constexpr int kMaxRadius = 8;

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Warp-strip stencils.  Each warp owns a strip of image columns, four per
// lane (one 128-bit load per row and lane), and slides down a band of rows:
// the vertical taps come from a window of rows kept in registers (each input
// row is loaded once), the horizontal taps from the neighbouring lanes'
// registers by warp shuffles, so there is no shared memory and no block
// barrier.  The HL lanes at each end of a warp are halo lanes: they load
// and filter the columns next to the strip (replicated at the image edge)
// but store nothing, so a strip is 4 (32 - 2 HL) columns wide.  Rows and
// columns outside the image take the nearest edge value (clamp-to-edge).
constexpr int kStWarps = 4;
constexpr int kStThreads = 32 * kStWarps;
constexpr unsigned kFull = 0xffffffffu;

// Pixels x .. x+3 of row y, clamped to the image; one 128-bit load when the
// four lie inside the image and rows are 16-byte aligned (vec).
__device__ __forceinline__ float4 load4_clamped(const float *__restrict__ in, int rows, int cols, bool vec, int y, int x)
{
    const float *row = in + (size_t)clampi(y, 0, rows - 1) * cols;
    if (vec && x >= 0 && x + 3 < cols) return __ldg(reinterpret_cast<const float4 *>(row + x));
    return make_float4(__ldg(row + clampi(x, 0, cols - 1)), __ldg(row + clampi(x + 1, 0, cols - 1)),
                       __ldg(row + clampi(x + 2, 0, cols - 1)), __ldg(row + clampi(x + 3, 0, cols - 1)));
}

// Store pixels x .. x+3 (x >= 0) of row y, those inside the image.
__device__ __forceinline__ void store4(float *__restrict__ out, int rows, int cols, bool vec, int y, int x, float4 v)
{
    if (y >= rows || x >= cols) return;
    float *o = out + (size_t)y * cols + x;
    if (vec && x + 3 < cols) {
        *reinterpret_cast<float4 *>(o) = v;
    } else {
        o[0] = v.x;
        if (x + 1 < cols) o[1] = v.y;
        if (x + 2 < cols) o[2] = v.z;
        if (x + 3 < cols) o[3] = v.w;
    }
}

__device__ __forceinline__ bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// Separable Gaussian blur of radius R.  Per output row a lane makes four
// outputs: the vertical pass (2R+1 taps on the row window, packed fp32x2
// FMAs) gives the four columns' vertical sums, the horizontal pass combines
// them with the 4 HL neighbouring columns on each side taken from the
// neighbour lanes.  The rows live in a ring of 2R+1+P registers slots: the
// row that output row y needs last, y + R, was loaded P rows earlier, so P
// loads per lane are always in flight.  The band of output rows is a
// multiple of the ring size and the row loop is unrolled by it, so every
// slot index is a compile-time constant.
template <int R> struct BlurShape {
    static constexpr int HL = (R + 3) / 4;             // halo lanes per side
    static constexpr int HALO = 4 * HL;                // halo columns per side
    static constexpr int OUTL = 32 - 2 * HL;           // lanes that store
    static constexpr int W = 2 * R + 1;
    // rows loaded ahead, and output rows per warp (a multiple of the
    // ring): a 4096 x 4096 image then gives each SM about 20 warps with P
    // rows in flight each, in one wave of resident blocks (the wider ring
    // of a larger radius costs registers, so fewer blocks fit an SM)
    static constexpr int P = R <= 2 ? 6 : 4;
    static constexpr int RING = W + P;
    static constexpr int TH = RING * (R <= 2 ? (45 / RING > 0 ? 45 / RING : 1) : (52 / RING > 0 ? 52 / RING : 1));
};

template <int R>
__global__ void __launch_bounds__(kStThreads) gauss_blur_kernel(const float *__restrict__ in, float *__restrict__ out,
                                                                const float *__restrict__ w, int rows, int cols)
{
    using S = BlurShape<R>;
    constexpr int W = S::W, HL = S::HL, HALO = S::HALO, P = S::P, RING = S::RING;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int x0 = (blockIdx.x * kStWarps + warp) * 4 * S::OUTL;
    if (x0 >= cols) return;  // the whole warp
    const int x = x0 + 4 * (lane - HL);
    const int y0 = blockIdx.y * S::TH;
    const bool vin = (cols & 3) == 0 && aligned16(in), vout = (cols & 3) == 0 && aligned16(out);
    const bool stores = lane >= HL && lane < 32 - HL;
    float wr[W];
#pragma unroll
    for (int k = 0; k < W; ++k) wr[k] = __ldg(w + k);
    float4 ring[RING];  // slot (y - y0 + R) % RING holds input row y
#pragma unroll
    for (int k = 0; k < W - 1 + P; ++k) ring[k] = load4_clamped(in, rows, cols, vin, y0 - R + k, x);
    for (int r0 = 0; r0 < S::TH; r0 += RING) {
        if (y0 + r0 >= rows) break;  // the whole warp
#pragma unroll
        for (int k = 0; k < RING; ++k) {
            const int y = y0 + r0 + k;
            // row y + R + P, P rows ahead, into slot (k + W - 1 + P) % RING
            ring[(k + W - 1 + P) % RING] = load4_clamped(in, rows, cols, vin, y + R + P, x);
            float2 lo = make_float2(0.f, 0.f), hi = lo;
#pragma unroll
            for (int j = 0; j < W; ++j) {  // input row y - R + j
                const float4 p = ring[(k + j) % RING];
                const float2 wj = make_float2(wr[j], wr[j]);
                lo = __ffma2_rn(wj, make_float2(p.x, p.y), lo);
                hi = __ffma2_rn(wj, make_float2(p.z, p.w), hi);
            }
            // columns x - HALO .. x + 3 + HALO of the vertical result
            float v[4 + 2 * HALO];
            v[HALO] = lo.x;
            v[HALO + 1] = lo.y;
            v[HALO + 2] = hi.x;
            v[HALO + 3] = hi.y;
#pragma unroll
            for (int h = 1; h <= HL; ++h) {
                v[HALO - 4 * h] = __shfl_up_sync(kFull, lo.x, h);
                v[HALO - 4 * h + 1] = __shfl_up_sync(kFull, lo.y, h);
                v[HALO - 4 * h + 2] = __shfl_up_sync(kFull, hi.x, h);
                v[HALO - 4 * h + 3] = __shfl_up_sync(kFull, hi.y, h);
                v[HALO + 4 * h] = __shfl_down_sync(kFull, lo.x, h);
                v[HALO + 4 * h + 1] = __shfl_down_sync(kFull, lo.y, h);
                v[HALO + 4 * h + 2] = __shfl_down_sync(kFull, hi.x, h);
                v[HALO + 4 * h + 3] = __shfl_down_sync(kFull, hi.y, h);
            }
            // outputs (0,1) and (2,3) take the taps whose input offset o is
            // even: their operand pairs (v[o], v[o+1]) sit in aligned
            // register pairs.  For odd o the aligned pair is (v[o+1],
            // v[o+2]), which feeds outputs (1,2); outputs 0 and 3 take that
            // tap with scalar FMAs.  The parities are compile-time.
            float2 a01 = make_float2(0.f, 0.f), a23 = a01, mid = a01;
            float e0 = 0.f, e3 = 0.f;
#pragma unroll
            for (int k2 = 0; k2 < W; ++k2) {
                const int o = HALO - R + k2;
                const float2 wk = make_float2(wr[k2], wr[k2]);
                if ((o & 1) == 0) {
                    a01 = __ffma2_rn(wk, make_float2(v[o], v[o + 1]), a01);
                    a23 = __ffma2_rn(wk, make_float2(v[o + 2], v[o + 3]), a23);
                } else {
                    mid = __ffma2_rn(wk, make_float2(v[o + 1], v[o + 2]), mid);
                    e0 = fmaf(wr[k2], v[o], e0);
                    e3 = fmaf(wr[k2], v[o + 3], e3);
                }
            }
            if (stores) store4(out, rows, cols, vout, y, x, make_float4(a01.x + e0, a01.y + mid.x, a23.x + mid.y, a23.y + e3));
        }
    }
}

// sqrt(gx^2 + gy^2) with the single-instruction approximate square root
// (relative error about 1e-7, far inside the 1e-5 tolerance; the outputs
// that are compared bit for bit downstream are min/max of these values
// themselves); exactly 0 for a flat neighbourhood.
__device__ __forceinline__ float sobel_mag(float gx, float gy)
{
    const float g2 = fmaf(gx, gx, gy * gy);
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(g2));
    return g2 > 0.f ? r : 0.f;
}

// Sobel magnitude, separably: per column the vertical smoothing
// sv = top + 2 mid + bottom and difference dv = bottom - top of three rows
// in registers; gx = sv(c+1) - sv(c-1), gy = dv(c-1) + 2 dv(c) + dv(c+1),
// the neighbouring columns of a lane's four from the next lanes (one halo
// lane per side).  Rows are loaded two ahead of their use.
constexpr int kSobelRows = 32;  // output rows per warp

__global__ void __launch_bounds__(kStThreads) sobel_kernel(const float *__restrict__ in, float *__restrict__ out,
                                                           int rows, int cols)
{
    constexpr int HL = 1, OUTL = 32 - 2 * HL;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int x0 = (blockIdx.x * kStWarps + warp) * 4 * OUTL;
    if (x0 >= cols) return;  // the whole warp
    const int x = x0 + 4 * (lane - HL);
    const int y0 = blockIdx.y * kSobelRows;
    const bool vin = (cols & 3) == 0 && aligned16(in), vout = (cols & 3) == 0 && aligned16(out);
    const bool stores = lane >= HL && lane < 32 - HL;
    float4 a = load4_clamped(in, rows, cols, vin, y0 - 1, x);
    float4 b = load4_clamped(in, rows, cols, vin, y0, x);
    float4 c1 = load4_clamped(in, rows, cols, vin, y0 + 1, x);
    float4 c2 = load4_clamped(in, rows, cols, vin, y0 + 2, x);
    for (int r = 0; r < kSobelRows; ++r) {
        const int y = y0 + r;
        if (y >= rows) break;  // the whole warp
        const float4 c = c1;
        c1 = c2;
        c2 = load4_clamped(in, rows, cols, vin, y + 3, x);
        const float4 sv = make_float4(fmaf(2.f, b.x, a.x + c.x), fmaf(2.f, b.y, a.y + c.y), fmaf(2.f, b.z, a.z + c.z),
                                      fmaf(2.f, b.w, a.w + c.w));
        const float4 dv = make_float4(c.x - a.x, c.y - a.y, c.z - a.z, c.w - a.w);
        const float svl = __shfl_up_sync(kFull, sv.w, 1), svr = __shfl_down_sync(kFull, sv.x, 1);
        const float dvl = __shfl_up_sync(kFull, dv.w, 1), dvr = __shfl_down_sync(kFull, dv.x, 1);
        const float4 m = make_float4(sobel_mag(sv.y - svl, fmaf(2.f, dv.x, dvl + dv.y)),
                                     sobel_mag(sv.z - sv.x, fmaf(2.f, dv.y, dv.x + dv.z)),
                                     sobel_mag(sv.w - sv.y, fmaf(2.f, dv.z, dv.y + dv.w)),
                                     sobel_mag(svr - sv.z, fmaf(2.f, dv.w, dv.z + dvr)));
        if (stores) store4(out, rows, cols, vout, y, x, m);
        a = b;
        b = c;
    }
}

// (min, max) of n floats -> mm[0], mm[1], in two kernels.  The first gives
// each block one chunk of sixteen 128-bit loads per thread, all issued
// before any is used (past kMmMaxBlocks chunks a block takes several,
// grid-strided), and writes the block's (min, max) pair; no block takes an
// arrival atomic.  The second, one block launched as a programmatic
// dependent, becomes resident early and waits on the device for the first
// grid to complete before it combines the pairs.  min and max round
// nothing, so the result is exact whatever the order.
constexpr int kMmThreads = 128;
constexpr int kMmV = 16;                      // float4 per thread per chunk
constexpr int kMmChunk4 = kMmThreads * kMmV;  // 2048 float4
constexpr int kMmMaxBlocks = 4096;
constexpr int kMmCombineThreads = 256;

inline unsigned minmax_grid(int64_t n)
{
    const int64_t chunks = ceil_div(n >> 2, kMmChunk4);
    return (unsigned)(chunks < 1 ? 1 : (chunks < kMmMaxBlocks ? chunks : kMmMaxBlocks));
}

size_t minmax_scratch_bytes() { return (size_t)kMmMaxBlocks * sizeof(float2) + 16; }

__global__ void __launch_bounds__(kMmThreads) minmax_kernel(const float *__restrict__ x, float2 *__restrict__ part,
                                                            int64_t n)
{
    // the combine kernel may start now: it waits for this grid to finish
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    __shared__ float smin[kMmThreads / 32], smax[kMmThreads / 32];
    const float kNaN = __int_as_float(0x7fffffff);
    float lo = INFINITY, hi = -INFINITY;
    if ((reinterpret_cast<uintptr_t>(x) & 15) == 0) {
        const float4 *x4 = reinterpret_cast<const float4 *>(x);
        const int64_t n4 = n >> 2, chunks = (n4 + kMmChunk4 - 1) / kMmChunk4;
        for (int64_t c = blockIdx.x; c < chunks; c += gridDim.x) {
            float4 v[kMmV];
#pragma unroll
            for (int u = 0; u < kMmV; ++u) {
                const int64_t i = c * kMmChunk4 + threadIdx.x + (int64_t)u * kMmThreads;
                v[u] = i < n4 ? x4[i] : make_float4(kNaN, kNaN, kNaN, kNaN);
            }
#pragma unroll
            for (int u = 0; u < kMmV; ++u) {
                // padding is NaN, which fminf and fmaxf pass over
                lo = fminf(lo, fminf(fminf(v[u].x, v[u].y), fminf(v[u].z, v[u].w)));
                hi = fmaxf(hi, fmaxf(fmaxf(v[u].x, v[u].y), fmaxf(v[u].z, v[u].w)));
            }
        }
        if (blockIdx.x == 0 && threadIdx.x < (n & 3)) {
            const float t = x[(n4 << 2) + threadIdx.x];
            lo = fminf(lo, t);
            hi = fmaxf(hi, t);
        }
    } else {
        for (int64_t i = (int64_t)blockIdx.x * kMmThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kMmThreads) {
            lo = fminf(lo, x[i]);
            hi = fmaxf(hi, x[i]);
        }
    }
    lo = warp_min(lo);
    hi = warp_max(hi);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        smin[warp] = lo;
        smax[warp] = hi;
    }
    __syncthreads();
    if (warp == 0) {
        lo = lane < kMmThreads / 32 ? smin[lane] : INFINITY;
        hi = lane < kMmThreads / 32 ? smax[lane] : -INFINITY;
        lo = warp_min(lo);
        hi = warp_max(hi);
        if (lane == 0) part[blockIdx.x] = make_float2(lo, hi);
    }
}

__global__ void __launch_bounds__(kMmCombineThreads) minmax_combine_kernel(const float2 *__restrict__ part,
                                                                           float *__restrict__ mm, int blocks)
{
    __shared__ float smin[kMmCombineThreads / 32], smax[kMmCombineThreads / 32];
    // the first grid has completed and its writes are visible
    asm volatile("griddepcontrol.wait;" ::: "memory");
    float lo = INFINITY, hi = -INFINITY;
    for (int b = threadIdx.x; b < blocks; b += kMmCombineThreads) {
        const float2 p = part[b];
        lo = fminf(lo, p.x);
        hi = fmaxf(hi, p.y);
    }
    lo = warp_min(lo);
    hi = warp_max(hi);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        smin[warp] = lo;
        smax[warp] = hi;
    }
    __syncthreads();
    if (warp == 0) {
        lo = lane < kMmCombineThreads / 32 ? smin[lane] : INFINITY;
        hi = lane < kMmCombineThreads / 32 ? smax[lane] : -INFINITY;
        lo = warp_min(lo);
        hi = warp_max(hi);
        if (lane == 0) {
            mm[0] = lo;
            mm[1] = hi;
        }
    }
}

// x := (x - mn) / (mx - mn) with (mn, mx) read from device memory; a flat
// image (mx == mn) maps to 0.
__global__ void __launch_bounds__(1024) extend_kernel(float *__restrict__ x, const float *__restrict__ mm, int64_t n)
{
    const float mn = mm[0], mx = mm[1];
    const bool flat = !(mx > mn);
    const float span = mx - mn;
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
                if (i < n4) {
                    float4 o;
                    o.x = flat ? 0.f : __fdiv_rn(v[k].x - mn, span);
                    o.y = flat ? 0.f : __fdiv_rn(v[k].y - mn, span);
                    o.z = flat ? 0.f : __fdiv_rn(v[k].z - mn, span);
                    o.w = flat ? 0.f : __fdiv_rn(v[k].w - mn, span);
                    x4[i] = o;
                }
            }
        }
        if (blockIdx.x == 0 && threadIdx.x < (n & 3)) {
            int64_t i = (n4 << 2) + threadIdx.x;
            x[i] = flat ? 0.f : __fdiv_rn(x[i] - mn, span);
        }
    } else {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
            x[i] = flat ? 0.f : __fdiv_rn(x[i] - mn, span);
    }
}

__device__ __forceinline__ float unsharp1(float a, float b, float alpha) { return fmaf(alpha, a - b, a); }

__global__ void __launch_bounds__(1024) unsharp_kernel(const float *__restrict__ img, const float *__restrict__ bl,
                                                       float *__restrict__ out, float alpha, int64_t n)
{
    if (((reinterpret_cast<uintptr_t>(img) | reinterpret_cast<uintptr_t>(bl) | reinterpret_cast<uintptr_t>(out)) & 15) ==
        0) {
        const float4 *a4 = reinterpret_cast<const float4 *>(img);
        const float4 *b4 = reinterpret_cast<const float4 *>(bl);
        float4 *o4 = reinterpret_cast<float4 *>(out);
        const int64_t n4 = n >> 2, bd = blockDim.x, tile = bd * kUnroll;
        for (int64_t base = (int64_t)blockIdx.x * tile; base < n4; base += (int64_t)gridDim.x * tile) {
            float4 a[kUnroll], b[kUnroll];
#pragma unroll
            for (int k = 0; k < kUnroll; ++k) {
                int64_t i = base + threadIdx.x + k * bd;
                if (i < n4) {
                    a[k] = a4[i];
                    b[k] = b4[i];
                }
            }
#pragma unroll
            for (int k = 0; k < kUnroll; ++k) {
                int64_t i = base + threadIdx.x + k * bd;
                if (i < n4)
                    o4[i] = make_float4(unsharp1(a[k].x, b[k].x, alpha), unsharp1(a[k].y, b[k].y, alpha),
                                        unsharp1(a[k].z, b[k].z, alpha), unsharp1(a[k].w, b[k].w, alpha));
            }
        }
        if (blockIdx.x == 0 && threadIdx.x < (n & 3)) {
            int64_t i = (n4 << 2) + threadIdx.x;
            out[i] = unsharp1(img[i], bl[i], alpha);
        }
    } else {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
            out[i] = unsharp1(img[i], bl[i], alpha);
    }
}

__device__ __forceinline__ float combine1(float s, float b5, float b9, float e5, float e9)
{
    return e5 * s + (1.f - e5) * (e9 * b5 + (1.f - e9) * b9);
}

__global__ void __launch_bounds__(1024) combine_kernel(const float *__restrict__ s, const float *__restrict__ b5,
                                                       const float *__restrict__ b9, const float *__restrict__ e5,
                                                       const float *__restrict__ e9, float *__restrict__ out,
                                                       int64_t n)
{
    const uintptr_t al = reinterpret_cast<uintptr_t>(s) | reinterpret_cast<uintptr_t>(b5) |
                         reinterpret_cast<uintptr_t>(b9) | reinterpret_cast<uintptr_t>(e5) |
                         reinterpret_cast<uintptr_t>(e9) | reinterpret_cast<uintptr_t>(out);
    if ((al & 15) == 0) {
        const int64_t n4 = n >> 2, bd = blockDim.x, tile = bd * 2;
        for (int64_t base = (int64_t)blockIdx.x * tile; base < n4; base += (int64_t)gridDim.x * tile) {
            float4 v[2][5];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                int64_t i = base + threadIdx.x + k * bd;
                if (i < n4) {
                    v[k][0] = reinterpret_cast<const float4 *>(s)[i];
                    v[k][1] = reinterpret_cast<const float4 *>(b5)[i];
                    v[k][2] = reinterpret_cast<const float4 *>(b9)[i];
                    v[k][3] = reinterpret_cast<const float4 *>(e5)[i];
                    v[k][4] = reinterpret_cast<const float4 *>(e9)[i];
                }
            }
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                int64_t i = base + threadIdx.x + k * bd;
                if (i < n4) {
                    float4 o;
                    o.x = combine1(v[k][0].x, v[k][1].x, v[k][2].x, v[k][3].x, v[k][4].x);
                    o.y = combine1(v[k][0].y, v[k][1].y, v[k][2].y, v[k][3].y, v[k][4].y);
                    o.z = combine1(v[k][0].z, v[k][1].z, v[k][2].z, v[k][3].z, v[k][4].z);
                    o.w = combine1(v[k][0].w, v[k][1].w, v[k][2].w, v[k][3].w, v[k][4].w);
                    reinterpret_cast<float4 *>(out)[i] = o;
                }
            }
        }
        if (blockIdx.x == 0 && threadIdx.x < (n & 3)) {
            int64_t i = (n4 << 2) + threadIdx.x;
            out[i] = combine1(s[i], b5[i], b9[i], e5[i], e9[i]);
        }
    } else {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
            out[i] = combine1(s[i], b5[i], b9[i], e5[i], e9[i]);
    }
}

namespace {

bool image_ok(const LaunchArgs &a, int i, int rows, int cols)
{
    return (size_t)rows * (size_t)cols <= a.bytes[i] / 4;
}

const char *validate_blur(const LaunchArgs &a)
{
    int rows = a.i32(3), cols = a.i32(4), R = a.i32(5);
    if (rows <= 0 || cols <= 0) return "rows and cols must be > 0";
    if (R < 1 || R > kMaxRadius) return "radius must be in 1..8";
    if (!image_ok(a, 0, rows, cols) || !image_ok(a, 1, rows, cols)) return "image smaller than rows x cols floats";
    if (a.bytes[2] / 4 < (size_t)(2 * R + 1)) return "weights smaller than 2R+1 floats";
    return nullptr;
}

// one resident wave of persistent blocks (at most one per tile)
template <int R> void blur_launch(const LaunchArgs &a, cudaStream_t s)
{
    using S = BlurShape<R>;
    const int rows = a.i32(3), cols = a.i32(4);
    const dim3 g((unsigned)ceil_div(ceil_div(cols, 4 * S::OUTL), kStWarps), (unsigned)ceil_div(rows, S::TH));
    gauss_blur_kernel<R><<<g, kStThreads, 0, s>>>(a.p<float>(0), a.p<float>(1), a.p<float>(2), rows, cols);
}
int launch_blur(const LaunchArgs &a, void *sv)
{
    cudaStream_t s = (cudaStream_t)sv;
    switch (a.i32(5)) {
    case 1: blur_launch<1>(a, s); break;
    case 2: blur_launch<2>(a, s); break;
    case 3: blur_launch<3>(a, s); break;
    case 4: blur_launch<4>(a, s); break;
    case 5: blur_launch<5>(a, s); break;
    case 6: blur_launch<6>(a, s); break;
    case 7: blur_launch<7>(a, s); break;
    default: blur_launch<8>(a, s); break;
    }
    return cudaGetLastError();
}

const char *validate_sobel(const LaunchArgs &a)
{
    int rows = a.i32(2), cols = a.i32(3);
    if (rows <= 0 || cols <= 0) return "rows and cols must be > 0";
    if (!image_ok(a, 0, rows, cols) || !image_ok(a, 1, rows, cols)) return "image smaller than rows x cols floats";
    return nullptr;
}

int launch_sobel(const LaunchArgs &a, void *s)
{
    int rows = a.i32(2), cols = a.i32(3);
    const dim3 g((unsigned)ceil_div(ceil_div(cols, 4 * 30), kStWarps), (unsigned)ceil_div(rows, kSobelRows));
    sobel_kernel<<<g, kStThreads, 0, (cudaStream_t)s>>>(a.p<float>(0), a.p<float>(1), rows, cols);
    return cudaGetLastError();
}

const char *validate_minmax(const LaunchArgs &a)
{
    int64_t n = a.i64(3);
    if (n <= 0) return "n must be > 0";
    if (a.bytes[0] / 4 < (size_t)n) return "input smaller than n floats";
    if (a.bytes[1] < 8) return "mm smaller than two floats";
    if (a.bytes[2] < minmax_scratch_bytes()) return "scratch smaller than gdag_scratch_bytes()";
    return nullptr;
}

int launch_minmax(const LaunchArgs &a, void *s)
{
    const int64_t n = a.i64(3);
    const unsigned g = minmax_grid(n);
    float2 *part = reinterpret_cast<float2 *>(a.p<double>(2));
    minmax_kernel<<<g, kMmThreads, 0, (cudaStream_t)s>>>(a.p<float>(0), part, n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the combine as a programmatic dependent of the block pairs
    return launch_dependent(minmax_combine_kernel, kMmCombineThreads, (cudaStream_t)s, (const float2 *)part,
                            a.p<float>(1), (int)g);
}

const char *validate_extend(const LaunchArgs &a)
{
    int64_t n = a.i64(2);
    if (n < 0) return "n < 0";
    if (a.bytes[0] / 4 < (size_t)n) return "x smaller than n floats";
    if (a.bytes[1] < 8) return "mm smaller than two floats";
    return nullptr;
}

int launch_extend(const LaunchArgs &a, void *s)
{
    int64_t n = a.i64(2);
    if (n == 0) return cudaSuccess;
    extend_kernel<<<stream_grid(n >> 2), kThreads, 0, (cudaStream_t)s>>>(a.p<float>(0), a.p<float>(1), n);
    return cudaGetLastError();
}

const char *validate_unsharp(const LaunchArgs &a)
{
    int64_t n = a.i64(4);
    if (n < 0) return "n < 0";
    for (int i = 0; i < 3; ++i)
        if (a.bytes[i] / 4 < (size_t)n) return "an image is smaller than n floats";
    return nullptr;
}

int launch_unsharp(const LaunchArgs &a, void *s)
{
    int64_t n = a.i64(4);
    if (n == 0) return cudaSuccess;
    unsharp_kernel<<<stream_grid(n >> 2), kThreads, 0, (cudaStream_t)s>>>(a.p<float>(0), a.p<float>(1),
                                                                          a.p<float>(2), a.f32(3), n);
    return cudaGetLastError();
}

const char *validate_combine(const LaunchArgs &a)
{
    int64_t n = a.i64(6);
    if (n < 0) return "n < 0";
    for (int i = 0; i < 6; ++i)
        if (a.bytes[i] / 4 < (size_t)n) return "an image is smaller than n floats";
    return nullptr;
}

int launch_combine(const LaunchArgs &a, void *s)
{
    int64_t n = a.i64(6);
    if (n == 0) return cudaSuccess;
    int64_t tiles = ceil_div(n >> 2 > 0 ? n >> 2 : 1, (int64_t)kThreads * 2);
    int64_t cap = (int64_t)sm_count() * kBlocksPerSm;
    combine_kernel<<<(unsigned)(tiles < cap ? tiles : cap), kThreads, 0, (cudaStream_t)s>>>(
        a.p<float>(0), a.p<float>(1), a.p<float>(2), a.p<float>(3), a.p<float>(4), a.p<float>(5), n);
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
    for (const auto &s : spec) e.spec[i++] = s;
    e.validate = v;
    e.launcher = l;
    return e;
}

}  // namespace

void append_img_kernels(std::vector<KernelEntry> &v)
{
    v.push_back(entry("gauss_blur", (const void *)gauss_blur_kernel<2>,
                      {arr(GDAG_MODE_IN), arr(GDAG_MODE_OUT), arr(GDAG_MODE_IN), scal(4), scal(4), scal(4)},
                      validate_blur, launch_blur));
    v.push_back(entry("sobel", (const void *)sobel_kernel, {arr(GDAG_MODE_IN), arr(GDAG_MODE_OUT), scal(4), scal(4)},
                      validate_sobel, launch_sobel));
    v.push_back(entry("minmax", (const void *)minmax_kernel,
                      {arr(GDAG_MODE_IN), arr(GDAG_MODE_OUT), arr(GDAG_MODE_INOUT), scal(8)}, validate_minmax,
                      launch_minmax));
    v.push_back(entry("extend", (const void *)extend_kernel, {arr(GDAG_MODE_INOUT), arr(GDAG_MODE_IN), scal(8)},
                      validate_extend, launch_extend));
    v.push_back(entry("unsharp", (const void *)unsharp_kernel,
                      {arr(GDAG_MODE_IN), arr(GDAG_MODE_IN), arr(GDAG_MODE_OUT), scal(4), scal(8)}, validate_unsharp,
                      launch_unsharp));
    v.push_back(entry("combine", (const void *)combine_kernel,
                      {arr(GDAG_MODE_IN), arr(GDAG_MODE_IN), arr(GDAG_MODE_IN), arr(GDAG_MODE_IN), arr(GDAG_MODE_IN),
                       arr(GDAG_MODE_OUT), scal(8)},
                      validate_combine, launch_combine));
}

}  // namespace gdag
