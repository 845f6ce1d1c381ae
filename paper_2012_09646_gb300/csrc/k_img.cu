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

constexpr int kTileW = 64, kTileH = 32;   // output tile of one 256-thread block
constexpr int kImgThreads = 256;
constexpr int kMaxRadius = 8;

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Stage rows y0-R .. y0+kTileH+R-1 and columns x0-HALO .. x0+kTileW+HALO-1 of
// the image into s (row stride IW = kTileW + 2 HALO, HALO a multiple of 4),
// clamping coordinates to the image.  Interior blocks of an image whose
// rows are 16-byte aligned use 128-bit loads; border blocks clamp per pixel.
template <int R, int HALO, int IW>
__device__ __forceinline__ void stage_tile(const float *__restrict__ in, float *s, int rows, int cols, int x0, int y0)
{
    constexpr int IH = kTileH + 2 * R;
    const bool fast = (cols & 3) == 0 && (reinterpret_cast<uintptr_t>(in) & 15) == 0 && x0 >= HALO &&
                      x0 + kTileW + HALO <= cols;
    if (fast) {
        constexpr int V = IW / 4;  // float4 per staged row
        constexpr int PER = (IH * V + kImgThreads - 1) / kImgThreads;
        float4 v[PER];  // every load of the thread in flight before any store
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int i = threadIdx.x + k * kImgThreads;
            if (i < IH * V) {
                const int r = i / V, c4 = i - r * V;
                const int y = clampi(y0 + r - R, 0, rows - 1);
                v[k] = *reinterpret_cast<const float4 *>(in + (size_t)y * cols + (x0 - HALO) + 4 * c4);
            }
        }
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int i = threadIdx.x + k * kImgThreads;
            if (i < IH * V) {
                const int r = i / V, c4 = i - r * V;
                *reinterpret_cast<float4 *>(s + r * IW + 4 * c4) = v[k];
            }
        }
    } else {
        for (int i = threadIdx.x; i < IH * IW; i += kImgThreads) {
            const int r = i / IW, c = i - r * IW;
            const int y = clampi(y0 + r - R, 0, rows - 1);
            s[r * IW + c] = in[(size_t)y * cols + clampi(x0 + c - HALO, 0, cols - 1)];
        }
    }
}

__device__ __forceinline__ void img_cp_async16(float *dst, const float *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}

// The same staged tile as stage_tile, copied asynchronously (cp.async,
// 16 bytes a copy, completion per thread by cp.async.wait_group) when the
// tile's columns plus halo lie inside an image whose rows are 16-byte
// aligned (rows are clamped whole, so only the columns decide); returns
// false, having issued nothing, for the other tiles, which the caller stages
// with stage_tile.  Uniform across the block.
template <int R, int HALO, int IW>
__device__ __forceinline__ bool stage_tile_async(const float *__restrict__ in, float *s, int rows, int cols, int x0,
                                                 int y0)
{
    constexpr int IH = kTileH + 2 * R;
    const bool fast = (cols & 3) == 0 && (reinterpret_cast<uintptr_t>(in) & 15) == 0 && x0 >= HALO &&
                      x0 + kTileW + HALO <= cols;
    if (!fast) return false;
    constexpr int V = IW / 4;
    for (int i = threadIdx.x; i < IH * V; i += kImgThreads) {
        const int r = i / V, c4 = i - r * V;
        const int y = clampi(y0 + r - R, 0, rows - 1);
        img_cp_async16(s + r * IW + 4 * c4, in + (size_t)y * cols + (x0 - HALO) + 4 * c4);
    }
    return true;
}

// Persistent blur blocks walk tiles t = blockIdx.x, + gridDim.x, ...
// (row-major tile order, so neighbouring tiles share their halos in L2),
// double-buffering the staged input: tile t+gridDim.x is copied while tile t
// is computed.  (Sobel, whose tile costs less arithmetic, measured faster
// with one tile per block and the hardware's block scheduler.)
__device__ __forceinline__ void tile_origin(int t, int ntx, int &x0, int &y0)
{
    x0 = (t % ntx) * kTileW;
    y0 = (t / ntx) * kTileH;
}

// Store two rows of four outputs (x .. x+3, rows y, y+1) with bounds checks.
__device__ __forceinline__ void store_2x4(float *__restrict__ out, int rows, int cols, int x, int y, float4 a, float4 b)
{
    const bool vec = (cols & 3) == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0 && x + 3 < cols;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int yy = y + h;
        if (yy >= rows) break;
        const float4 v = h ? b : a;
        float *o = out + (size_t)yy * cols + x;
        if (vec) {
            *reinterpret_cast<float4 *>(o) = v;
        } else {
            if (x < cols) o[0] = v.x;
            if (x + 1 < cols) o[1] = v.y;
            if (x + 2 < cols) o[2] = v.z;
            if (x + 3 < cols) o[3] = v.w;
        }
    }
}

// Separable Gaussian blur with radius R.  Horizontal pass: each thread makes
// four adjacent outputs of one staged row from 4 + 2R inputs (packed fp32x2
// FMAs); vertical pass: each thread makes a 4-column x 2-row block from
// 2 + 2R rows of the horizontal result.  Per output 2(2R+1) FMAs and about
// one 32-bit shared-memory access; DRAM: one read and one write of the image.
template <int R>
__global__ void __launch_bounds__(kImgThreads) gauss_blur_kernel(const float *__restrict__ in, float *__restrict__ out,
                                                                 const float *__restrict__ w, int rows, int cols)
{
    constexpr int HALO = (R + 3) / 4 * 4;
    constexpr int IW = kTileW + 2 * HALO, IH = kTileH + 2 * R;
    __shared__ __align__(16) float s_in[2][IH * IW];
    __shared__ __align__(16) float s_h[IH * kTileW];
    float wr[2 * R + 1];
#pragma unroll
    for (int k = 0; k <= 2 * R; ++k) wr[k] = w[k];
    const int ntx = (cols + kTileW - 1) / kTileW;
    const int ntiles = ntx * ((rows + kTileH - 1) / kTileH);
    int t = blockIdx.x, x0, y0;
    if (t >= ntiles) return;
    tile_origin(t, ntx, x0, y0);
    bool staged = stage_tile_async<R, HALO, IW>(in, s_in[0], rows, cols, x0, y0);
    asm volatile("cp.async.commit_group;" ::: "memory");
    for (int buf = 0; t < ntiles; t += gridDim.x, buf ^= 1) {
        tile_origin(t, ntx, x0, y0);
        // the next tile's copies go into the other buffer (last read before
        // the previous tile's second barrier)
        bool staged_next = false;
        if (t + (int)gridDim.x < ntiles) {
            int nx0, ny0;
            tile_origin(t + gridDim.x, ntx, nx0, ny0);
            staged_next = stage_tile_async<R, HALO, IW>(in, s_in[buf ^ 1], rows, cols, nx0, ny0);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 1;" ::: "memory");  // this tile's copies (this thread's) landed
        if (!staged) stage_tile<R, HALO, IW>(in, s_in[buf], rows, cols, x0, y0);  // border tile: clamped columns
        __syncthreads();
        const float *si = s_in[buf];
        // horizontal: IH rows x 16 groups of four columns
        for (int q = threadIdx.x; q < IH * (kTileW / 4); q += kImgThreads) {
            const int r = q >> 4, g = q & 15;
            const float *row = si + r * IW + 4 * g;  // inputs 4g .. 4g + 4 + 2 HALO
            float v[4 + 2 * HALO];
#pragma unroll
            for (int k = 0; k < (4 + 2 * HALO) / 4; ++k) {
                const float4 p = reinterpret_cast<const float4 *>(row)[k];
                v[4 * k] = p.x;
                v[4 * k + 1] = p.y;
                v[4 * k + 2] = p.z;
                v[4 * k + 3] = p.w;
            }
            // outputs (0,1) and (2,3) take the taps whose input offset o is
            // even: their operand pairs (v[o], v[o+1]) sit in aligned
            // register pairs.  For odd o the aligned pair is (v[o+1],
            // v[o+2]), which feeds outputs (1,2); outputs 0 and 3 take that
            // tap with scalar FMAs.  (Building misaligned pairs would cost two
            // register moves per pair.)  The parities are compile-time.
            float2 lo = make_float2(0.f, 0.f), hi = lo, mid = lo;
            float e0 = 0.f, e3 = 0.f;
#pragma unroll
            for (int k = 0; k <= 2 * R; ++k) {
                const int o = HALO - R + k;
                if ((o & 1) == 0) {
                    const float2 wk = make_float2(wr[k], wr[k]);
                    lo = __ffma2_rn(wk, make_float2(v[o], v[o + 1]), lo);
                    hi = __ffma2_rn(wk, make_float2(v[o + 2], v[o + 3]), hi);
                } else {
                    mid = __ffma2_rn(make_float2(wr[k], wr[k]), make_float2(v[o + 1], v[o + 2]), mid);
                    e0 = fmaf(wr[k], v[o], e0);
                    e3 = fmaf(wr[k], v[o + 3], e3);
                }
            }
            reinterpret_cast<float4 *>(s_h + r * kTileW)[g] =
                make_float4(lo.x + e0, lo.y + mid.x, hi.x + mid.y, hi.y + e3);
        }
        __syncthreads();
        // vertical: 16 column groups x 16 row pairs, one block per thread
        const int g = threadIdx.x & 15, rp = threadIdx.x >> 4;
        float4 col[2 + 2 * R];
#pragma unroll
        for (int k = 0; k < 2 + 2 * R; ++k) col[k] = reinterpret_cast<const float4 *>(s_h + (2 * rp + k) * kTileW)[g];
        float2 a01 = make_float2(0.f, 0.f), a23 = a01, b01 = a01, b23 = a01;
#pragma unroll
        for (int k = 0; k <= 2 * R; ++k) {
            const float2 wk = make_float2(wr[k], wr[k]);
            a01 = __ffma2_rn(wk, make_float2(col[k].x, col[k].y), a01);
            a23 = __ffma2_rn(wk, make_float2(col[k].z, col[k].w), a23);
            b01 = __ffma2_rn(wk, make_float2(col[k + 1].x, col[k + 1].y), b01);
            b23 = __ffma2_rn(wk, make_float2(col[k + 1].z, col[k + 1].w), b23);
        }
        store_2x4(out, rows, cols, x0 + 4 * g, y0 + 2 * rp, make_float4(a01.x, a01.y, a23.x, a23.y),
                  make_float4(b01.x, b01.y, b23.x, b23.y));
        staged = staged_next;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
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

// Sobel magnitude: gx = right column - left column with weights (1, 2, 1),
// gy = bottom row - top row with weights (1, 2, 1); out = sqrt(gx^2 + gy^2).
// Each thread makes a 4-column x 2-row block from a 6 x 4 window.
__global__ void __launch_bounds__(kImgThreads) sobel_kernel(const float *__restrict__ in, float *__restrict__ out,
                                                            int rows, int cols)
{
    constexpr int HALO = 4, IW = kTileW + 2 * HALO, IH = kTileH + 2;
    __shared__ __align__(16) float s[IH * IW];
    const int x0 = blockIdx.x * kTileW, y0 = blockIdx.y * kTileH;
    stage_tile<1, HALO, IW>(in, s, rows, cols, x0, y0);
    __syncthreads();
    const int g = threadIdx.x & 15, rp = threadIdx.x >> 4;
    float m[4][12];  // staged rows 2rp .. 2rp+3, columns 4g .. 4g+11 (pixel 4g+c-HALO)
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float4 q = reinterpret_cast<const float4 *>(s + (2 * rp + r) * IW + 4 * g)[k];
            m[r][4 * k] = q.x;
            m[r][4 * k + 1] = q.y;
            m[r][4 * k + 2] = q.z;
            m[r][4 * k + 3] = q.w;
        }
    float o[2][4];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = HALO + j;  // the output pixel's column in m
            const float a = m[h][c - 1], b = m[h][c], cc = m[h][c + 1];
            const float d = m[h + 1][c - 1], f = m[h + 1][c + 1];
            const float gg = m[h + 2][c - 1], hh = m[h + 2][c], i = m[h + 2][c + 1];
            const float gx = (cc + 2.f * f + i) - (a + 2.f * d + gg);
            const float gy = (gg + 2.f * hh + i) - (a + 2.f * b + cc);
            o[h][j] = sobel_mag(gx, gy);
        }
    store_2x4(out, rows, cols, x0 + 4 * g, y0 + 2 * rp, make_float4(o[0][0], o[0][1], o[0][2], o[0][3]),
              make_float4(o[1][0], o[1][1], o[1][2], o[1][3]));
}

// (min, max) of n floats -> mm[0], mm[1].  Exact (min and max round
// nothing); blocks publish their pair, the last block combines in order.
__global__ void __launch_bounds__(kThreads) minmax_kernel(const float *__restrict__ x, float *__restrict__ mm,
                                                          double *scratch, int64_t n)
{
    __shared__ float smin[kThreads / 32], smax[kThreads / 32];
    float lo = INFINITY, hi = -INFINITY;
    if ((reinterpret_cast<uintptr_t>(x) & 15) == 0) {
        const float4 *x4 = reinterpret_cast<const float4 *>(x);
        const int64_t n4 = n >> 2;
        const int64_t tile = (int64_t)kThreads * kUnroll;
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
                    lo = fminf(lo, fminf(fminf(v[k].x, v[k].y), fminf(v[k].z, v[k].w)));
                    hi = fmaxf(hi, fmaxf(fmaxf(v[k].x, v[k].y), fmaxf(v[k].z, v[k].w)));
                }
            }
        }
        if (blockIdx.x == 0 && threadIdx.x < (n & 3)) {
            float t = x[(n4 << 2) + threadIdx.x];
            lo = fminf(lo, t);
            hi = fmaxf(hi, t);
        }
    } else {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
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
    float2 *part = reinterpret_cast<float2 *>(scratch);
    if (threadIdx.x < 32) {
        lo = lane < kThreads / 32 ? smin[lane] : INFINITY;
        hi = lane < kThreads / 32 ? smax[lane] : -INFINITY;
        lo = warp_min(lo);
        hi = warp_max(hi);
        if (lane == 0) part[blockIdx.x] = make_float2(lo, hi);
    }
    unsigned *counter = reinterpret_cast<unsigned *>(scratch + 2 * kReduceMaxBlocks);
    if (!arrive_last(counter)) return;
    if (threadIdx.x < 32) {
        lo = INFINITY;
        hi = -INFINITY;
        for (unsigned b = lane; b < gridDim.x; b += 32) {
            const volatile float *pv = reinterpret_cast<volatile float *>(part + b);
            lo = fminf(lo, pv[0]);
            hi = fmaxf(hi, pv[1]);
        }
        lo = warp_min(lo);
        hi = warp_max(hi);
        if (lane == 0) {
            mm[0] = lo;
            mm[1] = hi;
            *counter = 0u;
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
unsigned stencil_grid(const void *fn, int &per_sm, int rows, int cols)
{
    const int64_t tiles = ceil_div(cols, kTileW) * ceil_div(rows, kTileH);
    return fused_grid(fn, kImgThreads, tiles, per_sm);
}

template <int R> void blur_launch(const LaunchArgs &a, cudaStream_t s)
{
    int rows = a.i32(3), cols = a.i32(4);
    static int per_sm = 0;
    const unsigned g = stencil_grid((const void *)gauss_blur_kernel<R>, per_sm, rows, cols);
    gauss_blur_kernel<R><<<g, kImgThreads, 0, s>>>(a.p<float>(0), a.p<float>(1), a.p<float>(2), rows, cols);
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
    dim3 g((unsigned)ceil_div(cols, kTileW), (unsigned)ceil_div(rows, kTileH));
    sobel_kernel<<<g, kImgThreads, 0, (cudaStream_t)s>>>(a.p<float>(0), a.p<float>(1), rows, cols);
    return cudaGetLastError();
}

const char *validate_minmax(const LaunchArgs &a)
{
    int64_t n = a.i64(3);
    if (n <= 0) return "n must be > 0";
    if (a.bytes[0] / 4 < (size_t)n) return "input smaller than n floats";
    if (a.bytes[1] < 8) return "mm smaller than two floats";
    if (a.bytes[2] < reduce_scratch_bytes<2>()) return "scratch smaller than gdag_scratch_bytes()";
    return nullptr;
}

int launch_minmax(const LaunchArgs &a, void *s)
{
    int64_t n = a.i64(3);
    minmax_kernel<<<reduce_grid(n >> 2), kThreads, 0, (cudaStream_t)s>>>(a.p<float>(0), a.p<float>(1),
                                                                         a.p<double>(2), n);
    return cudaGetLastError();
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
