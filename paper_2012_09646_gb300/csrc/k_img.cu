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
constexpr int kTx = 64, kTy = 4;          // block shape
constexpr int kMaxRadius = 8;

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Separable Gaussian blur with radius R: horizontal pass from the staged
// input into shared memory, vertical pass from there to the output.  Per
// output: 2(2R+1) FMAs; DRAM: one read and one write of the image.
template <int R>
__global__ void __launch_bounds__(kTx *kTy) gauss_blur_kernel(const float *__restrict__ in, float *__restrict__ out,
                                                              const float *__restrict__ w, int rows, int cols)
{
    constexpr int IW = kTileW + 2 * R, IH = kTileH + 2 * R;
    __shared__ float s_in[IH][IW];
    __shared__ float s_h[IH][kTileW];
    __shared__ float s_w[2 * R + 1];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kTx + tx;
    const int x0 = blockIdx.x * kTileW, y0 = blockIdx.y * kTileH;
    if (tid < 2 * R + 1) s_w[tid] = w[tid];
    for (int r = ty; r < IH; r += kTy) {
        const size_t row = (size_t)clampi(y0 + r - R, 0, rows - 1) * cols;
        for (int c = tx; c < IW; c += kTx) s_in[r][c] = in[row + clampi(x0 + c - R, 0, cols - 1)];
    }
    __syncthreads();
    for (int r = ty; r < IH; r += kTy) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k <= 2 * R; ++k) acc = fmaf(s_w[k], s_in[r][tx + k], acc);
        s_h[r][tx] = acc;
    }
    __syncthreads();
    const int x = x0 + tx;
    if (x >= cols) return;
    for (int r = ty; r < kTileH; r += kTy) {
        const int y = y0 + r;
        if (y >= rows) break;
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k <= 2 * R; ++k) acc = fmaf(s_w[k], s_h[r + k][tx], acc);
        out[(size_t)y * cols + x] = acc;
    }
}

// Sobel magnitude: gx = right column - left column with weights (1, 2, 1),
// gy = bottom row - top row with weights (1, 2, 1); out = sqrt(gx^2 + gy^2).
__global__ void __launch_bounds__(kTx *kTy) sobel_kernel(const float *__restrict__ in, float *__restrict__ out,
                                                         int rows, int cols)
{
    constexpr int IW = kTileW + 2, IH = kTileH + 2;
    __shared__ float s[IH][IW];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x0 = blockIdx.x * kTileW, y0 = blockIdx.y * kTileH;
    for (int r = ty; r < IH; r += kTy) {
        const size_t row = (size_t)clampi(y0 + r - 1, 0, rows - 1) * cols;
        for (int c = tx; c < IW; c += kTx) s[r][c] = in[row + clampi(x0 + c - 1, 0, cols - 1)];
    }
    __syncthreads();
    const int x = x0 + tx;
    if (x >= cols) return;
    for (int r = ty; r < kTileH; r += kTy) {
        const int y = y0 + r;
        if (y >= rows) break;
        const float a = s[r][tx], b = s[r][tx + 1], c = s[r][tx + 2];
        const float d = s[r + 1][tx], f = s[r + 1][tx + 2];
        const float g = s[r + 2][tx], h = s[r + 2][tx + 1], i = s[r + 2][tx + 2];
        const float gx = (c + 2.f * f + i) - (a + 2.f * d + g);
        const float gy = (g + 2.f * h + i) - (a + 2.f * b + c);
        out[(size_t)y * cols + x] = sqrtf(gx * gx + gy * gy);
    }
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

template <int R> void blur_launch(const LaunchArgs &a, cudaStream_t s)
{
    int rows = a.i32(3), cols = a.i32(4);
    dim3 g((unsigned)ceil_div(cols, kTileW), (unsigned)ceil_div(rows, kTileH));
    gauss_blur_kernel<R><<<g, dim3(kTx, kTy), 0, s>>>(a.p<float>(0), a.p<float>(1), a.p<float>(2), rows, cols);
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
    sobel_kernel<<<g, dim3(kTx, kTy), 0, (cudaStream_t)s>>>(a.p<float>(0), a.p<float>(1), rows, cols);
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
