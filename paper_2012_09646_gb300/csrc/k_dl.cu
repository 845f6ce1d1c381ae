// DL nodes (Section IV-B, DL): a convolutional network projects two images to
// low-dimensional embeddings and combines them with a dense layer.
//   conv3x3_relu_pool  3x3 convolution (3 -> 64 channels, zero padding 1) +
//                      bias + ReLU + 2x2 max-pool, bf16 NCHW in and out, fp32
//                      accumulation on the tcgen05 tensor cores
//   avgpool_global     mean of every (image, channel) plane -> f32 embedding
//   concat_dense       out = [e1 e2] wd + bd, fp32
//
// conv3x3_relu_pool is an implicit GEMM: one CTA owns two output rows x 64
// output columns of one image, i.e. M = 128 pixels, N = 64 channels and
// K = 27 taps (3 channels x 3 x 3) padded to 32.  The CTA stages its input
// halo in shared memory, builds the im2col tile A (128 x 32) and the weights B
// (64 x 32) in the canonical K-major layout without swizzle (8-row x 16-byte
// core matrices; 128 B between core matrices adjacent in K, 512 B between
// core matrices adjacent in M or N), and one thread issues two
// tcgen05.mma.cta_group::1.kind::f16 (K = 16 each) into a 128-lane x 64-column
// fp32 accumulator in tensor memory.  Completion comes through
// tcgen05.commit on an mbarrier; the epilogue reads the accumulator with
// tcgen05.ld (one pixel per thread, 64 channels), takes the 2x2 maximum
// (horizontal pairs by shuffle, the two rows through shared memory), adds the
// bias and applies ReLU after the pooling (both commute with the maximum),
// and writes the pooled bf16 outputs.  Every wait is bounded: past about one
// second the CTA records status[0] = 1, skips its epilogue, frees its tensor
// memory and returns.
#include <cuda_bf16.h>

#include <initializer_list>
#include <vector>

#include "catalog.h"
#include "kcommon.cuh"

namespace gdag {

constexpr int kConvM = 128, kConvN = 64, kConvK = 32, kConvTaps = 27;
constexpr int kConvCols = 64;  // output columns per CTA
constexpr int kConvThreads = 128;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of (row, k) in the canonical K-major, no-swizzle layout
__device__ __forceinline__ int umma_off(int row, int k)
{
    return ((row >> 3) * (kConvK / 8) + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// shared-memory matrix descriptor (sm_100): start >> 4, leading byte offset
// (between K-adjacent core matrices) >> 4 at bit 16, stride byte offset
// (between M/N-adjacent core matrices) >> 4 at bit 32, version 1 at bit 46,
// no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr)
{
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) |
           ((uint64_t)((kConvK / 8) * 128 >> 4) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: D f32, A and B bf16, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t kConvIdesc =
    (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kConvN >> 3) << 17) | ((uint32_t)(kConvM >> 4) << 24);

__global__ void __launch_bounds__(kConvThreads) conv3x3_relu_pool_kernel(const __nv_bfloat16 *__restrict__ x,
                                                                         const __nv_bfloat16 *__restrict__ wt,
                                                                         const float *__restrict__ bias,
                                                                         __nv_bfloat16 *__restrict__ out,
                                                                         int *status, int n, int h, int w)
{
    __shared__ __align__(128) unsigned char sa[kConvM * kConvK * 2];
    __shared__ __align__(128) unsigned char sb[kConvN * kConvK * 2];
    __shared__ __nv_bfloat16 s_in[3][4][kConvCols + 2];
    __shared__ float s_pool[kConvN][kConvCols / 2 + 1];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_x = w / kConvCols, rows2 = h / 2;
    const int bx = blockIdx.x % tiles_x;
    const int by = (blockIdx.x / tiles_x) % rows2;
    const int b = blockIdx.x / (tiles_x * rows2);
    const int y0 = 2 * by, x0 = bx * kConvCols;

    // input halo: channels 0..2, rows y0-1 .. y0+2, columns x0-1 .. x0+64
    for (int i = tid; i < 3 * 4 * (kConvCols + 2); i += kConvThreads) {
        const int ch = i / (4 * (kConvCols + 2)), rem = i - ch * 4 * (kConvCols + 2);
        const int r = rem / (kConvCols + 2), c = rem - r * (kConvCols + 2);
        const int yy = y0 - 1 + r, xx = x0 - 1 + c;
        const bool in = yy >= 0 && yy < h && xx >= 0 && xx < w;
        s_in[ch][r][c] = in ? x[(((size_t)b * 3 + ch) * h + yy) * w + xx] : __float2bfloat16(0.f);
    }
    // weights B: row co, column k = ci*9 + dy*3 + dx, zero past 27
    for (int i = tid; i < kConvN * kConvK; i += kConvThreads) {
        const int co = i / kConvK, k = i - co * kConvK;
        *reinterpret_cast<__nv_bfloat16 *>(sb + umma_off(co, k)) =
            k < kConvTaps ? wt[co * kConvTaps + k] : __float2bfloat16(0.f);
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(smem_addr(&tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    __syncthreads();

    // im2col row of this thread's pixel: p = r * 64 + c
    {
        const int r = tid >> 6, c = tid & 63;
        __nv_bfloat16 v[kConvK];
#pragma unroll
        for (int k = 0; k < kConvK; ++k) {
            if (k < kConvTaps) {
                const int ci = k / 9, dy = (k % 9) / 3, dx = k % 3;
                v[k] = s_in[ci][r + dy][c + dx];
            } else {
                v[k] = __float2bfloat16(0.f);
            }
        }
#pragma unroll
        for (int kc = 0; kc < kConvK / 8; ++kc) {
            uint4 q;
            q.x = (uint32_t)__bfloat16_as_ushort(v[8 * kc + 0]) | ((uint32_t)__bfloat16_as_ushort(v[8 * kc + 1]) << 16);
            q.y = (uint32_t)__bfloat16_as_ushort(v[8 * kc + 2]) | ((uint32_t)__bfloat16_as_ushort(v[8 * kc + 3]) << 16);
            q.z = (uint32_t)__bfloat16_as_ushort(v[8 * kc + 4]) | ((uint32_t)__bfloat16_as_ushort(v[8 * kc + 5]) << 16);
            q.w = (uint32_t)__bfloat16_as_ushort(v[8 * kc + 6]) | ((uint32_t)__bfloat16_as_ushort(v[8 * kc + 7]) << 16);
            *reinterpret_cast<uint4 *>(sa + umma_off(tid, 8 * kc)) = q;
        }
    }
    asm volatile("fence.proxy.async.shared::cta;");  // generic-proxy stores -> tensor core reads
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    if (tid == 0) {
#pragma unroll
        for (int ks = 0; ks < kConvK / 16; ++ks) {
            const uint64_t ad = umma_desc(smem_addr(sa) + ks * 256);
            const uint64_t bd = umma_desc(smem_addr(sb) + ks * 256);
            asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                         " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                         "l"(ad), "l"(bd), "r"(kConvIdesc), "r"((uint32_t)ks));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_addr(&mbar)));
    }
    // bounded wait for the accumulator (about 1 s at GB300 clocks)
    uint32_t ok = 0;
    const long long t0 = clock64();
    while (!ok) {
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(ok)
                     : "r"(smem_addr(&mbar)));
        if (!ok && clock64() - t0 > 2000000000LL) break;
    }
    ok = __syncthreads_and(ok);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!ok) {
        if (tid == 0) atomicExch(status, 1);
    } else {
        uint32_t acc[kConvN];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,"
            "%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
            : "=r"(acc[0]), "=r"(acc[1]), "=r"(acc[2]), "=r"(acc[3]), "=r"(acc[4]), "=r"(acc[5]), "=r"(acc[6]),
              "=r"(acc[7]), "=r"(acc[8]), "=r"(acc[9]), "=r"(acc[10]), "=r"(acc[11]), "=r"(acc[12]), "=r"(acc[13]),
              "=r"(acc[14]), "=r"(acc[15]), "=r"(acc[16]), "=r"(acc[17]), "=r"(acc[18]), "=r"(acc[19]),
              "=r"(acc[20]), "=r"(acc[21]), "=r"(acc[22]), "=r"(acc[23]), "=r"(acc[24]), "=r"(acc[25]),
              "=r"(acc[26]), "=r"(acc[27]), "=r"(acc[28]), "=r"(acc[29]), "=r"(acc[30]), "=r"(acc[31]),
              "=r"(acc[32]), "=r"(acc[33]), "=r"(acc[34]), "=r"(acc[35]), "=r"(acc[36]), "=r"(acc[37]),
              "=r"(acc[38]), "=r"(acc[39]), "=r"(acc[40]), "=r"(acc[41]), "=r"(acc[42]), "=r"(acc[43]),
              "=r"(acc[44]), "=r"(acc[45]), "=r"(acc[46]), "=r"(acc[47]), "=r"(acc[48]), "=r"(acc[49]),
              "=r"(acc[50]), "=r"(acc[51]), "=r"(acc[52]), "=r"(acc[53]), "=r"(acc[54]), "=r"(acc[55]),
              "=r"(acc[56]), "=r"(acc[57]), "=r"(acc[58]), "=r"(acc[59]), "=r"(acc[60]), "=r"(acc[61]),
              "=r"(acc[62]), "=r"(acc[63])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        // pixel p = warp*32 + lane: row p / 64, column p % 64; pool pairs of
        // columns (lanes l, l^1), then the two rows (warps w, w+2)
        float v[kConvN];
#pragma unroll
        for (int ch = 0; ch < kConvN; ++ch) {
            const float a = __uint_as_float(acc[ch]);
            v[ch] = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, 1));
        }
        const int c = (tid & 63), pc = c >> 1;
        if (warp >= 2 && (lane & 1) == 0) {
#pragma unroll
            for (int ch = 0; ch < kConvN; ++ch) s_pool[ch][pc] = v[ch];
        }
        __syncthreads();
        if (warp < 2 && (lane & 1) == 0) {
            const int ho = h / 2, wo = w / 2;
            __nv_bfloat16 *o = out + (((size_t)b * kConvN) * ho + by) * wo + (x0 >> 1) + pc;
#pragma unroll
            for (int ch = 0; ch < kConvN; ++ch) {
                const float m = fmaxf(v[ch], s_pool[ch][pc]) + bias[ch];
                o[(size_t)ch * ho * wo] = __float2bfloat16_rn(fmaxf(m, 0.f));
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem));
}

// e[p] = mean of plane p (hw bf16 values): 128-bit loads, fp32 per thread,
// fixed-order block tree; one block per plane.
__global__ void __launch_bounds__(256) avgpool_global_kernel(const __nv_bfloat16 *__restrict__ p,
                                                             float *__restrict__ e, int hw)
{
    __shared__ double sh[256 / 32];
    const uint4 *q = reinterpret_cast<const uint4 *>(p + (size_t)blockIdx.x * hw);
    float s = 0.f;
    for (int i = threadIdx.x; i < hw / 8; i += 256) {
        const uint4 v = q[i];
        const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            s += __uint_as_float(u[k] << 16);
            s += __uint_as_float(u[k] & 0xFFFF0000u);
        }
    }
    const double t = block_sum((double)s, sh);
    if (threadIdx.x == 0) e[blockIdx.x] = (float)(t / hw);
}

// out[b][j] = bd[j] + sum_i e1[b][i] wd[i][j] + sum_i e2[b][i] wd[c+i][j]
__global__ void concat_dense_kernel(const float *__restrict__ e1, const float *__restrict__ e2,
                                    const float *__restrict__ wd, const float *__restrict__ bd,
                                    float *__restrict__ out, int n, int c, int classes)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * classes) return;
    const int b = t / classes, j = t - b * classes;
    float s = bd[j];
    for (int i = 0; i < c; ++i) s = fmaf(e1[b * c + i], wd[i * classes + j], s);
    for (int i = 0; i < c; ++i) s = fmaf(e2[b * c + i], wd[(c + i) * classes + j], s);
    out[t] = s;
}

namespace {

const char *validate_conv(const LaunchArgs &a)
{
    const int n = a.i32(5), h = a.i32(6), w = a.i32(7);
    if (n < 1 || h < 2 || w < kConvCols) return "n >= 1, h >= 2, w >= 64 required";
    if (h % 2 || w % kConvCols) return "h must be even and w a multiple of 64";
    if ((int64_t)n * (h / 2) * (w / kConvCols) > INT32_MAX) return "too many tiles";
    if (a.bytes[0] / 2 / 3 / (size_t)h / (size_t)w < (size_t)n) return "x smaller than n x 3 x h x w bf16";
    if (a.bytes[1] < (size_t)kConvN * kConvTaps * 2) return "weights smaller than 64 x 3 x 3 x 3 bf16";
    if (a.bytes[2] < (size_t)kConvN * 4) return "bias smaller than 64 floats";
    if (a.bytes[3] / 2 / kConvN / (size_t)(h / 2) / (size_t)(w / 2) < (size_t)n)
        return "out smaller than n x 64 x h/2 x w/2 bf16";
    if (a.bytes[4] < 4) return "status smaller than one int32";
    return nullptr;
}

int launch_conv(const LaunchArgs &a, void *s)
{
    const int n = a.i32(5), h = a.i32(6), w = a.i32(7);
    const unsigned grid = (unsigned)((int64_t)n * (h / 2) * (w / kConvCols));
    conv3x3_relu_pool_kernel<<<grid, kConvThreads, 0, (cudaStream_t)s>>>(
        a.p<__nv_bfloat16>(0), a.p<__nv_bfloat16>(1), a.p<float>(2), a.p<__nv_bfloat16>(3), a.p<int>(4), n, h, w);
    return cudaGetLastError();
}

const char *validate_avgpool(const LaunchArgs &a)
{
    const int planes = a.i32(2), hw = a.i32(3);
    if (planes < 1 || hw < 8 || hw % 8) return "planes >= 1 and hw a positive multiple of 8 required";
    if (a.bytes[0] / 2 / (size_t)hw < (size_t)planes) return "input smaller than planes x hw bf16";
    if (a.bytes[1] / 4 < (size_t)planes) return "e smaller than planes floats";
    if ((reinterpret_cast<uintptr_t>(a.ptr[0]) & 15) != 0) return "input must be 16-byte aligned";
    return nullptr;
}

int launch_avgpool(const LaunchArgs &a, void *s)
{
    avgpool_global_kernel<<<(unsigned)a.i32(2), 256, 0, (cudaStream_t)s>>>(a.p<__nv_bfloat16>(0), a.p<float>(1),
                                                                           a.i32(3));
    return cudaGetLastError();
}

const char *validate_dense(const LaunchArgs &a)
{
    const int n = a.i32(5), c = a.i32(6), k = a.i32(7);
    if (n < 1 || c < 1 || k < 1) return "n, c and classes must be >= 1";
    if (a.bytes[0] / 4 / (size_t)c < (size_t)n || a.bytes[1] / 4 / (size_t)c < (size_t)n)
        return "e1 or e2 smaller than n x c floats";
    if (a.bytes[2] / 4 / (size_t)k < (size_t)2 * c) return "wd smaller than 2c x classes floats";
    if (a.bytes[3] / 4 < (size_t)k) return "bd smaller than classes floats";
    if (a.bytes[4] / 4 / (size_t)k < (size_t)n) return "out smaller than n x classes floats";
    return nullptr;
}

int launch_dense(const LaunchArgs &a, void *s)
{
    const int n = a.i32(5), k = a.i32(7);
    concat_dense_kernel<<<(unsigned)ceil_div((int64_t)n * k, 128), 128, 0, (cudaStream_t)s>>>(
        a.p<float>(0), a.p<float>(1), a.p<float>(2), a.p<float>(3), a.p<float>(4), n, a.i32(6), k);
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

void append_dl_kernels(std::vector<KernelEntry> &v)
{
    v.push_back(entry("conv3x3_relu_pool", (const void *)conv3x3_relu_pool_kernel,
                      {arr(GDAG_MODE_IN), arr(GDAG_MODE_IN), arr(GDAG_MODE_IN), arr(GDAG_MODE_OUT),
                       arr(GDAG_MODE_INOUT), scal(4), scal(4), scal(4)},
                      validate_conv, launch_conv));
    v.push_back(entry("avgpool_global", (const void *)avgpool_global_kernel,
                      {arr(GDAG_MODE_IN), arr(GDAG_MODE_OUT), scal(4), scal(4)}, validate_avgpool, launch_avgpool));
    v.push_back(entry("concat_dense", (const void *)concat_dense_kernel,
                      {arr(GDAG_MODE_IN), arr(GDAG_MODE_IN), arr(GDAG_MODE_IN), arr(GDAG_MODE_IN), arr(GDAG_MODE_OUT),
                       scal(4), scal(4), scal(4)},
                      validate_dense, launch_dense));
}

}  // namespace gdag
