// B&S node (Section IV-B, B&S): Black-Scholes price of a European call for
// every spot price of a vector, fp32.
//   d1 = (ln(S/K) + (r + sigma^2/2) T) / (sigma sqrt(T)),  d2 = d1 - sigma sqrt(T)
//   C  = S N(d1) - K exp(-rT) N(d2)
//
// N is evaluated through the Mills ratio R(z) = (1 - N(z)) / phi(z):
// N(x) = phi(x) R(-x) for x < 0 and 1 - phi(x) R(x) for x >= 0, with R a
// rational function P(z)/Q(z) of degrees 4/5 whose coefficients are all
// positive (fp32 Horner without cancellation); relative error of R about
// 4e-8 on [0, 4] and below 1e-6 on [0, 1e5] (beyond 4 the tail it scales is
// below 3e-5).  The fit is derived in fit_mills_ratio.py, which prints the
// coefficients rescaled to z with P pre-multiplied by 1/sqrt(2 pi), the
// constant of phi.
//
// GB300 specifics.  The kernel reads 4 and writes 4 bytes per option, so it
// is HBM-bound only if it stays near 35 instructions per option; therefore:
//  - d1 and d2 travel as one float2 through the packed fp32x2 FMA/MUL of
//    sm_100+ (__ffma2_rn, __fmul2_rn): both CDFs cost one Horner chain;
//  - the transcendentals are single MUFU operations written as PTX:
//    lg2.approx for the logarithm, ex2.approx for phi, rcp.approx for each
//    1/Q (five per option: the multiply pipe, not the MUFU pipe, is the
//    busier one, so one reciprocal of Q(z1) Q(z2) and a packed multiply to
//    split it would cost more than the reciprocal they save);
//  - d1 = lg2(S) (ln2 / (sigma sqrt T)) + (drift - ln K) / (sigma sqrt T) is
//    one FMA, with both constants computed in double on the host.
// Error: a shift e common to d1 and d2 (the logarithm's error, the rounding
// of the constants) changes C only to second order, because
// S phi(d1) = K exp(-rT) phi(d2); what remains is each N's own error.  (That
// is why phi(d2) is evaluated from d2 itself: deriving it from phi(d1) by the
// same identity would save an ex2 but lose this cancellation.)
// Conditioning: C is a difference of two terms of size ~S, so for
// sigma sqrt(T) well below 1e-2 an fp32 price near the strike carries an
// error of a few ulp of S, whatever the evaluation.
#include <cmath>
#include <vector>

#include "catalog.h"
#include "kcommon.cuh"

namespace gdag {

struct BsConst {
    float a, b;     // d1 = lg2(S) a + b
    float vol;      // sigma sqrt(T): d2 = d1 - vol
    float k_disc;   // K exp(-rT)
};

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }

__device__ __forceinline__ float lg2_approx(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// (N(d.x), N(d.y)).  |d| is clamped at 40, where phi has long underflowed to
// 0 in fp32 (and P, Q would overflow for |d| > 1e5).
__device__ __forceinline__ float2 norm_cdf2(float2 d)
{
    const float2 z = make_float2(fminf(fabsf(d.x), 40.0f), fminf(fabsf(d.y), 40.0f));
    float2 p = f2(5.286688848e-03f);
    p = __ffma2_rn(p, z, f2(4.807076126e-02f));
    p = __ffma2_rn(p, z, f2(2.045669649e-01f));
    p = __ffma2_rn(p, z, f2(4.659080207e-01f));
    p = __ffma2_rn(p, z, f2(5.000000162e-01f));
    float2 q = f2(1.325175100e-02f);
    q = __ffma2_rn(q, z, f2(1.204967448e-01f));
    q = __ffma2_rn(q, z, f2(5.259802458e-01f));
    q = __ffma2_rn(q, z, f2(1.289215420e+00f));
    q = __ffma2_rn(q, z, f2(1.729702769e+00f));
    q = __ffma2_rn(q, z, f2(1.000000000e+00f));
    const float2 t = __fmul2_rn(__fmul2_rn(z, z), f2(-7.213475204e-01f));  // -z^2 log2(e) / 2
    const float2 e = make_float2(ex2_approx(t.x), ex2_approx(t.y));
    const float2 inv_q = make_float2(rcp_approx(q.x), rcp_approx(q.y));
    const float2 tail = __fmul2_rn(__fmul2_rn(p, inv_q), e);                // phi(z) R(z)
    return make_float2(d.x < 0.f ? tail.x : 1.0f - tail.x, d.y < 0.f ? tail.y : 1.0f - tail.y);
}

__device__ __forceinline__ float bs_price(float s, const BsConst &c)
{
    const float d1 = fmaf(lg2_approx(s), c.a, c.b);
    const float2 n = norm_cdf2(make_float2(d1, d1 - c.vol));
    return s * n.x - c.k_disc * n.y;
}

__device__ __forceinline__ float4 bs_price4(float4 v, const BsConst &c)
{
    return make_float4(bs_price(v.x, c), bs_price(v.y, c), bs_price(v.z, c), bs_price(v.w, c));
}

// 8 bytes of HBM traffic per option (4 in, 4 out); streaming loads/stores
// (each byte is touched once).  A block works through chunks of
// kBsUnroll float4s per thread: all kBsUnroll loads of a thread are issued
// before any pricing (64 bytes in flight per thread), then the chunk is
// priced and stored.  At most 256 threads a block and at least four blocks
// an SM leave 64 registers a thread: enough to keep the rational function's
// constants (packed pairs) in registers instead of re-materialising them for
// every option, which at a 40-register cap cost about a quarter of the
// kernel's time.
constexpr int kBsThreads = 256;
constexpr int kBsUnroll = 4;

// Options [base4*4, ...) of one chunk: float4s base4 + threadIdx.x + k*bd
// for k < kBsUnroll, below n4.
__device__ __forceinline__ void bs_chunk(const float4 *__restrict__ S4, float4 *__restrict__ C4, int64_t n4,
                                         int64_t base4, int64_t bd, const BsConst &c)
{
    float4 v[kBsUnroll];
#pragma unroll
    for (int k = 0; k < kBsUnroll; ++k) {
        const int64_t i = base4 + threadIdx.x + k * bd;
        if (i < n4) v[k] = __ldcs(S4 + i);
    }
#pragma unroll
    for (int k = 0; k < kBsUnroll; ++k) {
        const int64_t i = base4 + threadIdx.x + k * bd;
        if (i < n4) __stcs(C4 + i, bs_price4(v[k], c));
    }
}

// Blocks stride over chunks.  TH > 0 fixes the block size at compile time
// (the automatic launch shape: 256 threads, two resident waves, so the
// index arithmetic folds to constants); TH = 0 takes blockDim.x (explicit
// launch shapes, e.g. from the autotuner).
template <int TH>
__global__ void __launch_bounds__(kBsThreads, 4) bs_call_kernel(const float *__restrict__ S, float *__restrict__ C,
                                                                int64_t n, BsConst c)
{
    const int64_t bd = TH > 0 ? TH : blockDim.x;
    if (((reinterpret_cast<uintptr_t>(S) | reinterpret_cast<uintptr_t>(C)) & 15) == 0) {
        const int64_t n4 = n >> 2, chunk = bd * kBsUnroll;
        for (int64_t base = (int64_t)blockIdx.x * chunk; base < n4; base += (int64_t)gridDim.x * chunk)
            bs_chunk(reinterpret_cast<const float4 *>(S), reinterpret_cast<float4 *>(C), n4, base, bd, c);
        if (blockIdx.x == 0 && threadIdx.x < (n & 3)) {
            const int64_t t = (n4 << 2) + threadIdx.x;
            C[t] = bs_price(S[t], c);
        }
    } else {
        for (int64_t i = (int64_t)blockIdx.x * bd + threadIdx.x; i < n; i += (int64_t)gridDim.x * bd)
            C[i] = bs_price(S[i], c);
    }
}

// Fused form: the work items are chunks of kBsChunk options (one bs_chunk
// of kBsThreads threads); member m owns chunks [start[m], start[m+1]), its
// last chunk also pricing the n & 3 scalar tail (or, when S or C is not
// 16-byte aligned, the chunk's options one by one).  Every option gets the
// same arithmetic as in bs_call_kernel, so each member's prices equal its
// plain launch's.  Each block takes one contiguous range of chunks and
// finds its first member by binary search, then steps to the next member
// as its range crosses one (the member table lives in parameter memory:
// one search per block, not per chunk).
constexpr int64_t kBsChunk4 = (int64_t)kBsThreads * kBsUnroll;
constexpr int64_t kBsChunk = kBsChunk4 * 4;

// CAP members at most: the table is a kernel parameter, so a small group
// launches with a small parameter block (32 members: 1.5 KB; 128: 6 KB)
template <int CAP> struct BsFused {
    int count;
    int64_t start[CAP + 1];
    const float *S[CAP];
    float *C[CAP];
    int64_t n[CAP];
    BsConst c[CAP];
};

template <int CAP>
__global__ void __launch_bounds__(kBsThreads, 4) bs_call_fused_kernel(const __grid_constant__ BsFused<CAP> t)
{
    const int64_t total = t.start[t.count];
    const int64_t per = (total + gridDim.x - 1) / gridDim.x;
    const int64_t it0 = (int64_t)blockIdx.x * per;
    const int64_t it1 = it0 + per < total ? it0 + per : total;
    if (it0 >= it1) return;
    int m = fused_member(t.start, t.count, it0);
    int64_t first = t.start[m], next = t.start[m + 1];
    const float *S = t.S[m];
    float *C = t.C[m];
    int64_t n = t.n[m];
    BsConst c = t.c[m];
    for (int64_t it = it0; it < it1; ++it) {
        while (it >= next) {  // uniform across the block
            ++m;
            first = next;
            next = t.start[m + 1];
            S = t.S[m];
            C = t.C[m];
            n = t.n[m];
            c = t.c[m];
        }
        const int64_t local = it - first;
        if (((reinterpret_cast<uintptr_t>(S) | reinterpret_cast<uintptr_t>(C)) & 15) == 0) {
            const int64_t n4 = n >> 2;
            bs_chunk(reinterpret_cast<const float4 *>(S), reinterpret_cast<float4 *>(C), n4, local * kBsChunk4,
                     kBsThreads, c);
            if (it == next - 1 && threadIdx.x < (n & 3)) {
                const int64_t i = (n4 << 2) + threadIdx.x;
                C[i] = bs_price(S[i], c);
            }
        } else {
            const int64_t hi = (local + 1) * kBsChunk < n ? (local + 1) * kBsChunk : n;
            for (int64_t i = local * kBsChunk + threadIdx.x; i < hi; i += kBsThreads) C[i] = bs_price(S[i], c);
        }
    }
}

namespace {

const char *validate_bs(const LaunchArgs &a)
{
    int64_t n = a.i64(2);
    if (n < 0) return "n < 0";
    if (a.bytes[0] / 4 < (size_t)n || a.bytes[1] / 4 < (size_t)n) return "S or C smaller than n floats";
    if (!(a.f32(3) > 0.f) || !(a.f32(5) > 0.f) || !(a.f32(6) > 0.f)) return "K, sigma and T must be > 0";
    if (!a.auto_cfg && (int64_t)a.block[0] * a.block[1] * a.block[2] > kBsThreads) return "blocks of at most 256 threads";
    return nullptr;
}

// The kernel's constants from (K, r, sigma, T), computed in double.
BsConst bs_const(const LaunchArgs &a)
{
    const double K = a.f32(3), r = a.f32(4), sigma = a.f32(5), T = a.f32(6);
    const double vol = sigma * std::sqrt(T);
    BsConst c;
    c.a = (float)(std::log(2.0) / vol);
    c.b = (float)(((r + 0.5 * sigma * sigma) * T - std::log(K)) / vol);
    c.vol = (float)vol;
    c.k_disc = (float)(K * std::exp(-r * T));
    return c;
}

int launch_bs(const LaunchArgs &a, void *s)
{
    int64_t n = a.i64(2);
    if (n == 0) return cudaSuccess;
    if (!a.auto_cfg) {
        bs_call_kernel<0><<<a.grid[0], a.block[0], 0, (cudaStream_t)s>>>(a.p<float>(0), a.p<float>(1), n,
                                                                        bs_const(a));
        return cudaGetLastError();
    }
    // four resident waves of 256-thread blocks (capped by the chunk count,
    // so at 1e7 options about one chunk a block): back to back on one
    // stream, replayed from a CUDA graph, 16.0 us per 1e7 options against
    // 17.1 us for two waves and 19.9 us for one; the hardware's block
    // scheduler fills the SMs that finish first
    static int per_sm = 0;
    const int64_t chunks = ceil_div((n >> 2) > 0 ? (n >> 2) : 1, kBsChunk4);
    const int64_t g1 = fused_grid((const void *)bs_call_kernel<kBsThreads>, kBsThreads, chunks, per_sm);
    const int64_t g = 4 * g1 < chunks ? 4 * g1 : chunks;
    bs_call_kernel<kBsThreads><<<(unsigned)g, kBsThreads, 0, (cudaStream_t)s>>>(a.p<float>(0), a.p<float>(1), n,
                                                                              bs_const(a));
    return cudaGetLastError();
}

template <int CAP> int fused_bs_cap(const LaunchArgs *a, int count, void *s)
{
    for (int off = 0; off < count; off += CAP) {
        BsFused<CAP> t;
        t.count = count - off < CAP ? count - off : CAP;
        t.start[0] = 0;
        for (int m = 0; m < t.count; ++m) {
            const LaunchArgs &la = a[off + m];
            t.S[m] = la.p<float>(0);
            t.C[m] = la.p<float>(1);
            t.n[m] = la.i64(2);
            t.c[m] = bs_const(la);
            t.start[m + 1] = t.start[m] + ceil_div(t.n[m], kBsChunk);
        }
        const int64_t total = t.start[t.count];
        if (total == 0) continue;
        static int per_sm = 0;
        const unsigned g = fused_grid((const void *)bs_call_fused_kernel<CAP>, kBsThreads, total, per_sm);
        bs_call_fused_kernel<CAP><<<g, kBsThreads, 0, (cudaStream_t)s>>>(t);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int fused_bs(const LaunchArgs *a, int count, void *s)
{
    return count <= kFuseSmall ? fused_bs_cap<kFuseSmall>(a, count, s) : fused_bs_cap<kFuseTable>(a, count, s);
}

}  // namespace

void append_bs_kernels(std::vector<KernelEntry> &v)
{
    KernelEntry e;
    e.name = "bs_call";
    e.fn = (const void *)bs_call_kernel<0>;
    e.nargs = 7;
    e.spec[0] = arr(GDAG_MODE_IN);
    e.spec[1] = arr(GDAG_MODE_OUT);
    e.spec[2] = scal(8);
    e.spec[3] = scal(4);
    e.spec[4] = scal(4);
    e.spec[5] = scal(4);
    e.spec[6] = scal(4);
    e.validate = validate_bs;
    e.launcher = launch_bs;
    e.fused = fused_bs;
    v.push_back(e);
}

}  // namespace gdag
