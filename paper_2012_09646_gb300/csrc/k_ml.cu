// ML nodes (Section IV-B, ML): naive-Bayes and ridge-regression classifiers
// combined by a softmax of each and the average of their scores.
//   dense_scores    S[i][c] = bias[c] + sum_f float(X[i][f]) T[f][c]
//                   (both classifiers: log-probability table + log prior,
//                   or weights + intercepts), X int32 row-major rows x feats
//   row_softmax     S[i][:] := exp(S[i][:] - max) / sum, in place
//   argmax_combine  labels[i] = argmax_c (P1[i][c] + P2[i][c]), ties -> lowest c
//
// dense_scores streams X once (4 bytes per feature per row) against a table
// of feats x classes floats kept in shared memory: HBM-bound at
// rows*feats*4 bytes.  Four lanes share a row, each summing a quarter of the
// features (contiguous 32-byte sectors per lane), the eight rows of a warp
// read the same table entries (shared-memory broadcast), class pairs are
// accumulated with the packed fp32x2 FMA of sm_100+, and the quarters are
// combined by a fixed shuffle tree (deterministic).
#include <initializer_list>
#include <vector>

#include "catalog.h"
#include "kcommon.cuh"

namespace gdag {

constexpr int kMlThreads = 256;
constexpr int kMlQuarters = 4;   // lanes per row
constexpr int kMlFeatStep = 8;   // features per lane per load (32 bytes)

// Shared-memory table layout: quarter q holds features [q F/4, (q+1) F/4),
// each feature a row of NC4*4 floats (classes padded to a multiple of 4);
// quarters are offset by 4 extra floats so that the four quarters' reads of
// one step fall into different banks.
__host__ __device__ constexpr int ml_quarter_stride(int feats, int nc4) { return (feats / kMlQuarters) * nc4 * 4 + 4; }

template <int NC4>
__global__ void __launch_bounds__(kMlThreads) dense_scores_kernel(const int *__restrict__ X, const float *__restrict__ T,
                                                                  const float *__restrict__ bias,
                                                                  float *__restrict__ S, int rows, int feats,
                                                                  int classes)
{
    extern __shared__ float4 smem4[];
    float *st = reinterpret_cast<float *>(smem4);
    const int fq = feats / kMlQuarters;  // features per quarter
    const int qs = ml_quarter_stride(feats, NC4);
    for (int i = threadIdx.x; i < kMlQuarters * qs; i += kMlThreads) {
        const int q = i / qs, rem = i - q * qs;
        const int f = rem / (NC4 * 4), c = rem - f * (NC4 * 4);
        st[i] = (f < fq && c < classes) ? T[(size_t)(q * fq + f) * classes + c] : 0.f;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = lane & 3;            // quarter of the features
    const int rsub = lane >> 2;        // rows rsub and rsub + 8 of the warp's 16
    const int warps_total = gridDim.x * (kMlThreads / 32);
    const float4 *tq = reinterpret_cast<const float4 *>(st + q * qs);
    for (int row0 = (blockIdx.x * (kMlThreads / 32) + warp) * 16; row0 < rows; row0 += warps_total * 16) {
        const int ra = row0 + rsub, rb = ra + 8;
        const bool la = ra < rows, lb = rb < rows;
        float2 acc_a[NC4 * 2], acc_b[NC4 * 2];
#pragma unroll
        for (int k = 0; k < NC4 * 2; ++k) acc_a[k] = acc_b[k] = make_float2(0.f, 0.f);
        const int4 *xa = reinterpret_cast<const int4 *>(X + (size_t)(la ? ra : 0) * feats + q * fq);
        const int4 *xb = reinterpret_cast<const int4 *>(X + (size_t)(lb ? rb : 0) * feats + q * fq);
        const int4 zero = make_int4(0, 0, 0, 0);
        // software pipeline: the next 8 features of both rows are in flight
        // while the current 8 are multiplied
        int4 a0 = la ? xa[0] : zero, a1 = la ? xa[1] : zero;
        int4 b0 = lb ? xb[0] : zero, b1 = lb ? xb[1] : zero;
        for (int f0 = 0; f0 < fq; f0 += kMlFeatStep) {
            const int nf = f0 + kMlFeatStep;
            int4 na0 = zero, na1 = zero, nb0 = zero, nb1 = zero;
            if (nf < fq) {
                if (la) {
                    na0 = xa[nf / 4];
                    na1 = xa[nf / 4 + 1];
                }
                if (lb) {
                    nb0 = xb[nf / 4];
                    nb1 = xb[nf / 4 + 1];
                }
            }
            const int va[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const int vb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float fa = __int2float_rn(va[j]), fb = __int2float_rn(vb[j]);
                const float2 xxa = make_float2(fa, fa), xxb = make_float2(fb, fb);
                const float4 *trow = tq + (f0 + j) * NC4;
#pragma unroll
                for (int k = 0; k < NC4; ++k) {
                    const float4 t = trow[k];
                    const float2 t01 = make_float2(t.x, t.y), t23 = make_float2(t.z, t.w);
                    acc_a[2 * k] = __ffma2_rn(xxa, t01, acc_a[2 * k]);
                    acc_a[2 * k + 1] = __ffma2_rn(xxa, t23, acc_a[2 * k + 1]);
                    acc_b[2 * k] = __ffma2_rn(xxb, t01, acc_b[2 * k]);
                    acc_b[2 * k + 1] = __ffma2_rn(xxb, t23, acc_b[2 * k + 1]);
                }
            }
            a0 = na0;
            a1 = na1;
            b0 = nb0;
            b1 = nb1;
        }
        // combine the four quarters: (q0 + q1) + (q2 + q3), same order on
        // every run
#pragma unroll
        for (int k = 0; k < NC4 * 2; ++k) {
            acc_a[k].x += __shfl_xor_sync(0xffffffffu, acc_a[k].x, 1);
            acc_a[k].y += __shfl_xor_sync(0xffffffffu, acc_a[k].y, 1);
            acc_a[k].x += __shfl_xor_sync(0xffffffffu, acc_a[k].x, 2);
            acc_a[k].y += __shfl_xor_sync(0xffffffffu, acc_a[k].y, 2);
            acc_b[k].x += __shfl_xor_sync(0xffffffffu, acc_b[k].x, 1);
            acc_b[k].y += __shfl_xor_sync(0xffffffffu, acc_b[k].y, 1);
            acc_b[k].x += __shfl_xor_sync(0xffffffffu, acc_b[k].x, 2);
            acc_b[k].y += __shfl_xor_sync(0xffffffffu, acc_b[k].y, 2);
        }
        if (q == 0) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int row = h ? rb : ra;
                if (!(h ? lb : la)) continue;
                const float2 *acc = h ? acc_b : acc_a;
                float *out = S + (size_t)row * classes;
#pragma unroll
                for (int k = 0; k < NC4 * 2; ++k) {
                    if (2 * k < classes) out[2 * k] = bias[2 * k] + acc[k].x;
                    if (2 * k + 1 < classes) out[2 * k + 1] = bias[2 * k + 1] + acc[k].y;
                }
            }
        }
    }
}

// Row softmax in place, one thread per row (classes <= 32), max-subtracted.
__global__ void __launch_bounds__(256) row_softmax_kernel(float *__restrict__ S, int rows, int classes)
{
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= rows) return;
    float v[32];
    float *s = S + (size_t)row * classes;
    float m = -INFINITY;
#pragma unroll
    for (int c = 0; c < 32; ++c)
        if (c < classes) {
            v[c] = s[c];
            m = fmaxf(m, v[c]);
        }
    float z = 0.f;
#pragma unroll
    for (int c = 0; c < 32; ++c)
        if (c < classes) {
            v[c] = expf(v[c] - m);
            z += v[c];
        }
    const float inv = 1.0f / z;
#pragma unroll
    for (int c = 0; c < 32; ++c)
        if (c < classes) s[c] = v[c] * inv;
}

// labels[i] = argmax_c (P1[i][c] + P2[i][c]), the lowest c among equals.
__global__ void __launch_bounds__(256) argmax_combine_kernel(const float *__restrict__ P1, const float *__restrict__ P2,
                                                             int *__restrict__ labels, int rows, int classes)
{
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= rows) return;
    const float *a = P1 + (size_t)row * classes, *b = P2 + (size_t)row * classes;
    int best = 0;
    float bv = a[0] + b[0];
    for (int c = 1; c < classes; ++c) {
        const float v = a[c] + b[c];
        if (v > bv) {
            bv = v;
            best = c;
        }
    }
    labels[row] = best;
}

namespace {

int nc4_of(int classes) { return (classes + 3) / 4; }

size_t dense_smem(int feats, int classes) { return (size_t)kMlQuarters * ml_quarter_stride(feats, nc4_of(classes)) * 4; }

const char *validate_scores(const LaunchArgs &a)
{
    const int rows = a.i32(4), feats = a.i32(5), classes = a.i32(6);
    if (rows < 0) return "rows < 0";
    if (feats <= 0 || feats % (kMlQuarters * kMlFeatStep)) return "feats must be a positive multiple of 32";
    if (classes < 1 || classes > 16) return "classes must be in 1..16";
    if (dense_smem(feats, classes) > 200 * 1024) return "feats x classes table exceeds shared memory";
    if (a.bytes[0] / 4 / (size_t)feats < (size_t)rows) return "X smaller than rows x feats int32";
    if (a.bytes[1] / 4 < (size_t)feats * classes) return "T smaller than feats x classes floats";
    if (a.bytes[2] / 4 < (size_t)classes) return "bias smaller than classes floats";
    if (a.bytes[3] / 4 / (size_t)classes < (size_t)rows) return "S smaller than rows x classes floats";
    if ((reinterpret_cast<uintptr_t>(a.ptr[0]) & 15) != 0) return "X must be 16-byte aligned";
    return nullptr;
}

template <int NC4> int scores_launch(const LaunchArgs &a, cudaStream_t s)
{
    const int rows = a.i32(4), feats = a.i32(5), classes = a.i32(6);
    if (rows == 0) return cudaSuccess;
    const size_t smem = dense_smem(feats, classes);
    // per process: raise the dynamic shared-memory limit once and remember
    // the occupancy of the last table size (no device queries on later
    // launches, so the launch can be stream-captured)
    static bool configured = false;
    static size_t occ_smem = 0;
    static int occ_blocks = 0;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(dense_scores_kernel<NC4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             200 * 1024);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    if (occ_smem != smem) {
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dense_scores_kernel<NC4>, kMlThreads, smem);
        if (e != cudaSuccess) return e;
        occ_blocks = per_sm < 1 ? 1 : per_sm;
        occ_smem = smem;
    }
    const int per_sm = occ_blocks;
    const int64_t groups = ceil_div(rows, 16 * (kMlThreads / 32));
    int64_t grid = (int64_t)sm_count() * per_sm;
    if (grid > groups) grid = groups;
    dense_scores_kernel<NC4><<<(unsigned)grid, kMlThreads, smem, s>>>(a.p<int>(0), a.p<float>(1), a.p<float>(2),
                                                                       a.p<float>(3), rows, feats, classes);
    return cudaGetLastError();
}

int launch_scores(const LaunchArgs &a, void *sv)
{
    cudaStream_t s = (cudaStream_t)sv;
    switch (nc4_of(a.i32(6))) {
    case 1: return scores_launch<1>(a, s);
    case 2: return scores_launch<2>(a, s);
    case 3: return scores_launch<3>(a, s);
    default: return scores_launch<4>(a, s);
    }
}

const char *validate_softmax(const LaunchArgs &a)
{
    const int rows = a.i32(1), classes = a.i32(2);
    if (rows < 0) return "rows < 0";
    if (classes < 1 || classes > 32) return "classes must be in 1..32";
    if (a.bytes[0] / 4 / (size_t)classes < (size_t)rows) return "S smaller than rows x classes floats";
    return nullptr;
}

int launch_softmax(const LaunchArgs &a, void *s)
{
    const int rows = a.i32(1);
    if (rows == 0) return cudaSuccess;
    row_softmax_kernel<<<(unsigned)ceil_div(rows, 256), 256, 0, (cudaStream_t)s>>>(a.p<float>(0), rows, a.i32(2));
    return cudaGetLastError();
}

const char *validate_argmax(const LaunchArgs &a)
{
    const int rows = a.i32(3), classes = a.i32(4);
    if (rows < 0) return "rows < 0";
    if (classes < 1) return "classes must be >= 1";
    if (a.bytes[0] / 4 / (size_t)classes < (size_t)rows || a.bytes[1] / 4 / (size_t)classes < (size_t)rows)
        return "P1 or P2 smaller than rows x classes floats";
    if (a.bytes[2] / 4 < (size_t)rows) return "labels smaller than rows int32";
    return nullptr;
}

int launch_argmax(const LaunchArgs &a, void *s)
{
    const int rows = a.i32(3);
    if (rows == 0) return cudaSuccess;
    argmax_combine_kernel<<<(unsigned)ceil_div(rows, 256), 256, 0, (cudaStream_t)s>>>(
        a.p<float>(0), a.p<float>(1), a.p<int>(2), rows, a.i32(4));
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

void append_ml_kernels(std::vector<KernelEntry> &v)
{
    v.push_back(entry("dense_scores", (const void *)dense_scores_kernel<3>,
                      {arr(GDAG_MODE_IN), arr(GDAG_MODE_IN), arr(GDAG_MODE_IN), arr(GDAG_MODE_OUT), scal(4), scal(4),
                       scal(4)},
                      validate_scores, launch_scores));
    v.push_back(entry("row_softmax", (const void *)row_softmax_kernel, {arr(GDAG_MODE_INOUT), scal(4), scal(4)},
                      validate_softmax, launch_softmax));
    v.push_back(entry("argmax_combine", (const void *)argmax_combine_kernel,
                      {arr(GDAG_MODE_IN), arr(GDAG_MODE_IN), arr(GDAG_MODE_OUT), scal(4), scal(4)}, validate_argmax,
                      launch_argmax));
}

}  // namespace gdag
