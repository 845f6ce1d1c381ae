// ML nodes (Section IV-B, ML): naive-Bayes and ridge-regression classifiers
// combined by a softmax of each and the average of their scores.
//   dense_scores    S[i][c] = bias[c] + sum_f float(X[i][f]) T[f][c]
//                   (both classifiers: log-probability table + log prior,
//                   or weights + intercepts), X int32 row-major rows x feats
//   row_softmax     S[i][:] := exp(S[i][:] - max) / sum, in place
//   argmax_combine  labels[i] = argmax_c (P1[i][c] + P2[i][c]), ties -> lowest c
//
// dense_scores runs on the tensor cores (k_ml_tc.cu) when feats is a
// multiple of 64 up to 1024; the CUDA-core forms below take the other
// shapes.  Either way it streams X once (4 bytes per feature per row)
// against a table kept in shared memory: HBM-bound at rows*feats*4 bytes.
// CUDA-core forms:  Four lanes share a row, each summing a quarter of the
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

// ---- pipelined form (tables that leave room for a staging ring): X is
// staged in shared memory in slices of kPipeSlice features x kPipeRows rows
// by cp.async, kPipeStages slices in flight per CTA, so the loads no longer
// wait in registers.  Four lanes share a row, the eight row groups of a warp
// share every table read (broadcast), and each lane carries four rows, so
// one table load serves 32 rows: a 128-bit shared load costs four wavefronts
// whatever its addresses, and the table loads are what bounds this form.
// Packed fp32x2 FMA, fixed shuffle tree, deterministic.  Lane q sums the
// features 32 s + 8 q .. 32 s + 8 q + 7 of every slice s instead of one
// contiguous quarter, so a general table rounds differently from the form
// above (a dyadic one, whose partial sums are exact, gives the same bits).
constexpr int kPipeSlice = 32;                            // features per stage
constexpr int kPipeThreads = 128;                         // four warps
constexpr int kPipeRowsPerLane = 4;                       // rows rsub, rsub+8, rsub+16, rsub+24 of a warp
constexpr int kPipeRows = 8 * kPipeRowsPerLane * (kPipeThreads / 32);  // 128 rows per tile
constexpr int kPipeRowBytes = kPipeSlice * 4 + 16;        // padded: the lanes' 16-byte reads spread over all banks
constexpr int kPipeStageBytes = kPipeRows * kPipeRowBytes;
constexpr int kPipeStages = 3;

// Table layout of the pipelined form: lane q handles features
// f = 32 s + 8 q + j (index i = 8 s + j of its quarter); the float4 of class
// group k of quarter q at index i sits at float4 slot (i * NC4 + k) * 4 + q,
// so the four quarters a warp reads at once share one 64-byte span: one
// shared-memory wavefront per table load, no bank conflict.
__host__ __device__ constexpr int pipe_table_floats(int feats, int nc4) { return feats * nc4 * 4; }

__device__ __forceinline__ void cp_async16(void *dst, const void *src, int src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(src_bytes)
                 : "memory");
}

template <int NC4>
__global__ void __launch_bounds__(kPipeThreads, 2)
    dense_scores_pipe_kernel(const int *__restrict__ X, const float *__restrict__ T, const float *__restrict__ bias,
                             float *__restrict__ S, int rows, int feats, int classes)
{
    extern __shared__ float4 smem4[];
    unsigned char *xs = reinterpret_cast<unsigned char *>(smem4);
    float *st = reinterpret_cast<float *>(xs + kPipeStages * kPipeStageBytes);
    for (int i = threadIdx.x; i < pipe_table_floats(feats, NC4); i += kPipeThreads) {
        const int c = i % 4, q = (i / 4) % 4, k = (i / 16) % NC4, idx = i / (16 * NC4);
        const int f = (idx / 8) * kPipeSlice + 8 * q + (idx % 8), cls = 4 * k + c;
        st[i] = cls < classes ? T[(size_t)f * classes + cls] : 0.f;
    }
    const int slices = feats / kPipeSlice;
    const int ntiles = (rows + kPipeRows - 1) / kPipeRows;
    const int my_tiles = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int total = my_tiles * slices;  // steps: (tile, slice) pairs of this CTA, tile-major

    // copy role: thread c copies chunk k = c % 8 of rows c / 8 + 16 j
    // (j = 0..7) of each slice; the row pointers are set once per tile
    constexpr int kCopies = kPipeRows * (kPipeSlice / 4) / kPipeThreads;  // 8
    constexpr int kCopyRowStep = kPipeThreads / (kPipeSlice / 4);        // 16
    const int ck = threadIdx.x % (kPipeSlice / 4), cr = threadIdx.x / (kPipeSlice / 4);
    const int *csrc[kCopies];
    int cbytes[kCopies];
    int i_tile = 0, i_slice = 0, i_buf = 0, issued = 0;  // next step to issue
    auto set_rows = [&](int tile_i) {
        const int tile = (int)blockIdx.x + tile_i * (int)gridDim.x;
#pragma unroll
        for (int j = 0; j < kCopies; ++j) {
            const int row = tile * kPipeRows + cr + j * kCopyRowStep;
            csrc[j] = X + (size_t)(row < rows ? row : 0) * feats + 4 * ck;
            cbytes[j] = row < rows ? 16 : 0;
        }
    };
    auto issue_next = [&]() {
        if (issued < total) {
            unsigned char *dst = xs + i_buf * kPipeStageBytes + cr * kPipeRowBytes + 16 * ck;
#pragma unroll
            for (int j = 0; j < kCopies; ++j)
                cp_async16(dst + j * kCopyRowStep * kPipeRowBytes, csrc[j] + i_slice * kPipeSlice,
                           cbytes[j]);
            ++issued;
            i_buf = i_buf + 1 == kPipeStages ? 0 : i_buf + 1;
            if (++i_slice == slices) {
                i_slice = 0;
                if (++i_tile < my_tiles) set_rows(i_tile);
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = lane & 3, rsub = lane >> 2;
    const int r0_l = warp * (8 * kPipeRowsPerLane) + rsub;  // rows r0_l + 8 m, m < kPipeRowsPerLane
    const float4 *tq = reinterpret_cast<const float4 *>(st) + q;
    float2 acc[kPipeRowsPerLane][NC4 * 2];
#pragma unroll
    for (int m = 0; m < kPipeRowsPerLane; ++m)
#pragma unroll
        for (int k = 0; k < NC4 * 2; ++k) acc[m][k] = make_float2(0.f, 0.f);
    if (my_tiles > 0) set_rows(0);
    for (int t = 0; t < kPipeStages - 1; ++t) issue_next();
    int sl = 0, tile_i = 0, buf = 0;  // step being computed
    for (int t = 0; t < total; ++t) {
        asm volatile("cp.async.wait_group %0;" ::"n"(kPipeStages - 2) : "memory");
        __syncthreads();  // step t landed for every thread; step t-1's buffer is free
        issue_next();
        const unsigned char *bufp = xs + buf * kPipeStageBytes + r0_l * kPipeRowBytes + 32 * q;
        const float4 *tsl = tq + 8 * sl * NC4 * 4;
#pragma unroll
        for (int h = 0; h < 2; ++h) {  // features 4h .. 4h+3 of the lane's eight
            float x[kPipeRowsPerLane][4];
#pragma unroll
            for (int m = 0; m < kPipeRowsPerLane; ++m) {
                const int4 v = *reinterpret_cast<const int4 *>(bufp + 8 * m * kPipeRowBytes + 16 * h);
                x[m][0] = __int2float_rn(v.x);
                x[m][1] = __int2float_rn(v.y);
                x[m][2] = __int2float_rn(v.z);
                x[m][3] = __int2float_rn(v.w);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float4 *trow = tsl + (4 * h + j) * NC4 * 4;
#pragma unroll
                for (int k = 0; k < NC4; ++k) {
                    const float4 tv = trow[4 * k];
                    const float2 t01 = make_float2(tv.x, tv.y), t23 = make_float2(tv.z, tv.w);
#pragma unroll
                    for (int m = 0; m < kPipeRowsPerLane; ++m) {
                        const float2 xx = make_float2(x[m][j], x[m][j]);
                        acc[m][2 * k] = __ffma2_rn(xx, t01, acc[m][2 * k]);
                        acc[m][2 * k + 1] = __ffma2_rn(xx, t23, acc[m][2 * k + 1]);
                    }
                }
            }
        }
        buf = buf + 1 == kPipeStages ? 0 : buf + 1;
        if (++sl == slices) {
            sl = 0;
            // combine the four quarters, (q0 + q1) + (q2 + q3), and write
            const int tile = (int)blockIdx.x + tile_i * (int)gridDim.x;
#pragma unroll
            for (int m = 0; m < kPipeRowsPerLane; ++m) {
#pragma unroll
                for (int k = 0; k < NC4 * 2; ++k) {
                    acc[m][k].x += __shfl_xor_sync(0xffffffffu, acc[m][k].x, 1);
                    acc[m][k].y += __shfl_xor_sync(0xffffffffu, acc[m][k].y, 1);
                    acc[m][k].x += __shfl_xor_sync(0xffffffffu, acc[m][k].x, 2);
                    acc[m][k].y += __shfl_xor_sync(0xffffffffu, acc[m][k].y, 2);
                }
                const int row = tile * kPipeRows + r0_l + 8 * m;
                if (q == 0 && row < rows) {
                    float *out = S + (size_t)row * classes;
#pragma unroll
                    for (int k = 0; k < NC4 * 2; ++k) {
                        if (2 * k < classes) out[2 * k] = bias[2 * k] + acc[m][k].x;
                        if (2 * k + 1 < classes) out[2 * k + 1] = bias[2 * k + 1] + acc[m][k].y;
                    }
                }
#pragma unroll
                for (int k = 0; k < NC4 * 2; ++k) acc[m][k] = make_float2(0.f, 0.f);
            }
            ++tile_i;
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
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

// the tcgen05 form (k_ml_tc.cu): classes <= 16, feats a multiple of 64 up to 1024
bool scores_tc_ok(int feats, int classes);
int launch_scores_tc(const LaunchArgs &a, cudaStream_t s);

namespace {

int nc4_of(int classes) { return (classes + 3) / 4; }

size_t dense_smem(int feats, int classes) { return (size_t)kMlQuarters * ml_quarter_stride(feats, nc4_of(classes)) * 4; }

size_t pipe_smem(int feats, int classes)
{
    return (size_t)kPipeStages * kPipeStageBytes + (size_t)pipe_table_floats(feats, nc4_of(classes)) * 4;
}

// the pipelined form when two CTAs with their staging rings fit an SM
bool use_pipe(int feats, int classes) { return pipe_smem(feats, classes) <= 110 * 1024; }

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

template <int NC4> int scores_pipe_launch(const LaunchArgs &a, cudaStream_t s)
{
    const int rows = a.i32(4), feats = a.i32(5), classes = a.i32(6);
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(dense_scores_pipe_kernel<NC4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             110 * 1024);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    // an equal number of tiles for every CTA (to within one): waves of two
    // CTAs per SM, then as many CTAs as that many tiles each need
    const int64_t ntiles = ceil_div(rows, kPipeRows), slots = 2 * (int64_t)sm_count();
    const int64_t per = ceil_div(ntiles, slots);
    const int64_t grid = ceil_div(ntiles, per);
    dense_scores_pipe_kernel<NC4><<<(unsigned)grid, kPipeThreads, pipe_smem(feats, classes), s>>>(
        a.p<int>(0), a.p<float>(1), a.p<float>(2), a.p<float>(3), rows, feats, classes);
    return cudaGetLastError();
}

template <int NC4> int scores_launch(const LaunchArgs &a, cudaStream_t s)
{
    const int rows = a.i32(4), feats = a.i32(5), classes = a.i32(6);
    if (rows == 0) return cudaSuccess;
    if (use_pipe(feats, classes)) return scores_pipe_launch<NC4>(a, s);
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
    if (scores_tc_ok(a.i32(5), a.i32(6))) return launch_scores_tc(a, s);
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
