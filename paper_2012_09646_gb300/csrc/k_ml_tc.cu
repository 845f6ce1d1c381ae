// ML node dense_scores on the tcgen05 tensor cores (Section IV-B, ML: the
// naive-Bayes and ridge scores are a dense matrix product):
//   S[i][c] = bias[c] + sum_f float(X[i][f]) T[f][c]
// for int32 X (rows x feats) and fp32 T (feats x classes), classes <= 16,
// feats a multiple of 64 up to 1024.
//
// Exactness.  bf16 holds every integer of magnitude <= 256 exactly, and an
// fp32 table entry t is the exact sum of three bf16 pieces t = hi + mid + lo
// (hi = bf16(t), mid = bf16(t - hi), lo = t - hi - mid; each difference is
// exact in fp32 and the last has at most 8 significant bits).  So with X in
// bf16 and B = [hi | mid | lo] every product on the tensor cores is exact;
// only the fp32 accumulation rounds, as it does in the CUDA-core form.  Any x
// with |x| > 256 makes its tile fall back to CUDA cores (below), so the
// result never depends on the input range.
//
// The pieces sit at column strides of 10 (N = 32) up to 10 classes and of 16
// (N = 48) up to 16; the narrower table leaves room for a fourth X stage.
//
// Data flow (one persistent CTA of 448 threads per SM, 128-row tiles):
//   warp 13 (loader, one lane) copies X into a ring of four (N = 32) or
//     three (N = 48) int32 stages with TMA (two 32-feature x 128-row boxes
//     per 64-feature stage, 128-byte swizzle, zeros past the last row), each
//     stage completing on its own mbarrier: 128 or 96 KB of loads in flight
//     per SM;
//   warps 1-12 first stage the table pieces B (resident for the whole
//     launch) while the loader already runs;
//   warps 1-8 (producers) read their pieces of a landed stage (the swizzle
//     makes the eight rows of a wavefront hit eight different bank groups),
//     release the stage to the loader, convert to bf16 (exact integer
//     conversion by the 1.5 x 2^23 bias, the bf16 bits being the top half of
//     the fp32 bits), check the range, and write 16-byte rows of core
//     matrices into a ring of kScStages A stages in the canonical K-major
//     layout (conflict-free: the eight lanes of a wavefront write the eight
//     rows of one core matrix).  They have no copies of their own in flight,
//     so the proxy fence before each A stage's release costs nothing;
//   warps 9-12 (epilogue) per tile read the N accumulator columns of their
//     TMEM lane quarter with tcgen05.ld, add the three pieces and the bias,
//     and store S (fp32);
//   warp 0, one lane, issues four tcgen05.mma (M 128, N 32 or 48, K 16) per
//     stage into one of two accumulator sets (so the next tile's MMAs run while the
//     epilogue drains the other set), committing each stage back to the ring
//     and each tile to the epilogue.
// The one HBM stream is X (4 bytes per feature per row); B is staged once per
// CTA from L2, and S is 4 bytes per class per row.
// Every mbarrier wait is bounded (about one second) and also ends when
// another role raises the shared abort flag; a role stops by vote, so no
// barrier is left half-arrived.  After an abort the epilogue writes NaN to
// the rows it could not finish (the output is visibly invalid), the control
// lane waits (bounded) for its MMAs in flight, and the CTA frees its tensor
// memory.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "catalog.h"
#include "kcommon.cuh"
#include "tcgen05.cuh"

namespace gdag {

constexpr int kScM = 128;                        // rows per tile (MMA M)
constexpr int kScKc = 64;                        // features per A stage
constexpr int kScMaxCls = 16;                    // classes the tensor-core form takes
constexpr int kScStages = 2;                     // A ring depth (bf16 operands)
constexpr int kScMaxFeats = 1024;
constexpr int kScCtl = 32, kScProd = 256, kScEpi = 128, kScLoad = 32;
constexpr int kScThreads = kScCtl + kScProd + kScEpi + kScLoad;
constexpr int kScStageBytes = kScM * kScKc * 2;  // 16 KB of bf16
constexpr int kScAccCols = 64;                   // one accumulator set (32 or 48 columns used)
constexpr int kScTmemCols = 2 * kScAccCols;
constexpr int kScXmax = 256;                     // |x| <= 256 is exact in bf16
constexpr int kScXStageBytes = kScM * kScKc * 4;  // 32 KB of int32: two 128-row boxes of 32 features
constexpr int kScXBoxFeats = 32;                    // 128 bytes of int32: the 128-byte swizzle span
constexpr int kScXBoxBytes = kScM * kScXBoxFeats * 4;
constexpr int kScOffX = kScStages * kScStageBytes;

// Shared-memory layout for an MMA width of kN columns.  Up to 10 classes the
// three pieces sit at column strides of 10 (N = 32), and the 32 KB that the
// narrower table frees holds a fourth X stage; up to 16 classes they sit at
// strides of 16 (N = 48) beside three X stages.
template <int kN>
struct ScLayout {
    static_assert(kN == 32 || kN == 48, "two table layouts");
    static constexpr int kPiece = kN == 32 ? 10 : 16;  // column stride of the pieces
    static constexpr int kXStages = kN == 32 ? 4 : 3;  // X ring depth
    static constexpr int kOffB = kScOffX + kXStages * kScXStageBytes;
    static constexpr int kOffBars = kOffB + kScMaxFeats * kN * 2;
    // a_full x stages, a_empty x stages, acc_full x2, acc_empty x2,
    // flags_ready x2, x_full x X stages, x_empty x X stages
    static constexpr int kNumBars = 2 * kScStages + 6 + 2 * kXStages;
    static constexpr size_t kSmem = kOffBars + kNumBars * 8 + 32;
    static_assert(kOffB % 1024 == 0 && kScOffX % 1024 == 0 && kOffBars % 8 == 0, "operand alignment");
    static_assert(kSmem <= 227 * 1024, "dense_scores shared memory");
    static_assert(3 * kPiece <= kN, "three pieces in N columns");
};

// offset of (row, k) in a canonical K-major, no-swizzle operand whose rows
// hold `kdim` values: core matrix (row / 8, k / 8), 128 bytes each
__device__ __forceinline__ int kmajor_off(int row, int k, int kdim)
{
    return ((row >> 3) * (kdim >> 3) + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// one row on CUDA cores (the fallback), in feature order, with compensated
// (Kahan) fp32 sums: an input with one huge term would otherwise round every
// later small term to the huge partial sum's ulp (a plain fp32 sum of 1024
// terms is only guaranteed to 1023 u sum |terms|; this one to about 2 u)
__device__ __noinline__ void scores_row_cuda(const int *__restrict__ X, const float *__restrict__ T,
                                             const float *__restrict__ bias, float *__restrict__ S, int row,
                                             int feats, int classes)
{
    float acc[kScMaxCls], cmp[kScMaxCls];
#pragma unroll
    for (int c = 0; c < kScMaxCls; ++c) acc[c] = cmp[c] = 0.f;
    const int *x = X + (size_t)row * feats;
    for (int f = 0; f < feats; ++f) {
        const float xv = (float)x[f];
        const float *t = T + (size_t)f * classes;
#pragma unroll
        for (int c = 0; c < kScMaxCls; ++c)
            if (c < classes) {
                const float y = __fmul_rn(xv, t[c]) - cmp[c];
                const float u = acc[c] + y;
                cmp[c] = (u - acc[c]) - y;
                acc[c] = u;
            }
    }
#pragma unroll
    for (int c = 0; c < kScMaxCls; ++c)
        if (c < classes) S[(size_t)row * classes + c] = bias[c] + acc[c];
}

// Stage the table as the MMA's B operand, resident for the whole launch:
// row n = piece * kPiece + c holds piece `piece` of column c of T (zero for
// c >= classes), K = feature, canonical K-major layout, 16 bytes (8
// features) per store; rows from 3 * kPiece to kN are zero.  Threads t of
// nthr share the items.
template <int kN>
__device__ __forceinline__ void stage_table(unsigned char *sb, const float *__restrict__ T, int feats, int classes,
                                            int t, int nthr)
{
    constexpr int kPiece = ScLayout<kN>::kPiece;
    for (int item = t; item < (feats / 8) * kPiece; item += nthr) {
        const int c = item % kPiece, f8 = item / kPiece;
        uint32_t pk[3][4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float hv[2], mv[2], lv[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int f = 8 * f8 + 2 * e + h;
                const float v = c < classes ? T[(size_t)f * classes + c] : 0.f;
                const float hi = __bfloat162float(__float2bfloat16_rn(v));
                const float r1 = v - hi;
                const float mid = __bfloat162float(__float2bfloat16_rn(r1));
                hv[h] = hi;
                mv[h] = mid;
                lv[h] = r1 - mid;  // at most 8 significant bits: exact in bf16
            }
            const __nv_bfloat162 bh = __floats2bfloat162_rn(hv[0], hv[1]);
            const __nv_bfloat162 bm = __floats2bfloat162_rn(mv[0], mv[1]);
            const __nv_bfloat162 bl = __floats2bfloat162_rn(lv[0], lv[1]);
            pk[0][e] = *reinterpret_cast<const uint32_t *>(&bh);
            pk[1][e] = *reinterpret_cast<const uint32_t *>(&bm);
            pk[2][e] = *reinterpret_cast<const uint32_t *>(&bl);
        }
#pragma unroll
        for (int piece = 0; piece < 3; ++piece)
            *reinterpret_cast<uint4 *>(sb + kmajor_off(piece * kPiece + c, 8 * f8, feats)) =
                make_uint4(pk[piece][0], pk[piece][1], pk[piece][2], pk[piece][3]);
    }
    constexpr int kPad = kN - 3 * kPiece;
    if constexpr (kPad > 0) {
        for (int item = t; item < (feats / 8) * kPad; item += nthr)
            *reinterpret_cast<uint4 *>(sb + kmajor_off(3 * kPiece + item % kPad, 8 * (item / kPad), feats)) =
                make_uint4(0u, 0u, 0u, 0u);
    }
}

template <int kN>
__global__ void __launch_bounds__(kScThreads, 1)
    dense_scores_tc_kernel(const __grid_constant__ CUtensorMap tx, const int *__restrict__ X,
                           const float *__restrict__ T, const float *__restrict__ bias, float *__restrict__ S, int rows,
                           int feats, int classes)
{
    extern __shared__ __align__(1024) unsigned char sc_smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = (rows + kScM - 1) / kScM;
    const int kchunks = feats / kScKc;
    using L = ScLayout<kN>;
    constexpr int kXSt = L::kXStages, kPiece = L::kPiece;
    if ((smem_addr(sc_smem) & 1023u) != 0) {
        // no swizzled TMA stages without a 1024-byte aligned window: CUDA
        // cores for every row of this CTA's tiles (uniform over the CTA)
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
            for (int r = tid; r < kScM; r += kScThreads)
                if (tile * kScM + r < rows) scores_row_cuda(X, T, bias, S, tile * kScM + r, feats, classes);
        return;
    }
    unsigned char *sa = sc_smem;
    unsigned char *sb = sc_smem + L::kOffB;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sc_smem + L::kOffBars);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + L::kNumBars);
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);
    volatile int *bad = reinterpret_cast<volatile int *>(tmem_slot + 2);  // [4]: last tile index with |x| > 256
    const uint32_t afull = smem_addr(&bars[0]);               // + 8 * stage: A stage written
    const uint32_t aempty = smem_addr(&bars[kScStages]);      // + 8 * stage: A stage read by the MMAs
    const uint32_t accfull = smem_addr(&bars[2 * kScStages]); // + 8 * set: tile's MMAs done
    const uint32_t accempty = accfull + 16;                   // + 8 * set: accumulators read
    const uint32_t flagsrdy = accfull + 32;                   // + 8 * set: the tile's range flags written
    const uint32_t xfull = accfull + 48;                      // + 8 * X stage: TMA landed
    const uint32_t xempty = xfull + 8 * kXSt;           // + 8 * X stage: producers read it
    const int my_tiles = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int total = my_tiles * kchunks;  // stages of this CTA, tile-major

    if (warp == 0) {
        if (lane == 0) {
            *abort = 0;
            for (int j = 0; j < 4; ++j) bad[j] = -1;
            for (int j = 0; j < kScStages; ++j) {
                asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(afull + 8 * j), "r"(kScProd / 32));
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(aempty + 8 * j));
            }
            for (int s = 0; s < 2; ++s) {
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(accfull + 8 * s));
                asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(accempty + 8 * s), "r"(kScEpi / 32));
                asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(flagsrdy + 8 * s), "r"(kScProd / 32));
            }
            for (int j = 0; j < kXSt; ++j) {
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(xfull + 8 * j));
                asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(xempty + 8 * j), "r"(kScProd / 32));
            }
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncwarp();
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "n"(kScTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();  // barriers initialised, tensor memory allocated
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;

    // The table first, by the producers and the epilogue together, while the
    // loader already fills the X ring; the MMAs start once it is staged.
    if (warp <= (kScProd + kScEpi) / 32) {
        if (warp >= 1) {
            stage_table<kN>(sb, T, feats, classes, tid - kScCtl, kScProd + kScEpi);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic stores -> tensor-core reads
        }
        asm volatile("bar.sync 3, %0;" ::"n"(kScCtl + kScProd + kScEpi) : "memory");
    }

    if (warp == 0) {
        // ---- control: MMA issue (one lane)
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16_f32(kScM, kN);
            const uint32_t b_sbo = (uint32_t)(feats / 8) * 128;
            int step = 0, issued = 0;
            for (int it = 0; it < my_tiles && !*abort; ++it) {
                const int s = it & 1;
                if (it >= 2 && !mbar_wait_bounded(accempty + 8 * s, ((it >> 1) - 1) & 1, abort)) {
                    *abort = 1;
                    break;
                }
                for (int kc = 0; kc < kchunks; ++kc, ++step) {
                    const int st = step % kScStages;
                    if (!mbar_wait_bounded(afull + 8 * st, (step / kScStages) & 1, abort)) {
                        *abort = 1;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
                    for (int ks = 0; ks < kScKc / 16; ++ks) {
                        const uint64_t ad = umma_desc_kmajor(smem_addr(sa + st * kScStageBytes) + ks * 256, 128,
                                                             (kScKc / 8) * 128);
                        const uint64_t bd = umma_desc_kmajor(smem_addr(sb) + (kc * (kScKc / 8) + ks * 2) * 128, 128,
                                                             b_sbo);
                        asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                                     " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
                                         tmem + s * kScAccCols),
                                     "l"(ad), "l"(bd), "r"(idesc), "r"((uint32_t)(kc | ks)));
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        aempty + 8 * st));
                    ++issued;
                }
                if (*abort) break;
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    accfull + 8 * s));
            }
            if (*abort && issued > 0) {
                // the MMAs in flight finish before the CTA frees tensor memory
                const volatile int no_abort = 0;
                const int last = issued - 1;
                mbar_wait_bounded(aempty + 8 * (last % kScStages), (last / kScStages) & 1, &no_abort);
            }
        }
        __syncwarp();
    } else if (warp <= kScProd / 32) {
        // ---- producers: rows j*32 + rb*8 + mlo (j < 4) of each stage, features 8g .. 8g+7
        // (box g / 4, 16-byte chunks 2(g % 4) and 2(g % 4) + 1 of the row,
        // stored at chunk ^ (row % 8) by the 128-byte swizzle)
        const int p = tid - kScCtl;
        const int mlo = p & 7, g = (p >> 3) & 7, rb = p >> 6;
        const int c0 = (2 * (g & 3)) ^ mlo, c1 = (2 * (g & 3) + 1) ^ mlo;  // rows m have m % 8 == mlo
        for (int step = 0; step < total; ++step) {
            const int xsl = step % kXSt, st = step % kScStages, it = step / kchunks, kc = step % kchunks;
            const bool xok = mbar_wait_bounded(xfull + 8 * xsl, (step / kXSt) & 1, abort);
            const bool wok = step < kScStages || mbar_wait_bounded(aempty + 8 * st, ((step / kScStages) - 1) & 1, abort);
            if (!__all_sync(0xffffffffu, xok && wok)) {  // warp-uniform stop
                if (lane == 0) *abort = 1;
                break;
            }
            const unsigned char *xb = sc_smem + kScOffX + xsl * kScXStageBytes + (g >> 2) * kScXBoxBytes;
            int4 lo4[4], hi4[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const unsigned char *row = xb + (j * 32 + rb * 8 + mlo) * 128;
                lo4[j] = *reinterpret_cast<const int4 *>(row + c0 * 16);
                hi4[j] = *reinterpret_cast<const int4 *>(row + c1 * 16);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(xempty + 8 * xsl);  // the stage's values are in registers
            unsigned char *A = sa + st * kScStageBytes;
            uint32_t vrange = 0;  // max of v + 256 as unsigned: above 512 iff |v| > 256 (INT_MIN included)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int v[8] = {lo4[j].x, lo4[j].y, lo4[j].z, lo4[j].w, hi4[j].x, hi4[j].y, hi4[j].z, hi4[j].w};
                uint32_t w[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    vrange = max(vrange, max((uint32_t)v[2 * e] + (uint32_t)kScXmax,
                                             (uint32_t)v[2 * e + 1] + (uint32_t)kScXmax));
                    // exact for |v| < 2^22: the float 1.5 * 2^23 + v, minus 1.5 * 2^23
                    const float2 f = __fadd2_rn(make_float2(__uint_as_float((uint32_t)v[2 * e] + 0x4B400000u),
                                                            __uint_as_float((uint32_t)v[2 * e + 1] + 0x4B400000u)),
                                                make_float2(-12582912.0f, -12582912.0f));
                    // integers up to 256 have zero low halves: bf16 = top 16 bits
                    w[e] = __byte_perm(__float_as_uint(f.x), __float_as_uint(f.y), 0x7632);
                }
                *reinterpret_cast<uint4 *>(A + kmajor_off(j * 32 + rb * 8 + mlo, 8 * g, kScKc)) =
                    make_uint4(w[0], w[1], w[2], w[3]);
            }
            if (vrange > 2u * kScXmax) bad[it & 3] = it;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic stores -> tensor-core reads
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(afull + 8 * st);
                if (kc == kchunks - 1) mbar_arrive(flagsrdy + 8 * (it & 1));
            }
        }
    } else if (warp == kScThreads / 32 - 1) {
        // ---- loader (one lane): X stages by TMA, kXSt ahead
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tx)) : "memory");
            int issued = 0;
            for (int step = 0; step < total; ++step) {
                const int xsl = step % kXSt;
                if (step >= kXSt &&
                    !mbar_wait_bounded(xempty + 8 * xsl, ((step / kXSt) - 1) & 1, abort)) {
                    *abort = 1;
                    break;
                }
                const int tile = (int)blockIdx.x + (step / kchunks) * (int)gridDim.x, kc = step % kchunks;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(xfull + 8 * xsl),
                             "r"(kScXStageBytes)
                             : "memory");
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    asm volatile(
                        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
                            smem_addr(sc_smem + kScOffX + xsl * kScXStageBytes + h * kScXBoxBytes)),
                        "l"(reinterpret_cast<uint64_t>(&tx)), "r"(kc * kScKc + h * kScXBoxFeats), "r"(tile * kScM),
                        "r"(xfull + 8 * xsl)
                        : "memory");
                ++issued;
            }
            if (*abort && issued > 0) {
                // the copies in flight land before the CTA frees its memory
                const volatile int no_abort = 0;
                for (int k = issued - kXSt < 0 ? 0 : issued - kXSt; k < issued; ++k)
                    mbar_wait_bounded(xfull + 8 * (k % kXSt), (k / kXSt) & 1, &no_abort);
            }
        }
        __syncwarp();
    } else {
        // ---- epilogue (warps 9-12): drain one accumulator set per tile
        const int quad = warp & 3;       // the TMEM lane quarter this warp may read
        const int r = quad * 32 + lane;  // row of the tile
        float bz[kScMaxCls];
#pragma unroll
        for (int c = 0; c < kScMaxCls; ++c) bz[c] = c < classes ? bias[c] : 0.f;
        int it = 0;
        for (; it < my_tiles; ++it) {
            const int s = it & 1, tile = (int)blockIdx.x + it * (int)gridDim.x;
            const bool ok = mbar_wait_bounded(accfull + 8 * s, (it >> 1) & 1, abort) &&
                            mbar_wait_bounded(flagsrdy + 8 * s, (it >> 1) & 1, abort);
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) *abort = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            uint32_t v[kN / 16][16];  // accumulator columns 16 q .. 16 q + 15
#pragma unroll
            for (int q = 0; q < kN / 16; ++q) {
                const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + s * kScAccCols + q * 16;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                    : "=r"(v[q][0]), "=r"(v[q][1]), "=r"(v[q][2]), "=r"(v[q][3]), "=r"(v[q][4]), "=r"(v[q][5]),
                      "=r"(v[q][6]), "=r"(v[q][7]), "=r"(v[q][8]), "=r"(v[q][9]), "=r"(v[q][10]), "=r"(v[q][11]),
                      "=r"(v[q][12]), "=r"(v[q][13]), "=r"(v[q][14]), "=r"(v[q][15])
                    : "r"(taddr));
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) mbar_arrive(accempty + 8 * s);
            const int row = tile * kScM + r;
            if (row < rows) {
                if (bad[it & 3] == it) {
                    scores_row_cuda(X, T, bias, S, row, feats, classes);
                } else {
                    float *out = S + (size_t)row * classes;
#pragma unroll
                    for (int c = 0; c < kPiece; ++c)
                        if (c < classes)  // piece p of class c is column p * kPiece + c
                            out[c] = bz[c] + ((__uint_as_float(v[c >> 4][c & 15]) +
                                               __uint_as_float(v[(kPiece + c) >> 4][(kPiece + c) & 15])) +
                                              __uint_as_float(v[(2 * kPiece + c) >> 4][(2 * kPiece + c) & 15]));
                }
            }
        }
        // after an abort: the rows this warp did not finish are invalid
        for (; it < my_tiles; ++it) {
            const int row = ((int)blockIdx.x + it * (int)gridDim.x) * kScM + quad * 32 + lane;
            if (row < rows)
                for (int c = 0; c < classes; ++c) S[(size_t)row * classes + c] = __int_as_float(0x7FC00000);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(kScTmemCols));
}

bool scores_tc_ok(int feats, int classes)
{
    return classes >= 1 && classes <= kScMaxCls && feats > 0 && feats % kScKc == 0 && feats <= kScMaxFeats;
}

int launch_scores_tc(const LaunchArgs &a, cudaStream_t s)
{
    const int rows = a.i32(4), feats = a.i32(5), classes = a.i32(6);
    if (rows == 0) return cudaSuccess;
    // per process: the shared-memory limit is raised once; the tensor maps
    // of the last few (X, shape) combinations are kept, so a repeated launch
    // makes no driver call (and can be stream-captured)
    struct XMap {
        const void *x = nullptr;
        int rows = 0, feats = 0;
        CUtensorMap map;
    };
    static std::mutex mu;
    static bool configured = false;  // both layouts' shared-memory limits raised
    static XMap cache[8];
    static int cache_next = 0;
    CUtensorMap tx;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!configured) {
            cudaError_t e = cudaFuncSetAttribute(dense_scores_tc_kernel<32>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)ScLayout<32>::kSmem);
            if (e != cudaSuccess) return e;
            e = cudaFuncSetAttribute(dense_scores_tc_kernel<48>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)ScLayout<48>::kSmem);
            if (e != cudaSuccess) return e;
            configured = true;
        }
        int hit = -1;
        for (int i = 0; i < 8; ++i)
            if (cache[i].x == a.ptr[0] && cache[i].rows == rows && cache[i].feats == feats) hit = i;
        if (hit < 0) {
            EncodeTiled fn = tma_encoder();
            if (!fn) return cudaErrorNotSupported;
            XMap m;
            m.x = a.ptr[0];
            m.rows = rows;
            m.feats = feats;
            std::memset(&m.map, 0, sizeof m.map);
            // X as a 2-D int32 tensor (feats innermost, rows), boxes of 32 x 128,
            // 128-byte swizzle, zeros past the last row
            const cuuint64_t dims[2] = {(cuuint64_t)feats, (cuuint64_t)rows};
            const cuuint64_t strides[1] = {(cuuint64_t)feats * 4};
            const cuuint32_t box[2] = {(cuuint32_t)kScXBoxFeats, (cuuint32_t)kScM};
            const cuuint32_t estr[2] = {1, 1};
            if (fn(&m.map, CU_TENSOR_MAP_DATA_TYPE_INT32, 2, a.ptr[0], dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return cudaErrorNotSupported;
            hit = cache_next;
            cache[hit] = m;
            cache_next = (cache_next + 1) % 8;
        }
        tx = cache[hit].map;
    }
    const int64_t ntiles = ceil_div(rows, kScM);
    const int64_t grid = ntiles < sm_count() ? ntiles : sm_count();
    if (classes <= ScLayout<32>::kPiece)
        dense_scores_tc_kernel<32><<<(unsigned)grid, kScThreads, ScLayout<32>::kSmem, s>>>(
            tx, a.p<int>(0), a.p<float>(1), a.p<float>(2), a.p<float>(3), rows, feats, classes);
    else
        dense_scores_tc_kernel<48><<<(unsigned)grid, kScThreads, ScLayout<48>::kSmem, s>>>(
            tx, a.p<int>(0), a.p<float>(1), a.p<float>(2), a.p<float>(3), rows, feats, classes);
    return cudaGetLastError();
}

}  // namespace gdag
