// Helpers shared by the tcgen05 kernels (shared-memory addresses, bounded
// mbarrier waits, named barriers that vote, the sm_100 shared-memory matrix
// descriptor).
#pragma once

#include <cuda.h>  // CUtensorMap and its enums (the encoder comes from the runtime's driver entry point)
#include <cuda_runtime.h>

#include <cstdint>

namespace gdag {

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// wait for phase `parity` of the mbarrier at `bar`; false after about one
// second or once another thread has raised *abort
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, const volatile int *abort)
{
    {
        // the common case, a phase that has already completed, costs one
        // test (no clock read, no abort load)
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (done) return true;
        if (*abort || clock64() - t0 > 2000000000LL) return false;
    }
}

// named barrier `id` over `n` threads that also ANDs v across them
__device__ __forceinline__ bool bar_and(int id, int n, bool v)
{
    uint32_t r;
    asm volatile("{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}"
                 : "=r"(r)
                 : "r"((uint32_t)v), "r"(id), "r"(n)
                 : "memory");
    return r != 0;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}


// shared-memory matrix descriptor (sm_100) of an operand in the canonical
// K-major layout without swizzle (core matrices of 8 rows x 16 bytes stored
// as 128 contiguous bytes): start address >> 4, leading byte offset (between
// K-adjacent core matrices) >> 4 at bit 16, stride byte offset (between
// M/N-adjacent core matrices) >> 4 at bit 32, version 1 at bit 46
__device__ __forceinline__ uint64_t umma_desc_kmajor(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of tcgen05.mma kind::f16 with an f32 accumulator,
// A and B bf16 and both K-major: N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int m, int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// the driver's tensor-map encoder, through the runtime (no link to libcuda)
inline EncodeTiled tma_encoder()
{
    static EncodeTiled fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

}  // namespace gdag
