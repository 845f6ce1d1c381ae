// B&S node (Section IV-B, B&S): Black-Scholes price of a European call for
// every spot price of a vector, fp32.
//   d1 = (ln(S/K) + (r + sigma^2/2) T) / (sigma sqrt(T)),  d2 = d1 - sigma sqrt(T)
//   C  = S N(d1) - K exp(-rT) N(d2)
// N is CUDA's normcdff; the logarithm CUDA's logf.
#include <vector>

#include "catalog.h"
#include "kcommon.cuh"

namespace gdag {

struct BsConst {
    float inv_k, drift, inv_vol, vol, k_disc;
};

__device__ __forceinline__ float bs_price(float s, const BsConst &c)
{
    float d1 = (logf(s * c.inv_k) + c.drift) * c.inv_vol;
    float d2 = d1 - c.vol;
    return s * normcdff(d1) - c.k_disc * normcdff(d2);
}

// 8 bytes of HBM traffic per option (4 in, 4 out); streaming loads/stores
// (each byte is touched once).
__global__ void __launch_bounds__(1024) bs_call_kernel(const float *__restrict__ S, float *__restrict__ C, int64_t n,
                                                       float K, float r, float sigma, float T)
{
    BsConst c;
    c.inv_k = 1.0f / K;
    c.vol = sigma * sqrtf(T);
    c.inv_vol = 1.0f / c.vol;
    c.drift = (r + 0.5f * sigma * sigma) * T;
    c.k_disc = K * expf(-r * T);
    if (((reinterpret_cast<uintptr_t>(S) | reinterpret_cast<uintptr_t>(C)) & 15) == 0) {
        const float4 *S4 = reinterpret_cast<const float4 *>(S);
        float4 *C4 = reinterpret_cast<float4 *>(C);
        const int64_t n4 = n >> 2;
        const int64_t bd = blockDim.x;
        const int64_t tile = bd * kUnroll;
        for (int64_t base = (int64_t)blockIdx.x * tile; base < n4; base += (int64_t)gridDim.x * tile) {
            float4 v[kUnroll];
#pragma unroll
            for (int k = 0; k < kUnroll; ++k) {
                int64_t i = base + threadIdx.x + k * bd;
                if (i < n4) v[k] = __ldcs(S4 + i);
            }
#pragma unroll
            for (int k = 0; k < kUnroll; ++k) {
                int64_t i = base + threadIdx.x + k * bd;
                if (i < n4) {
                    float4 o;
                    o.x = bs_price(v[k].x, c);
                    o.y = bs_price(v[k].y, c);
                    o.z = bs_price(v[k].z, c);
                    o.w = bs_price(v[k].w, c);
                    __stcs(C4 + i, o);
                }
            }
        }
        if (blockIdx.x == 0 && threadIdx.x < (n & 3)) {
            int64_t i = (n4 << 2) + threadIdx.x;
            C[i] = bs_price(S[i], c);
        }
    } else {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
            C[i] = bs_price(S[i], c);
    }
}

namespace {

const char *validate_bs(const LaunchArgs &a)
{
    int64_t n = a.i64(2);
    if (n < 0) return "n < 0";
    if (a.bytes[0] / 4 < (size_t)n || a.bytes[1] / 4 < (size_t)n) return "S or C smaller than n floats";
    if (!(a.f32(3) > 0.f) || !(a.f32(5) > 0.f) || !(a.f32(6) > 0.f)) return "K, sigma and T must be > 0";
    return nullptr;
}

int launch_bs(const LaunchArgs &a, void *s)
{
    int64_t n = a.i64(2);
    if (n == 0) return cudaSuccess;
    unsigned g = a.auto_cfg ? stream_grid(n >> 2) : a.grid[0];
    unsigned b = a.auto_cfg ? kThreads : a.block[0];
    bs_call_kernel<<<g, b, 0, (cudaStream_t)s>>>(a.p<float>(0), a.p<float>(1), n, a.f32(3), a.f32(4), a.f32(5),
                                                 a.f32(6));
    return cudaGetLastError();
}

}  // namespace

void append_bs_kernels(std::vector<KernelEntry> &v)
{
    KernelEntry e;
    e.name = "bs_call";
    e.fn = (const void *)bs_call_kernel;
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
    v.push_back(e);
}

}  // namespace gdag
