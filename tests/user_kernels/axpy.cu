// A user's own kernel, built outside the library, for the test that
// registers a __global__ function with gdag_kernel_register and launches it
// as a DAG element (the paper's user kernels with argument annotations,
// Section III-D).
#include <cstdint>

__global__ void user_axpy(const float *__restrict__ x, float *__restrict__ y, float a, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = a * x[i] + y[i];
}

// The host handle of the kernel, as cudaLaunchKernel takes it.
extern "C" const void *user_axpy_handle() { return (const void *)user_axpy; }
