// Kernel table shared by the runtime and the built-in kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cstring>
#include <string>

#include "gdag.h"

namespace gdag {

constexpr int kMaxArgs = 16;

// Resolved arguments of one launch: device pointers for arrays, raw scalar
// bits for scalars, plus the array sizes for bounds validation.
struct LaunchArgs {
    void *ptr[kMaxArgs];
    size_t bytes[kMaxArgs];
    uint64_t val[kMaxArgs];
    int nargs = 0;
    bool auto_cfg = true;  // grid chosen by the kernel
    unsigned grid[3] = {0, 0, 0};
    unsigned block[3] = {0, 0, 0};
    size_t smem = 0;

    template <class T> T *p(int i) const { return static_cast<T *>(ptr[i]); }
    int64_t i64(int i) const { return static_cast<int64_t>(val[i]); }
    int32_t i32(int i) const {
        int32_t v;
        std::memcpy(&v, &val[i], 4);
        return v;
    }
    float f32(int i) const {
        float v;
        std::memcpy(&v, &val[i], 4);
        return v;
    }
};

// Validate sizes before anything is issued; return nullptr if fine, else a
// static message.
typedef const char *(*ValidateFn)(const LaunchArgs &);
// Issue the node's kernel launch(es) on `stream` (a cudaStream_t); returns a
// cudaError_t value.
typedef int (*LauncherFn)(const LaunchArgs &, void *stream);
// Issue `count` launches of the kernel (each validated, automatic launch
// shape) as one persistent launch on `stream` (more than one only when
// `count` exceeds the kernel's table capacity); returns a cudaError_t value.
typedef int (*FusedLauncherFn)(const LaunchArgs *members, int count, void *stream);

struct KernelEntry {
    std::string name;
    const void *fn = nullptr;  // user kernels: the __global__ handle
    int nargs = 0;
    gdag_argspec spec[kMaxArgs];
    ValidateFn validate = nullptr;  // built-ins only
    LauncherFn launcher = nullptr;  // built-ins only
    FusedLauncherFn fused = nullptr;  // built-ins with a fused form only
};

// Built-in kernels (defined by the kernel translation units).
int builtin_count();
const KernelEntry &builtin(int i);

// Helpers for the table.
inline gdag_argspec arr(int mode) { return gdag_argspec{GDAG_ARG_ARRAY, mode, 0, 0}; }
inline gdag_argspec scal(int size) { return gdag_argspec{GDAG_ARG_SCALAR, 0, size, 0}; }

// Scratch sizes of the built-in kernels that need one (0 if none).
size_t scratch_bytes(const char *kernel, int64_t n);

}  // namespace gdag
