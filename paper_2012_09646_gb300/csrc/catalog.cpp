// Table of built-in kernels, in a fixed order.
#include <cstring>
#include <vector>

#include "catalog.h"
#include "kcommon.cuh"

namespace gdag {

void append_vec_kernels(std::vector<KernelEntry> &v);
void append_bs_kernels(std::vector<KernelEntry> &v);
void append_img_kernels(std::vector<KernelEntry> &v);
void append_ml_kernels(std::vector<KernelEntry> &v);

namespace {
const std::vector<KernelEntry> &table()
{
    static const std::vector<KernelEntry> t = [] {
        std::vector<KernelEntry> v;
        append_vec_kernels(v);
        append_bs_kernels(v);
        append_img_kernels(v);
        append_ml_kernels(v);
        return v;
    }();
    return t;
}
}  // namespace

int builtin_count() { return (int)table().size(); }
const KernelEntry &builtin(int i) { return table()[(size_t)i]; }

size_t scratch_bytes(const char *kernel, int64_t n)
{
    (void)n;
    if (!std::strcmp(kernel, "vec_reduce_diff")) return reduce_scratch_bytes<1>();
    if (!std::strcmp(kernel, "minmax")) return reduce_scratch_bytes<2>();
    return 0;
}

}  // namespace gdag
