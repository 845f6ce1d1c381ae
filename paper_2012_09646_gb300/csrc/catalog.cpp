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
void append_hits_kernels(std::vector<KernelEntry> &v);
void append_dl_kernels(std::vector<KernelEntry> &v);
size_t spmv_part_bytes(int64_t rows_plus_nnz);
size_t seg_norm_scratch_bytes(int64_t G);
size_t l2norm_scratch_bytes();
size_t minmax_scratch_bytes();
size_t spmv_carry_bytes(int64_t rows_plus_nnz);

namespace {
const std::vector<KernelEntry> &table()
{
    static const std::vector<KernelEntry> t = [] {
        std::vector<KernelEntry> v;
        append_vec_kernels(v);
        append_bs_kernels(v);
        append_img_kernels(v);
        append_ml_kernels(v);
        append_hits_kernels(v);
        append_dl_kernels(v);
        return v;
    }();
    return t;
}
}  // namespace

int builtin_count() { return (int)table().size(); }
const KernelEntry &builtin(int i) { return table()[(size_t)i]; }

size_t scratch_bytes(const char *kernel, int64_t n)
{
    if (!std::strcmp(kernel, "vec_reduce_diff")) return reduce_scratch_bytes<1>();
    if (!std::strcmp(kernel, "minmax")) return minmax_scratch_bytes();
    if (!std::strcmp(kernel, "l2norm")) return l2norm_scratch_bytes();
    // for seg_l2norm n is the number of segments
    if (!std::strcmp(kernel, "seg_l2norm")) return seg_norm_scratch_bytes(n);
    // for the two SpMV buffers n is nrows + nnz
    if (!std::strcmp(kernel, "spmv_partition")) return spmv_part_bytes(n);
    if (!std::strcmp(kernel, "spmv_csr")) return spmv_carry_bytes(n);
    return 0;
}

}  // namespace gdag
