// Instantiations of the scan kernel: packed text, batch launches, and the dispatch.
#include "scan_kernel.cuh"

namespace acgb {
namespace kern {
KernelFn kernels_packed_single(bool hybrid, uint32_t bx, uint32_t C);

KernelFn kernels_packed(bool batch, bool hybrid, uint32_t bx, uint32_t C) {
    return batch ? pick_variant<FMT_P2, ALPHA_MAP, true>(hybrid, bx, C) : kernels_packed_single(hybrid, bx, C);
}
}  // namespace kern
}  // namespace acgb
