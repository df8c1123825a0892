// Instantiations of the scan kernel: u8 map text, batch launches, and the dispatch.
#include "scan_kernel.cuh"

namespace acgb {
namespace kern {
KernelFn kernels_u8_map_single(bool hybrid, uint32_t bx, uint32_t C);

KernelFn kernels_u8_map(bool batch, bool hybrid, uint32_t bx, uint32_t C) {
    return batch ? pick_variant<FMT_U8, ALPHA_MAP, true>(hybrid, bx, C) : kernels_u8_map_single(hybrid, bx, C);
}
}  // namespace kern
}  // namespace acgb
