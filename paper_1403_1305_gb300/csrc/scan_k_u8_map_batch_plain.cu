// Instantiations of the scan kernel: u8 map text, batch launches, flag tracking off.
#include "scan_kernel.cuh"

namespace acgb {
namespace kern {
KernelFn kernels_u8_map_batch_plain(int mode, uint32_t bx, uint32_t C) {
    return pick_variant<FMT_U8, ALPHA_MAP, true, false>(mode, bx, C);
}
}  // namespace kern
}  // namespace acgb
