// Instantiations of the scan kernel: u8 map text, single launches, flag tracking off.
#include "scan_kernel.cuh"

namespace acgb {
namespace kern {
KernelFn kernels_u8_map_single_plain(int mode, uint32_t bx, uint32_t C) {
    return pick_variant<FMT_U8, ALPHA_MAP, false, false>(mode, bx, C);
}
}  // namespace kern
}  // namespace acgb
