// Instantiations of the scan kernel: u8 map text, single launches, flag tracking on.
#include "scan_kernel.cuh"

namespace acgb {
namespace kern {
KernelFn kernels_u8_map_single_track(int mode, uint32_t bx, uint32_t C) {
    return pick_variant<FMT_U8, ALPHA_MAP, false, true>(mode, bx, C);
}
}  // namespace kern
}  // namespace acgb
