// Instantiations of the scan kernel: packed text, single launches, flag tracking off.
#include "scan_kernel.cuh"

namespace acgb {
namespace kern {
KernelFn kernels_packed_single_plain(int mode, uint32_t bx, uint32_t C) {
    return pick_variant<FMT_P2, ALPHA_MAP, false, false>(mode, bx, C);
}
}  // namespace kern
}  // namespace acgb
