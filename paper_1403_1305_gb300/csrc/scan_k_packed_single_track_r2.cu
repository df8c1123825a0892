// Instantiations of the scan kernel: packed text, single launches, flag tracking on,
// two symbols per lookup.
#include "scan_kernel.cuh"

namespace acgb {
namespace kern {
KernelFn kernels_packed_single_track_r2(int mode, uint32_t bx, uint32_t C) {
    return pick_variant<FMT_P2, ALPHA_MAP, false, true, 2>(mode, bx, C);
}
}  // namespace kern
}  // namespace acgb
