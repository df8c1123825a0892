// Lean scan kernels: packed text, smem32 table placement (one translation unit per
// variant so they compile in parallel).
#include "scan_lean.cuh"

namespace acgb {
namespace kern {
LeanFn lean_packed_smem32(uint32_t threads, uint32_t C) { return pick_lean_shape<FMT_P2, LEAN_SMEM32>(threads, C); }
}  // namespace kern
}  // namespace acgb
