// Lean scan kernels: u8 text, smem32 table placement (one translation unit per
// variant so they compile in parallel).
#include "scan_lean.cuh"

namespace acgb {
namespace kern {
LeanFn lean_u8_smem32(uint32_t threads, uint32_t C) { return pick_lean_shape<FMT_U8, LEAN_SMEM32>(threads, C); }
}  // namespace kern
}  // namespace acgb
