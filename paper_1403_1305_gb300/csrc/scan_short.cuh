// Declarations of the short-text scan kernel (scan_short.cu).
#pragma once

#include "scan_kernel.cuh"

namespace acgb {
namespace kern {

enum { SHORT_FULL = kShortFull, SHORT_E16 = kShortE16 };
constexpr uint32_t kShortMaxWords = 9;  // warm-up words + row words a thread holds
using ShortFn = void (*)(ScanParams);
// words = warm-up words + row words of a thread's window
// acgt: the machine's alphabet is exactly A, C, G, T (bytes decoded without the symbol map)
ShortFn short_u8_full(uint32_t words, bool acgt);
ShortFn short_u8_e16(uint32_t words, bool acgt);
ShortFn short_packed_full(uint32_t words);
ShortFn short_packed_e16(uint32_t words);

}  // namespace kern
}  // namespace acgb
