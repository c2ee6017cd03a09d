// Kernel instantiations for ring degree N = 2^8: one variant per register
// layout (coefficients per thread 2^EL) and digit width.
#include "fdfb_inst.cuh"

namespace fdfb {
// Variants whose last template argument is true are also built with balanced
// blind-rotation digits (the only ones a set with signed_digits uses).
const Ops* ops_n8(int w, int variant) {
  static const Ops a0 = Inst<8, 3, 2, uint32_t, uint16_t, false, br_min_blocks(2 << (8 - 3)), 1, false, false, 1, true>::ops();
  // lazy prime family: paired with 64-bit sums, and single with per-product reduction
  static const Ops a1 = Inst<8, 3, 2, uint32_t, uint16_t, true, br_min_blocks(2 << (8 - 3)), 2, true, false, 1, true>::ops();
  static const Ops a2 = Inst<8, 3, 2, uint32_t, uint16_t, false, br_min_blocks(2 << (8 - 3)), 1, true>::ops();
  static const Ops b0 = Inst<8, 3, 3, uint64_t, uint16_t, false, br_min_blocks(3 << (8 - 3)), 1, false, false, 1, true>::ops();
  if (w == 32) {
    switch (variant) {
      case 0: return &a0;
      case 1: return &a1;
      case 2: return &a2;
      default: return nullptr;
    }
  }
  if (w == 64) {
    switch (variant) {
      case 0: return &b0;
      default: return nullptr;
    }
  }
  return nullptr;
}
}  // namespace fdfb
