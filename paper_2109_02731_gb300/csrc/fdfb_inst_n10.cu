// Kernel instantiations for ring degree N = 2^10: one variant per register
// layout (coefficients per thread 2^EL) and digit width.
#include "fdfb_inst.cuh"

namespace fdfb {
const Ops* ops_n10(int w, int variant) {
  static const Ops a0 = Inst<10, 4, 2, uint32_t, uint16_t>::ops();
  static const Ops b0 = Inst<10, 4, 3, uint64_t, uint16_t>::ops();
  static const Ops a1 = Inst<10, 5, 2, uint32_t, uint8_t>::ops();
  static const Ops a2 = Inst<10, 5, 2, uint32_t, uint16_t>::ops();
  static const Ops a3 = Inst<10, 4, 2, uint32_t, uint16_t, true, 3>::ops();
  static const Ops b1 = Inst<10, 5, 3, uint64_t, uint16_t>::ops();
  static const Ops b2 = Inst<10, 4, 3, uint64_t, uint16_t, true>::ops();
  if (w == 32) {
    switch (variant) {
      case 0: return &a0;
      case 1: return &a1;
      case 2: return &a2;
      case 3: return &a3;
      default: return nullptr;
    }
  }
  if (w == 64) {
    switch (variant) {
      case 0: return &b0;
      case 1: return &b1;
      case 2: return &b2;
      default: return nullptr;
    }
  }
  return nullptr;
}
}  // namespace fdfb
