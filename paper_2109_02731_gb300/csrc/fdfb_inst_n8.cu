// Kernel instantiations for ring degree N = 2^8: one variant per register
// layout (coefficients per thread 2^EL).
#include "fdfb_inst.cuh"

namespace fdfb {
const Ops* ops_n8(int w, int variant) {
  static const Ops a0 = Inst<8, 3, 2, uint32_t>::ops();
  static const Ops b0 = Inst<8, 3, 3, uint64_t>::ops();
  switch (variant) {
    case 0: return w == 32 ? &a0 : (w == 64 ? &b0 : nullptr);
    default: return nullptr;
  }
}
}  // namespace fdfb
