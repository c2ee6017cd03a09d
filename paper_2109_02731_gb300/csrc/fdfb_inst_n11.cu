// Kernel instantiations for ring degree N = 2^11.
#include "fdfb_inst.cuh"

namespace fdfb {
const Ops* ops_n11(int w) {
  static const Ops o32 = Inst<11, 4, 2, uint32_t>::ops();
  static const Ops o64 = Inst<11, 4, 3, uint64_t>::ops();
  return w == 32 ? &o32 : (w == 64 ? &o64 : nullptr);
}
}  // namespace fdfb
