// Kernel instantiations for ring degree N = 2^9.
#include "fdfb_inst.cuh"

namespace fdfb {
const Ops* ops_n9(int w) {
  static const Ops o32 = Inst<9, 4, 2, uint32_t>::ops();
  static const Ops o64 = Inst<9, 4, 3, uint64_t>::ops();
  return w == 32 ? &o32 : (w == 64 ? &o64 : nullptr);
}
}  // namespace fdfb
