// Kernel instantiations for ring degree N = 2^12: one blind-rotation variant per
// register layout (coefficients per thread), digit width, accumulation
// (Montgomery-reduced 32-bit or 64-bit) and polynomials per transform pass.
#include "fdfb_inst.cuh"

namespace fdfb {
// Variants whose last template argument is true are also built with balanced
// blind-rotation digits (the only ones a set with signed_digits uses).
const Ops* ops_n12(int w, int variant) {
  static const Ops a0 = Inst<12, 4, 2, uint32_t, uint16_t, false, br_min_blocks(2 << (12 - 4)), 1, false, false, 1, true>::ops();
  static const Ops a1 = Inst<12, 5, 2, uint32_t, uint8_t>::ops();
  static const Ops a2 = Inst<12, 4, 2, uint32_t, uint16_t, true, br_blocks_for_regs(2 << (12 - 4), 168)>::ops();
  static const Ops a3 = Inst<12, 4, 2, uint32_t, uint8_t, false, br_blocks_for_regs(2 << (12 - 4), 128), 2>::ops();
  static const Ops a4 = Inst<12, 4, 2, uint32_t, uint16_t, true, br_blocks_for_regs(2 << (12 - 4), 168), 2>::ops();
  // lazy prime family (variant 5): a4 with unreduced forward transforms
  static const Ops a5 = Inst<12, 4, 2, uint32_t, uint16_t, true, br_blocks_for_regs(2 << (12 - 4), 168), 2, true>::ops();
  static const Ops b0 = Inst<12, 4, 3, uint64_t, uint16_t, false, br_min_blocks(3 << (12 - 4)), 1, false, false, 1, true>::ops();
  static const Ops b1 = Inst<12, 5, 3, uint64_t, uint16_t>::ops();
  static const Ops b2 = Inst<12, 4, 3, uint64_t, uint16_t, true>::ops();
  static const Ops b3 = Inst<12, 4, 3, uint64_t, uint16_t, false, br_min_blocks(3 << (12 - 4)), 2>::ops();
  static const Ops b4 = Inst<12, 4, 3, uint64_t, uint16_t, true, br_min_blocks(3 << (12 - 4)), 2>::ops();
  // 64-bit key words split into 32-bit halves over two primes (two groups of threads)
  static const Ops b5 = Inst<12, 4, 2, uint64_t, uint16_t, false, 1, 2, false, false, 2, true>::ops();
  // split keys with single forward transforms (fewer live registers at 128 per thread)
  static const Ops b6 = Inst<12, 4, 2, uint64_t, uint16_t, false, 1, 1, false, false, 2>::ops();
  static const Ops* const v32[] = {&a0, &a1, &a2, &a3, &a4, &a5};
  static const Ops* const v64[] = {&b0, &b1, &b2, &b3, &b4, &b5, &b6};
  if (variant < 0) return nullptr;
  if (w == 32) return variant < 6 ? v32[variant] : nullptr;
  if (w == 64) return variant < 7 ? v64[variant] : nullptr;
  return nullptr;
}
}  // namespace fdfb
