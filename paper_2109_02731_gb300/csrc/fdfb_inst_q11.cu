// Kernel instantiations for the prime-modulus parameter sets (Table 1) at
// N = 2^11: the blind rotation built with MQ (residues mod Q, exact digits,
// the products lifted to the exact integer and reduced mod Q).  Variant 0
// uses three 30-bit primes and also serves PubMux and key generation; the
// others split the centred key words into 32-bit halves over two primes,
// except 3: three primes with 64-bit sums of the 2l products (and, at
// N = 2^11, ping-pong exchange buffers).
#include "fdfb_inst.cuh"

namespace fdfb {
const Ops* ops_q_n11(int variant) {
  static const Ops v0 = Inst<11, 4, 3, uint64_t, uint16_t, false, br_min_blocks(3 << (11 - 4)), 2, false, false, 1, false, false, true>::ops();
  static const Ops v1 = Inst<11, 4, 2, uint64_t, uint16_t, false, 1, 2, false, true, 2, false, false, true>::ops();
  static const Ops v2 = Inst<11, 4, 2, uint64_t, uint16_t, false, 2, 1, false, false, 2, false, false, true>::ops();
  static const Ops v3 = Inst<11, 4, 3, uint64_t, uint16_t, true, br_min_blocks(3 << (11 - 4)), 2, false, true, 1, false, false, true>::ops();
  static const Ops* const v[] = {&v0, &v1, &v2, &v3};
  return variant >= 0 && variant < 4 ? v[variant] : nullptr;
}
}  // namespace fdfb
