// Kernel instantiations for the prime-modulus parameter sets (Table 1) at
// N = 2^8: the blind rotation built with MQ (residues mod Q, exact digits,
// the products lifted to the exact integer and reduced mod Q).  Variant 0
// uses three 30-bit primes and also serves PubMux and key generation; 1
// pairs the forward transforms; 2 splits the centred key words into 32-bit
// halves over two primes; 3 sums the 2l products of a column in 64 bits
// (three primes, paired); 4 uses two primes with whole key words, kept only
// where that lift is exact (Q_4).
#include "fdfb_inst.cuh"

namespace fdfb {
const Ops* ops_q_n8(int variant) {
  static const Ops v0 = Inst<8, 3, 3, uint64_t, uint16_t, false, br_min_blocks(3 << (8 - 3)), 1, false, false, 1, false, false, true>::ops();
  static const Ops v1 = Inst<8, 3, 3, uint64_t, uint16_t, false, br_min_blocks(3 << (8 - 3)), 2, false, false, 1, false, false, true>::ops();
  static const Ops v2 = Inst<8, 3, 2, uint64_t, uint16_t, false, br_min_blocks(2 << (8 - 3)), 1, false, false, 2, false, false, true>::ops();
  static const Ops v3 = Inst<8, 3, 3, uint64_t, uint16_t, true, br_min_blocks(3 << (8 - 3)), 2, false, false, 1, false, false, true>::ops();
  // two primes with whole key words: kept only where that lift is exact (Q_4)
  static const Ops v4 = Inst<8, 3, 2, uint64_t, uint16_t, false, br_min_blocks(2 << (8 - 3)), 1, false, false, 1, false, false, true>::ops();
  static const Ops* const v[] = {&v0, &v1, &v2, &v3, &v4};
  return variant >= 0 && variant < 5 ? v[variant] : nullptr;
}
}  // namespace fdfb
