// Kernel instantiations for the prime-modulus parameter sets (Table 1) at
// N = 2^10 (the TFHE columns): the blind rotation built with MQ (residues
// mod Q, exact digits, the products lifted to the exact integer and reduced
// mod Q).  Variant 0 uses three 30-bit primes and also serves PubMux and key
// generation; 1 splits the centred key words into 32-bit halves over two
// primes; 2 sums the 2l products of a column in 64 bits (three primes,
// paired transforms); 3 and 4 use two primes with whole key words, which
// registration keeps only where the sums lift exactly from two primes
// (Q_4 = 2^32 - 139263: 2 l N (B - 1) Q / 2 < 2^55).
#include "fdfb_inst.cuh"

namespace fdfb {
const Ops* ops_q_n10(int variant) {
  static const Ops v0 = Inst<10, 4, 3, uint64_t, uint16_t, false, br_min_blocks(3 << (10 - 4)), 1, false, false, 1, false, false, true>::ops();
  static const Ops v1 = Inst<10, 4, 2, uint64_t, uint16_t, false, br_min_blocks(2 << (10 - 4)), 1, false, false, 2, false, false, true>::ops();
  static const Ops v2 = Inst<10, 4, 3, uint64_t, uint16_t, true, br_min_blocks(3 << (10 - 4)), 2, false, false, 1, false, false, true>::ops();
  // two primes, whole key words (Q_4: the sums lift from two primes), single
  // and paired forward transforms
  static const Ops v3 = Inst<10, 4, 2, uint64_t, uint16_t, false, br_min_blocks(2 << (10 - 4)), 1, false, false, 1, false, false, true>::ops();
  static const Ops v4 = Inst<10, 4, 2, uint64_t, uint16_t, true, br_min_blocks(2 << (10 - 4)), 2, false, false, 1, false, false, true>::ops();
  static const Ops* const v[] = {&v0, &v1, &v2, &v3, &v4};
  return variant >= 0 && variant < 5 ? v[variant] : nullptr;
}
}  // namespace fdfb
