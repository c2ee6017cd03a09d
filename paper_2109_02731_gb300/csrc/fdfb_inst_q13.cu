// Kernel instantiations for the prime-modulus parameter sets (Table 1) at
// N = 2^13 (fdfb_n13.cuh: split transforms, one CTA per item).  Variant 0
// keeps 16 coefficients per thread (768 threads), variant 1 32 (384
// threads, twice the registers per thread), both with three 30-bit primes
// (variant 0 also serves PubMux and key generation); variant 2 splits the
// key words into 32-bit halves over two primes (512 threads).
#include "fdfb_n13.cuh"
#include "fdfb_ops.hpp"

namespace fdfb {

template <int EL, int P = 3, int MINB = 1, int KH = 1>
struct InstN13 {
  static constexpr int THREADS = P << (12 - EL);
  static constexpr size_t XB = (size_t)P * n13_xwords<EL>() * 4;
  static constexpr size_t region_bytes() {
    return (size_t)P * kN13 * 4 > XB ? (size_t)P * kN13 * 4 : XB;
  }
  // d | a_N | one region: exchange buffers, then the lift's stage [P][8192]
  static size_t br_smem(int n, int, uint32_t* r1, uint32_t* ex) {
    const size_t d = 2 * (size_t)kN13 * 8;
    const size_t an = ((size_t)n * 2 + 15) & ~(size_t)15;
    *r1 = *ex = (uint32_t)(d + an);
    return d + an + region_bytes();
  }
  static cudaError_t br_prepare(size_t smem) {
    return cudaFuncSetAttribute(blind_rotate_n13_kernel<EL, P, MINB, KH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
  }
  static cudaError_t br(const BRParams& prm, int64_t batch, size_t smem, cudaStream_t st) {
    if (batch <= 0) return cudaSuccess;
    if (prm.signed_digits || !prm.half_y || prm.mq.Q == 0) return cudaErrorInvalidValue;
    blind_rotate_n13_kernel<EL, P, MINB, KH><<<(unsigned)batch, THREADS, smem, st>>>(prm);
    return cudaGetLastError();
  }
  // the power-of-two PubMux and encryption do not exist at N = 2^13
  static cudaError_t pubmux(const PubMuxParams&, int64_t, cudaStream_t) { return cudaErrorInvalidValue; }
  static cudaError_t rlwe_enc(const RlweEncParams&, int64_t, cudaStream_t) { return cudaErrorInvalidValue; }
  static cudaError_t bsk_ntt(const PrimeSet& S, const void* bsk, int64_t rows, int R, uint32_t* out, uint64_t Q,
                             cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    if (Q == 0) return cudaErrorInvalidValue;
    if (XB > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(bsk_to_ntt_n13_kernel<EL, P, KH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)XB);
      if (e != cudaSuccess) return e;
    }
    bsk_to_ntt_n13_kernel<EL, P, KH><<<(unsigned)rows, THREADS, XB, st>>>(S, bsk, R, out, Q);
    return cudaGetLastError();
  }
  static int br_blocks_per_sm(size_t smem) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, blind_rotate_n13_kernel<EL, P, MINB, KH>, THREADS, smem) !=
        cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return b;
  }
  // PubMux and key generation: three primes (their products reach 2^87)
  static cudaError_t pubmux_q(const PubMuxQParams& prm, int64_t batch, cudaStream_t st) {
    if (P != 3) return cudaErrorInvalidValue;
    if (batch <= 0) return cudaSuccess;
    const size_t sm = (size_t)2 * P * kN13h * 4 + region_bytes();
    cudaError_t e = cudaFuncSetAttribute(pubmux_q_n13_kernel<EL, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    pubmux_q_n13_kernel<EL, P><<<(unsigned)batch, THREADS, sm, st>>>(prm);
    return cudaGetLastError();
  }
  static cudaError_t rlwe_enc_q(const RlweEncQParams& prm, int64_t count, cudaStream_t st) {
    if (P != 3) return cudaErrorInvalidValue;
    if (count <= 0) return cudaSuccess;
    const size_t sm = (size_t)2 * P * kN13h * 4 + region_bytes();
    cudaError_t e = cudaFuncSetAttribute(rlwe_encrypt_q_n13_kernel<EL, P>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    rlwe_encrypt_q_n13_kernel<EL, P><<<(unsigned)count, THREADS, sm, st>>>(prm);
    return cudaGetLastError();
  }
  static Ops ops() {
    return Ops{13, EL, P, 64, THREADS, 16, &br_smem, &br_prepare, &br, &pubmux, &rlwe_enc, &bsk_ntt, 0,
               &br_blocks_per_sm, KH, 0, 1, &pubmux_q, &rlwe_enc_q};
  }
};

const Ops* ops_q_n13(int variant) {
  static const Ops v0 = InstN13<4>::ops();
  static const Ops v1 = InstN13<5>::ops();
  static const Ops v2 = InstN13<4, 2, 1, 2>::ops();
  static const Ops* const v[] = {&v0, &v1, &v2};
  return variant >= 0 && variant < 3 ? v[variant] : nullptr;
}

}  // namespace fdfb
