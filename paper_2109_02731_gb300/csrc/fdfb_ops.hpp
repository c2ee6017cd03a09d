// Per-(ring degree, word size) table of launchers for the templated kernels.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "fdfb_kernels.cuh"

namespace fdfb {

struct Ops {
  int L, EL, P, w, threads;
  int max_log2B;  // widest digit the blind rotation's digit buffer holds
  size_t (*br_smem)(int n, int lg, uint32_t* r1_off, uint32_t* exch_off);
  cudaError_t (*br_prepare)(size_t smem);
  cudaError_t (*br)(const BRParams& prm, int64_t batch, size_t smem, cudaStream_t st);
  cudaError_t (*pubmux)(const PubMuxParams& prm, int64_t batch, cudaStream_t st);
  cudaError_t (*rlwe_enc)(const RlweEncParams& prm, int64_t count, cudaStream_t st);
  cudaError_t (*bsk_ntt)(const PrimeSet& S, const void* bsk, int64_t rows, int R, uint32_t* out,
                         uint64_t Q, cudaStream_t st);
  int family;  // NTT prime family of the blind rotation (0: 30-bit primes, 1: lazy family)
  int (*br_blocks_per_sm)(size_t smem);  // resident blind-rotation CTAs per SM
  int key_halves;  // 2: 64-bit key words split into 32-bit halves over two primes
  int has_signed;  // also built with balanced blind-rotation digits
  int mq;          // built for the prime-modulus sets (words mod Q, exact digits)
  cudaError_t (*pubmux_q)(const PubMuxQParams& prm, int64_t batch, cudaStream_t st);
  cudaError_t (*rlwe_enc_q)(const RlweEncQParams& prm, int64_t count, cudaStream_t st);
};

// Returns the launcher table of register-layout variant `variant` for
// N = 2^L and word size w, or nullptr past the last variant; find_ops_q the
// variants built for the prime-modulus sets (64-bit words).
const Ops* find_ops(int L, int w, int variant);
const Ops* find_ops_q(int L, int variant);

}  // namespace fdfb
