// Explicit instantiation of the kernels for one (L, EL, P, W) combination.
#pragma once
#include "fdfb_ops.hpp"

namespace fdfb {

template <int L, int EL, int P, typename W, typename DT = uint16_t, bool WIDE = false,
          int MINB = br_min_blocks(P * (1 << (L - EL))), int M = 1, bool LZ = false, bool PP = false,
          int KH = 1, bool SGV = false, bool TK = false, bool MQ = false>
struct Inst {
  // SGV: also build the blind rotation with balanced digits (parameter sets
  // with signed_digits only use variants that have it)
  template <bool SG>
  static constexpr auto kernel() { return blind_rotate_kernel<L, EL, P, W, DT, WIDE, MINB, M, LZ, PP, KH, SG, TK, MQ>; }
  using Sh = BRShape<L, EL, P, W, DT, M, PP, KH, TK, MQ>;
  static constexpr int THREADS = Sh::THREADS;
  static size_t br_smem(int n, int lg, uint32_t* r1, uint32_t* ex) { return Sh::smem_bytes(n, lg, r1, ex); }
  static cudaError_t br_prepare(size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(kernel<false>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess || !SGV) return e;
    return cudaFuncSetAttribute(kernel<SGV>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  static cudaError_t br(const BRParams& prm, int64_t batch, size_t smem, cudaStream_t st) {
    if (batch <= 0) return cudaSuccess;
    if (prm.signed_digits) {
      if (!SGV) return cudaErrorInvalidValue;
      kernel<SGV>()<<<(unsigned)batch, THREADS, smem, st>>>(prm);
    } else {
      kernel<false>()<<<(unsigned)batch, THREADS, smem, st>>>(prm);
    }
    return cudaGetLastError();
  }
  static cudaError_t pubmux(const PubMuxParams& prm, int64_t batch, cudaStream_t st) {
    if (batch <= 0) return cudaSuccess;
    constexpr size_t sm = product_smem_bytes<L, EL, P>();
    if (sm > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(pubmux_kernel<L, EL, P, W>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
    }
    pubmux_kernel<L, EL, P, W><<<(unsigned)batch, THREADS, sm, st>>>(prm);
    return cudaGetLastError();
  }
  static cudaError_t rlwe_enc(const RlweEncParams& prm, int64_t count, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    constexpr size_t sm = product_smem_bytes<L, EL, P>();
    if (sm > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(rlwe_encrypt_kernel<L, EL, P, W>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
    }
    rlwe_encrypt_kernel<L, EL, P, W><<<(unsigned)count, THREADS, sm, st>>>(prm);
    return cudaGetLastError();
  }
  static cudaError_t bsk_ntt(const PrimeSet& S, const void* bsk, int64_t rows, int R, uint32_t* out,
                             uint64_t Q, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    constexpr size_t sm = (size_t)P * (((size_t)Xch<L, EL>::kWords + 3) & ~(size_t)3) * 4;
    if (sm > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(bsk_to_ntt_kernel<L, EL, P, W, KH>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
    }
    bsk_to_ntt_kernel<L, EL, P, W, KH><<<(unsigned)rows, THREADS, sm, st>>>(S, bsk, R, out, Q);
    return cudaGetLastError();
  }
  static int br_blocks_per_sm(size_t smem) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel<false>(), THREADS, smem) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return b;
  }
  // prime-modulus PubMux and key generation (three primes: exact to 2^89)
  static cudaError_t pubmux_q(const PubMuxQParams& prm, int64_t batch, cudaStream_t st) {
    if constexpr (P != 3) {
      return cudaErrorInvalidValue;
    } else {
      if (batch <= 0) return cudaSuccess;
      constexpr size_t sm = product_smem_bytes<L, EL, P>();
      if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(pubmux_q_kernel<L, EL, P>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
      }
      pubmux_q_kernel<L, EL, P><<<(unsigned)batch, THREADS, sm, st>>>(prm);
      return cudaGetLastError();
    }
  }
  static cudaError_t rlwe_enc_q(const RlweEncQParams& prm, int64_t count, cudaStream_t st) {
    if constexpr (P != 3) {
      return cudaErrorInvalidValue;
    } else {
      if (count <= 0) return cudaSuccess;
      constexpr size_t sm = product_smem_bytes<L, EL, P>();
      if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(rlwe_encrypt_q_kernel<L, EL, P>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
      }
      rlwe_encrypt_q_kernel<L, EL, P><<<(unsigned)count, THREADS, sm, st>>>(prm);
      return cudaGetLastError();
    }
  }
  static Ops ops() {
    return Ops{L, EL, P, (int)(sizeof(W) * 8), THREADS, (int)(sizeof(DT) * 8), &br_smem, &br_prepare, &br,
               &pubmux, &rlwe_enc, &bsk_ntt, LZ ? 1 : 0, &br_blocks_per_sm, KH, SGV ? 1 : 0,
               MQ ? 1 : 0, MQ ? &pubmux_q : nullptr, MQ ? &rlwe_enc_q : nullptr};
  }
};

}  // namespace fdfb
