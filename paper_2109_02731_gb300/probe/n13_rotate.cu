// Small-case driver of the N = 2^13 blind rotation (blind_rotate_n13_kernel
// of csrc/fdfb_n13.cuh, the layout of variant 0: 16 coefficients per thread,
// three primes), for timing and profiler captures on a case that holds a few
// hundred MB on the device.  The full FDFB:80:8 parameter set keeps about
// 21 GB of keys on the device, too much for a capture that saves and restores
// device memory between passes.  The key words here are random transform-
// domain residues and the ciphertexts random words mod 2N: the kernel does
// the same work for any values.  Sign mode, l_g = 7, B_g = 2^9, Q = Q_2.
//
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -lineinfo -std c++17 \
//        --expt-relaxed-constexpr -I include -I paper_2109_02731_gb300/csrc \
//        -o n13_rotate paper_2109_02731_gb300/probe/n13_rotate.cu
//   ./n13_rotate [items = 152] [n = 64] [launches = 3]
//
// Prints the best time per launch (after the first) and a checksum of the
// outputs; exits non-zero on a CUDA error.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "fdfb_host.hpp"
#include "fdfb_n13.cuh"

using namespace fdfb;

namespace {
bool ok(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return true;
  fprintf(stderr, "%s: %s\n", what, cudaGetErrorString(e));
  return false;
}
}  // namespace

int main(int argc, char** argv) {
  const int batch = argc > 1 ? atoi(argv[1]) : 152;
  const int n = argc > 2 ? atoi(argv[2]) : 64;
  const int reps = argc > 3 ? atoi(argv[3]) : 3;
  if (batch < 1 || n < 1 || n > 1536 || reps < 1) {
    fprintf(stderr, "items >= 1, 1 <= n <= 1536, launches >= 1\n");
    return 1;
  }
  constexpr int EL = 4, P = 3;
  const int lg = 7, log2Bg = 9, R = 2 * lg;
  const uint64_t Q = (1ull << 63) - 278527, c = 278527;
  PrimeSet S{};
  std::vector<uint2> tf, ti;
  host::make_prime_set_n13(P, EL, S, tf, ti);
  std::mt19937_64 g(1);
  const size_t kwords = (size_t)n * P * 2 * R * 2 * kN13h;
  std::vector<uint32_t> hk(kwords);
  for (size_t i = 0; i < kwords; ++i) hk[i] = (uint32_t)(g() % S.p[(i / ((size_t)2 * R * 2 * kN13h)) % P]);
  std::vector<uint64_t> hct((size_t)batch * (n + 1));
  for (auto& x : hct) x = g() % (2 * kN13);
  uint2* dtw = nullptr;
  uint32_t *dk = nullptr, *dy = nullptr;
  uint64_t *dct = nullptr, *dout = nullptr;
  int* derr = nullptr;
  if (!ok(cudaMalloc(&dtw, (tf.size() + ti.size()) * sizeof(uint2)), "cudaMalloc") ||
      !ok(cudaMalloc(&dk, kwords * 4), "cudaMalloc") || !ok(cudaMalloc(&dct, hct.size() * 8), "cudaMalloc") ||
      !ok(cudaMalloc(&dout, (size_t)batch * (kN13 + 1) * 8), "cudaMalloc") ||
      !ok(cudaMalloc(&dy, (size_t)batch * n13_scratch_words<P>() * 4), "cudaMalloc") ||
      !ok(cudaMalloc(&derr, 4), "cudaMalloc"))
    return 2;
  cudaMemcpy(dtw, tf.data(), tf.size() * sizeof(uint2), cudaMemcpyHostToDevice);
  cudaMemcpy(dtw + tf.size(), ti.data(), ti.size() * sizeof(uint2), cudaMemcpyHostToDevice);
  cudaMemcpy(dk, hk.data(), kwords * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(dct, hct.data(), hct.size() * 8, cudaMemcpyHostToDevice);
  cudaMemset(derr, 0, 4);
  S.tw_fwd = dtw;
  S.tw_inv = dtw + tf.size();
  BRParams prm{};
  prm.S = S;
  prm.bsk = dk;
  prm.ct = dct;
  prm.lwe_out = dout;
  prm.n = n;
  prm.lg = lg;
  prm.log2Bg = log2Bg;
  prm.batch = batch;
  prm.sign_mode = 1;
  const size_t d = 2 * (size_t)kN13 * 8, an = ((size_t)n * 2 + 15) & ~(size_t)15;
  prm.smem_r1 = prm.smem_exch = (uint32_t)(d + an);
  const size_t smem = d + an + (size_t)P * kN13 * 4;
  prm.rep = 1;
  prm.err = derr;
  prm.mq = ModQ{Q, c, 63, modq_folds(Q, c, 63), modq_folds64(Q, c, 63)};
  for (int i = 0; i < 8; ++i) prm.sgn_scale[i] = g() % Q;
  prm.half_y = dy;
  auto k = blind_rotate_n13_kernel<EL, P, 1>;
  if (!ok(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "smem attribute"))
    return 3;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float best = 1e30f;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(a);
    k<<<batch, P << (12 - EL), smem>>>(prm);
    cudaEventRecord(b);
    if (!ok(cudaGetLastError(), "launch") || !ok(cudaEventSynchronize(b), "kernel")) return 4;
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    if ((r > 0 || reps == 1) && ms < best) best = ms;
  }
  std::vector<uint64_t> ho((size_t)batch * (kN13 + 1));
  cudaMemcpy(ho.data(), dout, ho.size() * 8, cudaMemcpyDeviceToHost);
  uint64_t chk = 0;
  for (auto x : ho) chk = chk * 1000003 + x;
  printf("blind_rotate_n13_kernel, %d items, n %d: %.3f ms per launch (%.4f ms per step and wave of 152), "
         "checksum %016llx\n",
         batch, n, best, best / ((double)n * ((batch + 151) / 152)), (unsigned long long)chk);
  return 0;
}
