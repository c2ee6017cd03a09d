// Throughput probe of the SM pipes the blind rotation could use, run by
// bench.py on the GPU it measures.  Two purposes:
//   1. The roofline's denominator.  The exact negacyclic products of the
//      blind rotation are built from three operations -- the forward
//      (Harvey) and inverse (Gentleman-Sande) Shoup butterflies of
//      fdfb_core.cuh and the 32 x 32 -> 64 multiply-add of the transform-
//      domain key products -- and each is timed here, on registers only, at
//      full occupancy with several independent chains per thread, so the rate
//      is set by the pipes and not by latency.  Every kernel below calls the
//      very functions the library's kernels call.  Several chain counts are
//      timed and the fastest kept.
//   2. The split-precision alternatives of the products: FP64 fused
//      multiply-add (an FFT over small key limbs) and 8-bit integer tensor
//      products (mma.sync m16n8k32, the IMMA form sm_103a accepts; tcgen05's
//      kind::i8 is rejected by ptxas for this target).
// Single plain instructions (mad.lo, mad.hi, a three-input logic op) are
// timed too, for the derived integer-multiplier peak.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../csrc/fdfb_core.cuh"

namespace {

constexpr int kIter = 2048;

template <int C>
__global__ void imad_kernel(uint32_t* out, uint32_t x, uint32_t y) {
  uint32_t a[C];
#pragma unroll
  for (int k = 0; k < C; ++k) a[k] = threadIdx.x + k;
  for (int i = 0; i < kIter; ++i) {
#pragma unroll
    for (int k = 0; k < C; ++k) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[k]) : "r"(x), "r"(y));
  }
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < C; ++k) s ^= a[k];
  if (s == 0x12345678u) out[0] = s;
}

template <int C>
__global__ void imadhi_kernel(uint32_t* out, uint32_t x, uint32_t y) {
  uint32_t a[C];
#pragma unroll
  for (int k = 0; k < C; ++k) a[k] = threadIdx.x + k;
  for (int i = 0; i < kIter; ++i) {
#pragma unroll
    for (int k = 0; k < C; ++k) asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(a[k]) : "r"(x), "r"(y));
  }
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < C; ++k) s ^= a[k];
  if (s == 0x12345678u) out[0] = s;
}

// Three-input XOR of neighbouring chains (one LOP3 each); the chains feed
// each other, so nothing folds away.
template <int C>
__global__ void lop_kernel(uint32_t* out, uint32_t x, uint32_t y) {
  uint32_t a[C];
#pragma unroll
  for (int k = 0; k < C; ++k) a[k] = threadIdx.x * 0x9e3779b9u + k * x + y;
  for (int i = 0; i < kIter; ++i) {
#pragma unroll
    for (int k = 0; k < C; ++k)
      asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[k]) : "r"(a[(k + 3) % C]), "r"(a[(k + 5) % C]));
  }
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < C; ++k) s ^= a[k];
  if (s == 0x12345678u) out[0] = s;
}

// Butterflies on 2C registers with a fixed twiddle: C independent chains.
// KIND 0: Harvey forward (fdfb::bfly_fwd), 1: Gentleman-Sande inverse
// (fdfb::bfly_inv), 2: the lazy family's forward (fdfb::bfly_fwd_lazy).
template <int KIND, int C>
__global__ void bfly_kernel(uint32_t* out, uint32_t w, uint32_t wp, uint32_t p, uint32_t z) {
  uint32_t v[2 * C];
#pragma unroll
  for (int k = 0; k < 2 * C; ++k) v[k] = (threadIdx.x * 2 * C + k) % p;
  const uint2 tw{w, wp};
  for (int i = 0; i < kIter / C; ++i) {
#pragma unroll
    for (int k = 0; k < C; ++k) {
      if (KIND == 0) fdfb::bfly_fwd(v[k], v[k + C], tw, p, z);
      if (KIND == 1) fdfb::bfly_inv(v[k], v[k + C], tw, p, z);
      if (KIND == 2) fdfb::bfly_fwd_lazy(v[k], v[k + C], tw, p, z);  // values wrap: only the rate matters
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < 2 * C; ++k) s ^= v[k];
  if (s == 0x12345678u) out[0] = s;
}

// Transform-domain key products: C independent 64-bit sums of 32 x 32 -> 64
// products (the "wide" sums of the blind rotation), the multiplicands
// changing every step so nothing is hoisted.
template <int C>
__global__ void mac_kernel(uint32_t* out, uint32_t x, uint32_t y) {
  uint64_t acc[C];
  uint32_t a[C];
#pragma unroll
  for (int k = 0; k < C; ++k) {
    acc[k] = threadIdx.x + k;
    a[k] = threadIdx.x * 0x9e3779b9u + k;
  }
  for (int i = 0; i < kIter; ++i) {
#pragma unroll
    for (int k = 0; k < C; ++k) {
      acc[k] += (uint64_t)a[k] * (x + (uint32_t)i);
      a[k] ^= y;
    }
  }
  uint64_t s = 0;
#pragma unroll
  for (int k = 0; k < C; ++k) s ^= acc[k];
  if (s == 0x12345678ull) out[0] = (uint32_t)s;
}

// FP64 fused multiply-add chains (2 flops each).
template <int C>
__global__ void dfma_kernel(double* out, double x, double y) {
  double a[C];
#pragma unroll
  for (int k = 0; k < C; ++k) a[k] = threadIdx.x + k;
  for (int i = 0; i < kIter; ++i) {
#pragma unroll
    for (int k = 0; k < C; ++k) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(a[k]) : "d"(x), "d"(y));
  }
  double s = 0;
#pragma unroll
  for (int k = 0; k < C; ++k) s += a[k];
  if (s == 1234.5) out[0] = s;
}

// 8-bit integer tensor products: C independent accumulators of
// mma.sync.m16n8k32 (s8 x s8 -> s32), 16 * 8 * 32 multiply-adds per warp each.
template <int C>
__global__ void imma_kernel(int* out, uint32_t a0, uint32_t b0) {
  int c[C][4];
#pragma unroll
  for (int k = 0; k < C; ++k)
#pragma unroll
    for (int j = 0; j < 4; ++j) c[k][j] = 0;
  const uint32_t a[4] = {a0, a0 ^ 0x01010101u, a0 ^ 0x02020202u, a0 ^ 0x03030303u};
  const uint32_t b[2] = {b0, b0 ^ 0x05050505u};
  for (int i = 0; i < kIter / 4; ++i) {
#pragma unroll
    for (int k = 0; k < C; ++k)
      asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                   "{%0,%1,%2,%3};"
                   : "+r"(c[k][0]), "+r"(c[k][1]), "+r"(c[k][2]), "+r"(c[k][3])
                   : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  }
  int s = 0;
#pragma unroll
  for (int k = 0; k < C; ++k) s += c[k][0] + c[k][1] + c[k][2] + c[k][3];
  if (s == 0x12345678) out[0] = s;
}

template <typename F>
float best_ms(F launch) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(a);
    launch();
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    if (rep > 0 && ms < best) best = ms;  // the first launch warms up
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return best;
}

}  // namespace

// Number of rates probe_pipe_rates writes.
extern "C" int probe_pipe_count() { return 9; }

// rates[i], operations per second over the whole GPU:
//   0 mad.lo.u32     1 mad.hi.u32     2 lop3 (three-input logic)
//   3 Harvey forward butterflies (bfly_fwd, 30-bit prime)
//   4 Gentleman-Sande inverse butterflies (bfly_inv)
//   5 lazy-family forward butterflies (bfly_fwd_lazy)
//   6 32 x 32 -> 64 multiply-adds into 64-bit sums
//   7 FP64 flops (fma.rn.f64 = 2 flops)
//   8 8-bit integer tensor ops (mma.sync m16n8k32 s8: 2 ops per multiply-add)
// Every rate is the best of the chain counts tried.  Returns 0 or a CUDA
// error code.
extern "C" int probe_pipe_rates(int device, double* rates) {
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return (int)e;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  void* out = nullptr;
  if ((e = cudaMalloc(&out, 64)) != cudaSuccess) return (int)e;
  uint32_t* o32 = (uint32_t*)out;
  const int blocks = sms * 8, threads = 256;  // 2048 threads per SM
  const double thr = (double)blocks * threads;
  const uint32_t p = fdfb::kPrimes[0], w = 123456789u, wp = fdfb::host_shoup(w, p);
  const uint32_t pl = fdfb::kPrimesLazy[0], wl = 12345679u, wpl = fdfb::host_shoup(wl, pl);
  auto rate = [&](double ops_per_thread, float ms) { return thr * ops_per_thread / (ms / 1e3); };
  double r;
#define FD_BEST(idx, expr) do { r = (expr); if (r > rates[idx]) rates[idx] = r; } while (0)
  for (int i = 0; i < 9; ++i) rates[i] = 0.0;
  FD_BEST(0, rate(kIter * 8.0, best_ms([&] { imad_kernel<8><<<blocks, threads>>>(o32, 3, 7); })));
  FD_BEST(0, rate(kIter * 16.0, best_ms([&] { imad_kernel<16><<<blocks, threads>>>(o32, 3, 7); })));
  FD_BEST(1, rate(kIter * 8.0, best_ms([&] { imadhi_kernel<8><<<blocks, threads>>>(o32, 0x9e3779b9u, 7); })));
  FD_BEST(1, rate(kIter * 16.0, best_ms([&] { imadhi_kernel<16><<<blocks, threads>>>(o32, 0x9e3779b9u, 7); })));
  FD_BEST(2, rate(kIter * 8.0, best_ms([&] { lop_kernel<8><<<blocks, threads>>>(o32, 0x9e3779b9u, 7); })));
  FD_BEST(2, rate(kIter * 16.0, best_ms([&] { lop_kernel<16><<<blocks, threads>>>(o32, 0x9e3779b9u, 7); })));
  // butterflies: (kIter / C) iterations of C butterflies
  FD_BEST(3, rate(kIter, best_ms([&] { bfly_kernel<0, 4><<<blocks, threads>>>(o32, w, wp, p, 0u); })));
  FD_BEST(3, rate(kIter, best_ms([&] { bfly_kernel<0, 8><<<blocks, threads>>>(o32, w, wp, p, 0u); })));
  FD_BEST(3, rate(kIter, best_ms([&] { bfly_kernel<0, 16><<<blocks, threads>>>(o32, w, wp, p, 0u); })));
  FD_BEST(4, rate(kIter, best_ms([&] { bfly_kernel<1, 4><<<blocks, threads>>>(o32, w, wp, p, 0u); })));
  FD_BEST(4, rate(kIter, best_ms([&] { bfly_kernel<1, 8><<<blocks, threads>>>(o32, w, wp, p, 0u); })));
  FD_BEST(4, rate(kIter, best_ms([&] { bfly_kernel<1, 16><<<blocks, threads>>>(o32, w, wp, p, 0u); })));
  FD_BEST(5, rate(kIter, best_ms([&] { bfly_kernel<2, 8><<<blocks, threads>>>(o32, wl, wpl, pl, 0u); })));
  FD_BEST(5, rate(kIter, best_ms([&] { bfly_kernel<2, 16><<<blocks, threads>>>(o32, wl, wpl, pl, 0u); })));
  FD_BEST(6, rate(kIter * 4.0, best_ms([&] { mac_kernel<4><<<blocks, threads>>>(o32, 0x9e3779b9u, 7); })));
  FD_BEST(6, rate(kIter * 8.0, best_ms([&] { mac_kernel<8><<<blocks, threads>>>(o32, 0x9e3779b9u, 7); })));
  FD_BEST(6, rate(kIter * 16.0, best_ms([&] { mac_kernel<16><<<blocks, threads>>>(o32, 0x9e3779b9u, 7); })));
  FD_BEST(7, rate(kIter * 8.0 * 2, best_ms([&] { dfma_kernel<8><<<blocks, threads>>>((double*)out, 1.0000001, 1e-9); })));
  FD_BEST(7, rate(kIter * 16.0 * 2, best_ms([&] { dfma_kernel<16><<<blocks, threads>>>((double*)out, 1.0000001, 1e-9); })));
  // one mma per warp = 16 * 8 * 32 multiply-adds = 8192 ops, i.e. 256 per thread
  FD_BEST(8, rate((kIter / 4) * 2.0 * 256, best_ms([&] { imma_kernel<2><<<blocks, threads>>>((int*)out, 0x01020304u, 0x05060708u); })));
  FD_BEST(8, rate((kIter / 4) * 4.0 * 256, best_ms([&] { imma_kernel<4><<<blocks, threads>>>((int*)out, 0x01020304u, 0x05060708u); })));
#undef FD_BEST
  e = cudaGetLastError();
  cudaFree(out);
  return e == cudaSuccess ? 0 : (int)e;
}
