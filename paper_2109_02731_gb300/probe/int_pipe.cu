// Throughput probe of the SM integer pipes on the local GPU, used by bench.py
// to report the measured peak next to the derived one.  Each kernel keeps 8
// independent dependency chains per thread at full occupancy, so the rate is
// set by pipe width, not latency.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../csrc/fdfb_core.cuh"

namespace {

constexpr int kIter = 2048;

__global__ void imad_kernel(uint32_t* out, uint32_t x, uint32_t y) {
  uint32_t a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = threadIdx.x + k;
  for (int i = 0; i < kIter; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[k]) : "r"(x), "r"(y));
  }
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s ^= a[k];
  if (s == 0x12345678u) out[0] = s;
}

__global__ void imadhi_kernel(uint32_t* out, uint32_t x, uint32_t y) {
  uint32_t a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = threadIdx.x + k;
  for (int i = 0; i < kIter; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(a[k]) : "r"(x), "r"(y));
  }
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s ^= a[k];
  if (s == 0x12345678u) out[0] = s;
}

// Three-input XOR of neighbouring chains (one LOP3 each); the chains feed
// each other, so nothing folds away.
__global__ void lop_kernel(uint32_t* out, uint32_t x, uint32_t y) {
  uint32_t a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = threadIdx.x * 0x9e3779b9u + k * x + y;
  for (int i = 0; i < kIter; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k)
      asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[k]) : "r"(a[(k + 3) & 7]), "r"(a[(k + 5) & 7]));
  }
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s ^= a[k];
  if (s == 0x12345678u) out[0] = s;
}

// Harvey forward butterflies on registers with a fixed twiddle.
__global__ void bfly_kernel(uint32_t* out, uint32_t w, uint32_t wp, uint32_t p, uint32_t z) {
  uint32_t v[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = (threadIdx.x * 16 + k) % p;
  const uint2 tw{w, wp};
  for (int i = 0; i < kIter / 8; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) fdfb::bfly_fwd(v[k], v[k + 8], tw, p, z);
  }
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) s ^= v[k];
  if (s == 0x12345678u) out[0] = s;
}

}  // namespace

// rates[0..3]: IMAD (mad.lo.u32), IMAD.HI (mad.hi.u32), LOP (xor), Harvey
// butterflies, all per second over the whole GPU.  Returns 0 or a CUDA error.
extern "C" int probe_int_rates(int device, double* rates) {
  cudaSetDevice(device);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  uint32_t* out = nullptr;
  if (cudaMalloc(&out, 16) != cudaSuccess) return 1;
  const int blocks = sms * 8, threads = 256;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  for (int kind = 0; kind < 4; ++kind) {
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
      cudaEventRecord(a);
      if (kind == 0) imad_kernel<<<blocks, threads>>>(out, 3, 7);
      if (kind == 1) imadhi_kernel<<<blocks, threads>>>(out, 0x9e3779b9u, 7);
      if (kind == 2) lop_kernel<<<blocks, threads>>>(out, 0x9e3779b9u, 7);
      if (kind == 3) bfly_kernel<<<blocks, threads>>>(out, 123456789u, fdfb::host_shoup(123456789u, 1073692673u), 1073692673u, 0u);
      cudaEventRecord(b);
      cudaEventSynchronize(b);
      float ms = 0;
      cudaEventElapsedTime(&ms, a, b);
      if (rep > 0 && ms < best) best = ms;
    }
    const double ops = (double)blocks * threads * (kind == 3 ? (kIter / 8) * 8 : kIter * 8);
    rates[kind] = ops / (best / 1e3);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(out);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}
