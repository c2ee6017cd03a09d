// Exact key switching on the tensor cores (tcgen05.mma, kind::f16): see
// fdfb_ks_tc.hpp for the arithmetic.  One CTA computes a 128 x BN tile of
// the output (128 ciphertexts x BN output words; BN = 128 for the
// power-of-two form, 64 for the exact form, whose 128-bit sums take twice
// the registers):
//   - warp 0 allocates 2 BN columns of tensor memory (two fp32 accumulators);
//     its lane 0 issues the TMA loads of the digit tile (128 x 64 f16) and
//     the key-limb tile (BN x 64 f16) into a four-stage shared-memory ring
//     and the MMAs (M = 128, N = BN, K = 16 each) that accumulate one (digit
//     half, limb, chunk) unit into one accumulator;
//   - warps 1-8 drain each finished accumulator with tcgen05.ld (warp w reads
//     the 32 rows of tensor-memory lane quarter w mod 4 and half of the
//     columns), convert the exact fp32 integers and add them, shifted by the
//     unit's bits, into per-thread 64-bit (power-of-two form) or 128-bit
//     (exact form) sums, while the MMAs of the next unit fill the other
//     accumulator.
// Every wait on an mbarrier is bounded in time; on expiry the thread latches
// FDFB_ETIMEOUT, raises an abort flag the other roles poll, waits (again
// bounded) for the copies it issued, and the CTA releases its tensor memory.
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "fdfb.h"
#include "fdfb_ks_tc.hpp"

namespace fdfb {
namespace {

constexpr int TC_BM = 128, TC_BK = 64, TC_STAGES = 4;
constexpr int TC_EPI_WARPS = 8;
constexpr int TC_THREADS = 32 * (1 + TC_EPI_WARPS);
constexpr uint32_t TC_A_BYTES = TC_BM * TC_BK * 2;  // 16 KB
constexpr long long kWaitCycles = 1ll << 32;         // about two seconds at 2 GHz

// Shapes of a CTA with a BN-wide output tile.
template <int BN>
struct TcTile {
  static constexpr uint32_t STAGE = TC_A_BYTES + (uint32_t)BN * TC_BK * 2;  // 32 or 24 KB (multiples of 1 KB)
  static constexpr uint32_t TMEM_COLS = 2 * BN;
  static constexpr size_t SMEM = 1024 + (size_t)TC_STAGES * STAGE + 256;
  static constexpr int CPW = BN / 2;  // columns per epilogue warp (two warps per lane quarter)
  // instruction descriptor: fp32 accumulator, f16 A and B, both K-major, N = BN, M = 128
  static constexpr uint32_t IDESC = (1u << 4) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
};

struct TcArgs {
  const void* ct;   // [batch][n_in + 1] words; b_m is word 0 of row m
  void* out;        // [batch][cols] words, or the exact form's [batch][2 cols] sums
  int* err;
  int64_t batch;
  int n_in, cols, S, b, chunks, ksteps, halves, h;
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
// Waits for phase `parity` of the mbarrier; false if the abort flag rises or
// the time budget runs out first.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, volatile int* abort_flag) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}" : "=r"(done) : "r"(a), "r"(parity) : "memory");
    if (done) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > kWaitCycles) return false;
  }
}
__device__ __forceinline__ void tma_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t mbar) {
  asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
               ::"r"(dst), "l"(map), "r"(x), "r"(y), "r"(mbar) : "memory");
}
__device__ __forceinline__ void tma_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t mbar) {
  asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
               ::"r"(dst), "l"(map), "r"(x), "r"(y), "r"(z), "r"(mbar) : "memory");
}
// Shared-memory matrix descriptor of a K-major operand tile whose rows are 128
// bytes (64 f16) in the 128-byte swizzle TMA writes: 8-row atoms of 1024
// bytes (stride between atoms 1024 B), descriptor version 1, swizzle mode 2.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
               " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
               ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive fp32 columns of this warp's 32 tensor-memory lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

// EXACT: the prime-modulus form (128-bit sums of the exact integer products,
// written as S mod 2^32 and S >> 32); else the power-of-two form.
template <typename W, int BN, bool EXACT>
__global__ void __launch_bounds__(TC_THREADS, 1)
tc_ks_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const TcArgs a) {
  using T = TcTile<BN>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t raw = smem_addr(smem_raw);
  const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
  unsigned char* smem = smem_raw + pad;
  const uint32_t sbase = raw + pad;  // 1024-byte aligned: the swizzle atoms start on it
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)TC_STAGES * T::STAGE);
  const uint32_t bar0 = smem_addr(bars);
  auto full = [&](int s) { return bar0 + 8u * s; };
  auto empty = [&](int s) { return bar0 + 8u * (TC_STAGES + s); };
  auto accfull = [&](int b) { return bar0 + 8u * (2 * TC_STAGES + b); };
  auto accempty = [&](int b) { return bar0 + 8u * (2 * TC_STAGES + 2 + b); };
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2 * TC_STAGES + 4);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accfull(b), 1);
      mbar_init(accempty(b), TC_EPI_WARPS * 32);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                 "r"(T::TMEM_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const int64_t m0 = (int64_t)blockIdx.x * TC_BM;
  const int n0 = blockIdx.y * BN;
  // after an expired wait anywhere in the launch (latched until fdfb_sync),
  // the remaining CTAs skip their work instead of waiting out their budgets
  const bool dead = *reinterpret_cast<volatile int*>(a.err) == FDFB_ETIMEOUT;
  // unit u: digit half u / (S chunks), limb (u / chunks) mod S, chunk u mod chunks
  const int units = dead ? 0 : a.halves * a.S * a.chunks;
  const int total = units * a.ksteps;

  if (warp == 0) {
    if (lane == 0) {
      // loads of iteration i (unit i / ksteps, k-step i % ksteps) into stage i % STAGES
      auto load = [&](int i) {
        const int st = i % TC_STAGES, unit = i / a.ksteps, kk = i - unit * a.ksteps;
        const int hs = unit / a.chunks, c = unit - hs * a.chunks;  // hs = half * S + limb
        const int half = hs / a.S, s = hs - half * a.S;
        const int kx = (c * a.ksteps + kk) * TC_BK;
        const uint32_t sa = sbase + (uint32_t)st * T::STAGE;
        mbar_expect_tx(full(st), T::STAGE);
        tma_3d(sa, &tmA, kx, (int)m0, half, full(st));
        tma_3d(sa + TC_A_BYTES, &tmB, kx, n0, s, full(st));
      };
      const int pre = total < TC_STAGES ? total : TC_STAGES;
      for (int i = 0; i < pre; ++i) load(i);
      int issued = pre;  // loads issued so far
      int consumed = 0;  // loads whose MMAs were issued
      bool ok = true;
      for (int it = 0; it < total && ok; ++it) {
        const int st = it % TC_STAGES, unit = it / a.ksteps, kk = it - unit * a.ksteps, buf = unit & 1;
        if (kk == 0 && unit >= 2) ok = mbar_wait(accempty(buf), ((unit >> 1) - 1) & 1, abort_flag);
        if (ok) ok = mbar_wait(full(st), (it / TC_STAGES) & 1, abort_flag);
        if (!ok) break;
        tc_fence_after();
        const uint32_t sa = sbase + (uint32_t)st * T::STAGE, sb = sa + TC_A_BYTES;
        const uint32_t d = tmem + (uint32_t)buf * BN;
#pragma unroll
        for (int j = 0; j < TC_BK / 16; ++j)
          mma_f16(d, sw128_desc(sa + 32u * j), sw128_desc(sb + 32u * j), T::IDESC, (kk | j) != 0);
        mma_commit(empty(st));
        if (kk == a.ksteps - 1) mma_commit(accfull(buf));
        consumed = it + 1;
        // refill the stage the previous iteration read, once its MMAs are done
        if (it >= 1 && issued < total) {
          const int pst = (it - 1) % TC_STAGES;
          ok = mbar_wait(empty(pst), ((it - 1) / TC_STAGES) & 1, abort_flag);
          if (ok) {
            load(issued);
            ++issued;
          }
        }
      }
      if (!ok) {
        atomicExch(a.err, FDFB_ETIMEOUT);
        *abort_flag = 1;
        // bounded wait for the copies still in flight into the ring
        for (int i = consumed; i < issued; ++i) mbar_wait(full(i % TC_STAGES), (i / TC_STAGES) & 1, abort_flag);
      }
    }
  } else {
    constexpr int CPW = T::CPW, NLD = CPW / 32;
    const int q = warp & 3;                // tensor-memory lane quarter of this warp
    const int half = (warp - 1) >> 2;      // columns [CPW half, CPW half + CPW) of the tile
    const int64_t row = m0 + 32 * q + lane;
    using Sum = typename std::conditional<EXACT, unsigned __int128, uint64_t>::type;
    Sum sum[CPW];
#pragma unroll
    for (int j = 0; j < CPW; ++j) sum[j] = 0;
    bool ok = true;
    for (int u = 0; u < units; ++u) {
      const int buf = u & 1, hs = u / a.chunks;
      const int dh = hs / a.S, s = hs - dh * a.S;
      ok = mbar_wait(accfull(buf), (u >> 1) & 1, abort_flag);
      if (!ok) break;
      tc_fence_after();
      uint32_t r[NLD][32];
      const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)buf * BN + (uint32_t)half * CPW;
#pragma unroll
      for (int l = 0; l < NLD; ++l) tmem_ld32(ta + 32 * l, r[l]);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      tc_fence_before();
      mbar_arrive(accempty(buf));
      const int sh = a.b * s + a.h * dh;
#pragma unroll
      for (int l = 0; l < NLD; ++l)
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int v = __float2int_rn(__uint_as_float(r[l][j]));
          if constexpr (EXACT) sum[32 * l + j] += (unsigned __int128)(__int128)v << sh;
          else sum[32 * l + j] += (uint64_t)(int64_t)v << sh;
        }
    }
    if (!ok) {
      atomicExch(a.err, FDFB_ETIMEOUT);
      *abort_flag = 1;
    } else if (row < a.batch && !dead) {
      const int c0 = n0 + half * CPW;
      if constexpr (EXACT) {
        uint64_t* out = reinterpret_cast<uint64_t*>(a.out) + row * 2 * a.cols;
#pragma unroll
        for (int j = 0; j < CPW; ++j) {
          const int c = c0 + j;
          if (c < a.cols) {
            out[c] = (uint64_t)sum[j] & 0xffffffffull;
            out[a.cols + c] = (uint64_t)(sum[j] >> 32);
          }
        }
      } else {
        const W* ct = reinterpret_cast<const W*>(a.ct);
        W* out = reinterpret_cast<W*>(a.out) + row * a.cols;
#pragma unroll
        for (int j = 0; j < CPW; ++j) {
          const int c = c0 + j;
          if (c < a.cols) {
            W v = (W)(0 - (W)sum[j]);
            if (c == 0) v = (W)(v + ct[row * (a.n_in + 1)]);
            out[c] = v;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(T::TMEM_COLS) : "memory");
}

// Digit matrix of the key switch: A[m][i l + j] = digit j (least significant
// first) of the rounded mask word a_{m,i}, as f16 (exact below 2^11).  With
// two halves, A[0] holds the digit's low h bits and A[1] the rest.
template <typename W>
__global__ void tc_digits_kernel(const W* __restrict__ ct, int64_t batch, int n_in, int ell, int log2B,
                                 int rtrunc, int halves, int h, __half* __restrict__ A) {
  const int64_t K = (int64_t)n_in * ell;
  const uint32_t mask = (1u << log2B) - 1;
  const W half_rt = rtrunc ? ((W)1 << (rtrunc - 1)) : (W)0;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < batch * n_in;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = idx / n_in;
    const int i = (int)(idx - m * n_in);
    const W x = ct[m * (n_in + 1) + 1 + i];
    const W xt = rtrunc ? (W)((W)(x + half_rt) >> rtrunc) : x;
    __half* dst = A + m * K + (int64_t)i * ell;
    if (halves == 1) {
      for (int j = 0; j < ell; ++j) dst[j] = __uint2half_rn((uint32_t)(xt >> (j * log2B)) & mask);
    } else {
      const uint32_t lmask = (1u << h) - 1;
      __half* dst_hi = dst + batch * K;
      for (int j = 0; j < ell; ++j) {
        const uint32_t d = (uint32_t)(xt >> (j * log2B)) & mask;
        dst[j] = __uint2half_rn(d & lmask);
        dst_hi[j] = __uint2half_rn(d >> h);
      }
    }
  }
}

// Key limbs, transposed: out[s][c][k] = limb s of key[k][c], balanced
// base-2^b digits of the word mod 2^w (a limb of at least 2^(b-1) becomes
// limb - 2^b with a carry into the next; the carry out of the top limb is a
// multiple of 2^w).  32 x 32 tiles through shared memory.
template <typename W>
__global__ void tc_limbs_kernel(const W* __restrict__ key, int K, int cols, int S, int b, __half* __restrict__ out) {
  __shared__ W tile[32][33];
  const int k0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int k = k0 + r, c = c0 + threadIdx.x;
    tile[r][threadIdx.x] = (k < K && c < cols) ? key[(size_t)k * cols + c] : (W)0;
  }
  __syncthreads();
  const uint32_t lmask = (1u << b) - 1, halfb = 1u << (b - 1);
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int c = c0 + r, k = k0 + threadIdx.x;
    if (c >= cols || k >= K) continue;
    const W x = tile[threadIdx.x][r];
    uint32_t carry = 0;
    for (int s = 0; s < S; ++s) {
      const int sh = b * s;
      const uint32_t v = (sh < (int)(8 * sizeof(W)) ? (uint32_t)(x >> sh) & lmask : 0u) + carry;
      carry = v >= halfb ? 1u : 0u;
      const int limb = (int)v - (int)(carry << b);
      out[((size_t)s * cols + c) * K + k] = __int2half_rn(limb);
    }
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

int cuda_rc(cudaError_t e) {
  if (e == cudaSuccess) return FDFB_OK;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? FDFB_ENOMEM : FDFB_ECUDA;
}

}  // namespace

bool tc_ks_split(int dbits, int span, int n_in, int ell, int* b, int* S, int* kappa) {
  if (dbits < 1 || dbits > 11 || n_in < 64 || (n_in & (n_in - 1)) || ell < 1) return false;
  const double Bm1 = (double)((1u << dbits) - 1);
  double best = 1e300;
  bool found = false;
  for (int bb = 2; bb <= 12; ++bb) {
    // every partial sum of a chunk: at most kappa (2^dbits - 1) 2^(b-1) <= 2^23
    const double kmax = 8388608.0 / (Bm1 * (double)(1u << (bb - 1)));
    if (kmax < 64) continue;
    int kap = 64;
    while ((double)kap * 2 <= kmax && kap * 2 <= n_in) kap *= 2;  // divides K = n_in ell
    const int SS = (span + bb - 1) / bb;
    const double cost = SS * (1.0 + 128.0 / kap);  // MMA work plus one drain per chunk
    if (cost < best) {
      best = cost;
      *b = bb;
      *S = SS;
      *kappa = kap;
      found = true;
    }
  }
  return found;
}

void tc_ks_release(TcKsKey& k) {
  if (k.limbs) cudaFree(k.limbs);
  k.limbs = nullptr;
  k.bytes = 0;
  k.ready = false;
}

namespace {
template <typename W, int BN, bool EXACT>
cudaError_t tc_set_smem() {
  return cudaFuncSetAttribute(tc_ks_kernel<W, BN, EXACT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)TcTile<BN>::SMEM);
}
}  // namespace

int tc_ks_prepare(TcKsKey& k, const void* key, int w, int n_in, int ell, int log2B, int cols, cudaStream_t s,
                  bool exact) {
  k.ready = false;
  int b = 0, S = 0, kappa = 0;
  EncodeTiledFn enc = encode_fn();
  if (!enc || (w != 32 && w != 64) || (exact && w != 64)) return FDFB_EINVAL;
  // exact form: digits above 11 bits in two halves; limbs over 65 bits, so
  // that a word below 2^63 is their sum as an integer (the balanced top limb
  // then never carries out)
  const int halves = (exact && log2B > 11) ? 2 : 1;
  const int h = halves == 2 ? (log2B + 1) / 2 : 0;
  const int dbits = halves == 2 ? h : log2B;
  if (log2B > 22 || !tc_ks_split(dbits, exact ? 65 : w, n_in, ell, &b, &S, &kappa)) return FDFB_EINVAL;
  const int BN = exact ? 64 : 128;
  const int K = n_in * ell;
  const size_t bytes = (size_t)S * cols * K * 2;
  if (k.bytes < bytes) {
    tc_ks_release(k);
    if (cudaMalloc(&k.limbs, bytes) != cudaSuccess) {
      cudaGetLastError();
      k.limbs = nullptr;
      return FDFB_ENOMEM;
    }
    k.bytes = bytes;
  }
  dim3 grid((unsigned)((K + 31) / 32), (unsigned)((cols + 31) / 32)), block(32, 8);
  if (w == 32)
    tc_limbs_kernel<uint32_t><<<grid, block, 0, s>>>((const uint32_t*)key, K, cols, S, b, (__half*)k.limbs);
  else
    tc_limbs_kernel<uint64_t><<<grid, block, 0, s>>>((const uint64_t*)key, K, cols, S, b, (__half*)k.limbs);
  int rc = cuda_rc(cudaGetLastError());
  if (rc != FDFB_OK) return rc;
  rc = cuda_rc(cudaStreamSynchronize(s));
  if (rc != FDFB_OK) return rc;
  const cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)cols, (cuuint64_t)S};
  const cuuint64_t strides[2] = {(cuuint64_t)K * 2, (cuuint64_t)K * cols * 2};
  const cuuint32_t box[3] = {TC_BK, (cuuint32_t)BN, 1}, estr[3] = {1, 1, 1};
  if (enc(&k.tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, k.limbs, dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return FDFB_ECUDA;
  if (tc_set_smem<uint32_t, 128, false>() != cudaSuccess || tc_set_smem<uint64_t, 128, false>() != cudaSuccess ||
      tc_set_smem<uint64_t, 64, true>() != cudaSuccess) {
    cudaGetLastError();
    return FDFB_ECUDA;
  }
  k.S = S;
  k.b = b;
  k.kappa = kappa;
  k.K = K;
  k.cols = cols;
  k.w = w;
  k.ell = ell;
  k.log2B = log2B;
  k.n_in = n_in;
  k.exact = exact;
  k.halves = halves;
  k.h = h;
  k.ready = true;
  return FDFB_OK;
}

size_t tc_ks_digits_bytes(const TcKsKey& k, int64_t batch) { return (size_t)k.halves * batch * k.K * 2; }

int tc_keyswitch(const TcKsKey& k, const void* ct, int64_t batch, int rtrunc, void* out, void* digits, int* err,
                 cudaStream_t s) {
  if (!k.ready || !digits) return FDFB_EINVAL;
  if (batch <= 0) return FDFB_OK;
  const int64_t work = batch * k.n_in;
  const unsigned blocks = (unsigned)std::min<int64_t>((work + 255) / 256, 4096);
  if (k.w == 32)
    tc_digits_kernel<uint32_t><<<blocks, 256, 0, s>>>((const uint32_t*)ct, batch, k.n_in, k.ell, k.log2B, rtrunc,
                                                      k.halves, k.h, (__half*)digits);
  else
    tc_digits_kernel<uint64_t><<<blocks, 256, 0, s>>>((const uint64_t*)ct, batch, k.n_in, k.ell, k.log2B, rtrunc,
                                                      k.halves, k.h, (__half*)digits);
  int rc = cuda_rc(cudaGetLastError());
  if (rc != FDFB_OK) return rc;
  CUtensorMap tmA;
  const cuuint64_t dims[3] = {(cuuint64_t)k.K, (cuuint64_t)batch, (cuuint64_t)k.halves};
  const cuuint64_t strides[2] = {(cuuint64_t)k.K * 2, (cuuint64_t)batch * k.K * 2};
  const cuuint32_t box[3] = {TC_BK, TC_BM, 1}, estr[3] = {1, 1, 1};
  if (encode_fn()(&tmA, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, digits, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return FDFB_ECUDA;
  TcArgs a;
  a.ct = ct;
  a.out = out;
  a.err = err;
  a.batch = batch;
  a.n_in = k.n_in;
  a.cols = k.cols;
  a.S = k.S;
  a.b = k.b;
  a.chunks = k.K / k.kappa;
  a.ksteps = k.kappa / TC_BK;
  a.halves = k.halves;
  a.h = k.h;
  const int BN = k.exact ? 64 : 128;
  dim3 grid((unsigned)((batch + TC_BM - 1) / TC_BM), (unsigned)((k.cols + BN - 1) / BN));
  if (k.exact)
    tc_ks_kernel<uint64_t, 64, true><<<grid, TC_THREADS, TcTile<64>::SMEM, s>>>(tmA, k.tmap, a);
  else if (k.w == 32)
    tc_ks_kernel<uint32_t, 128, false><<<grid, TC_THREADS, TcTile<128>::SMEM, s>>>(tmA, k.tmap, a);
  else
    tc_ks_kernel<uint64_t, 128, false><<<grid, TC_THREADS, TcTile<128>::SMEM, s>>>(tmA, k.tmap, a);
  return cuda_rc(cudaGetLastError());
}

}  // namespace fdfb
