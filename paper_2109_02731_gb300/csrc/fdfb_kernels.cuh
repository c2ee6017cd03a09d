// Device kernels of the FDFB pipeline (templated on the ring degree 2^L, the
// registers per thread 2^EL, the prime count P and the word type W).
#pragma once
#include <stdint.h>

#include <type_traits>

#include "fdfb_core.cuh"

namespace fdfb {

template <typename W> struct Word;
template <> struct Word<uint32_t> { static constexpr int bits = 32; };
template <> struct Word<uint64_t> { static constexpr int bits = 64; };

// 128-bit read-only load that does not allocate in L1: the key rows stream
// through once per ciphertext and step, and must not evict the twiddles.
__device__ __forceinline__ uint4 ldg_stream(const uint4* p) {
  uint4 v;
  asm("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(p));
  return v;
}

// Asks the bulk-copy engine to bring `bytes` (a multiple of 16, 16-byte
// aligned) into L2; no completion to wait for.
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) from
// global to shared memory by the copy engine, completing on an mbarrier.
__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(mbar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// orders this thread's earlier generic-proxy accesses of shared memory before
// its later bulk copies into it
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  const uint32_t m = (uint32_t)__cvta_generic_to_shared(mbar);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(m), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(d), "l"(src), "r"(bytes), "r"(m) : "memory");
}
// Waits for phase `parity` of the mbarrier to complete, giving up after
// `limit` polls (the caller latches FDFB_ETIMEOUT): returns whether it completed.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, uint32_t limit) {
  const uint32_t m = (uint32_t)__cvta_generic_to_shared(mbar);
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}" : "=r"(done) : "r"(m), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void named_bar(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Synchronises the G threads of one transform: a warp barrier when the group
// is one warp, else the group's named barrier.
template <int G>
__device__ __forceinline__ void group_sync(int bar) {
  if constexpr (G == 32) {
    __syncwarp();
  } else {
    named_bar(bar, G);
  }
}

// Moves the E registers of every thread of a group from the layout of pass
// FROM to the layout of pass TO through the group's exchange buffer.
template <int L, int EL, int FROM, int TO>
__device__ __forceinline__ void exchange(uint32_t (&v)[1 << EL], int t, uint32_t* xb, int bar) {
  using Y = Layout<L, EL>;
  using X = Xch<L, EL>;
  const uint32_t wb = X::addr(Y::j_of(FROM, t, 0));
#pragma unroll
  for (int r = 0; r < Y::E; ++r) xb[X::join(wb, X::addr(Y::j_of(FROM, 0, r)))] = v[r];
  group_sync<Y::G>(bar);
  const uint32_t rb = X::addr(Y::j_of(TO, t, 0));
#pragma unroll
  for (int r = 0; r < Y::E; ++r) v[r] = xb[X::join(rb, X::addr(Y::j_of(TO, 0, r)))];
  group_sync<Y::G>(bar);
}

// Exchange / transforms of M polynomials at once.  M = 1: one buffer of XW
// words.  M = 2: the two words of a position travel as one 64-bit word
// (Xch64), in a buffer of XW 64-bit entries; with PP the exchanges between
// passes 0 and 1 and between passes 1 and 2 use two such buffers, so a
// buffer is rewritten only after the other buffer's exchange has synchronised
// the group, and the barrier that protects the reads can be dropped.  That
// needs three passes per transform and a block-wide barrier between the last
// forward and the first inverse exchange and between the last inverse and the
// next forward exchange (the blind rotation has both).
template <int L, int EL, int FROM, int TO, int M, int XW, bool PP = false>
__device__ __forceinline__ void exchange_m(uint32_t (&v)[M][1 << EL], int t, uint32_t* xb, int bar) {
  using Y = Layout<L, EL>;
  if constexpr (M == 2) {
    static_assert(!PP || Y::K == 3, "ping-pong exchange buffers need three passes");
    using X = Xch64<L, EL>;
    uint2* b = reinterpret_cast<uint2*>(xb) + (PP ? ((FROM < TO ? FROM : TO) & 1) * XW : 0);
    const uint32_t wb = X::addr(Y::j_of(FROM, t, 0));
#pragma unroll
    for (int r = 0; r < Y::E; ++r) b[X::join(wb, X::addr(Y::j_of(FROM, 0, r)))] = make_uint2(v[0][r], v[1][r]);
    group_sync<Y::G>(bar);
    const uint32_t rb = X::addr(Y::j_of(TO, t, 0));
#pragma unroll
    for (int r = 0; r < Y::E; ++r) {
      const uint2 x = b[X::join(rb, X::addr(Y::j_of(TO, 0, r)))];
      v[0][r] = x.x;
      v[1][r] = x.y;
    }
    if constexpr (!PP) group_sync<Y::G>(bar);
  } else {
    using X = Xch<L, EL>;
    const uint32_t wb = X::addr(Y::j_of(FROM, t, 0));
#pragma unroll
    for (int r = 0; r < Y::E; ++r) {
      const uint32_t a = X::join(wb, X::addr(Y::j_of(FROM, 0, r)));
#pragma unroll
      for (int m = 0; m < M; ++m) xb[m * XW + a] = v[m][r];
    }
    group_sync<Y::G>(bar);
    const uint32_t rb = X::addr(Y::j_of(TO, t, 0));
#pragma unroll
    for (int r = 0; r < Y::E; ++r) {
      const uint32_t a = X::join(rb, X::addr(Y::j_of(TO, 0, r)));
#pragma unroll
      for (int m = 0; m < M; ++m) v[m][r] = xb[m * XW + a];
    }
    group_sync<Y::G>(bar);
  }
}

template <int L, int EL, int PASS, int M, int XW, bool LZ = false, bool PP = false>
__device__ __forceinline__ void ntt_fwd_m(uint32_t (&v)[M][1 << EL], int t, const uint2* tw, uint32_t p,
                                          uint32_t* xb, int bar, uint32_t z) {
  using Y = Layout<L, EL>;
  if constexpr (PASS < Y::K) {
    if constexpr (PASS > 0) exchange_m<L, EL, PASS - 1, PASS, M, XW, PP>(v, t, xb, bar);
    fwd_pass_m<L, EL, PASS, M, LZ>(v, t, tw, p, z);
    ntt_fwd_m<L, EL, PASS + 1, M, XW, LZ, PP>(v, t, tw, p, xb, bar, z);
  }
}

template <int L, int EL, int PASS, int M, int XW, bool PP = false>
__device__ __forceinline__ void ntt_inv_m(uint32_t (&v)[M][1 << EL], int t, const uint2* tw, uint32_t p,
                                          uint32_t* xb, int bar, uint32_t z) {
  if constexpr (PASS >= 0) {
    inv_pass_m<L, EL, PASS, M>(v, t, tw, p, z);
    if constexpr (PASS > 0) exchange_m<L, EL, PASS, PASS - 1, M, XW, PP>(v, t, xb, bar);
    ntt_inv_m<L, EL, PASS - 1, M, XW, PP>(v, t, tw, p, xb, bar, z);
  }
}

// Forward negacyclic NTT of one polynomial by one thread group: v holds the
// pass-0 layout (natural order) on entry and the last-pass layout
// (bit-reversed order, values in [0, 4p)) on exit.  xb is the group's
// exchange buffer (Xch::kWords words), bar its named barrier.
template <int L, int EL, int PASS>
__device__ __forceinline__ void ntt_fwd(uint32_t (&v)[1 << EL], int t, const uint2* tw, uint32_t p,
                                        uint32_t* xb, int bar, uint32_t z) {
  using Y = Layout<L, EL>;
  if constexpr (PASS < Y::K) {
    if constexpr (PASS > 0) exchange<L, EL, PASS - 1, PASS>(v, t, xb, bar);
    fwd_pass<L, EL, PASS>(v, t, tw, p, z);
    ntt_fwd<L, EL, PASS + 1>(v, t, tw, p, xb, bar, z);
  }
}

// Inverse transform: last-pass layout, values in [0, 2p) -> pass-0 layout
// (natural order), values in [0, 2p).  The 1/N factor is not applied.
template <int L, int EL, int PASS>
__device__ __forceinline__ void ntt_inv(uint32_t (&v)[1 << EL], int t, const uint2* tw, uint32_t p,
                                        uint32_t* xb, int bar, uint32_t z) {
  if constexpr (PASS >= 0) {
    inv_pass<L, EL, PASS>(v, t, tw, p, z);
    if constexpr (PASS > 0) exchange<L, EL, PASS, PASS - 1>(v, t, xb, bar);
    ntt_inv<L, EL, PASS - 1>(v, t, tw, p, xb, bar, z);
  }
}

// Coefficient j of poly * X^k (k in [0, 2N)): reads poly[j - k] with the sign
// of the wrap (X^N = -1).  get(m) returns coefficient m.
template <int L>
__device__ __forceinline__ int rot_src(int j, int k, bool& neg) {
  constexpr int N = 1 << L;
  int m = j - k;
  neg = false;
  if (m < 0) { m += N; neg = true; }
  if (m < 0) { m += N; neg = false; }
  return m;
}

// ModSwitch q = 2^w -> 2N = 2^(L+1), round half up (appendix figure
// "Modulus switching algorithm").
template <typename W, int L>
__device__ __forceinline__ uint32_t modswitch_2n(W x) {
  constexpr int sh = Word<W>::bits - (L + 1);
  return (uint32_t)((W)(x + ((W)1 << (sh - 1))) >> sh);
}

// ---------------------------------------------------------------------------
// Blind rotation (appendix figure "Blind Rotation and its setup", u = {1}):
// one CTA per item (a ciphertext, or an (input, table) pair when rep > 1), P
// thread groups of G threads, group g computing every product modulo prime g.
// For i = 1..n:
//   d = acc * X^{-a_i} - acc;  D = Decomp(d) (2 lg digit polynomials);
//   acc += sum_r D_r * bsk[i][r]    (CMux = extProd(C, g - h) + h)
// The digits are transformed on the fly; the key rows are pre-transformed
// (centred, scaled by N^-1 in Montgomery form) and stored so that thread t's
// E outputs of the transform meet their key words in E/4 128-bit loads that
// are contiguous across the warp.
// ---------------------------------------------------------------------------
struct BRParams {
  PrimeSet S;
  const uint32_t* bsk;    // [n][P][2 lg][2][KH][N]
  const void* ct;         // [batch / rep][n+1] words (input LWE, modulus q)
  const void* acc0;       // function mode: [batch][2N] words; sign mode: nullptr
  void* lwe_out;          // [batch][N+1] words: SampleExtract(acc, 0) (+ Delta/2 in sign mode)
  uint32_t* ctN_out;      // optional [batch][n+1]: ModSwitch(ct, q, 2N) (rep = 1 only)
  int n, lg, log2Bg, rtrunc;
  int64_t batch;
  uint64_t delta_half;
  int sign_mode;
  uint32_t smem_r1, smem_exch;  // byte offsets inside dynamic shared memory
  int rep;                      // items per input ciphertext: item i rotates by ct[i / rep]
  int signed_digits;            // balanced digits: the launcher picks the kernel built with SG
  int* err;                     // device error latch (FDFB_ETIMEOUT if a key copy never lands)
  // test hook (fdfb_test_hooks): TK issues no key copies, so its bounded wait
  // expires with nothing in flight; key_wait_polls bounds that wait (0: 2^20)
  int test_skip_key_copy;
  uint32_t key_wait_polls;
  // prime-modulus sets (the kernel built with MQ): words are residues mod
  // Q, the input LWE words already lie in [0, 2N) (q = 2N), and sign item i
  // starts from (and adds after extraction) sgn_scale[i % rep] instead of
  // delta_half
  ModQ mq;
  uint64_t sgn_scale[8];
  // N = 2^13 (fdfb_n13.cuh): per item global scratch, the residues of the
  // halves' inverse transforms and the accumulator (n13_scratch_words)
  uint32_t* half_y;
};

template <int L, int EL, int P, typename W, typename DT, int M = 1, bool PP = false, int KH = 1,
          bool TK = false, bool MQ = false>
struct BRShape {
  using Y = Layout<L, EL>;
  static constexpr int N = Y::N, E = Y::E, G = Y::G, THREADS = P * G;
  // acc | a_N | (digits, or the staged residues) | exchange buffers
  static size_t smem_bytes(int n, int lg, uint32_t* r1_off, uint32_t* exch_off) {
    size_t acc = 2 * (size_t)N * sizeof(W);
    size_t an = ((size_t)n * 2 + 15) & ~(size_t)15;
    // MQ keeps d itself ([2][N] words) and cuts the digits out as it loads them
    size_t dig = MQ ? 2 * (size_t)N * sizeof(W) : (2 * (size_t)lg * N * sizeof(DT) + 15) & ~(size_t)15;
    size_t stage = (size_t)2 * (P - 1) * KH * N * 4;
    size_t r1 = dig > stage ? dig : stage;
    *r1_off = (uint32_t)(acc + an);
    *exch_off = (uint32_t)(acc + an + r1);
    return acc + an + r1 + (size_t)P * group_words() * 4 + kstage_bytes();
  }
  // TK: per group, the key rows of one pair (2M rows x N words), then one
  // mbarrier per group
  static constexpr size_t kpair_words() { return (size_t)2 * M * KH * N; }
  static constexpr size_t kstage_bytes() { return TK ? (size_t)P * kpair_words() * 4 + (size_t)P * 8 : 0; }
  // 32-bit words of one polynomial's exchange buffer (M = 1)
  static constexpr size_t xwords() { return ((size_t)Xch<L, EL>::kWords + 3) & ~(size_t)3; }
  // 64-bit entries of one paired exchange buffer (M = 2)
  static constexpr size_t x64entries() { return ((size_t)Xch64<L, EL>::kEntries + 1) & ~(size_t)1; }
  // 32-bit words of one group's exchange region
  static constexpr size_t group_words() {
    return (M == 2 || KH == 2) ? (PP ? 2 : 1) * 2 * x64entries() : (size_t)M * xwords();
  }
};

// Resident CTAs per SM the register budget is sized for (512 threads per SM).
constexpr int br_min_blocks(int threads) { return threads >= 512 ? 1 : 512 / threads; }
// Resident CTAs per SM that leave each thread `regs` registers.
constexpr int br_blocks_for_regs(int threads, int regs) {
  return 65536 / (threads * regs) > 0 ? 65536 / (threads * regs) : 1;
}

// Transform-domain sum -> inverse-transform input in [0, 2p).  A 64-bit sum
// of at most 8 products is Montgomery-reduced: with transform values below p
// (< 8 p^2 -> below 3p) it is corrected once; with the lazy family's
// unreduced transform values (below 2^32: < 2^35 p -> below 9p) it is
// brought into [0, 2p) by Shoup's product by 1.  R14: up to 14 products (the
// exact decompositions of the prime-modulus sets, l <= 7): < 14 p^2 < 2^63.8
// reduces below 4.5p and is corrected twice.
template <bool WIDE, bool LZ, typename Acc, bool R14 = false>
__device__ __forceinline__ uint32_t acc_to_inv(Acc a, uint32_t p, uint32_t pneg, uint32_t ones) {
  if constexpr (WIDE) {
    const uint32_t r = redc((uint64_t)a, p, pneg);
    if constexpr (LZ) {
      return mul_shoup(r, 1u, ones, p);
    } else {
      const uint32_t r1 = umin32(r, r - 2 * p);
      return R14 ? umin32(r1, r1 - 2 * p) : r1;
    }
  } else {
    return (uint32_t)a;
  }
}

// Staging slot of group g's residues of output column c (g != c): the owner
// of column c (group c) reads the other P-1 groups' residues there.
template <int P>
__device__ __forceinline__ int stage_slot(int g, int c) {
  return c * (P - 1) + (g < c ? g : g - 1);
}

// WIDE: sum the pointwise products of all 2l digits in 64 bits and reduce
// once (fewer instructions, twice the accumulator registers); otherwise each
// product is Montgomery-reduced as it is formed.  MINB: resident CTAs per SM
// the register budget is sized for.
// M: polynomials transformed together by one thread group (1 or 2).
// LZ: the prime set is the lazy family; the forward transforms of the digits
// skip all intermediate reductions and their outputs (below 2^32) enter the
// pointwise products unreduced.
// PP: two exchange buffers per group used in turn (M = 2 only), one group
// barrier per exchange instead of two.
// KH = 2 (q = 2^64, two primes): every key word K is split into centred
// 32-bit halves, K = K_lo + 2^32 K_hi; both halves share the digits' forward
// transforms, and each half's product sum (at most 2l N (B-1) 2^31) is lifted
// exactly from two primes: acc += X_lo + 2^32 X_hi mod 2^64.
// SG: balanced digits in [-B/2, B/2) (a parameter set's signed_digits).
// TK: each group's key rows of the next pair (2M rows) are copied into shared
// memory by the bulk-copy engine while the group transforms that pair's
// digits; one thread per group issues the copy, completion is an mbarrier
// phase (bounded wait, FDFB_ETIMEOUT on expiry).
// MQ: prime modulus Q (Table 1): d = acc X^{-a} - acc mod Q, exact digits
// (l log2 B >= log2 Q), the products lifted to the exact integer and reduced
// mod Q; the input ciphertext is already modulo 2N.  With P = 2 and whole
// key words (KH = 1) the lift fits 64 bits (k = 32: |X| < 2^55).
template <int L, int EL, int P, typename W, typename DT, bool WIDE = false,
          int MINB = br_min_blocks(P * (1 << (L - EL))), int M = 1, bool LZ = false, bool PP = false,
          int KH = 1, bool SG = false, bool TK = false, bool MQ = false>
__global__ void __launch_bounds__(P * (1 << (L - EL)), MINB)
blind_rotate_kernel(const BRParams prm) {
  using Y = Layout<L, EL>;
  constexpr int N = Y::N, E = Y::E, G = Y::G, THREADS = P * G;
  static_assert(P >= 2, "the column owners are groups 0 and 1");
  static_assert(!LZ || (L <= 12 && sizeof(DT) <= 2), "lazy bound: 2^16 + 2 L p < 2^32");
  static_assert(KH == 1 || (KH == 2 && P == 2 && !WIDE && sizeof(W) == 8),
                "split keys: q = 2^64, two primes, per-product reduction");
  static_assert(!MQ || (sizeof(W) == 8 && !SG && !LZ), "prime modulus: 64-bit words, unsigned digits");
  extern __shared__ __align__(16) unsigned char smem[];
  W* acc = reinterpret_cast<W*>(smem);                                     // [2][N]
  uint16_t* aN = reinterpret_cast<uint16_t*>(smem + 2 * N * sizeof(W));     // [n]
  DT* dig = reinterpret_cast<DT*>(smem + prm.smem_r1);                      // [2 lg][N]
  W* dq = reinterpret_cast<W*>(smem + prm.smem_r1);                         // MQ: [2][N]
  uint32_t* stage = reinterpret_cast<uint32_t*>(smem + prm.smem_r1);        // [2 (P-1)][N]
  uint32_t* exch = reinterpret_cast<uint32_t*>(smem + prm.smem_exch);       // [P][xwords]

  const int tid = threadIdx.x;
  const int grp = tid / G;
  const int t = tid - grp * G;
  const int64_t ci = blockIdx.x;
  const int n = prm.n, lg = prm.lg, log2Bg = prm.log2Bg;
  const W* ct = reinterpret_cast<const W*>(prm.ct) + (ci / prm.rep) * (n + 1);

  // ModSwitch of the mask; b_N for the sign accumulator.
  const uint64_t Qm = prm.mq.Q;
  for (int i = tid; i < n; i += THREADS) {
    uint32_t a = MQ ? (uint32_t)ct[1 + i] & (2 * N - 1) : modswitch_2n<W, L>(ct[1 + i]);
    aN[i] = (uint16_t)a;
    if (prm.ctN_out) prm.ctN_out[ci * (n + 1) + 1 + i] = a;
  }
  if (prm.sign_mode) {
    const int bN = MQ ? (int)((uint32_t)ct[0] & (2 * N - 1)) : (int)modswitch_2n<W, L>(ct[0]);
    if (prm.ctN_out && tid == 0) prm.ctN_out[ci * (n + 1)] = (uint32_t)bN;
    // acc = [(Delta/2) sgnP X^{b_N}, 0], sgnP = 1 - sum_{i>=2} X^{i-1}
    // (MQ: item i of an input carries L_boot^i Delta/2)
    const W h = MQ ? (W)prm.sgn_scale[ci % prm.rep] : (W)prm.delta_half;
    for (int j = tid; j < N; j += THREADS) {
      bool neg;
      int m = rot_src<L>(j, bN, neg);
      if constexpr (MQ) {
        const W c = (m == 0) ? h : (W)negq(h, Qm);
        acc[j] = neg ? (W)negq(c, Qm) : c;
      } else {
        W c = (m == 0) ? h : (W)(0 - h);
        acc[j] = neg ? (W)(0 - c) : c;
      }
      acc[N + j] = 0;
    }
  } else {
    const W* a0 = reinterpret_cast<const W*>(prm.acc0) + ci * 2 * N;
    for (int j = tid; j < 2 * N; j += THREADS) acc[j] = a0[j];
  }
  // TK: the staged pair of key rows of each group, and its mbarrier
  constexpr uint32_t kPairWords = (uint32_t)(2 * M * KH * N);
  uint32_t* kst = reinterpret_cast<uint32_t*>(
      smem + prm.smem_exch + (size_t)P * BRShape<L, EL, P, W, DT, M, PP, KH, TK, MQ>::group_words() * 4);
  uint64_t* kmb = reinterpret_cast<uint64_t*>(kst + (size_t)P * kPairWords) + (tid / G);
  kst += (size_t)(tid / G) * kPairWords;
  if constexpr (TK) {
    if (tid % G == 0) {
      mbar_init(kmb, 1);
      fence_mbar_init();
    }
  }
  __syncthreads();

  const uint32_t p = prm.S.p[grp];
  const uint32_t pneg = prm.S.pneg[grp];
  const uint32_t ones = prm.S.ones[grp];
  const uint32_t z = prm.S.zero;
  const uint2* twf = prm.S.tw_fwd + (size_t)grp * N;
  const uint2* twi = prm.S.tw_inv + (size_t)grp * N;
  static_assert(!PP || M == 2, "ping-pong buffers are for paired transforms");
  using Sh = BRShape<L, EL, P, W, DT, M, PP, KH, TK, MQ>;
  // forward transforms: M polynomials per pass; inverse transforms: both
  // columns together whenever the forward is paired or the key is split
  constexpr int MI = (M == 2 || KH == 2) ? 2 : 1;
  constexpr int XW = (int)(M == 2 ? Sh::x64entries() : Sh::xwords());
  constexpr int XWI = (int)(MI == 2 ? Sh::x64entries() : Sh::xwords());
  uint32_t* xb = exch + grp * (int)Sh::group_words();
  const int bar = 1 + grp;
  const int rt = prm.rtrunc;
  const W half_rt = rt ? ((W)1 << (rt - 1)) : (W)0;
  const uint32_t dmask = (1u << log2Bg) - 1;
  const uint32_t halfB = 1u << (log2Bg - 1);
  const int R = 2 * lg;

  // Each group's key block of a step is contiguous (R rows x 2 columns x KH
  // halves x N words); one thread per group prefetches the next step's block
  // into L2 while this step computes (the keys of the q = 2^64 sets do not fit
  // in L2).
  const uint32_t kblock = (uint32_t)(R * 2 * KH * N * 4);
  if (t == 0) prefetch_l2_bulk(prm.bsk + (size_t)grp * R * 2 * KH * N, kblock);
  // TK: the first pair's rows; kph is the parity of the staged pair's phase,
  // kfail latches an expired wait (no further copies or waits after it)
  uint32_t kph = 0, kfph = 0;
  bool kfail = false;
  const uint32_t kWaitLimit = prm.key_wait_polls ? prm.key_wait_polls : (1u << 20);
  const bool kcopy = !prm.test_skip_key_copy;
  if constexpr (TK) {
    if (t == 0 && n > 0 && kcopy)
      bulk_copy_g2s(kst, prm.bsk + (size_t)grp * R * 2 * KH * N, kPairWords * 4, kmb);
  }
  for (int i = 0; i < n; ++i) {
    const int a = aN[i];
    if (t == 0 && i + 1 < n) prefetch_l2_bulk(prm.bsk + ((size_t)(i + 1) * P + grp) * R * 2 * KH * N, kblock);
    // d = acc X^{-a} - acc, rounded and split into digits (component major).
    // Coefficient j of acc X^{-a} is acc[(j + a) mod 2N], negated when that
    // index lies in [N, 2N) (X^N = -1).
#pragma unroll 4
    for (int idx = tid; idx < 2 * N; idx += THREADS) {
      const int c = idx >> L, j = idx & (N - 1);
      const int m = (j + a) & (2 * N - 1);
      const W neg = (W)0 - (W)(m >> L);  // all ones when negated
      const W* ac = acc + c * N;
      if constexpr (MQ) {
        const uint64_t v = ac[m & (N - 1)];
        dq[idx] = subq(neg ? negq(v, Qm) : v, ac[j], Qm);
        continue;
      }
      const W rv = (W)((ac[m & (N - 1)] ^ neg) - neg);
      const W d = (W)(rv - ac[j]);
      const W xt = (W)((W)(d + half_rt) >> rt);
      DT* dp = dig + c * lg * N + j;
      if constexpr (SG) {
        // balanced digits: a digit (plus the carry) of at least B/2 becomes
        // digit - B with a carry into the next one; stored as two's complement
        uint32_t carry = 0;
#pragma unroll
        for (int l = 0; l < 4; ++l)  // lg <= 4
          if (l < lg) {
            const uint32_t dv = ((uint32_t)(xt >> (l * log2Bg)) & dmask) + carry;
            carry = dv >= halfB ? 1u : 0u;
            dp[l * N] = (DT)(dv - (carry << log2Bg));
          }
      } else {
#pragma unroll
        for (int l = 0; l < 4; ++l)  // lg <= 4
          if (l < lg) dp[l * N] = (DT)((uint32_t)(xt >> (l * log2Bg)) & dmask);
      }
    }
    __syncthreads();

    // Pointwise products summed in the transform domain: each product is
    // Montgomery-reduced to [0, 2p) as it is formed (the key word carries the
    // factor 2^32 N^-1), and the running sum is kept in [0, 2p).
    // Group 0 accumulates column 1 in macc[0] and column 0 in macc[1], the
    // other groups column c in macc[c]: the column a group lifts (its own
    // index, for groups 0 and 1) always ends up in macc[1].
    using Acc = typename std::conditional<WIDE, uint64_t, uint32_t>::type;
    Acc macc[KH][2][E];
#pragma unroll
    for (int h = 0; h < KH; ++h)
#pragma unroll
      for (int k = 0; k < E; ++k) { macc[h][0][k] = 0; macc[h][1][k] = 0; }
    const int swap = (grp == 0) ? 1 : 0;
    const uint32_t* krow = prm.bsk + ((size_t)i * P + grp) * R * 2 * KH * N;
    for (int r0 = 0; r0 < R; r0 += M) {
      uint32_t v[M][E];
#pragma unroll
      for (int m = 0; m < M; ++m)
#pragma unroll
        for (int k = 0; k < E; ++k) {
          uint32_t dv;
          if constexpr (MQ) {
            // row r = c lg + l: digit l of component c of d
            const int r = r0 + m, cc = r >= lg ? 1 : 0, l = r - cc * lg;
            dv = (uint32_t)(dq[cc * N + Y::j_of(0, t, k)] >> (l * log2Bg)) & dmask;
          } else {
            dv = dig[(r0 + m) * N + Y::j_of(0, t, k)];
          }
          if constexpr (SG) {
            // a negative balanced digit enters the transform as d + p
            using SDT = typename std::make_signed<DT>::type;
            const int sd = (int)(SDT)dv;
            v[m][k] = sd < 0 ? (uint32_t)(sd + (int)p) : (uint32_t)sd;
          } else {
            v[m][k] = dv;
          }
        }
      ntt_fwd_m<L, EL, 0, M, XW, LZ, PP>(v, t, twf, p, xb, bar, z);
      if constexpr (WIDE && !LZ) {
#pragma unroll
        for (int m = 0; m < M; ++m)
#pragma unroll
          for (int k = 0; k < E; ++k) v[m][k] = csub(csub(v[m][k], 2 * p), p);
      }
      if constexpr (TK) {
        if (!kfail && !mbar_wait(kmb, kph, kWaitLimit)) {
          kfail = true;
          kfph = kph;
          if (prm.err) atomicExch(prm.err, -4);  // FDFB_ETIMEOUT
        }
        kph ^= 1u;
      }
#pragma unroll
      for (int c = 0; c < 2; ++c) {
#pragma unroll
        for (int h = 0; h < KH; ++h) {
#pragma unroll
          for (int m = 0; m < M; ++m) {
            const uint4* kp =
                TK ? reinterpret_cast<const uint4*>(kst + (((size_t)m * 2 + (c ^ swap)) * KH + h) * N) + t
                   : reinterpret_cast<const uint4*>(krow + (((size_t)(r0 + m) * 2 + (c ^ swap)) * KH + h) * N) + t;
#pragma unroll
            for (int q4 = 0; q4 < E / 4; ++q4) {
              const uint4 kk = TK ? kp[q4 * G] : ldg_stream(kp + q4 * G);
              const uint32_t kv[4] = {kk.x, kk.y, kk.z, kk.w};
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                if constexpr (WIDE) {
                  // K < p, and v < p (or, lazy family, v < 2^32 and p < 2^28):
                  // 2l <= 8 products stay below 2^63
                  macc[h][c][q4 * 4 + u] += (uint64_t)v[m][q4 * 4 + u] * kv[u];
                } else {
                  const uint32_t mm = redc((uint64_t)v[m][q4 * 4 + u] * kv[u], p, pneg);  // < 2p
                  uint32_t s2 = (uint32_t)macc[h][c][q4 * 4 + u] + mm + z;
                  macc[h][c][q4 * 4 + u] = umin32(s2, s2 - 2 * p + z);
                }
              }
            }
          }
        }
      }
      if constexpr (TK) {
        // the group is done with the staged rows: stage the next pair (this
        // step's, else the next step's first)
        named_bar(bar, G);
        if (t == 0 && !kfail && kcopy) {
          const bool more = r0 + M < R;
          if (more || i + 1 < n) {
            const uint32_t* src = more ? krow + (size_t)(r0 + M) * 2 * KH * N
                                       : prm.bsk + ((size_t)(i + 1) * P + grp) * R * 2 * KH * N;
            fence_proxy_async_smem();
            bulk_copy_g2s(kst, src, kPairWords * 4, kmb);
          }
        }
      }
    }
    __syncthreads();  // every group is done with the digits: the region becomes `stage`

    // Inverse transforms.  Column c is lifted by group c, which keeps its own
    // residues in registers; every other group stages its residues for it.
    // (staging slot s of key half h at stage + (s KH + h) N)
    uint32_t own[KH][E];
    if constexpr (MI == 2) {
#pragma unroll
      for (int h = 0; h < KH; ++h) {
        uint32_t v[2][E];
#pragma unroll
        for (int k = 0; k < E; ++k) {
          v[0][k] = acc_to_inv<WIDE, LZ, Acc, MQ>(macc[h][0][k], p, pneg, ones);
          v[1][k] = acc_to_inv<WIDE, LZ, Acc, MQ>(macc[h][1][k], p, pneg, ones);
        }
        ntt_inv_m<L, EL, Y::K - 1, 2, XWI, PP>(v, t, twi, p, xb, bar, z);
        uint32_t* dst0 = stage + (stage_slot<P>(grp, swap) * KH + h) * N;
#pragma unroll
        for (int k = 0; k < E; ++k) dst0[Y::j_of(0, t, k)] = csub(v[0][k], p);
        if (grp < 2) {
#pragma unroll
          for (int k = 0; k < E; ++k) own[h][k] = csub(v[1][k], p);
        } else {
          uint32_t* dst1 = stage + (stage_slot<P>(grp, 1) * KH + h) * N;
#pragma unroll
          for (int k = 0; k < E; ++k) dst1[Y::j_of(0, t, k)] = csub(v[1][k], p);
        }
      }
    } else {
      {
        uint32_t v[E];
#pragma unroll
        for (int k = 0; k < E; ++k) v[k] = acc_to_inv<WIDE, LZ, Acc, MQ>(macc[0][0][k], p, pneg, ones);
        ntt_inv<L, EL, Y::K - 1>(v, t, twi, p, xb, bar, z);
        uint32_t* dst = stage + stage_slot<P>(grp, swap) * N;
#pragma unroll
        for (int k = 0; k < E; ++k) dst[Y::j_of(0, t, k)] = csub(v[k], p);
      }
      {
        uint32_t v[E];
#pragma unroll
        for (int k = 0; k < E; ++k) v[k] = acc_to_inv<WIDE, LZ, Acc, MQ>(macc[0][1][k], p, pneg, ones);
        ntt_inv<L, EL, Y::K - 1>(v, t, twi, p, xb, bar, z);
        if (grp < 2) {
#pragma unroll
          for (int k = 0; k < E; ++k) own[0][k] = csub(v[k], p);
        } else {
          uint32_t* dst = stage + stage_slot<P>(grp, 1) * N;
#pragma unroll
          for (int k = 0; k < E; ++k) dst[Y::j_of(0, t, k)] = csub(v[k], p);
        }
      }
    }
    __syncthreads();
    if (grp < 2) {
      const int c = grp;
#pragma unroll
      for (int k = 0; k < E; ++k) {
        const int j = Y::j_of(0, t, k);
        if constexpr (MQ) {
          // the exact sum (one lift over P primes, or X_lo + 2^32 X_hi) mod Q
          __int128 X = 0;
#pragma unroll
          for (int h = 0; h < KH; ++h) {
            uint32_t x[P];
#pragma unroll
            for (int g = 0; g < P; ++g)
              x[g] = (g == c) ? own[h][k] : stage[(stage_slot<P>(g, c) * KH + h) * N + j];
            const __int128 Xh = garner_exact<P>(x, prm.S);
            X += h == 0 ? Xh : Xh * ((__int128)1 << 32);
          }
          // two primes, whole key words: registration admits this layout only
          // where the sum lifts exactly from two primes, |X| < 2^59, so the
          // 64-bit reduction serves (k = 32, Q_4)
          const uint64_t r = (P == 2 && KH == 1) ? modq_lift64((int64_t)X, prm.mq) : modq_lift(X, prm.mq);
          acc[c * N + j] = (W)addq(acc[c * N + j], r, Qm);
          continue;
        }
        W add = 0;
#pragma unroll
        for (int h = 0; h < KH; ++h) {
          uint32_t x[P];
#pragma unroll
          for (int g = 0; g < P; ++g)
            x[g] = (g == c) ? own[h][k] : stage[(stage_slot<P>(g, c) * KH + h) * N + j];
          const W X = (W)garner_p<P>(x, prm.S);
          add = (W)(add + (h == 0 ? X : (W)((uint64_t)X << 32)));
        }
        acc[c * N + j] = (W)(acc[c * N + j] + add);
      }
    }
    __syncthreads();
  }

  if constexpr (TK) {
    // an expired wait leaves at most the copy it waited for in flight: give it
    // a bounded chance to land before the CTA's shared memory is released
    if (kfail && t == 0) mbar_wait(kmb, kfph, kWaitLimit);
  }

  // SampleExtract of coefficient 0 (appendix figure "Sample and key
  // extraction", NSgn(x) = 1 iff x > 0): b' = b_0, a'_0 = a_0, a'_k = -a_{N-k}.
  W* out = reinterpret_cast<W*>(prm.lwe_out) + ci * (N + 1);
  for (int k = tid; k <= N; k += THREADS) {
    W v;
    if constexpr (MQ) {
      if (k == 0) v = (W)addq(acc[0], prm.sign_mode ? prm.sgn_scale[ci % prm.rep] : 0, Qm);
      else if (k == 1) v = acc[N];
      else v = (W)negq(acc[N + (N - (k - 1))], Qm);
    } else {
      if (k == 0) v = (W)(acc[0] + (prm.sign_mode ? (W)prm.delta_half : (W)0));
      else if (k == 1) v = acc[N];
      else v = (W)(0 - acc[N + (N - (k - 1))]);
    }
    out[k] = v;
  }
}

// ---------------------------------------------------------------------------
// Exact product of a small unsigned polynomial (coefficients < 2^16) with one
// or two word polynomials, all modulo X^N + 1 and 2^w, plus an addend.  Used
// by PubMux (BuildAcc, figure "cmux-accumulator-builder") and by RLWE
// encryption during key generation.  One CTA per item, P groups.
// ---------------------------------------------------------------------------
template <int L, int EL, int P, typename W, typename SmallF, typename WordF, typename OutF>
__device__ __forceinline__ void small_word_product(const PrimeSet& S, int ncols, SmallF small,
                                                   WordF word, OutF out, unsigned char* smem) {
  using Y = Layout<L, EL>;
  constexpr int N = Y::N, E = Y::E, G = Y::G, THREADS = P * G;
  constexpr int XW = (Xch<L, EL>::kWords + 3) & ~3;
  uint32_t* stage = reinterpret_cast<uint32_t*>(smem);          // [P][2][N]
  uint32_t* exch = stage + P * 2 * N;                           // [P][XW]
  const int tid = threadIdx.x;
  const int grp = tid / G;
  const int t = tid - grp * G;
  const uint32_t p = S.p[grp];
  const uint32_t pneg = S.pneg[grp];
  const uint2* twf = S.tw_fwd + (size_t)grp * N;
  const uint2* twi = S.tw_inv + (size_t)grp * N;
  uint32_t* xb = exch + grp * XW;
  const int bar = 1 + grp;

  uint32_t sv[E];
#pragma unroll
  for (int k = 0; k < E; ++k) sv[k] = small(Y::j_of(0, t, k));
  ntt_fwd<L, EL, 0>(sv, t, twf, p, xb, bar, S.zero);
#pragma unroll
  for (int k = 0; k < E; ++k) sv[k] = csub(csub(sv[k], 2 * p), p);
  for (int c = 0; c < ncols; ++c) {
    uint32_t v[E];
#pragma unroll
    for (int k = 0; k < E; ++k) v[k] = mod_word<W>(word(c, Y::j_of(0, t, k)), S, grp);
    ntt_fwd<L, EL, 0>(v, t, twf, p, xb, bar, S.zero);
#pragma unroll
    for (int k = 0; k < E; ++k) {
      const uint32_t x = csub(csub(v[k], 2 * p), p);
      const uint32_t m = csub(redc((uint64_t)x * sv[k], p, pneg), p);          // x s 2^-32
      v[k] = csub(mul_shoup(m, S.ninv_m[grp], S.ninv_ms[grp], p), p);         // * N^-1 2^32
    }
    ntt_inv<L, EL, Y::K - 1>(v, t, twi, p, xb, bar, S.zero);
#pragma unroll
    for (int k = 0; k < E; ++k) stage[(grp * 2 + c) * N + Y::j_of(0, t, k)] = csub(v[k], p);
  }
  __syncthreads();
  for (int idx = tid; idx < ncols * N; idx += THREADS) {
    uint32_t x[P];
#pragma unroll
    for (int g = 0; g < P; ++g) x[g] = stage[g * 2 * N + idx];
    out(idx / N, idx % N, (W)garner_p<P>(x, S));
  }
}

template <int L, int EL, int P>
constexpr size_t product_smem_bytes() {
  return (size_t)P * 2 * (1 << L) * 4 + (size_t)P * (((size_t)Xch<L, EL>::kWords + 3) & ~(size_t)3) * 4;
}

// PubMux with L_boot = t (one digit): acc_F = [Delta p0, 0] + ((p1 - p0) mod t) * c_R
// with (p0, p1) = (rotP'_1, rotP'_0), rotP'_j = rotP_j X^{b_N}.
struct PubMuxParams {
  PrimeSet S;
  const void* cR;          // [batch / rep][2N]
  const void* ct;          // [batch / rep][n+1] input LWE (for b_N)
  int rep;                 // tables per input: item i reads cR and ct of input i / rep
  const int32_t* lut_ids;  // [batch]
  const int16_t* luts;     // [n_luts][2][N]  (rotP_0, rotP_1)
  int n_luts;
  void* accF;              // [batch][2N]
  int n, t;
  uint64_t delta;
  int* err;                // device error latch
};

template <int L, int EL, int P, typename W>
__global__ void __launch_bounds__(P * (1 << (L - EL))) pubmux_kernel(const PubMuxParams prm) {
  constexpr int N = 1 << L;
  extern __shared__ __align__(16) unsigned char smem[];
  const int64_t ci = blockIdx.x;
  const int64_t src = ci / prm.rep;
  const W* ct = reinterpret_cast<const W*>(prm.ct) + src * (prm.n + 1);
  const int bN = (int)modswitch_2n<W, L>(ct[0]);
  int lut = prm.lut_ids[ci];
  if (lut < 0 || lut >= prm.n_luts) {
    if (threadIdx.x == 0) atomicExch(prm.err, -6);
    lut = 0;
  }
  const int16_t* r0 = prm.luts + (size_t)lut * 2 * N;
  const int16_t* r1 = r0 + N;
  const int tmask = prm.t - 1;
  auto rotated = [&](const int16_t* poly, int j) -> int {
    bool neg;
    int m = rot_src<L>(j, bN, neg);
    int v = poly[m];
    return neg ? -v : v;
  };
  const W* cR = reinterpret_cast<const W*>(prm.cR) + src * 2 * N;
  W* out = reinterpret_cast<W*>(prm.accF) + ci * 2 * N;
  const W delta = (W)prm.delta;
  small_word_product<L, EL, P, W>(
      prm.S, 2,
      [&](int j) -> uint32_t { return (uint32_t)((rotated(r0, j) - rotated(r1, j)) & tmask); },
      [&](int c, int j) -> W { return cR[c * N + j]; },
      [&](int c, int j, W x) {
        if (c == 0) x = (W)(x + delta * (W)(int64_t)rotated(r1, j));
        out[c * N + j] = x;
      },
      smem);
}

// Accumulator of the TFHE bootstrap (figure "TFHE Bootstrapping", lines
// 1-3): b_N = ModSwitch(b, q, 2N) and acc = [poly X^{b_N}, 0] for ciphertext
// blockIdx.x, poly = polys[ids[blockIdx.x]] ([N] words mod q).  An id out of
// range latches FDFB_EBADLUT and uses polynomial 0.
template <typename W, int L>
__global__ void __launch_bounds__(256)
tfhe_acc_kernel(const W* __restrict__ ct, int n, const int32_t* __restrict__ ids,
                const W* __restrict__ polys, int n_polys, W* __restrict__ acc, int* err, uint64_t Q) {
  constexpr int N = 1 << L;
  const int64_t ci = blockIdx.x;
  // prime-modulus sets (Q != 0): the input is already mod 2N, negation mod Q
  const int bN = Q ? (int)((uint64_t)ct[ci * (n + 1)] & (2 * N - 1)) : (int)modswitch_2n<W, L>(ct[ci * (n + 1)]);
  int id = ids[ci];
  if (id < 0 || id >= n_polys) {
    if (threadIdx.x == 0) atomicExch(err, -6);
    id = 0;
  }
  const W* poly = polys + (size_t)id * N;
  W* out = acc + ci * 2 * N;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    bool neg;
    const int m = rot_src<L>(j, bN, neg);
    const W v = poly[m];
    out[j] = neg ? (Q ? (W)negq((uint64_t)v, Q) : (W)(0 - v)) : v;
    out[N + j] = 0;
  }
}

// RLWE encryption: out[item] = [a sk + e, a], then mu[item] added to the
// constant coefficient of component comp[item] (GGSW rows and packing-key
// samples).  sk is binary.
struct RlweEncParams {
  PrimeSet S;
  const uint8_t* sk;       // [N]
  const void* a;           // [count][N] words
  const int64_t* e;        // [count][N]
  const uint64_t* mu;      // [count]
  const uint8_t* comp;     // [count]
  void* out;               // [count][2][N]
};

template <int L, int EL, int P, typename W>
__global__ void __launch_bounds__(P * (1 << (L - EL))) rlwe_encrypt_kernel(const RlweEncParams prm) {
  constexpr int N = 1 << L;
  extern __shared__ __align__(16) unsigned char smem[];
  const int64_t it = blockIdx.x;
  const W* a = reinterpret_cast<const W*>(prm.a) + it * N;
  const int64_t* e = prm.e + it * N;
  W* out = reinterpret_cast<W*>(prm.out) + it * 2 * N;
  const W mu = (W)prm.mu[it];
  const int comp = prm.comp[it];
  small_word_product<L, EL, P, W>(
      prm.S, 1, [&](int j) -> uint32_t { return prm.sk[j]; },
      [&](int, int j) -> W { return a[j]; },
      [&](int, int j, W x) {
        W b = (W)(x + (W)e[j]);
        W av = a[j];
        if (j == 0) {
          if (comp == 0) b = (W)(b + mu); else av = (W)(av + mu);
        }
        out[j] = b;
        out[N + j] = av;
      },
      smem);
}

// Converts canonical GGSW rows [n][2 lg][2][N] into the transform domain:
// out[i][g][r][c][h][.] = NTT(centred(half h of bsk[i][r][c]) mod p_g) * N^-1 * 2^32
// mod p_g, with KH = 1 (the whole word) or KH = 2 (q = 2^64: the centred
// halves K_lo = (int32) K and K_hi = (K >> 32) + [K_lo < 0], arithmetic
// shift, so that K = K_lo + 2^32 K_hi with |K_lo|, |K_hi| <= 2^31).
// Transform output j = t E + k (thread t of the last pass, register k) is
// stored at (k / 4) 4G + 4t + k % 4, so that the blind rotation's 128-bit
// key loads are contiguous across a warp.  With Q != 0 (prime-modulus sets)
// the words are residues mod Q and are centred in (-Q/2, Q/2] first.
template <int L, int EL, int P, typename W, int KH = 1>
__global__ void __launch_bounds__(P * (1 << (L - EL)))
bsk_to_ntt_kernel(PrimeSet S, const void* bsk, int R, uint32_t* out, uint64_t Q) {
  static_assert(KH == 1 || sizeof(W) == 8, "key halves are for 64-bit words");
  using Y = Layout<L, EL>;
  constexpr int N = Y::N, E = Y::E, G = Y::G;
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int XW = (Xch<L, EL>::kWords + 3) & ~3;
  uint32_t* exch = reinterpret_cast<uint32_t*>(smem);
  const int64_t row = blockIdx.x;  // i * R + r
  const int64_t i = row / R;
  const int r = (int)(row % R);
  const int tid = threadIdx.x, grp = tid / G, t = tid - grp * G;
  const uint32_t p = S.p[grp];
  const W* src = reinterpret_cast<const W*>(bsk) + row * 2 * N;
  for (int c = 0; c < 2; ++c) {
    for (int h = 0; h < KH; ++h) {
      uint32_t v[E];
#pragma unroll
      for (int k = 0; k < E; ++k) {
        W x = src[c * N + Y::j_of(0, t, k)];
        if (Q) x = (W)centre_q((uint64_t)x, Q);
        if (KH == 1) {
          v[k] = mod_centred<W>(x, S, grp);
        } else {
          const uint64_t u = (uint64_t)x;
          if (h == 0) {
            v[k] = mod_centred<uint32_t>((uint32_t)u, S, grp);  // K_lo = (int32) K
          } else {
            const int64_t hi = ((int64_t)u >> 32) + (((uint32_t)u >> 31) ? 1 : 0);
            v[k] = mod_centred<uint64_t>((uint64_t)hi, S, grp);
          }
        }
      }
      ntt_fwd<L, EL, 0>(v, t, S.tw_fwd + (size_t)grp * N, p, exch + grp * XW, 1 + grp, S.zero);
      uint32_t* dst = out + ((((size_t)i * P + grp) * R + r) * 2 + c) * KH * N + (size_t)h * N;
#pragma unroll
      for (int k = 0; k < E; ++k) {
        const uint32_t y = csub(csub(v[k], 2 * p), p);
        dst[(k >> 2) * 4 * G + t * 4 + (k & 3)] = csub(mul_shoup(y, S.ninv_m[grp], S.ninv_ms[grp], p), p);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Key switching (appendix figure "Key switching algorithm and its setup"):
//   out[m] = [b_m, 0, ..] - sum_{i<n_in} sum_{j<l} Decomp(a_{m,i})_j key[i][j]
// as a tiled integer GEMM: rows m (ciphertexts), columns (output words),
// reduction over (i, j) with the digits generated on the fly.
// ---------------------------------------------------------------------------
constexpr int KS_BM = 64, KS_BN = 128, KS_BK = 32, KS_THREADS = 256;  // 8 x 4 outputs per thread

__device__ __forceinline__ void atomic_add_word(uint32_t* p, uint32_t v) { atomicAdd(p, v); }
__device__ __forceinline__ void atomic_add_word(uint64_t* p, uint64_t v) {
  atomicAdd(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
}

// CTA (blockIdx.x, blockIdx.y, blockIdx.z): ciphertexts [64 x, 64 x + 64),
// output columns [128 y, 128 y + 128), and slice z of `ksplit` equal slices of the
// reduction (K = n_in l, in steps of 32).  Thread (ty, tx) = (tid / 32,
// tid % 32) owns rows 8 ty.. and columns 4 tx..; per reduction index it reads
// its 8 digits as one broadcast 128-bit shared load and its 4 key words as
// one (u32) or two (u64) 128-bit loads, then does 32 multiply-adds.  With
// ksplit = 1 each output is written once; otherwise `out` must be zero and the
// slices add their parts atomically (integer addition mod 2^w: exact in any
// order), slice 0 adding b.
//
// KW = uint32_t with W = uint64_t (prime-modulus sets, raw = 1): the key holds
// the 32-bit halves of the words mod Q as separate columns and the kernel
// writes the exact 64-bit column sums (no negation, no b): every term
// d K_half < 2^16 2^32 and n_in l <= 2^18 terms keep them below 2^64;
// ks_finalize_q_kernel recombines and reduces them.
template <typename W, typename KW = W>
__global__ void __launch_bounds__(KS_THREADS)
keyswitch_kernel(const W* __restrict__ ct, int64_t batch, int n_in, const KW* __restrict__ key,
                 int ell, int log2B, int rtrunc, int out_len, W* __restrict__ out, int ksplit,
                 int raw = 0) {
  __shared__ __align__(16) uint16_t sa[KS_BK][KS_BM];
  __shared__ __align__(16) KW sb[KS_BK][KS_BN];
  const int tid = threadIdx.x, ty = tid >> 5, tx = tid & 31;
  const int64_t m0 = (int64_t)blockIdx.x * KS_BM;
  const int c0 = blockIdx.y * KS_BN;
  const int K = n_in * ell;
  const int kt = (K + KS_BK - 1) / KS_BK;
  const int kb = (int)((int64_t)kt * blockIdx.z / ksplit) * KS_BK;
  const int ke = min(K, (int)((int64_t)kt * (blockIdx.z + 1) / ksplit) * KS_BK);
  W acc[8][4];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0;
  const W half_rt = rtrunc ? ((W)1 << (rtrunc - 1)) : (W)0;
  const uint32_t dmask = (1u << log2B) - 1;
  for (int k0 = kb; k0 < ke; k0 += KS_BK) {
    // digits of the tile's ciphertexts: KS_BK x KS_BM, 8 per thread
#pragma unroll
    for (int e = tid; e < KS_BK * KS_BM; e += KS_THREADS) {
      const int kk = e / KS_BM, mm = e % KS_BM;
      const int k = k0 + kk;
      const int64_t m = m0 + mm;
      uint16_t d = 0;
      if (k < ke && m < batch) {
        const int i = k / ell, j = k - i * ell;
        const W x = ct[m * (n_in + 1) + 1 + i];
        const W xt = rtrunc ? (W)((W)(x + half_rt) >> rtrunc) : x;
        d = (uint16_t)((uint32_t)(xt >> (j * log2B)) & dmask);
      }
      sa[kk][mm] = d;
    }
    // key rows: KS_BK x KS_BN words, 16 per thread, coalesced along a row
#pragma unroll
    for (int e = tid; e < KS_BK * KS_BN; e += KS_THREADS) {
      const int kk = e / KS_BN, cc = e % KS_BN;
      const int k = k0 + kk, c = c0 + cc;
      sb[kk][cc] = (k < ke && c < out_len) ? key[(size_t)k * out_len + c] : (KW)0;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < KS_BK; ++kk) {
      const uint4 dq = *reinterpret_cast<const uint4*>(&sa[kk][ty * 8]);
      const uint32_t dw[4] = {dq.x, dq.y, dq.z, dq.w};
      W kv[4];
      if constexpr (sizeof(KW) == 4) {
        const uint4 q = *reinterpret_cast<const uint4*>(&sb[kk][tx * 4]);
        kv[0] = q.x; kv[1] = q.y; kv[2] = q.z; kv[3] = q.w;
      } else {
        const ulonglong2 q0 = *reinterpret_cast<const ulonglong2*>(&sb[kk][tx * 4]);
        const ulonglong2 q1 = *reinterpret_cast<const ulonglong2*>(&sb[kk][tx * 4 + 2]);
        kv[0] = q0.x; kv[1] = q0.y; kv[2] = q1.x; kv[3] = q1.y;
      }
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const uint32_t d = (dw[a >> 1] >> ((a & 1) * 16)) & 0xffffu;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          if constexpr (sizeof(W) == 4 || sizeof(KW) == 4) {
            acc[a][b] += (W)d * kv[b];
          } else {
            // d < 2^16: d K = d K_lo + 2^32 d K_hi, a 32x32->64 multiply-add
            // and a 32-bit multiply-add into the high word
            const uint64_t lo = (uint64_t)d * (uint32_t)kv[b];
            const uint32_t hi = d * (uint32_t)(kv[b] >> 32);
            acc[a][b] += lo + ((uint64_t)hi << 32);
          }
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int64_t m = m0 + ty * 8 + a;
    if (m >= batch) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int c = c0 + tx * 4 + b;
      if (c >= out_len) continue;
      W v = raw ? acc[a][b] : (W)(0 - acc[a][b]);
      if (!raw && c == 0 && blockIdx.z == 0) v = (W)(v + ct[m * (n_in + 1)]);
      if (ksplit == 1) out[m * out_len + c] = v;
      else atomic_add_word(&out[m * out_len + c], v);
    }
  }
}

// LWE encryption b = <a, s> + e + Delta m, one warp per ciphertext.
// Words are taken mod q = 2^logq (logq = w for the power-of-two sets; 2N
// for the prime-modulus sets, whose LWE side lives mod q = 2N).
template <typename W>
__global__ void lwe_encrypt_kernel(const uint8_t* s, const W* a, const int64_t* e, const int64_t* m,
                                   int64_t count, int n, uint64_t delta, W* out, int logq) {
  const int64_t c = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (c >= count) return;
  W acc = 0;
  for (int i = lane; i < n; i += 32) {
    const W ai = a[c * n + i];
    acc = (W)(acc + ai * (W)s[i]);
    out[c * (n + 1) + 1 + i] = ai;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc = (W)(acc + __shfl_xor_sync(0xffffffffu, acc, o));
  if (lane == 0) {
    const W mask = logq >= Word<W>::bits ? (W)~(W)0 : (W)(((W)1 << logq) - 1);
    out[c * (n + 1)] = (W)((acc + (W)e[c] + (W)delta * (W)m[c]) & mask);
  }
}

// Decryption round(t * phase / q) mod t (round half up): power-of-two t
// (t = 2^logt) by shifts, or any t (t_any > 0, the prime-modulus sets' CRT
// moduli) as ((phase t + q/2) >> logq) mod t.
template <typename W>
__global__ void lwe_decrypt_kernel(const uint8_t* s, const W* ct, int64_t count, int n, int logt,
                                   int32_t* m, int logq, int t_any) {
  const int64_t c = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (c >= count) return;
  W acc = 0;
  for (int i = lane; i < n; i += 32) acc = (W)(acc + ct[c * (n + 1) + 1 + i] * (W)s[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc = (W)(acc + __shfl_xor_sync(0xffffffffu, acc, o));
  if (lane == 0) {
    const W mask = logq >= Word<W>::bits ? (W)~(W)0 : (W)(((W)1 << logq) - 1);
    const W ph = (W)(ct[c * (n + 1)] - acc);
    if (t_any > 0) {  // logq <= 14 here: the product fits 64 bits
      const uint64_t phq = (uint64_t)(ph & mask);
      m[c] = (int32_t)(((phq * (uint64_t)t_any + (1ull << (logq - 1))) >> logq) % (uint64_t)t_any);
    } else {
      const W r = (W)((W)((W)(ph + ((W)1 << (logq - logt - 1))) & mask) >> (logq - logt));
      m[c] = (int32_t)r;
    }
  }
}

// y[b][o][k] = sum_i W[o][i] x[b][i][k] mod q: one block per (b, o-tile, k-tile).
constexpr int AFF_TO = 8, AFF_TK = 128;
template <typename W>
__global__ void __launch_bounds__(AFF_TK)
lwe_affine_kernel(const int32_t* __restrict__ Wm, int n_in, int n_out, const W* __restrict__ x,
                  int len, W* __restrict__ y) {
  const int64_t b = blockIdx.z;
  const int o0 = blockIdx.y * AFF_TO;
  const int k = blockIdx.x * AFF_TK + threadIdx.x;
  __shared__ int32_t sw[AFF_TO][64];
  W acc[AFF_TO];
#pragma unroll
  for (int o = 0; o < AFF_TO; ++o) acc[o] = 0;
  for (int i0 = 0; i0 < n_in; i0 += 64) {
    for (int e = threadIdx.x; e < AFF_TO * 64; e += AFF_TK) {
      const int oo = e / 64, ii = e % 64;
      sw[oo][ii] = (o0 + oo < n_out && i0 + ii < n_in) ? Wm[(size_t)(o0 + oo) * n_in + i0 + ii] : 0;
    }
    __syncthreads();
    if (k < len) {
      const int iend = min(64, n_in - i0);
      for (int ii = 0; ii < iend; ++ii) {
        const W xv = x[((size_t)b * n_in + i0 + ii) * len + k];
#pragma unroll
        for (int o = 0; o < AFF_TO; ++o) acc[o] = (W)(acc[o] + (W)(int64_t)sw[o][ii] * xv);
      }
    }
    __syncthreads();
  }
  if (k < len)
#pragma unroll
    for (int o = 0; o < AFF_TO; ++o)
      if (o0 + o < n_out) y[((size_t)b * n_out + o0 + o) * len + k] = acc[o];
}


// ---------------------------------------------------------------------------
// Prime-modulus sets (Table 1): the pieces of the pipeline that differ from
// the power-of-two path.
// ---------------------------------------------------------------------------

// out[m][c] = ([b_m, 0, ..] - S[m][c]) mod Q, S = sums[m][c] + 2^32
// sums[m][out_len + c] (the raw key-switch sums of the two key halves), and
// with logq > 0 then ModSwitch(Q -> q = 2^logq): round(q v / Q) mod q, round
// half up (appendix figure "Modulus switching algorithm").
static __global__ void ks_finalize_q_kernel(const uint64_t* __restrict__ ct, int n_in, int64_t batch,
                                     const uint64_t* __restrict__ sums, int out_len, ModQ mq, int logq,
                                     uint64_t* __restrict__ out) {
  const int64_t total = batch * out_len;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = idx / out_len;
    const int c = (int)(idx - m * out_len);
    const uint64_t* row = sums + m * 2 * out_len;
    const unsigned __int128 S = (unsigned __int128)row[c] + ((unsigned __int128)row[out_len + c] << 32);
    const uint64_t r = modq_u128(S, mq);
    uint64_t v = c == 0 ? subq(ct[m * (n_in + 1)], r, mq.Q) : negq(r, mq.Q);
    if (logq > 0) {
      const unsigned __int128 num = ((unsigned __int128)v << (logq + 1)) + mq.Q;
      v = (uint64_t)(num / ((unsigned __int128)2 * mq.Q)) & ((1ull << logq) - 1);
    }
    out[idx] = v;
  }
}

// Key words mod Q, [rows][cols], to the key-switch layout [rows][2 cols] of
// their 32-bit halves (low halves first).
static __global__ void split_halves_kernel(const uint64_t* __restrict__ in, int64_t rows, int cols,
                                    uint32_t* __restrict__ out) {
  const int64_t total = rows * cols;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / cols;
    const int c = (int)(idx - r * cols);
    const uint64_t x = in[idx];
    out[r * 2 * cols + c] = (uint32_t)x;
    out[r * 2 * cols + cols + c] = (uint32_t)(x >> 32);
  }
}

// PubMux over l_boot RLWE samples (figure "cmux-accumulator-builder"):
// p = p_1 - p_0 in Z_Q with (p_0, p_1) = (rotP'_1, rotP'_0), its base-L_boot
// digits p[i], acc_F = [Delta p_0, 0] + sum_i p[i] * c_R,i mod Q.  The l_boot
// products of each column are summed in the transform domain (exact while
// l_boot N (L_boot - 1) Q / 2 stays below half the primes' product) and
// lifted once.  cR: [batch / rep][lboot][2][N] words mod Q.
struct PubMuxQParams {
  PrimeSet S;
  ModQ mq;
  const uint64_t* cR;
  const uint64_t* ct;      // [batch / rep][n+1] input LWE mod 2N (for b_N)
  int rep;
  const int32_t* lut_ids;  // [batch]
  const int16_t* luts;     // [n_luts][2][N]
  int n_luts;
  uint64_t* accF;          // [batch][2N]
  int n, lboot, log2Lboot;
  uint64_t delta;          // round(Q / t)
  int* err;
};

template <int L, int EL, int P>
__global__ void __launch_bounds__(P * (1 << (L - EL))) pubmux_q_kernel(const PubMuxQParams prm) {
  using Y = Layout<L, EL>;
  constexpr int N = Y::N, E = Y::E, G = Y::G, THREADS = P * G;
  constexpr int XW = (Xch<L, EL>::kWords + 3) & ~3;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* stage = reinterpret_cast<uint32_t*>(smem);  // [P][2][N]
  uint32_t* exch = stage + P * 2 * N;                   // [P][XW]
  const int64_t ci = blockIdx.x;
  const int64_t src = ci / prm.rep;
  const uint64_t Q = prm.mq.Q;
  const uint64_t* ct = prm.ct + src * (prm.n + 1);
  const int bN = (int)(ct[0] & (2 * N - 1));
  int lut = prm.lut_ids[ci];
  if (lut < 0 || lut >= prm.n_luts) {
    if (threadIdx.x == 0) atomicExch(prm.err, -6);
    lut = 0;
  }
  const int16_t* r0 = prm.luts + (size_t)lut * 2 * N;
  const int16_t* r1 = r0 + N;
  auto rotated = [&](const int16_t* poly, int j) -> int {
    bool neg;
    int m = rot_src<L>(j, bN, neg);
    int v = poly[m];
    return neg ? -v : v;
  };
  const int tid = threadIdx.x;
  const int grp = tid / G;
  const int t = tid - grp * G;
  const uint32_t p = prm.S.p[grp];
  const uint32_t pneg = prm.S.pneg[grp];
  const uint32_t z = prm.S.zero;
  const uint2* twf = prm.S.tw_fwd + (size_t)grp * N;
  const uint2* twi = prm.S.tw_inv + (size_t)grp * N;
  uint32_t* xb = exch + grp * XW;
  const int bar = 1 + grp;
  const uint64_t dmask = (1ull << prm.log2Lboot) - 1;
  const uint64_t* cR = prm.cR + src * (size_t)prm.lboot * 2 * N;

  uint32_t accm[2][E];
#pragma unroll
  for (int k = 0; k < E; ++k) accm[0][k] = accm[1][k] = 0;
  for (int i = 0; i < prm.lboot; ++i) {
    uint32_t sv[E];
#pragma unroll
    for (int k = 0; k < E; ++k) {
      const int j = Y::j_of(0, t, k);
      const int pd = rotated(r0, j) - rotated(r1, j);  // p_1 - p_0, |pd| < 2t
      const uint64_t pq = pd >= 0 ? (uint64_t)pd : Q - (uint64_t)(-pd);
      sv[k] = (uint32_t)((pq >> (i * prm.log2Lboot)) & dmask);
    }
    ntt_fwd<L, EL, 0>(sv, t, twf, p, xb, bar, z);
#pragma unroll
    for (int k = 0; k < E; ++k) sv[k] = csub(csub(sv[k], 2 * p), p);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      uint32_t v[E];
#pragma unroll
      for (int k = 0; k < E; ++k)
        v[k] = mod_centred<uint64_t>(centre_q(cR[((size_t)i * 2 + c) * N + Y::j_of(0, t, k)], Q), prm.S, grp);
      ntt_fwd<L, EL, 0>(v, t, twf, p, xb, bar, z);
#pragma unroll
      for (int k = 0; k < E; ++k) {
        const uint32_t x = csub(csub(v[k], 2 * p), p);
        const uint32_t m = redc((uint64_t)x * sv[k], p, pneg);  // x s 2^-32, < 2p
        const uint32_t s2 = accm[c][k] + m;
        accm[c][k] = umin32(s2, s2 - 2 * p);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    uint32_t v[E];
#pragma unroll
    for (int k = 0; k < E; ++k)
      v[k] = csub(mul_shoup(csub(accm[c][k], p), prm.S.ninv_m[grp], prm.S.ninv_ms[grp], p), p);
    ntt_inv<L, EL, Y::K - 1>(v, t, twi, p, xb, bar, z);
#pragma unroll
    for (int k = 0; k < E; ++k) stage[(grp * 2 + c) * N + Y::j_of(0, t, k)] = csub(v[k], p);
  }
  __syncthreads();
  uint64_t* out = prm.accF + ci * 2 * N;
  for (int idx = tid; idx < 2 * N; idx += THREADS) {
    uint32_t x[P];
#pragma unroll
    for (int g = 0; g < P; ++g) x[g] = stage[g * 2 * N + idx];
    uint64_t r = modq_lift(garner_exact<P>(x, prm.S), prm.mq);
    if (idx < N) {
      const int p0 = rotated(r1, idx);
      const uint64_t p0q = p0 >= 0 ? (uint64_t)p0 : Q - (uint64_t)(-p0);
      r = addq(r, mulq(prm.delta, p0q, prm.mq), Q);
    }
    out[idx] = r;
  }
}

// RLWE samples mod Q with a uniform key sk in Z_Q^N (key generation of the
// prime-modulus sets): out = [b = a sk + e + mu, a], mu added to coefficient
// 0 of component comp.  a sk is exact as sum_k 2^(13 k) (a * sk_k) over the
// balanced 13-bit limbs sk_k of the centred key (|sk_k| <= 2^12, five limbs
// for |sk| < 2^62): each limb product is below N 2^12 2^62 <= 2^86 in
// magnitude and lifts exactly from three primes.  skl: the limbs in the
// transform domain, [5][P][2][N] in the blind rotation's key layout
// (bsk_to_ntt_kernel with R = 1 on rows [limb, 0]: times N^-1 2^32).
struct RlweEncQParams {
  PrimeSet S;
  ModQ mq;
  const uint32_t* skl;
  const uint64_t* a;       // [count][N] mod Q
  const int64_t* e;        // [count][N]
  const uint64_t* mu;      // [count] mod Q
  const uint8_t* comp;     // [count]
  uint64_t* out;           // [count][2][N]
};
constexpr int kSkLimbs = 5, kSkLimbBits = 13;

template <int L, int EL, int P>
__global__ void __launch_bounds__(P * (1 << (L - EL))) rlwe_encrypt_q_kernel(const RlweEncQParams prm) {
  using Y = Layout<L, EL>;
  constexpr int N = Y::N, E = Y::E, G = Y::G, THREADS = P * G;
  constexpr int XW = (Xch<L, EL>::kWords + 3) & ~3;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* stage = reinterpret_cast<uint32_t*>(smem);  // [P][N]
  uint32_t* exch = stage + P * 2 * N;                   // [P][XW]
  const int64_t it = blockIdx.x;
  const uint64_t Q = prm.mq.Q;
  const uint64_t* a = prm.a + it * N;
  const int64_t* e = prm.e + it * N;
  uint64_t* out = prm.out + it * 2 * N;
  const int tid = threadIdx.x;
  const int grp = tid / G;
  const int t = tid - grp * G;
  const uint32_t p = prm.S.p[grp];
  const uint32_t pneg = prm.S.pneg[grp];
  const uint32_t z = prm.S.zero;
  uint32_t* xb = exch + grp * XW;
  const int bar = 1 + grp;
  // b starts as e + mu (component 0), a as given (+ mu on component 1)
  for (int j = tid; j < N; j += THREADS) {
    const int64_t ev = e[j];
    uint64_t b = ev >= 0 ? (uint64_t)ev % Q : negq((uint64_t)(-ev) % Q, Q);
    uint64_t av = a[j];
    if (j == 0) {
      if (prm.comp[it] == 0) b = addq(b, prm.mu[it], Q);
      else av = addq(av, prm.mu[it], Q);
    }
    out[j] = b;
    out[N + j] = av;
  }
  uint32_t va[E];
#pragma unroll
  for (int k = 0; k < E; ++k) va[k] = mod_centred<uint64_t>(centre_q(a[Y::j_of(0, t, k)], Q), prm.S, grp);
  ntt_fwd<L, EL, 0>(va, t, prm.S.tw_fwd + (size_t)grp * N, p, xb, bar, z);
#pragma unroll
  for (int k = 0; k < E; ++k) va[k] = csub(csub(va[k], 2 * p), p);
  for (int l = 0; l < kSkLimbs; ++l) {
    const uint32_t* kl = prm.skl + ((size_t)l * P + grp) * 2 * N;  // component 0 of limb row l
    uint32_t v[E];
#pragma unroll
    for (int k = 0; k < E; ++k) {
      const uint32_t kv = kl[(k >> 2) * 4 * G + t * 4 + (k & 3)];
      v[k] = csub(redc((uint64_t)va[k] * kv, p, pneg), p);  // a sk_l N^-1
    }
    ntt_inv<L, EL, Y::K - 1>(v, t, prm.S.tw_inv + (size_t)grp * N, p, xb, bar, z);
    __syncthreads();  // the previous limb's lift has read the staging area
#pragma unroll
    for (int k = 0; k < E; ++k) stage[grp * N + Y::j_of(0, t, k)] = csub(v[k], p);
    __syncthreads();
    const uint64_t w = modq_u128((unsigned __int128)1 << (kSkLimbBits * l), prm.mq);  // 2^(13 l) mod Q
    for (int j = tid; j < N; j += THREADS) {
      uint32_t x[P];
#pragma unroll
      for (int g = 0; g < P; ++g) x[g] = stage[g * N + j];
      const uint64_t X = modq_lift(garner_exact<P>(x, prm.S), prm.mq);
      out[j] = addq(out[j], mulq(X, w, prm.mq), Q);
    }
  }
}

// The balanced 13-bit limbs of the centred key as rows [5][2][N] of words
// mod Q (a negative limb d stored as Q + d; component 1 left zero), for
// bsk_to_ntt_kernel.
static __global__ void sk_limbs_kernel(const uint64_t* __restrict__ sk, int N, ModQ mq, uint64_t* __restrict__ out) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
    int64_t x = (int64_t)centre_q(sk[j], mq.Q);
    for (int l = 0; l < kSkLimbs; ++l) {
      const int64_t d = ((x + (1 << (kSkLimbBits - 1))) & ((1 << kSkLimbBits) - 1)) - (1 << (kSkLimbBits - 1));
      out[(size_t)l * 2 * N + j] = d >= 0 ? (uint64_t)d : mq.Q - (uint64_t)(-d);
      out[(size_t)l * 2 * N + N + j] = 0;
      x = (x - d) >> kSkLimbBits;
    }
  }
}

// LWE samples mod Q under the binary key s (the key-switching key of the
// prime-modulus sets): out = [b = <a, s> + e + mu, a], one warp per sample.
static __global__ void lwe_encrypt_q_kernel(const uint8_t* s, const uint64_t* a, const int64_t* e,
                                     const uint64_t* mu, int64_t count, int n, ModQ mq, uint64_t* out) {
  const int64_t c = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (c >= count) return;
  const uint64_t Q = mq.Q;
  uint64_t acc = 0;
  for (int i = lane; i < n; i += 32) {
    const uint64_t ai = a[c * n + i];
    if (s[i]) acc = addq(acc, ai, Q);
    out[c * (n + 1) + 1 + i] = ai;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc = addq(acc, __shfl_xor_sync(0xffffffffu, acc, o), Q);
  if (lane == 0) {
    const int64_t ev = e[c];
    const uint64_t eq = ev >= 0 ? (uint64_t)ev % Q : negq((uint64_t)(-ev) % Q, Q);
    out[c * (n + 1)] = addq(addq(acc, eq, Q), mu[c], Q);
  }
}

}  // namespace fdfb
