// Ring degree N = 2^13 on the prime-modulus parameter sets (Table 1:
// FDFB:80:8 and FDFB:100:8).
//
// At N = 8192 one item's accumulator (2N words mod Q, 128 KB) takes more
// than half of an SM's shared memory, and the register layouts of N <= 4096
// (three primes, one thread group per prime) would need 1,536 threads at 16
// coefficients per thread.  So every negacyclic transform of 8192 points is
// cut at its first Cooley-Tukey stage.  That stage pairs coefficient j with
// j + 4096 under a single twiddle w (psi^4096, entry 1 of the bit-reversed
// table); its outputs x_j + w x_{j+4096} and x_j - w x_{j+4096} are the
// inputs of two independent 4096-point transforms, the halves h = 0, 1 of
// the spectrum, whose stage-s twiddles are the 8192-point table's entries
// 2^(s+1) + h 2^s + i.  The inverse mirrors it: two 4096-point inverse
// transforms, then the last Gentleman-Sande stage (X + Y, (X - Y) w^-1) on
// the pairs (j, j + 4096).  The half tables (host::make_prime_set_n13) are
// laid out so that the 4096-point register transforms of Layout<12, EL> run
// unchanged on them; entry 0 of each holds the split stage's twiddle.
//
// One CTA per item runs the two halves one after the other, so a CTA holds
// the same thread groups as at N = 4096 (one group of 4096 / E threads per
// prime).  Shared memory: d = acc X^{-a} - acc of the current step ([2][8192]
// words, from which every transform cuts its digits), the mask a_N, and one
// region that is the groups' exchange buffers during the transforms and the
// lift's staging area [P][8192] afterwards (227 KB for n <= 1536).  The
// accumulator itself lives in the item's global scratch (L2): it is read
// once per step to form d and updated once by the lift, while d is read
// 2 x 2 l_g times per step (every digit row, in both halves).  The halves'
// inverse results wait there too until both exist.
#pragma once
#include "fdfb_kernels.cuh"

namespace fdfb {

constexpr int kN13 = 8192, kN13h = 4096;

// 32-bit words of one item's global scratch of blind_rotate_n13_kernel.
template <int P, int KH = 1>
constexpr int n13_scratch_words() {
  return P * 4 * KH * kN13h + 4 * kN13;
}

template <int EL>
constexpr int n13_xwords() {
  return (Xch<12, EL>::kWords + 3) & ~3;
}

// Half h of the forward transform of the 8192 values x(j) (each below 4p):
// the split stage on (j, j + 4096) at the pass-0 positions of thread t,
// then the 4096-point transform; v ends in the last-pass layout, in [0, 4p).
template <int EL, typename X>
__device__ __forceinline__ void n13_fwd_half(uint32_t (&v)[1 << EL], int h, X x, int t, const uint2* tw,
                                             uint32_t p, uint32_t* xb, int bar, uint32_t z) {
  using Y = Layout<12, EL>;
  const uint2 w = tw[0];
#pragma unroll
  for (int k = 0; k < Y::E; ++k) {
    const int j = Y::j_of(0, t, k);
    uint32_t a = x(j), b = x(j + kN13h);
    bfly_fwd(a, b, w, p, z);
    v[k] = h ? b : a;
  }
  ntt_fwd<12, EL, 0>(v, t, tw, p, xb, bar, z);
}

// The last inverse stage of one prime's residues: y0 (half 0, [0, p)) and
// y1 (half 1) of pass-0 position j give the coefficients j and j + 4096 in
// [0, p), written to out[j] and out[j + 4096].
__device__ __forceinline__ void n13_join(uint32_t y0, uint32_t y1, uint2 wi, uint32_t p, uint32_t z,
                                         uint32_t* out, int j) {
  bfly_inv(y0, y1, wi, p, z);
  out[j] = csub(y0, p);
  out[j + kN13h] = csub(y1, p);
}

// ---------------------------------------------------------------------------
// Blind rotation (appendix figure "Blind Rotation and its setup"), prime
// modulus, N = 8192: for i = 1..n, d = acc X^{-a_i} - acc mod Q, its exact
// digits D_r (r = c lg + l), acc += sum_r D_r * bsk[i][r] mod Q.  Per step
// and half, each group transforms the 2 lg digit polynomials modulo its
// prime, sums the pointwise products with the key rows (each reduced as it
// is formed), and transforms the two column sums back into the item's
// global scratch; the joined residues of all primes are lifted to the exact
// integer (Garner) and reduced mod Q.
// Key rows: [n][P][2][2 lg][2][KH][4096] words, half h of row r, column c
// and key half kh in the 4096-point last-pass order of bsk_to_ntt_n13_kernel.
// Global scratch per item (half_y, n13_scratch_words): [P][2 halves][2][KH]
// [4096] residues, then the accumulator [2][8192] words.
// KH = 2 (two primes): every key word K is split into centred 32-bit halves,
// K = K_lo + 2^32 K_hi, both sharing the digits' transforms; each half's
// product sum (at most 2 l N (B - 1) 2^31 < 2^57) lifts exactly from two
// primes and acc += X_lo + 2^32 X_hi mod Q.
// ---------------------------------------------------------------------------
template <int EL, int P, int MINB, int KH = 1>
__global__ void __launch_bounds__(P * (1 << (12 - EL)), MINB) blind_rotate_n13_kernel(const BRParams prm) {
  static_assert(KH == 1 || P == 2, "split keys: two primes");
  using Y = Layout<12, EL>;
  constexpr int NF = kN13, NH = kN13h, E = Y::E, G = Y::G, THREADS = P * G;
  constexpr int XW = n13_xwords<EL>();
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* dq = reinterpret_cast<uint64_t*>(smem);                     // [2][NF] d of the step
  uint16_t* aN = reinterpret_cast<uint16_t*>(smem + 2 * NF * 8);       // [n]
  uint32_t* region = reinterpret_cast<uint32_t*>(smem + prm.smem_r1);  // [P][XW] exchange | [P][NF] stage

  const int tid = threadIdx.x;
  const int grp = tid / G;
  const int t = tid - grp * G;
  const int64_t ci = blockIdx.x;
  const int n = prm.n, lg = prm.lg, log2Bg = prm.log2Bg;
  const uint64_t Q = prm.mq.Q;
  const uint64_t* ct = reinterpret_cast<const uint64_t*>(prm.ct) + (ci / prm.rep) * (n + 1);
  // the item's global scratch: half results, then the accumulator
  uint32_t* scratch = prm.half_y + (size_t)ci * n13_scratch_words<P, KH>();
  uint64_t* acc = reinterpret_cast<uint64_t*>(scratch + P * 4 * KH * NH);  // [2][NF]

  // the input words already lie in [0, 2N) (q = 2N)
  for (int i = tid; i < n; i += THREADS) aN[i] = (uint16_t)((uint32_t)ct[1 + i] & (2 * NF - 1));
  if (prm.sign_mode) {
    // acc = [L_boot^(i mod l_boot) Delta/2 sgnP X^{b_N}, 0], sgnP = 1 - sum_{i>=2} X^{i-1}
    const int bN = (int)((uint32_t)ct[0] & (2 * NF - 1));
    const uint64_t hv = prm.sgn_scale[ci % prm.rep];
    for (int j = tid; j < NF; j += THREADS) {
      bool neg;
      const int m = rot_src<13>(j, bN, neg);
      const uint64_t c = (m == 0) ? hv : negq(hv, Q);
      acc[j] = neg ? negq(c, Q) : c;
      acc[NF + j] = 0;
    }
  } else {
    const uint64_t* a0 = reinterpret_cast<const uint64_t*>(prm.acc0) + ci * 2 * NF;
    for (int j = tid; j < 2 * NF; j += THREADS) acc[j] = a0[j];
  }
  __syncthreads();

  const uint32_t p = prm.S.p[grp];
  const uint32_t pneg = prm.S.pneg[grp];
  const uint32_t z = prm.S.zero;
  uint32_t* xb = region + grp * XW;
  const int bar = 1 + grp;
  const int R = 2 * lg;
  const uint32_t dmask = (1u << log2Bg) - 1;
  uint32_t* ys = scratch + (size_t)grp * 4 * KH * NH;  // this group's [2 halves][2][KH][NH]
  const size_t kblk = (size_t)R * 2 * KH * NH;              // words of one (step, prime, half) block
  const uint2 wfi = prm.S.tw_inv[(size_t)grp * 2 * NH];         // the split stage's inverse twiddle
  if (t == 0 && n > 0) prefetch_l2_bulk(prm.bsk + (size_t)grp * 2 * kblk, (uint32_t)(kblk * 4));

  for (int i = 0; i < n; ++i) {
    const int a = aN[i];
    // d = acc X^{-a} - acc mod Q: (acc X^{-a})_j = acc_{j+a}, negated when j +
    // a wraps past N (X^N = -1); the previous step's lift ended in a barrier,
    // so every thread's accumulator writes are visible here
    for (int idx = tid; idx < 2 * NF; idx += THREADS) {
      const int c = idx >> 13, j = idx & (NF - 1);
      const int m = (j + a) & (2 * NF - 1);
      const uint64_t sv = acc[c * NF + (m & (NF - 1))];
      dq[idx] = subq((m & NF) ? negq(sv, Q) : sv, acc[idx], Q);
    }
    __syncthreads();
    for (int h = 0; h < 2; ++h) {
      const uint2* twf = prm.S.tw_fwd + ((size_t)grp * 2 + h) * NH;
      const uint2* twi = prm.S.tw_inv + ((size_t)grp * 2 + h) * NH;
      const uint32_t* kb = prm.bsk + (((size_t)i * P + grp) * 2 + h) * kblk;
      if (t == 0) {  // into L2: this step's second half, else the next step's first
        if (h == 0) prefetch_l2_bulk(kb + kblk, (uint32_t)(kblk * 4));
        else if (i + 1 < n) prefetch_l2_bulk(prm.bsk + ((size_t)(i + 1) * P + grp) * 2 * kblk, (uint32_t)(kblk * 4));
      }
      uint32_t macc[KH][2][E];
#pragma unroll
      for (int kh = 0; kh < KH; ++kh)
#pragma unroll
        for (int k = 0; k < E; ++k) { macc[kh][0][k] = 0; macc[kh][1][k] = 0; }
      for (int r = 0; r < R; ++r) {
        const int cc = r >= lg ? 1 : 0;
        const int sh = (r - cc * lg) * log2Bg;
        const uint64_t* dc = dq + cc * NF;  // digit l of coefficient j of d_cc
        auto digit = [&](int j) -> uint32_t { return (uint32_t)(dc[j] >> sh) & dmask; };
        uint32_t v[E];
        n13_fwd_half<EL>(v, h, digit, t, twf, p, xb, bar, z);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
#pragma unroll
          for (int kh = 0; kh < KH; ++kh) {
            const uint4* kp = reinterpret_cast<const uint4*>(kb + (((size_t)r * 2 + c) * KH + kh) * NH) + t;
#pragma unroll
            for (int q4 = 0; q4 < E / 4; ++q4) {
              const uint4 kk = ldg_stream(kp + q4 * G);
              const uint32_t kv[4] = {kk.x, kk.y, kk.z, kk.w};
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                // v < 4p, K < p: v K < 2^62, reduced below 2p; the sum stays in [0, 2p)
                const uint32_t mm = redc((uint64_t)v[q4 * 4 + u] * kv[u], p, pneg);
                const uint32_t s2 = macc[kh][c][q4 * 4 + u] + mm + z;
                macc[kh][c][q4 * 4 + u] = umin32(s2, s2 - 2 * p + z);
              }
            }
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 2; ++c) {
#pragma unroll
        for (int kh = 0; kh < KH; ++kh) {
          uint32_t v[E];
#pragma unroll
          for (int k = 0; k < E; ++k) v[k] = macc[kh][c][k];
          ntt_inv<12, EL, Y::K - 1>(v, t, twi, p, xb, bar, z);
#pragma unroll
          for (int k = 0; k < E; ++k) ys[((h * 2 + c) * KH + kh) * NH + Y::j_of(0, t, k)] = csub(v[k], p);
        }
      }
    }
    __syncthreads();  // every group is done with its exchange buffer: the region becomes the stage
    for (int ck = 0; ck < 2 * KH; ++ck) {  // column c, key half kh
      const int c = ck / KH, kh = ck - c * KH;
      // the same thread wrote ys at these positions: no barrier needed for it
#pragma unroll
      for (int k = 0; k < E; ++k) {
        const int j = Y::j_of(0, t, k);
        n13_join(ys[(c * KH + kh) * NH + j], ys[((2 + c) * KH + kh) * NH + j], wfi, p, z, region + grp * NF, j);
      }
      __syncthreads();
      for (int j = tid; j < NF; j += THREADS) {
        uint32_t x[P];
#pragma unroll
        for (int g = 0; g < P; ++g) x[g] = region[g * NF + j];
        __int128 X = garner_exact<P>(x, prm.S);
        if (kh) X *= (__int128)1 << 32;
        acc[c * NF + j] = addq(acc[c * NF + j], modq_lift(X, prm.mq), Q);
      }
      __syncthreads();
    }
  }

  // SampleExtract of coefficient 0 (+ the sign item's constant in sign mode)
  uint64_t* out = reinterpret_cast<uint64_t*>(prm.lwe_out) + ci * (NF + 1);
  for (int k = tid; k <= NF; k += THREADS) {
    uint64_t v;
    if (k == 0) v = addq(acc[0], prm.sign_mode ? prm.sgn_scale[ci % prm.rep] : 0, Q);
    else if (k == 1) v = acc[NF];
    else v = negq(acc[NF + (NF - (k - 1))], Q);
    out[k] = v;
  }
}

// Canonical GGSW rows [n][2 lg][2][8192] words mod Q to the transform domain
// of blind_rotate_n13_kernel: out[i][g][h][r][c][kh][.] = half h of
// NTT(centred(bsk[i][r][c]) mod p_g) * 8192^-1 * 2^32 mod p_g (KH = 2: of the
// centred 32-bit halves K_lo = (int32) K and K_hi = (K >> 32) + [K_lo < 0]
// of the centred word K), output j = t E + k of the 4096-point last pass
// stored at (k / 4) 4G + 4t + k % 4.  With R = 1 and KH = 1 it converts the
// key limbs of rlwe_encrypt_q_n13_kernel.
template <int EL, int P, int KH = 1>
__global__ void __launch_bounds__(P * (1 << (12 - EL)))
bsk_to_ntt_n13_kernel(PrimeSet S, const void* bsk, int R, uint32_t* out, uint64_t Q) {
  using Y = Layout<12, EL>;
  constexpr int NF = kN13, NH = kN13h, E = Y::E, G = Y::G;
  constexpr int XW = n13_xwords<EL>();
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* exch = reinterpret_cast<uint32_t*>(smem);
  const int64_t row = blockIdx.x;  // i * R + r
  const int64_t i = row / R;
  const int r = (int)(row % R);
  const int tid = threadIdx.x, grp = tid / G, t = tid - grp * G;
  const uint32_t p = S.p[grp];
  const uint64_t* src = reinterpret_cast<const uint64_t*>(bsk) + row * 2 * NF;
  for (int c = 0; c < 2; ++c) {
    for (int h = 0; h < 2 * KH; ++h) {
      const int hh = h / KH, kh = h - hh * KH;  // spectrum half, key half
      const uint2* twf = S.tw_fwd + ((size_t)grp * 2 + hh) * NH;
      uint32_t v[E];
      n13_fwd_half<EL>(v, hh,
                       [&](int j) -> uint32_t {
                         const uint64_t u = centre_q(src[c * NF + j], Q);
                         if (KH == 1) return mod_centred<uint64_t>(u, S, grp);
                         if (kh == 0) return mod_centred<uint32_t>((uint32_t)u, S, grp);
                         const int64_t hi = ((int64_t)u >> 32) + (((uint32_t)u >> 31) ? 1 : 0);
                         return mod_centred<uint64_t>((uint64_t)hi, S, grp);
                       },
                       t, twf, p, exch + grp * XW, 1 + grp, S.zero);
      uint32_t* dst = out + (((((size_t)i * P + grp) * 2 + hh) * R + r) * 2 + c) * KH * NH + (size_t)kh * NH;
#pragma unroll
      for (int k = 0; k < E; ++k) {
        const uint32_t y = csub(csub(v[k], 2 * p), p);
        dst[(k >> 2) * 4 * G + t * 4 + (k & 3)] = csub(mul_shoup(y, S.ninv_m[grp], S.ninv_ms[grp], p), p);
      }
    }
  }
}

// PubMux over l_boot RLWE samples (figure "cmux-accumulator-builder"), N =
// 8192: the same computation as pubmux_q_kernel (p = p_1 - p_0 in Z_Q, its
// base-L_boot digits p[i], acc_F = [Delta p_0, 0] + sum_i p[i] * c_R,i mod Q)
// with the split transforms, one output column at a time.  Shared memory:
// both halves' inverse results [2][P][4096], then the exchange buffers /
// lift stage [P][8192].
template <int EL, int P>
__global__ void __launch_bounds__(P * (1 << (12 - EL))) pubmux_q_n13_kernel(const PubMuxQParams prm) {
  using Y = Layout<12, EL>;
  constexpr int NF = kN13, NH = kN13h, E = Y::E, G = Y::G, THREADS = P * G;
  constexpr int XW = n13_xwords<EL>();
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* ysh = reinterpret_cast<uint32_t*>(smem);  // [2 halves][P][NH]
  uint32_t* region = ysh + 2 * P * NH;                // [P][XW] exchange | [P][NF] stage
  const int64_t ci = blockIdx.x;
  const int64_t src = ci / prm.rep;
  const uint64_t Q = prm.mq.Q;
  const uint64_t* ct = prm.ct + src * (prm.n + 1);
  const int bN = (int)(ct[0] & (2 * NF - 1));
  int lut = prm.lut_ids[ci];
  if (lut < 0 || lut >= prm.n_luts) {
    if (threadIdx.x == 0) atomicExch(prm.err, -6);
    lut = 0;
  }
  const int16_t* r0 = prm.luts + (size_t)lut * 2 * NF;
  const int16_t* r1 = r0 + NF;
  auto rotated = [&](const int16_t* poly, int j) -> int {
    bool neg;
    const int m = rot_src<13>(j, bN, neg);
    const int v = poly[m];
    return neg ? -v : v;
  };
  const int tid = threadIdx.x;
  const int grp = tid / G;
  const int t = tid - grp * G;
  const uint32_t p = prm.S.p[grp];
  const uint32_t pneg = prm.S.pneg[grp];
  const uint32_t z = prm.S.zero;
  uint32_t* xb = region + grp * XW;
  const int bar = 1 + grp;
  const uint64_t dmask = (1ull << prm.log2Lboot) - 1;
  const uint64_t* cR = prm.cR + src * (size_t)prm.lboot * 2 * NF;
  const uint2 wfi = prm.S.tw_inv[(size_t)grp * 2 * NH];
  uint64_t* out = prm.accF + ci * 2 * NF;

  for (int c = 0; c < 2; ++c) {
    for (int h = 0; h < 2; ++h) {
      const uint2* twf = prm.S.tw_fwd + ((size_t)grp * 2 + h) * NH;
      const uint2* twi = prm.S.tw_inv + ((size_t)grp * 2 + h) * NH;
      uint32_t accm[E];
#pragma unroll
      for (int k = 0; k < E; ++k) accm[k] = 0;
      for (int i = 0; i < prm.lboot; ++i) {
        uint32_t sv[E];
        n13_fwd_half<EL>(sv, h,
                         [&](int j) -> uint32_t {
                           const int pd = rotated(r0, j) - rotated(r1, j);  // p_1 - p_0, |pd| < 2t
                           const uint64_t pq = pd >= 0 ? (uint64_t)pd : Q - (uint64_t)(-pd);
                           return (uint32_t)((pq >> (i * prm.log2Lboot)) & dmask);
                         },
                         t, twf, p, xb, bar, z);
        const uint64_t* w = cR + ((size_t)i * 2 + c) * NF;
        uint32_t v[E];
        n13_fwd_half<EL>(v, h, [&](int j) -> uint32_t { return mod_centred<uint64_t>(centre_q(w[j], Q), prm.S, grp); },
                         t, twf, p, xb, bar, z);
#pragma unroll
        for (int k = 0; k < E; ++k) {
          const uint32_t x = csub(csub(v[k], 2 * p), p);
          const uint32_t m = redc((uint64_t)x * csub(csub(sv[k], 2 * p), p), p, pneg);  // x s 2^-32, < 2p
          const uint32_t s2 = accm[k] + m;
          accm[k] = umin32(s2, s2 - 2 * p);
        }
      }
      uint32_t v[E];
#pragma unroll
      for (int k = 0; k < E; ++k) v[k] = csub(mul_shoup(csub(accm[k], p), prm.S.ninv_m[grp], prm.S.ninv_ms[grp], p), p);
      ntt_inv<12, EL, Y::K - 1>(v, t, twi, p, xb, bar, z);
#pragma unroll
      for (int k = 0; k < E; ++k) ysh[(h * P + grp) * NH + Y::j_of(0, t, k)] = csub(v[k], p);
    }
    __syncthreads();  // the exchange buffers become the stage
#pragma unroll
    for (int k = 0; k < E; ++k) {
      const int j = Y::j_of(0, t, k);
      n13_join(ysh[grp * NH + j], ysh[(P + grp) * NH + j], wfi, p, z, region + grp * NF, j);
    }
    __syncthreads();
    for (int j = tid; j < NF; j += THREADS) {
      uint32_t x[P];
#pragma unroll
      for (int g = 0; g < P; ++g) x[g] = region[g * NF + j];
      uint64_t r = modq_lift(garner_exact<P>(x, prm.S), prm.mq);
      if (c == 0) {
        const int p0 = rotated(r1, j);
        const uint64_t p0q = p0 >= 0 ? (uint64_t)p0 : Q - (uint64_t)(-p0);
        r = addq(r, mulq(prm.delta, p0q, prm.mq), Q);
      }
      out[c * NF + j] = r;
    }
    __syncthreads();  // the stage becomes the exchange buffers again
  }
}

// RLWE samples mod Q with a uniform key (key generation), N = 8192: the
// computation of rlwe_encrypt_q_kernel (a sk as the sum over the key's
// balanced 13-bit limbs of 2^(13 l) (a * sk_l), each limb product exact from
// three primes) with the split transforms.  skl: the limbs converted by
// bsk_to_ntt_n13_kernel with R = 1.  Shared memory: both halves' inverse
// results [2][P][4096], then the exchange buffers / lift stage [P][8192].
template <int EL, int P>
__global__ void __launch_bounds__(P * (1 << (12 - EL))) rlwe_encrypt_q_n13_kernel(const RlweEncQParams prm) {
  using Y = Layout<12, EL>;
  constexpr int NF = kN13, NH = kN13h, E = Y::E, G = Y::G, THREADS = P * G;
  constexpr int XW = n13_xwords<EL>();
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* ysh = reinterpret_cast<uint32_t*>(smem);  // [2 halves][P][NH]
  uint32_t* region = ysh + 2 * P * NH;                // [P][XW] exchange | [P][NF] stage
  const int64_t it = blockIdx.x;
  const uint64_t Q = prm.mq.Q;
  const uint64_t* a = prm.a + it * NF;
  const int64_t* e = prm.e + it * NF;
  uint64_t* out = prm.out + it * 2 * NF;
  const int tid = threadIdx.x;
  const int grp = tid / G;
  const int t = tid - grp * G;
  const uint32_t p = prm.S.p[grp];
  const uint32_t pneg = prm.S.pneg[grp];
  const uint32_t z = prm.S.zero;
  uint32_t* xb = region + grp * XW;
  const int bar = 1 + grp;
  // b starts as e + mu (component 0), a as given (+ mu on component 1); the
  // lift below visits the same j with the same thread
  for (int j = tid; j < NF; j += THREADS) {
    const int64_t ev = e[j];
    uint64_t b = ev >= 0 ? (uint64_t)ev % Q : negq((uint64_t)(-ev) % Q, Q);
    uint64_t av = a[j];
    if (j == 0) {
      if (prm.comp[it] == 0) b = addq(b, prm.mu[it], Q);
      else av = addq(av, prm.mu[it], Q);
    }
    out[j] = b;
    out[NF + j] = av;
  }
  const uint2 wfi = prm.S.tw_inv[(size_t)grp * 2 * NH];
  for (int l = 0; l < kSkLimbs; ++l) {
    for (int h = 0; h < 2; ++h) {
      const uint2* twf = prm.S.tw_fwd + ((size_t)grp * 2 + h) * NH;
      const uint2* twi = prm.S.tw_inv + ((size_t)grp * 2 + h) * NH;
      uint32_t v[E];
      n13_fwd_half<EL>(v, h, [&](int j) -> uint32_t { return mod_centred<uint64_t>(centre_q(a[j], Q), prm.S, grp); },
                       t, twf, p, xb, bar, z);
      const uint32_t* kl = prm.skl + (((size_t)l * P + grp) * 2 + h) * 2 * NH;  // component 0 of limb row l
#pragma unroll
      for (int k = 0; k < E; ++k) {
        const uint32_t x = csub(csub(v[k], 2 * p), p);
        const uint32_t kv = kl[(k >> 2) * 4 * G + t * 4 + (k & 3)];
        v[k] = csub(redc((uint64_t)x * kv, p, pneg), p);  // a sk_l N^-1
      }
      ntt_inv<12, EL, Y::K - 1>(v, t, twi, p, xb, bar, z);
#pragma unroll
      for (int k = 0; k < E; ++k) ysh[(h * P + grp) * NH + Y::j_of(0, t, k)] = csub(v[k], p);
    }
    __syncthreads();  // the exchange buffers become the stage
#pragma unroll
    for (int k = 0; k < E; ++k) {
      const int j = Y::j_of(0, t, k);
      n13_join(ysh[grp * NH + j], ysh[(P + grp) * NH + j], wfi, p, z, region + grp * NF, j);
    }
    __syncthreads();
    const uint64_t w = modq_u128((unsigned __int128)1 << (kSkLimbBits * l), prm.mq);  // 2^(13 l) mod Q
    for (int j = tid; j < NF; j += THREADS) {
      uint32_t x[P];
#pragma unroll
      for (int g = 0; g < P; ++g) x[g] = region[g * NF + j];
      const uint64_t X = modq_lift(garner_exact<P>(x, prm.S), prm.mq);
      out[j] = addq(out[j], mulq(X, w, prm.mq), Q);
    }
    __syncthreads();  // the stage becomes the exchange buffers again
  }
}

}  // namespace fdfb
