// Core arithmetic shared by every kernel of the FDFB library: 30-bit NTT
// primes, Shoup and Montgomery modular products, Garner reconstruction into
// Z_{2^w}, and the register/shared-memory layouts of the negacyclic NTT.
//
// The negacyclic products of the method (extProd of Definition "External
// Product", PubMux, RLWE encryption) are computed exactly: the integer
// product is formed modulo P primes p_i = 1 (mod 2^14), p_i < 2^30, by a
// merged-twist negacyclic NTT, then lifted to the centred integer by Garner's
// mixed-radix algorithm and reduced mod 2^w.  The lift is exact whenever
// |result| < prod(p_i)/2, which the host checks for each parameter set.
//
// Everything here is __host__ __device__ so the index arithmetic of the
// transform can be exercised on the CPU.
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#include <cuda_runtime.h>
#define FD_HD __host__ __device__ __forceinline__
#else
#define FD_HD inline
struct uint2 { uint32_t x, y; };
#endif

namespace fdfb {

constexpr int kMaxPrimes = 4;
// Largest primes below 2^30 that are 1 mod 2^14 (so 2N | p - 1 for N <= 8192).
constexpr uint32_t kPrimes[kMaxPrimes] = {1073692673u, 1073643521u, 1073479681u, 1073430529u};
// Largest primes below (2^32 - 2^16) / 25 that are 1 mod 2^14 (the "lazy"
// family): a forward transform of inputs below 2^16 keeps every value below
// 2^16 + 24 p < 2^32 through 12 stages without reducing (bfly_fwd_lazy).
constexpr uint32_t kPrimesLazy[kMaxPrimes] = {171737089u, 171687937u, 171491329u, 171048961u};
// Prime family 0: kPrimes, 1: kPrimesLazy (host side).
inline uint32_t family_prime(int family, int i) { return family ? kPrimesLazy[i] : kPrimes[i]; }

FD_HD uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

FD_HD uint32_t umin32(uint32_t a, uint32_t b) { return a < b ? a : b; }

// x < 2m (m < 2^31)  ->  x mod m, via the unsigned-wrap minimum.
FD_HD uint32_t csub(uint32_t x, uint32_t m) { return umin32(x, x - m); }

// Shoup's product a*w mod p with precomputed wp = floor(w 2^32 / p):
// result in [0, 2p) for any 32-bit a (w < p < 2^31).
FD_HD uint32_t mul_shoup(uint32_t a, uint32_t w, uint32_t wp, uint32_t p) {
  uint32_t q = mulhi32(a, wp);
  return a * w - q * p;
}

// Shoup companion floor(w 2^32 / p) (host side helper).
inline uint32_t host_shoup(uint32_t w, uint32_t p) { return (uint32_t)(((uint64_t)w << 32) / p); }

// Montgomery reduction: x * 2^-32 mod p for x < 2^63, pneg = -p^-1 mod 2^32.
// Result < x/2^32 + p.
FD_HD uint32_t redc(uint64_t x, uint32_t p, uint32_t pneg) {
  uint32_t m = (uint32_t)x * pneg;
  return (uint32_t)((x + (uint64_t)m * p) >> 32);
}

// Per-(prime set, ring degree) constants, passed to kernels by value.
struct PrimeSet {
  int P;                             // number of primes in use
  uint32_t p[kMaxPrimes];
  uint32_t pneg[kMaxPrimes];         // -p^-1 mod 2^32
  uint32_t ones[kMaxPrimes];         // floor(2^32 / p): Shoup companion of 1
  uint32_t r32[kMaxPrimes];          // 2^32 mod p
  uint32_t r32s[kMaxPrimes];         // Shoup companion of r32
  uint32_t r64[kMaxPrimes];          // 2^64 mod p
  uint32_t ninv_m[kMaxPrimes];       // N^-1 * 2^32 mod p  (Montgomery form of N^-1)
  uint32_t ninv_ms[kMaxPrimes];      // Shoup companion of ninv_m
  uint32_t gc[kMaxPrimes][kMaxPrimes];   // Garner: p_i^-1 mod p_j (i < j)
  uint32_t gcs[kMaxPrimes][kMaxPrimes];  // Shoup companions
  uint64_t M[kMaxPrimes + 1];        // prefix products of the primes, mod 2^64
  uint32_t half_top;                 // p_{P-1} / 2: sign threshold of the top digit
  uint32_t zero;                     // always 0 (see bfly_fwd)
  const uint2* tw_fwd;               // [P][N] (psi^brv(k), Shoup) forward twiddles
  const uint2* tw_inv;               // [P][N] (psi^-brv(k), Shoup) inverse twiddles
};

// Residue of a w-bit word (unsigned) modulo p.
FD_HD uint32_t mod_u32(uint32_t x, const PrimeSet& S, int i) {
  // Shoup's product by 1 (companion floor(2^32/p)) lands in [0, 2p).
  const uint32_t p = S.p[i];
  return csub(mul_shoup(x, 1u, S.ones[i], p), p);
}
FD_HD uint32_t mod_u64(uint64_t x, const PrimeSet& S, int i) {
  uint32_t p = S.p[i];
  uint32_t hi = mul_shoup((uint32_t)(x >> 32), S.r32[i], S.r32s[i], p);  // [0, 2p)
  uint32_t lo = mod_u32((uint32_t)x, S, i);                               // [0, p)
  return csub(csub(hi, p) + lo, p);
}
// Residue of the centred value of a w-bit word (x in [-2^{w-1}, 2^{w-1})).
template <typename W>
FD_HD uint32_t mod_centred(W x, const PrimeSet& S, int i);
template <>
FD_HD uint32_t mod_centred<uint32_t>(uint32_t x, const PrimeSet& S, int i) {
  uint32_t r = mod_u32(x, S, i);
  uint32_t c = (x >> 31) ? S.r32[i] : 0u;
  return csub(r + S.p[i] - c, S.p[i]);
}
template <>
FD_HD uint32_t mod_centred<uint64_t>(uint64_t x, const PrimeSet& S, int i) {
  uint32_t r = mod_u64(x, S, i);
  uint32_t c = (x >> 63) ? S.r64[i] : 0u;
  return csub(r + S.p[i] - c, S.p[i]);
}
template <typename W>
FD_HD uint32_t mod_word(W x, const PrimeSet& S, int i);
template <>
FD_HD uint32_t mod_word<uint32_t>(uint32_t x, const PrimeSet& S, int i) { return mod_u32(x, S, i); }
template <>
FD_HD uint32_t mod_word<uint64_t>(uint64_t x, const PrimeSet& S, int i) { return mod_u64(x, S, i); }

// Garner reconstruction for a compile-time prime count P.
template <int P>
FD_HD uint64_t garner_p(const uint32_t* x, const PrimeSet& S) {
  uint32_t y[P];
  y[0] = x[0];
  uint64_t X = y[0];
#pragma unroll
  for (int j = 1; j < P; ++j) {
    const uint32_t pj = S.p[j];
    uint32_t v = x[j];
#pragma unroll
    for (int i = 0; i < j; ++i) {
      const uint32_t d = v + 2 * pj - y[i];
      v = csub(mul_shoup(d, S.gc[i][j], S.gcs[i][j], pj), pj);
    }
    y[j] = v;
    X += S.M[j] * (uint64_t)v;
  }
  if (y[P - 1] > S.half_top) X -= S.M[P];
  return X;
}

// Garner reconstruction of the centred integer with residues x[i] in [0, p_i),
// reduced mod 2^64 (callers truncate to w bits).
FD_HD uint64_t garner(const uint32_t* x, const PrimeSet& S) {
  uint32_t y[kMaxPrimes];
  y[0] = x[0];
  uint64_t X = y[0];
#pragma unroll
  for (int j = 1; j < kMaxPrimes; ++j) {
    if (j < S.P) {
      uint32_t pj = S.p[j];
      uint32_t v = x[j];
#pragma unroll
      for (int i = 0; i < kMaxPrimes; ++i) {
        if (i < j) {
          // v <- (v - y_i) * p_i^-1 mod p_j ; y_i < p_i < 2 p_j
          uint32_t d = v + 2 * pj - y[i];
          v = csub(mul_shoup(d, S.gc[i][j], S.gcs[i][j], pj), pj);
        }
      }
      y[j] = v;
      X += S.M[j] * (uint64_t)v;
    }
  }
  if (y[S.P - 1] > S.half_top) X -= S.M[S.P];
  return X;
}

// ---------------------------------------------------------------------------
// Arithmetic modulo a pseudo-Mersenne modulus Q = 2^k - c (32 <= k <= 63,
// odd c < 2^20): the prime moduli of the paper's parameter sets (Table 1).
// Residues are uint64_t in [0, Q).
// ---------------------------------------------------------------------------
struct ModQ {
  uint64_t Q;  // 0: the set works modulo 2^w instead
  uint64_t c;  // Q = 2^k - c
  int k;
  int folds;   // folds that bring any value below 2^98 under 2Q (modq_lift)
  int folds64; // folds that bring any value below 2^62 under 2Q (modq_lift64)
};

// The fold count of modq_lift: the smallest f with F^f(2^98 - 1) < 2Q for
// the bound map F(u) = (u >> k) c + 2^k - 1 (1 for Q_1 and Q_2, 2 for Q_3,
// 5 for Q_4).
inline int modq_folds(uint64_t Q, uint64_t c, int k) {
  unsigned __int128 ub = (((unsigned __int128)1) << 98) - 1;
  int f = 0;
  while (ub >= (unsigned __int128)2 * Q && f < 16) {
    ub = (ub >> k) * c + ((((unsigned __int128)1) << k) - 1);
    ++f;
  }
  return f;
}

// The fold count of modq_lift64: the same map started from 2^62 - 1 (3 for
// Q_4; only used where registration has shown |x| < 2^59).
inline int modq_folds64(uint64_t Q, uint64_t c, int k) {
  unsigned __int128 ub = (((unsigned __int128)1) << 62) - 1;
  int f = 0;
  while (ub >= (unsigned __int128)2 * Q && f < 16) {
    ub = (ub >> k) * c + ((((unsigned __int128)1) << k) - 1);
    ++f;
  }
  return f;
}

// x mod Q for any x < 2^128: replace x by (x >> k) c + (x mod 2^k) while x
// has bits at or above 2^k (each fold divides the excess by 2^k / c >= 2^12,
// so a 128-bit x needs at most 11 folds; x < 2^96, the lifts' range, needs at
// most 6 at k = 32 and 2 at k >= 48), then one conditional subtraction
// (x < 2^k = Q + c <= 2Q).
FD_HD uint64_t modq_u128(unsigned __int128 x, const ModQ& m) {
  const unsigned __int128 lo_mask = (((unsigned __int128)1) << m.k) - 1;
#pragma unroll 1
  for (int it = 0; it < 12 && (x >> m.k) != 0; ++it) x = (x >> m.k) * m.c + (x & lo_mask);
  uint64_t r = (uint64_t)x;
  return r >= m.Q ? r - m.Q : r;
}
// residue of a signed integer |x| < 2^127
FD_HD uint64_t modq_i128(__int128 x, const ModQ& m) {
  if (x >= 0) return modq_u128((unsigned __int128)x, m);
  const uint64_t r = modq_u128((unsigned __int128)(-x), m);
  return r ? m.Q - r : 0;
}
// Residue of a lifted product sum, |x| < 2^96, without data-dependent
// branches: x + Q 2^(97-k) lies in (0, 2^98), m.folds folds (the same count
// for every thread) bring it below 2Q, one conditional subtraction ends it.
FD_HD uint64_t modq_lift(__int128 x, const ModQ& m) {
  const unsigned __int128 lo_mask = (((unsigned __int128)1) << m.k) - 1;
  unsigned __int128 y = (unsigned __int128)(x + (__int128)((unsigned __int128)m.Q << (97 - m.k)));
#pragma unroll 1
  for (int f = 0; f < m.folds; ++f) y = (y >> m.k) * m.c + (y & lo_mask);
  const uint64_t r = (uint64_t)y;
  return r >= m.Q ? r - m.Q : r;
}
// Residue of a lifted sum that fits 64 bits, |x| < 2^59 (two primes at k =
// 32): x + Q 2^(60-k) lies in (0, 2^62) (Q 2^(60-k) is in [2^59, 2^60)), and
// m.folds64 folds of the 64-bit value bring it below 2Q.  Needs k <= 60.
FD_HD uint64_t modq_lift64(int64_t x, const ModQ& m) {
  const uint64_t lo_mask = (1ull << m.k) - 1;
  uint64_t y = (uint64_t)(x + (int64_t)(m.Q << (60 - m.k)));
#pragma unroll 1
  for (int f = 0; f < m.folds64; ++f) y = (y >> m.k) * m.c + (y & lo_mask);
  return y >= m.Q ? y - m.Q : y;
}
FD_HD uint64_t addq(uint64_t a, uint64_t b, uint64_t Q) {
  const uint64_t s = a + b;  // < 2Q < 2^64
  return s >= Q ? s - Q : s;
}
FD_HD uint64_t subq(uint64_t a, uint64_t b, uint64_t Q) { return a >= b ? a - b : a + (Q - b); }
FD_HD uint64_t negq(uint64_t a, uint64_t Q) { return a ? Q - a : 0; }
FD_HD uint64_t mulq(uint64_t a, uint64_t b, const ModQ& m) {
  return modq_u128((unsigned __int128)a * b, m);
}
// centred representative of a residue in [0, Q), as a 64-bit two's complement
FD_HD uint64_t centre_q(uint64_t x, uint64_t Q) { return x > Q / 2 ? x - Q : x; }

// The exact integer X in (-M/2, M/2), M = p_0 .. p_{P-1}, with residues
// x[i] in [0, p_i): Garner's mixed-radix digits y_j, X = sum_j y_j M_j,
// minus M when the top digit puts X in the upper half.
template <int P>
FD_HD __int128 garner_exact(const uint32_t* x, const PrimeSet& S) {
  uint32_t y[P];
  y[0] = x[0];
  unsigned __int128 X = y[0];
  unsigned __int128 Mj = 1;
#pragma unroll
  for (int j = 1; j < P; ++j) {
    const uint32_t pj = S.p[j];
    uint32_t v = x[j];
#pragma unroll
    for (int i = 0; i < j; ++i) {
      const uint32_t d = v + 2 * pj - y[i];
      v = csub(mul_shoup(d, S.gc[i][j], S.gcs[i][j], pj), pj);
    }
    y[j] = v;
    Mj *= S.p[j - 1];
    X += Mj * v;
  }
  if (y[P - 1] > S.half_top) X -= Mj * S.p[P - 1];
  return (__int128)X;
}

// ---------------------------------------------------------------------------
// NTT register layouts.
//
// One NTT of size N = 2^L is computed by G = 2^(L-EL) threads, each holding
// E = 2^EL coefficients in registers.  The L butterfly stages are split into
// K passes of at most EL stages; inside a pass all butterflies are between
// registers of one thread, and between passes the coefficients are exchanged
// through shared memory.  Pass k < K-1 holds, in thread t and register r, the
// element
//     j = (t_hi << (L - k EL)) | (r << (L - (k+1) EL)) | t_lo,
// t_lo the low L-(k+1)EL bits of t; the last pass holds j = t E + r.
// The forward transform (Cooley-Tukey, merged psi twist, natural order in,
// bit-reversed order out) runs the passes 0..K-1; the inverse
// (Gentleman-Sande, bit-reversed in, natural out) runs them backwards.
// Stage s of the forward transform pairs bit L-1-s of j and uses twiddle
// index 2^s + (j >> (L - s)); the inverse stage on bit b uses
// (N >> (b+1)) + (j >> (b+1)).
// ---------------------------------------------------------------------------
template <int L, int EL>
struct Layout {
  static constexpr int N = 1 << L;
  static constexpr int E = 1 << EL;
  static constexpr int G = 1 << (L - EL);
  static constexpr int K = (L + EL - 1) / EL;
  static constexpr int LAST = L - (K - 1) * EL;  // stages in the last pass

  FD_HD static int j_of(int pass, int t, int r) {
    if (pass == K - 1) return t * E + r;
    const int lo_bits = L - (pass + 1) * EL;
    const int tlo = t & ((1 << lo_bits) - 1);
    const int thi = t >> lo_bits;
    return (thi << (L - pass * EL)) | (r << lo_bits) | tlo;
  }
  // stages of pass k: [first, first + len)
  FD_HD static constexpr int first(int pass) { return pass * EL; }
  FD_HD static constexpr int len(int pass) { return pass == K - 1 ? LAST : EL; }
  // register-bit of the butterfly partner for stage s of pass k
  FD_HD static constexpr int rbit(int pass, int s) {
    return pass == K - 1 ? (LAST - 1 - (s - first(pass))) : (EL - 1 - (s - first(pass)));
  }
};

// The butterflies' additions take a third operand z that is always zero but
// unknown to the compiler (a kernel argument): as three-input additions they
// issue on the ALU pipe instead of being turned into multiply-adds, which
// leaves the multiplier pipe to the Shoup products.
//
// Forward Cooley-Tukey butterfly (Harvey's lazy form): X, Y in [0, 4p) ->
// X + WY, X - WY + 2p, both in [0, 4p).
FD_HD void bfly_fwd(uint32_t& X, uint32_t& Y, uint2 w, uint32_t p, uint32_t z) {
  uint32_t x = umin32(X, X - 2 * p + z);
  uint32_t t = mul_shoup(Y, w.x, w.y, p);
  X = x + t + z;
  Y = x - t + 2 * p;
}
// Forward butterfly for the lazy prime family: X is not reduced, so each
// stage raises the bound on both outputs by less than 2p (X + WY and
// X - WY + 2p with WY in [0, 2p)).
FD_HD void bfly_fwd_lazy(uint32_t& X, uint32_t& Y, uint2 w, uint32_t p, uint32_t z) {
  const uint32_t x = X;
  const uint32_t t = mul_shoup(Y, w.x, w.y, p);
  X = x + t + z;
  Y = x - t + 2 * p;
}
// Inverse Gentleman-Sande butterfly: X, Y in [0, 2p) -> X + Y, (X - Y) W.
FD_HD void bfly_inv(uint32_t& X, uint32_t& Y, uint2 w, uint32_t p, uint32_t z) {
  uint32_t s = X + Y + z;
  s = umin32(s, s - 2 * p + z);
  uint32_t d = X - Y + 2 * p;
  X = s;
  Y = mul_shoup(d, w.x, w.y, p);
}

// Twiddle table position used by butterfly (thread t, register r) of stage s
// (forward stage s, or the inverse stage on bit L-1-s; both read the block
// [2^s, 2^(s+1)) at the same offsets).  The natural position is
// 2^s + (j >> (L - s)).  In the last pass j = t E + r, so thread t needs the
// C = 2^s / G consecutive entries 2^s + t C + c, c = r >> (L - s); the host
// stores those blocks transposed, at 2^s + c G + t, so the lanes of a warp
// read consecutive entries.
template <int L, int EL, int PASS>
FD_HD int tw_index(int s, int t, int r) {
  using Y = Layout<L, EL>;
  if (PASS == Y::K - 1) {
    const int c = r >> (L - s);
    return (1 << s) + c * Y::G + t;
  }
  return (1 << s) + (Y::j_of(PASS, t, r) >> (L - s));
}

#ifdef __CUDA_ARCH__
#define FD_LDG(ptr) __ldg(ptr)
#else
#define FD_LDG(ptr) (*(ptr))
#endif

// All stages of forward pass `pass` on the E registers of thread t.
template <int L, int EL, int PASS>
FD_HD void fwd_pass(uint32_t (&v)[1 << EL], int t, const uint2* tw, uint32_t p, uint32_t z) {
  using Y = Layout<L, EL>;
  constexpr int F = Y::first(PASS), LEN = Y::len(PASS);
#pragma unroll
  for (int s = F; s < F + LEN; ++s) {
    const int rb = Y::rbit(PASS, s);
#pragma unroll
    for (int r = 0; r < Y::E; ++r) {
      if (!(r & (1 << rb))) {
        const int ti = tw_index<L, EL, PASS>(s, t, r);
        const uint2 w = FD_LDG(tw + ti);
        bfly_fwd(v[r], v[r | (1 << rb)], w, p, z);
      }
    }
  }
}

// All stages of inverse pass `pass` (bits ascending) on thread t.
template <int L, int EL, int PASS>
FD_HD void inv_pass(uint32_t (&v)[1 << EL], int t, const uint2* tw, uint32_t p, uint32_t z) {
  using Y = Layout<L, EL>;
  constexpr int F = Y::first(PASS), LEN = Y::len(PASS);
  // stage s of the forward order touches j-bit L-1-s; run them in reverse
#pragma unroll
  for (int s = F + LEN - 1; s >= F; --s) {
    const int b = L - 1 - s;
    const int rb = Y::rbit(PASS, s);
#pragma unroll
    for (int r = 0; r < Y::E; ++r) {
      if (!(r & (1 << rb))) {
        const int ti = tw_index<L, EL, PASS>(L - 1 - b, t, r);
        const uint2 w = FD_LDG(tw + ti);
        bfly_inv(v[r], v[r | (1 << rb)], w, p, z);
      }
    }
  }
}

// The same passes on M polynomials held by the same threads at once: every
// twiddle is loaded once for the M butterflies that use it, and the M
// independent butterfly chains give the scheduler M times the parallelism.
template <int L, int EL, int PASS, int M, bool LZ = false>
FD_HD void fwd_pass_m(uint32_t (&v)[M][1 << EL], int t, const uint2* tw, uint32_t p, uint32_t z) {
  using Y = Layout<L, EL>;
  constexpr int F = Y::first(PASS), LEN = Y::len(PASS);
#pragma unroll
  for (int s = F; s < F + LEN; ++s) {
    const int rb = Y::rbit(PASS, s);
#pragma unroll
    for (int r = 0; r < Y::E; ++r) {
      if (!(r & (1 << rb))) {
        const int ti = tw_index<L, EL, PASS>(s, t, r);
        const uint2 w = FD_LDG(tw + ti);
#pragma unroll
        for (int m = 0; m < M; ++m) {
          if constexpr (LZ) bfly_fwd_lazy(v[m][r], v[m][r | (1 << rb)], w, p, z);
          else bfly_fwd(v[m][r], v[m][r | (1 << rb)], w, p, z);
        }
      }
    }
  }
}

template <int L, int EL, int PASS, int M>
FD_HD void inv_pass_m(uint32_t (&v)[M][1 << EL], int t, const uint2* tw, uint32_t p, uint32_t z) {
  using Y = Layout<L, EL>;
  constexpr int F = Y::first(PASS), LEN = Y::len(PASS);
#pragma unroll
  for (int s = F + LEN - 1; s >= F; --s) {
    const int b = L - 1 - s;
    const int rb = Y::rbit(PASS, s);
#pragma unroll
    for (int r = 0; r < Y::E; ++r) {
      if (!(r & (1 << rb))) {
        const int ti = tw_index<L, EL, PASS>(L - 1 - b, t, r);
        const uint2 w = FD_LDG(tw + ti);
#pragma unroll
        for (int m = 0; m < M; ++m) bfly_inv(v[m][r], v[m][r | (1 << rb)], w, p, z);
      }
    }
  }
}

// Shared-memory swizzle for the exchange buffers: XORs the five bank bits of
// j with a GF(2)-linear function of its higher bits, so that for every pass
// layout the 32 lanes of a warp hit 32 distinct banks for each register
// index.  Row b-5 of the table is the 5-bit mask that bit b of j flips; the
// tables were found by exhaustive search over the lane-bit patterns of the
// layouts above.
template <int L, int EL>
FD_HD constexpr uint32_t swz_mask(int b) {
  if (L == 8 && EL == 3) { constexpr uint8_t m[] = {4, 9, 18}; return m[b - 5]; }
  if (L == 9 && EL == 4) { constexpr uint8_t m[] = {2, 4, 8, 17}; return m[b - 5]; }
  if (L == 10 && EL == 4) { constexpr uint8_t m[] = {1, 4, 8, 18, 0}; return m[b - 5]; }
  if (L == 10 && EL == 5) { constexpr uint8_t m[] = {1, 2, 4, 8, 16}; return m[b - 5]; }
  if (L == 11 && EL == 4) { constexpr uint8_t m[] = {1, 2, 8, 20, 0, 0}; return m[b - 5]; }
  if (L == 11 && EL == 5) { constexpr uint8_t m[] = {1, 2, 4, 8, 16, 0}; return m[b - 5]; }
  if (L == 12 && EL == 4) { constexpr uint8_t m[] = {1, 2, 4, 24, 0, 0, 0}; return m[b - 5]; }
  return 0;
}

template <int L, int EL>
FD_HD uint32_t swz(uint32_t j) {
  uint32_t h = 0;
#pragma unroll
  for (int b = 5; b < L; ++b)
    if ((j >> b) & 1u) h ^= swz_mask<L, EL>(b);
  return j ^ h;
}

// Address of element j in a group's exchange buffer.  With 32 coefficients
// per thread the padded address j + (j >> 5) is bank-conflict free for every
// pass layout, and since the thread part and the register part of j occupy
// disjoint bits it splits into base(t) + offset(r), the offset a compile-time
// constant.  Other shapes use the XOR swizzle above (base(t) ^ offset(r)).
template <int L, int EL>
struct Xch {
  static constexpr bool kAdditive = (EL == 5);
  static constexpr int kWords = kAdditive ? (1 << L) + ((1 << L) >> 5) : (1 << L);
  FD_HD static uint32_t addr(uint32_t j) { return kAdditive ? j + (j >> 5) : swz<L, EL>(j); }
  FD_HD static uint32_t join(uint32_t base, uint32_t off) { return kAdditive ? base + off : base ^ off; }
};

// Exchange buffer of two polynomials transformed together: the two words of
// position j form one 64-bit word at index addr(j).  A 64-bit shared access
// is served per half-warp, so for every pass layout and register index the
// 16 lanes of each half-warp must hit 16 distinct 8-byte banks (addr mod 16).
// With 16 coefficients per thread the padded index j + (j >> 4) does this
// (checked exhaustively for N = 2^9 .. 2^12); it is additive over the
// disjoint thread and register bits of j, so each access is a per-thread
// base plus a compile-time offset.  N = 2^8 with 8 coefficients per thread has
// no such padding and uses an XOR swizzle of the low four bits instead
// (masks found by exhaustive search).
template <int L, int EL>
struct Xch64 {
  static constexpr bool kAdditive = (EL == 4);
  static constexpr int kEntries = kAdditive ? (1 << L) + ((1 << L) >> 4) : (1 << L);
  FD_HD static constexpr uint32_t mask(int b) {
    if (L == 8 && EL == 3) { constexpr uint8_t m[] = {1, 4, 10, 0}; return m[b - 4]; }
    return 0u;
  }
  FD_HD static uint32_t addr(uint32_t j) {
    if (kAdditive) return j + (j >> 4);
    uint32_t h = 0;
#pragma unroll
    for (int b = 4; b < L; ++b)
      if ((j >> b) & 1u) h ^= mask(b);
    return j ^ h;
  }
  FD_HD static uint32_t join(uint32_t base, uint32_t off) { return kAdditive ? base + off : base ^ off; }
};

}  // namespace fdfb
