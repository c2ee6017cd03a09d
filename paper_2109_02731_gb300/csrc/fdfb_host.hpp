// Host-side construction of the NTT constants: roots of unity, bit-reversed
// twiddle tables with Shoup companions, Montgomery and Garner constants.
#pragma once
#include <stdint.h>

#include <vector>

#include "fdfb_core.cuh"

namespace fdfb {
namespace host {

inline uint64_t mulmod(uint64_t a, uint64_t b, uint64_t m) {
  return (uint64_t)((unsigned __int128)a * b % m);
}
inline uint64_t powmod(uint64_t a, uint64_t e, uint64_t m) {
  uint64_t r = 1 % m;
  a %= m;
  while (e) {
    if (e & 1) r = mulmod(r, a, m);
    a = mulmod(a, a, m);
    e >>= 1;
  }
  return r;
}
inline uint32_t shoup(uint32_t w, uint32_t p) { return (uint32_t)(((uint64_t)w << 32) / p); }
inline uint32_t inv_mod(uint32_t a, uint32_t p) { return (uint32_t)powmod(a, p - 2, p); }
inline uint32_t bitrev(uint32_t x, int bits) {
  uint32_t r = 0;
  for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1u) << (bits - 1 - i);
  return r;
}

// Smallest generator of Z_p^* (p prime).
inline uint32_t generator(uint32_t p) {
  uint32_t m = p - 1;
  std::vector<uint32_t> fac;
  for (uint32_t d = 2; (uint64_t)d * d <= m; ++d)
    if (m % d == 0) {
      fac.push_back(d);
      while (m % d == 0) m /= d;
    }
  if (m > 1) fac.push_back(m);
  for (uint32_t g = 2;; ++g) {
    bool ok = true;
    for (uint32_t f : fac)
      if (powmod(g, (p - 1) / f, p) == 1) { ok = false; break; }
    if (ok) return g;
  }
}

// Stores the blocks [2^s, 2^(s+1)) of one 2^L-entry twiddle table that the
// last register pass of a transform with 2^EL coefficients per thread reads
// transposed: entry 2^s + t C + c moves to 2^s + c G + t (see tw_index).
inline void transpose_last_pass(uint2* tab, int L, int EL) {
  const int K = (L + EL - 1) / EL, last = L - (K - 1) * EL;
  const uint32_t G = 1u << (L - EL);
  for (int s = L - last; s < L; ++s) {
    const uint32_t base = 1u << s, C = base / G;
    std::vector<uint2> blk(tab + base, tab + 2 * base);
    for (uint32_t t = 0; t < G; ++t)
      for (uint32_t c = 0; c < C; ++c) tab[base + c * G + t] = blk[t * C + c];
  }
}

// Fills S (except the table pointers) and the [P][N] forward/inverse twiddle
// tables for ring degree N = 2^L with the first P primes, for transforms that
// keep 2^EL coefficients per thread: the blocks [2^s, 2^(s+1)) read by the
// last register pass are stored transposed (see tw_index).
inline void make_prime_set(int P, int L, int EL, PrimeSet& S, std::vector<uint2>& fwd,
                           std::vector<uint2>& inv, int family = 0) {
  const uint32_t N = 1u << L;
  S.P = P;
  fwd.assign((size_t)P * N, uint2{0, 0});
  inv.assign((size_t)P * N, uint2{0, 0});
  for (int i = 0; i < kMaxPrimes; ++i) {
    const uint32_t p = family_prime(family, i);
    S.p[i] = p;
    uint32_t x = 1;  // Newton iteration for p^-1 mod 2^32
    for (int it = 0; it < 5; ++it) x *= 2u - p * x;
    S.pneg[i] = 0u - x;
    S.ones[i] = shoup(1, p);
    S.r32[i] = (uint32_t)(((uint64_t)1 << 32) % p);
    S.r32s[i] = shoup(S.r32[i], p);
    S.r64[i] = (uint32_t)mulmod(S.r32[i], S.r32[i], p);
    const uint32_t ninv = inv_mod(N % p, p);
    S.ninv_m[i] = (uint32_t)mulmod(ninv, S.r32[i], p);
    S.ninv_ms[i] = shoup(S.ninv_m[i], p);
    for (int j = 0; j < kMaxPrimes; ++j) {
      S.gc[i][j] = 0;
      S.gcs[i][j] = 0;
    }
  }
  for (int i = 0; i < kMaxPrimes; ++i)
    for (int j = i + 1; j < kMaxPrimes; ++j) {
      S.gc[i][j] = inv_mod(family_prime(family, i) % family_prime(family, j), family_prime(family, j));
      S.gcs[i][j] = shoup(S.gc[i][j], family_prime(family, j));
    }
  S.M[0] = 1;
  for (int i = 0; i < kMaxPrimes; ++i) S.M[i + 1] = S.M[i] * (uint64_t)family_prime(family, i);
  S.half_top = family_prime(family, P - 1) / 2;
  S.zero = 0;
  for (int i = 0; i < P; ++i) {
    const uint32_t p = family_prime(family, i);
    const uint32_t g = generator(p);
    const uint32_t psi = (uint32_t)powmod(g, (p - 1) / (2 * N), p);  // primitive 2N-th root
    const uint32_t psi_inv = inv_mod(psi, p);
    for (uint32_t k = 0; k < N; ++k) {
      uint32_t e = bitrev(k, L);
      uint32_t wf = (uint32_t)powmod(psi, e, p);
      uint32_t wi = (uint32_t)powmod(psi_inv, e, p);
      fwd[(size_t)i * N + k] = uint2{wf, shoup(wf, p)};
      inv[(size_t)i * N + k] = uint2{wi, shoup(wi, p)};
    }
    transpose_last_pass(&fwd[(size_t)i * N], L, EL);
    transpose_last_pass(&inv[(size_t)i * N], L, EL);
  }
}

// Constants and twiddle tables of the N = 2^13 transforms (fdfb_n13.cuh),
// which run as one split stage plus two 4096-point transforms: per prime a
// [2][4096] table for each direction whose half h holds, at 2^s + i (s < 12,
// i < 2^s), the N = 8192 table's entry 2^(s+1) + h 2^s + i (the twiddles the
// 8192-point transform applies to that half), with the last-pass blocks
// transposed for 2^EL coefficients per thread, and at entry 0 (read by no
// 4096-point pass) the split stage's twiddle, entry 1 of the 8192 table.
// S.ninv_m is 8192^-1 2^32.
inline void make_prime_set_n13(int P, int EL, PrimeSet& S, std::vector<uint2>& fwd, std::vector<uint2>& inv) {
  constexpr uint32_t NF = 8192, NH = 4096;
  std::vector<uint2> f12, i12;
  make_prime_set(P, 12, EL, S, f12, i12, 0);
  for (int i = 0; i < kMaxPrimes; ++i) {
    const uint32_t p = kPrimes[i];
    S.ninv_m[i] = (uint32_t)mulmod(inv_mod(NF % p, p), S.r32[i], p);
    S.ninv_ms[i] = shoup(S.ninv_m[i], p);
  }
  fwd.assign((size_t)P * NF, uint2{0, 0});
  inv.assign((size_t)P * NF, uint2{0, 0});
  std::vector<uint32_t> ff(NF), fi(NF);
  for (int i = 0; i < P; ++i) {
    const uint32_t p = kPrimes[i];
    const uint32_t psi = (uint32_t)powmod(generator(p), (p - 1) / (2 * NF), p);  // primitive 2N-th root
    const uint32_t psi_inv = inv_mod(psi, p);
    for (uint32_t k = 0; k < NF; ++k) {
      ff[k] = (uint32_t)powmod(psi, bitrev(k, 13), p);
      fi[k] = (uint32_t)powmod(psi_inv, bitrev(k, 13), p);
    }
    for (uint32_t h = 0; h < 2; ++h) {
      uint2* hf = &fwd[((size_t)i * 2 + h) * NH];
      uint2* hi = &inv[((size_t)i * 2 + h) * NH];
      hf[0] = uint2{ff[1], shoup(ff[1], p)};
      hi[0] = uint2{fi[1], shoup(fi[1], p)};
      for (int s = 0; s < 12; ++s)
        for (uint32_t x = 0; x < (1u << s); ++x) {
          const uint32_t e = (2u << s) + h * (1u << s) + x;
          hf[(1u << s) + x] = uint2{ff[e], shoup(ff[e], p)};
          hi[(1u << s) + x] = uint2{fi[e], shoup(fi[e], p)};
        }
      transpose_last_pass(hf, 12, EL);
      transpose_last_pass(hi, 12, EL);
    }
  }
}

// log2 of the largest |centred result| the prime set can lift exactly:
// the top Garner digit must stay below p_{P-1}/2 - 1 for both signs.
inline bool lift_is_exact(int P, long double max_abs, int family = 0) {
  long double m = 1;
  for (int i = 0; i < P - 1; ++i) m *= (long double)family_prime(family, i);
  return max_abs / m + 2.0L < (long double)(family_prime(family, P - 1) / 2);
}

}  // namespace host
}  // namespace fdfb
