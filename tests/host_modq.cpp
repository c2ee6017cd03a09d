// Host check of the library's mod-Q helpers (paper_2109_02731_gb300/csrc/
// fdfb_core.cuh, compiled as plain C++): the lift reduction modq_lift with
// the fold counts registration computes, the generic modq_u128 / modq_i128,
// and Garner's exact lift garner_exact against the integer it must return.
// Prints "ok" and exits 0 when every value matches.
#include <stdio.h>
#include <stdint.h>

#include <random>
#include <vector>

#include "fdfb_host.hpp"

using namespace fdfb;

static uint64_t ref_mod(__int128 x, uint64_t Q) {
  __int128 r = x % (__int128)Q;
  if (r < 0) r += Q;
  return (uint64_t)r;
}

int main() {
  const uint64_t Qs[4][2] = {{(1ull << 62) - 65535, 65535},
                             {(1ull << 63) - 278527, 278527},
                             {(1ull << 48) - 163839, 163839},
                             {(1ull << 32) - 139263, 139263}};
  const int ks[4] = {62, 63, 48, 32};
  const int want_folds[4] = {1, 1, 2, 5};
  std::mt19937_64 g(2109);
  long bad = 0;
  for (int i = 0; i < 4; ++i) {
    ModQ m{Qs[i][0], Qs[i][1], ks[i], modq_folds(Qs[i][0], Qs[i][1], ks[i]), 0};
    if (m.folds != want_folds[i]) {
      printf("k=%d: %d folds, expected %d\n", m.k, m.folds, want_folds[i]);
      ++bad;
    }
    const __int128 lim = (__int128)1 << 96;
    const __int128 edges[] = {0, 1, -1, lim - 1, -(lim - 1), (__int128)m.Q, -(__int128)m.Q,
                              (__int128)m.Q - 1, (__int128)m.Q + 1};
    for (__int128 x : edges) {
      bad += modq_lift(x, m) != ref_mod(x, m.Q);
      bad += modq_i128(x, m) != ref_mod(x, m.Q);
    }
    for (int it = 0; it < 300000; ++it) {
      const unsigned __int128 u = ((unsigned __int128)g() << 64) | g();
      const int bits = 1 + (int)(g() % 96);
      __int128 x = (__int128)(u & ((((unsigned __int128)1) << bits) - 1));
      if (g() & 1) x = -x;
      bad += modq_lift(x, m) != ref_mod(x, m.Q);
      bad += modq_i128(x, m) != ref_mod(x, m.Q);
      const uint64_t a = g() % m.Q, b = g() % m.Q;
      bad += mulq(a, b, m) != (uint64_t)(((unsigned __int128)a * b) % m.Q);
      bad += addq(a, b, m.Q) != (uint64_t)(((unsigned __int128)a + b) % m.Q);
      bad += subq(a, b, m.Q) != ref_mod((__int128)a - (__int128)b, m.Q);
    }
  }
  // the 64-bit lift reduction of the two-prime layouts (k <= 60, |x| < 2^59)
  for (int i = 2; i < 4; ++i) {
    ModQ m{Qs[i][0], Qs[i][1], ks[i], modq_folds(Qs[i][0], Qs[i][1], ks[i]),
           modq_folds64(Qs[i][0], Qs[i][1], ks[i])};
    const int64_t lim = ((int64_t)1 << 59) - 1;
    const int64_t edges[] = {0, 1, -1, lim, -lim, (int64_t)m.Q, -(int64_t)m.Q, (int64_t)m.Q - 1};
    for (int64_t x : edges) bad += modq_lift64(x, m) != ref_mod(x, m.Q);
    for (int it = 0; it < 300000; ++it) {
      const int bits = 1 + (int)(g() % 59);
      int64_t x = (int64_t)(g() & (((uint64_t)1 << bits) - 1));
      if (g() & 1) x = -x;
      bad += modq_lift64(x, m) != ref_mod(x, m.Q);
    }
  }
  // Garner's exact lift with two and three 30-bit primes
  for (int P = 2; P <= 3; ++P) {
    PrimeSet S{};
    std::vector<uint2> fwd, inv;
    host::make_prime_set(P, 8, 3, S, fwd, inv);
    // the range registration guarantees (host::lift_is_exact): the top
    // mixed-radix digit decides the sign, so |X| / (p_0 .. p_{P-2}) + 2 must
    // stay below p_{P-1} / 2
    unsigned __int128 m = 1;
    for (int j = 0; j < P - 1; ++j) m *= S.p[j];
    const __int128 lim = (__int128)(m * (S.p[P - 1] / 2 - 3));
    for (int it = 0; it < 200000; ++it) {
      const unsigned __int128 u = ((unsigned __int128)g() << 64) | g();
      __int128 X = (__int128)(u % (unsigned __int128)(2 * lim + 1)) - lim;  // in [-lim, lim]
      if (it == 0) X = -lim;
      if (it == 1) X = lim;
      uint32_t r[4];
      for (int j = 0; j < P; ++j) r[j] = (uint32_t)ref_mod(X, S.p[j]);
      const __int128 got = P == 2 ? garner_exact<2>(r, S) : garner_exact<3>(r, S);
      bad += got != X;
    }
  }
  // NTT constants of both prime families (fdfb_host.hpp make_prime_set):
  // p = 1 mod 2N, psi^N = -1 (psi = the twiddle at bit-reversed index 1),
  // Shoup companions floor(w 2^32 / p), -p^-1 mod 2^32, N^-1 2^32 mod p,
  // Garner's p_i^-1 mod p_j and the prefix products
  for (int family = 0; family <= 1; ++family)
    for (int L = 8; L <= 12; ++L) {
      const uint32_t N = 1u << L;
      const int EL = L == 8 ? 3 : 4;
      PrimeSet S{};
      std::vector<uint2> fwd, inv;
      host::make_prime_set(family ? 2 : 3, L, EL, S, fwd, inv, family);
      for (int i = 0; i < S.P; ++i) {
        const uint64_t p = S.p[i];
        bad += (p - 1) % (2 * N) != 0;
        bad += fwd[(size_t)i * N].x != 1;
        const uint64_t w1 = fwd[(size_t)i * N + 1].x;  // psi^(N/2)
        bad += host::mulmod(w1, w1, p) != p - 1;     // psi^N = -1
        bad += host::mulmod(w1, inv[(size_t)i * N + 1].x, p) != 1;
        bad += fwd[(size_t)i * N + 1].y != (uint32_t)((w1 << 32) / p);
        bad += (uint32_t)(S.pneg[i] * (uint32_t)p) != 0xffffffffu;
        bad += host::mulmod(S.ninv_m[i], N, p) != ((uint64_t)1 << 32) % p;
        for (int j = i + 1; j < S.P; ++j) bad += host::mulmod(S.gc[i][j], p % S.p[j], S.p[j]) != 1;
        bad += S.M[i + 1] != S.M[i] * p;
      }
    }
  if (bad) {
    printf("%ld mismatches\n", bad);
    return 1;
  }
  printf("ok\n");
  return 0;
}
