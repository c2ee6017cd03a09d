// Host check of the N = 2^13 split transforms (paper_2109_02731_gb300/csrc/
// fdfb_n13.cuh and host::make_prime_set_n13, compiled as plain C++): one
// negacyclic product of 8192-coefficient polynomials modulo each prime, computed
// the way the kernels do -- the split stage on (j, j + 4096), the 4096-point
// register passes of Layout<12, EL> on each half with the half tables (the
// exchanges between passes emulated through an array indexed like the
// kernels' shared buffers), pointwise products scaled by 8192^-1, the
// 4096-point inverse passes and the joining stage -- against the schoolbook
// product mod p.  Prints "ok" and exits 0 when every coefficient matches.
#include <stdio.h>
#include <stdint.h>

#include <random>
#include <vector>

#include "fdfb_host.hpp"

using namespace fdfb;

constexpr int NF = 8192, NH = 4096;

using Regs = std::vector<std::vector<uint32_t>>;  // [G][E]

// the register arrays of the kernels are fixed-size; copy in and out
template <int EL, int PASS, bool FWD>
void run_pass(Regs& v, const uint2* tw, uint32_t p) {
  using Y = Layout<12, EL>;
  for (int t = 0; t < Y::G; ++t) {
    uint32_t r[1 << EL];
    for (int k = 0; k < Y::E; ++k) r[k] = v[t][k];
    if (FWD) fwd_pass<12, EL, PASS>(r, t, tw, p, 0u);
    else inv_pass<12, EL, PASS>(r, t, tw, p, 0u);
    for (int k = 0; k < Y::E; ++k) v[t][k] = r[k];
  }
}

// moves every thread's registers from the layout of pass `from` to that of `to`
template <int EL>
void exchange(Regs& v, int from, int to) {
  using Y = Layout<12, EL>;
  std::vector<uint32_t> buf(NH);
  for (int t = 0; t < Y::G; ++t)
    for (int k = 0; k < Y::E; ++k) buf[Y::j_of(from, t, k)] = v[t][k];
  for (int t = 0; t < Y::G; ++t)
    for (int k = 0; k < Y::E; ++k) v[t][k] = buf[Y::j_of(to, t, k)];
}

template <int EL, int PASS>
void fwd(Regs& v, const uint2* tw, uint32_t p) {
  using Y = Layout<12, EL>;
  if constexpr (PASS < Y::K) {
    if (PASS > 0) exchange<EL>(v, PASS - 1, PASS);
    run_pass<EL, PASS, true>(v, tw, p);
    fwd<EL, PASS + 1>(v, tw, p);
  }
}

template <int EL, int PASS>
void inv(Regs& v, const uint2* tw, uint32_t p) {
  if constexpr (PASS >= 0) {
    run_pass<EL, PASS, false>(v, tw, p);
    if (PASS > 0) exchange<EL>(v, PASS, PASS - 1);
    inv<EL, PASS - 1>(v, tw, p);
  }
}

// half h of the forward transform of x (values < p): the split stage, then
// the 4096-point passes; returns the registers in the last-pass layout
template <int EL>
Regs fwd_half(const std::vector<uint32_t>& x, int h, const uint2* tw, uint32_t p) {
  using Y = Layout<12, EL>;
  Regs v(Y::G, std::vector<uint32_t>(Y::E));
  for (int t = 0; t < Y::G; ++t)
    for (int k = 0; k < Y::E; ++k) {
      const int j = Y::j_of(0, t, k);
      uint32_t a = x[j], b = x[j + NH];
      bfly_fwd(a, b, tw[0], p, 0u);
      v[t][k] = h ? b : a;
    }
  fwd<EL, 0>(v, tw, p);
  return v;
}

template <int EL>
long check(int P, std::mt19937_64& g) {
  using Y = Layout<12, EL>;
  PrimeSet S{};
  std::vector<uint2> tf, ti;
  host::make_prime_set_n13(P, EL, S, tf, ti);
  long bad = 0;
  for (int gi = 0; gi < P; ++gi) {
    const uint32_t p = S.p[gi];
    std::vector<uint32_t> a(NF), b(NF);
    for (int j = 0; j < NF; ++j) {
      a[j] = (uint32_t)(g() % 512);  // a digit polynomial
      b[j] = (uint32_t)(g() % p);    // a key residue polynomial
    }
    a[NF - 1] = 511;
    b[NF - 1] = p - 1;
    // 8192^-1 from the Montgomery form the kernels fold into the key words
    const uint32_t ninv = (uint32_t)host::mulmod(S.ninv_m[gi], host::inv_mod(S.r32[gi], p), p);
    std::vector<uint32_t> y[2];
    for (int h = 0; h < 2; ++h) {
      const uint2* tw = &tf[((size_t)gi * 2 + h) * NH];
      const uint2* tv = &ti[((size_t)gi * 2 + h) * NH];
      Regs A = fwd_half<EL>(a, h, tw, p), B = fwd_half<EL>(b, h, tw, p);
      for (int t = 0; t < Y::G; ++t)
        for (int k = 0; k < Y::E; ++k)
          A[t][k] = (uint32_t)host::mulmod(host::mulmod(A[t][k] % p, B[t][k] % p, p), ninv, p);
      inv<EL, Y::K - 1>(A, tv, p);
      y[h].assign(NH, 0);
      for (int t = 0; t < Y::G; ++t)
        for (int k = 0; k < Y::E; ++k) y[h][Y::j_of(0, t, k)] = A[t][k] % p;
    }
    const uint2 wi = ti[(size_t)gi * 2 * NH];
    std::vector<uint32_t> got(NF);
    for (int j = 0; j < NH; ++j) {
      uint32_t x0 = y[0][j], x1 = y[1][j];
      bfly_inv(x0, x1, wi, p, 0u);
      got[j] = x0 % p;
      got[j + NH] = x1 % p;
    }
    // schoolbook negacyclic product mod p
    std::vector<uint64_t> want(NF, 0);
    for (int i = 0; i < NF; ++i) {
      if (!a[i]) continue;
      for (int j = 0; j < NF; ++j) {
        const uint64_t pr = (uint64_t)a[i] * b[j] % p;
        const int k = i + j;
        if (k < NF) want[k] = (want[k] + pr) % p;
        else want[k - NF] = (want[k - NF] + p - pr) % p;
      }
    }
    long bp = 0;
    for (int j = 0; j < NF; ++j) bp += got[j] != want[j];
    if (bp) printf("EL=%d prime %d: %ld mismatches\n", EL, gi, bp);
    bad += bp;
  }
  return bad;
}

int main() {
  std::mt19937_64 g(8192);
  long bad = check<4>(3, g) + check<5>(3, g);
  if (bad) return 1;
  printf("ok\n");
  return 0;
}
