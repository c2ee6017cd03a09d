// Key switching on the fifth-generation tensor cores (tcgen05), exact.
//
// The key switch of the appendix figure "Key switching algorithm and its
// setup",
//   out[m][c] = [c = 0] b_m - sum_{i < n_in} sum_{j < l} Decomp(a_{m,i})_j key[i l + j][c]  (mod 2^w),
// is a dense integer contraction D (batch x K digits, K = n_in l) times key
// (K x cols words).  Tensor cores multiply f16 operands into fp32 sums, so
// the contraction is made exact by splitting:
//   - every key word into S balanced limbs of b bits, key = sum_s 2^{b s}
//     k_s (mod 2^w) with k_s in [-2^{b-1}, 2^{b-1}), exact in f16 (b <= 12);
//   - the K digits (in [0, B), B <= 2^11, exact in f16) into chunks of kappa
//     terms with kappa (B - 1) 2^{b-1} <= 2^23, so that every partial fp32
//     sum of a chunk is an integer of magnitude at most 2^23 and therefore
//     exact whatever the order of accumulation.
// Each (limb, chunk) sum is read back from tensor memory, converted to an
// integer and added, shifted by b s bits, into 64-bit sums mod 2^w.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace fdfb {

// Tensor-core form of one key-switching key.
//
// Two kinds.  Power-of-two sets (exact = false): the words are residues mod
// 2^w and the result is [b, 0] - D K mod 2^w.  Prime-modulus sets (exact =
// true): the words are residues mod Q < 2^63 and the kernel writes the exact
// non-negative integer S = D K (below 2^96) as the two 64-bit words S mod
// 2^32 and S >> 32, the layout of the CUDA-core contraction's sums, for the
// reduction mod Q that follows; digits of more than 11 bits are split into
// two halves below 2^h and 2^(log2B - h) (D = D_lo + 2^h D_hi), and the limbs
// cover 65 bits so that their sum is the key word as an integer, not only
// modulo a power of two.
struct TcKsKey {
  void* limbs = nullptr;   // device [S][cols][K] f16
  size_t bytes = 0;
  CUtensorMap tmap;        // 3-D map of `limbs`: {K, cols, S}, 64 x BN x 1 boxes, 128-byte swizzle
  int S = 0, b = 0, kappa = 0;
  int K = 0, cols = 0, w = 0, ell = 0, log2B = 0, n_in = 0;
  bool exact = false;      // prime-modulus form
  int halves = 1, h = 0;   // digit halves (exact form, log2B > 11) and the low half's bits
  bool ready = false;
};

// Limb width, limb count and chunk length for digits below 2^dbits, K =
// n_in * ell terms and limbs covering `span` bits (host).  Returns false if
// no split keeps the chunks at least 64 terms long.
bool tc_ks_split(int dbits, int span, int n_in, int ell, int* b, int* S, int* kappa);

// Builds the limb form of a key given on the device in canonical layout
// [K][cols] words (K = n_in ell) and its tensor map; synchronises `s`.
// exact selects the prime-modulus form (w = 64, words in [0, Q), Q < 2^63).
// FDFB_ENOMEM / FDFB_ECUDA / FDFB_EINVAL on failure (then k.ready is false).
int tc_ks_prepare(TcKsKey& k, const void* key, int w, int n_in, int ell, int log2B, int cols, cudaStream_t s,
                  bool exact = false);
void tc_ks_release(TcKsKey& k);

// Bytes of the digit matrix a call on `batch` rows needs (f16 [halves][batch][K]).
size_t tc_ks_digits_bytes(const TcKsKey& k, int64_t batch);

// KeySwitch of ct[m] for m < batch: ct device [batch][n_in + 1] words,
// digits device scratch of tc_ks_digits_bytes(k, batch) bytes, rtrunc the
// decomposition's rounding bits (w - l log2 B when positive; 0 for the exact
// form).  Power-of-two form: out device [batch][cols] words, the key-switched
// samples.  Exact form: out device [batch][2 cols] uint64, the sums (S mod
// 2^32 at [m][c], S >> 32 at [m][cols + c]).  A bounded device-side wait
// that expires latches FDFB_ETIMEOUT in *err.  Stream ordered.
int tc_keyswitch(const TcKsKey& k, const void* ct, int64_t batch, int rtrunc, void* out, void* digits,
                 int* err, cudaStream_t s);

}  // namespace fdfb
