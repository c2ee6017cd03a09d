/*
 * FDFB oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, deliberately unoptimised CPU implementation of full-domain
 * functional bootstrapping (Kluczniak and Schild, "FDFB: Full Domain
 * Functional Bootstrapping Towards Practical Fully Homomorphic Encryption",
 * arXiv 2109.02731).  It exists to check the CUDA library: only the tests,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.
 * It shares no code, table or header with the CUDA library.
 *
 * Conventions
 *   - Every ring element lives in Z_q with q = 2^w (w <= 64); values are held
 *     in uint64_t and reduced with the mask 2^w - 1 (wrap-around arithmetic).
 *   - Polynomials are arrays of N coefficients in ascending powers of X
 *     (Notation paragraph of Section 2, Coefs()).
 *   - LWE ciphertexts are [b, a_1 .. a_n] and RLWE ciphertexts are the two
 *     polynomials [b, a] (Definition "Generalized Learning With Errors":
 *     b = <a, s> + e + m).  The phase is b - <a, s> (Definition "Phase").
 *   - Negacyclic products are computed by the schoolbook definition of
 *     multiplication in Z_q[X]/(X^N + 1): no transform of any kind.
 *
 * Readings of the paper (where it is silent, garbled or inconsistent):
 *   G1  lookup tables hold unscaled f(m) in Z_t; Delta enters once.
 *   G2  Bootstrap calls PubMux with (p_0, p_1) := (rotP'_1, rotP'_0), so an
 *       encrypted sign bit 1 (phase in [0, N)) selects rotP_0.
 *   G3  L_boot = t and l_boot = 1: one sign blind rotation, and the PubMux
 *       selector polynomial is (p_1 - p_0) mod t, a single digit.
 *   G4  BlindRotate applies X^{-sum a_i s_i} only; the X^{b_N} rotation is
 *       applied to the accumulator polynomials beforehand (Bootstrap figure).
 *   G5  Decomposition is truncated and unsigned: with r = max(0, w - l*beta),
 *       x~ = ((x + 2^{r-1}) mod 2^w) >> r, digit j = (x~ >> beta*(j-1)) & (B-1)
 *       against gadget value B^{j-1} * 2^r; GGSW rows are component major.
 *   G6  Every rounding is round-half-up.
 *   G7  NSgn(x) = 1 iff x > 0 (the LaTeX source redefines \ge as >).
 *   G8  SetupPolynomial runs m ascending, then e ascending; later writes win.
 *   G20 Several functions of one input share the sign part (ModSwitch, sign
 *       rotation, SampleExtract + Delta/2, packing KeySwitch); PubMux, the
 *       function rotation and the LWE KeySwitch run per function.
 *   G21 Optional balanced blind-rotation digits: the same x~ written with
 *       digits in [-B/2, B/2), carrying upward; the top carry is dropped
 *       (B^l 2^r = 2^w).  The key switches keep unsigned digits.
 *   G23 Optional output modulus t' (f: Z_t -> Z_t'): Delta' = q / t' scales
 *       the sign LWE and PubMux, the PubMux selector is reduced mod t', and
 *       SetupPolynomial's windows stay those of t.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef uint64_t u64;
typedef int64_t i64;
typedef uint8_t u8;

typedef struct {
    int32_t n, N, w, t;
    int32_t log2Bg, lg, log2Bks, lks, log2Bpk, lpk;
    int32_t signed_digits;  /* blind rotation decomposes into balanced digits (G21) */
    int32_t t_out;          /* output plaintext modulus t' (0: t' = t), G23 */
} or_params;

/* The output space Z_t' of f: Z_t -> Z_t' (footnote of Section 1.1: the
 * same method with a different message scaling). */
static int out_mod(const or_params* P) { return P->t_out > 0 ? P->t_out : P->t; }

static inline u64 wmask(int w) { return w >= 64 ? ~(u64)0 : (((u64)1 << w) - 1); }

static int g_threads = 1;

void or_set_threads(int n) { g_threads = n > 0 ? n : 1; }

int or_max_threads(void) {
#ifdef _OPENMP
    return omp_get_num_procs();
#else
    return 1;
#endif
}

static int in_parallel(void) {
#ifdef _OPENMP
    return omp_in_parallel();
#else
    return 0;
#endif
}

/* ------------------------------------------------------------------------
 * Ring arithmetic in R_{N,q} = Z_q[X]/(X^N + 1)  (Notation, Section 2)
 * ---------------------------------------------------------------------- */

/* out = a * b in Z_q[X]/(X^N+1), by the definition of the product:
 * coefficient k collects a_j b_{k-j} for j <= k, and -a_j b_{N+k-j} for j > k
 * (the wrapped terms pick up X^N = -1).  out may not alias a or b. */
void or_poly_mul(int w, int N, const u64* a, const u64* b, u64* out) {
    const u64 m = wmask(w);
    const int par = (N >= 512) && !in_parallel() && g_threads > 1;
#pragma omp parallel for if (par) num_threads(g_threads) schedule(static)
    for (int k = 0; k < N; ++k) {
        u64 acc = 0;
        for (int j = 0; j <= k; ++j) acc += a[j] * b[k - j];
        for (int j = k + 1; j < N; ++j) acc -= a[j] * b[N + k - j];
        out[k] = acc & m;
    }
}

/* out = p * X^k for any integer k (the monomials X^k form a cyclic group of
 * order 2N, X^N = -1: Section 1.2, footnote on the group G).  Term p_j X^j
 * moves to X^{j+k}; every full turn by N flips its sign. */
void or_poly_mul_xk(int w, int N, const u64* p, i64 k, u64* out) {
    const u64 m = wmask(w);
    i64 kk = k % (2 * (i64)N);
    if (kk < 0) kk += 2 * (i64)N;
    for (int j = 0; j < N; ++j) out[j] = 0;
    for (int j = 0; j < N; ++j) {
        i64 e = (i64)j + kk;             /* exponent in [0, 3N) */
        int neg = 0;
        while (e >= N) { e -= N; neg ^= 1; }
        out[e] = (neg ? (0 - p[j]) : p[j]) & m;
    }
}

/* Same rotation on a polynomial with signed integer coefficients (used for
 * the lookup-table polynomials, which live in Z before scaling). */
void or_poly_mul_xk_signed(int N, const i64* p, i64 k, i64* out) {
    i64 kk = k % (2 * (i64)N);
    if (kk < 0) kk += 2 * (i64)N;
    for (int j = 0; j < N; ++j) out[j] = 0;
    for (int j = 0; j < N; ++j) {
        i64 e = (i64)j + kk;
        int neg = 0;
        while (e >= N) { e -= N; neg ^= 1; }
        out[e] = neg ? -p[j] : p[j];
    }
}

/* ------------------------------------------------------------------------
 * Gadget and decomposition (Definitions "Gadget Matrix" and "Decomposition";
 * truncated unsigned reading G5)
 * ---------------------------------------------------------------------- */

static int trunc_bits(int w, int log2B, int ell) {
    int r = w - ell * log2B;
    return r > 0 ? r : 0;
}

/* The rounded, truncated value x~ whose base-B digits are the decomposition. */
u64 or_decomp_round(int w, int log2B, int ell, u64 x) {
    const u64 m = wmask(w);
    int r = trunc_bits(w, log2B, ell);
    if (r == 0) return x & m;
    return ((x + ((u64)1 << (r - 1))) & m) >> r;
}

/* Digits d_1..d_l of x (out[j-1] = d_j, d_1 least significant). */
void or_decomp(int w, int log2B, int ell, u64 x, u64* out) {
    u64 xt = or_decomp_round(w, log2B, ell, x);
    u64 bm = ((u64)1 << log2B) - 1;
    for (int j = 0; j < ell; ++j) {
        int sh = log2B * j;
        out[j] = sh < 64 ? ((xt >> sh) & bm) : 0;
    }
}

/* Balanced digits (reading G21) of x: the same rounded value x~, written as
 * sum_j d_j B^{j-1} with every d_j in [-B/2, B/2): take the base-B digits
 * from the least significant up, and whenever a digit plus the incoming carry
 * reaches B/2, subtract B and carry 1 into the next digit.  The carry out of
 * the top digit is dropped: B^l 2^r = 2^w vanishes mod 2^w, so
 * sum_j d_j g_j = x~ 2^r (mod 2^w) still holds. */
void or_decomp_signed(int w, int log2B, int ell, u64 x, i64* out) {
    u64 xt = or_decomp_round(w, log2B, ell, x);
    const i64 B = (i64)1 << log2B;
    i64 carry = 0;
    for (int j = 0; j < ell; ++j) {
        int sh = log2B * j;
        i64 d = (sh < 64 ? (i64)((xt >> sh) & (u64)(B - 1)) : 0) + carry;
        carry = d >= B / 2 ? 1 : 0;
        out[j] = d - carry * B;
    }
}

/* Gadget value g_j = B^{j-1} * 2^r mod 2^w for j = jj+1. */
u64 or_gadget(int w, int log2B, int ell, int jj) {
    int sh = trunc_bits(w, log2B, ell) + log2B * jj;
    if (sh >= w) return 0;
    return ((u64)1 << sh) & wmask(w);
}

/* ------------------------------------------------------------------------
 * Encryption, phase, decryption (Definitions "Generalized Learning With
 * Errors" and "Phase and Error"; Regev decryption of Section 1.2)
 * ---------------------------------------------------------------------- */

/* out = [b = <a,s> + e + mu, a_1..a_n] */
void or_lwe_encrypt(int w, int n, const u8* s, const u64* a, i64 e, u64 mu, u64* out) {
    const u64 m = wmask(w);
    u64 b = 0;
    for (int i = 0; i < n; ++i) b += a[i] * (u64)s[i];
    b += (u64)e + mu;
    out[0] = b & m;
    for (int i = 0; i < n; ++i) out[1 + i] = a[i] & m;
}

u64 or_lwe_phase(int w, int n, const u8* s, const u64* ct) {
    u64 ph = ct[0];
    for (int i = 0; i < n; ++i) ph -= ct[1 + i] * (u64)s[i];
    return ph & wmask(w);
}

/* Round(t * phase / q) mod t for power-of-two t (round half up, G6). */
u64 or_lwe_decrypt(int w, int n, int t, const u8* s, const u64* ct) {
    int logt = 0;
    while ((1 << logt) < t) ++logt;
    u64 ph = or_lwe_phase(w, n, s, ct);
    u64 half = (u64)1 << (w - logt - 1);
    return ((ph + half) & wmask(w)) >> (w - logt);
}

/* RLWE: out = [b = a*sk + e + mu, a] (two polynomials of N words). */
void or_rlwe_encrypt(int w, int N, const u8* sk, const u64* a, const i64* e,
                     const u64* mu, u64* out) {
    const u64 m = wmask(w);
    u64* skw = (u64*)calloc((size_t)N, sizeof(u64));
    for (int j = 0; j < N; ++j) skw[j] = sk[j];
    or_poly_mul(w, N, a, skw, out);
    for (int j = 0; j < N; ++j) {
        out[j] = (out[j] + (u64)e[j] + (mu ? mu[j] : 0)) & m;
        out[N + j] = a[j] & m;
    }
    free(skw);
}

/* Phase of an RLWE sample: b - a*sk. */
void or_rlwe_phase(int w, int N, const u8* sk, const u64* ct, u64* out) {
    const u64 m = wmask(w);
    u64* skw = (u64*)calloc((size_t)N, sizeof(u64));
    for (int j = 0; j < N; ++j) skw[j] = sk[j];
    or_poly_mul(w, N, ct + N, skw, out);
    for (int j = 0; j < N; ++j) out[j] = (ct[j] - out[j]) & m;
    free(skw);
}

/* ------------------------------------------------------------------------
 * Key generation
 * ---------------------------------------------------------------------- */

/* BRKeyGen (appendix figure "Blind Rotation and its setup") with u = {1}
 * (binary s, Table 1): brK[i] = RGSW(s[i]) = A + s[i] * G, every row of A a
 * GLWE(0) sample (Definition "Generalized-GSW Sample"), G = I_2 (x) g
 * (Definition "Gadget Matrix").  Row r = c*l + (j-1) adds s[i] * g_j to
 * component c (0 = b, 1 = a).
 * bsk_a, bsk_e: [n][2l][N];  out: [n][2l][2][N]. */
void or_keygen_bsk_row(const or_params* P, const u8* s, const u8* sk, const u64* a_row,
                       const i64* e_row, int i, int r, u64* out) {
    const int N = P->N, w = P->w, l = P->lg;
    or_rlwe_encrypt(w, N, sk, a_row, e_row, NULL, out);
    int c = r / l, j = r % l;
    u64 g = or_gadget(w, P->log2Bg, l, j);
    out[(size_t)c * N + 0] = (out[(size_t)c * N + 0] + (u64)s[i] * g) & wmask(w);
}

void or_keygen_bsk(const or_params* P, const u8* s, const u8* sk, const u64* bsk_a,
                   const i64* bsk_e, u64* out) {
    const int n = P->n, N = P->N, l = P->lg;
#pragma omp parallel for num_threads(g_threads) schedule(dynamic, 1) if (g_threads > 1)
    for (int i = 0; i < n; ++i)
        for (int r = 0; r < 2 * l; ++r) {
            size_t row = (size_t)i * 2 * l + r;
            or_keygen_bsk_row(P, s, sk, bsk_a + row * N, bsk_e + row * N, i, r, out + row * 2 * N);
        }
}

/* KeySwitchSetup (appendix figure "Key switching algorithm and its setup")
 * for the packing key pK: pK[i][j] = RLWE_sk(s_F[i] * g_j) with s_F =
 * KeyExtract(sk) = Coefs(sk), the message a constant polynomial.
 * pk_a, pk_e: [N][lpk][N];  out: [N][lpk][2][N]. */
void or_keygen_pk_row(const or_params* P, const u8* sk, const u64* a_row, const i64* e_row,
                      int i, int j, u64* out) {
    const int N = P->N, w = P->w, l = P->lpk;
    or_rlwe_encrypt(w, N, sk, a_row, e_row, NULL, out);
    out[0] = (out[0] + (u64)sk[i] * or_gadget(w, P->log2Bpk, l, j)) & wmask(w);
}

void or_keygen_pk(const or_params* P, const u8* sk, const u64* pk_a, const i64* pk_e, u64* out) {
    const int N = P->N, l = P->lpk;
#pragma omp parallel for num_threads(g_threads) schedule(dynamic, 1) if (g_threads > 1)
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < l; ++j) {
            size_t row = (size_t)i * l + j;
            or_keygen_pk_row(P, sk, pk_a + row * N, pk_e + row * N, i, j, out + row * 2 * N);
        }
}

/* KeySwitchSetup for the LWE key-switching key: ksK[i][j] = LWE_s(s_F[i] g_j).
 * ksk_a: [N][lks][n]; ksk_e: [N][lks];  out: [N][lks][n+1]. */
void or_keygen_ksk(const or_params* P, const u8* sk, const u8* s, const u64* ksk_a,
                   const i64* ksk_e, u64* out) {
    const int n = P->n, N = P->N, w = P->w, l = P->lks;
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < l; ++j) {
            size_t row = (size_t)i * l + j;
            u64 mu = (u64)sk[i] * or_gadget(w, P->log2Bks, l, j);
            or_lwe_encrypt(w, n, s, ksk_a + row * n, ksk_e[row], mu, out + row * (n + 1));
        }
}

/* ------------------------------------------------------------------------
 * Homomorphic primitives (Section 2 and Appendix A)
 * ---------------------------------------------------------------------- */

/* ModSwitch (appendix figure "Modulus switching algorithm") from q = 2^w to
 * 2^k: x -> round(2^k x / 2^w) mod 2^k, round half up (G6).  ct has n+1
 * words; out receives n+1 values in [0, 2^k). */
void or_modswitch(int w, int k, int n, const u64* ct, u64* out) {
    const u64 m = wmask(w);
    int sh = w - k;
    for (int i = 0; i <= n; ++i) {
        u64 x = ct[i] & m;
        out[i] = sh == 0 ? x : (((x + ((u64)1 << (sh - 1))) & m) >> sh);
    }
}

/* External product (Definition "External Product"): Decomp(d^T) * C.
 * C = one GGSW sample, [2l][2][N]; d = RLWE [2][N]; out = RLWE [2][N].
 * Row r = c*l + (j-1) of Decomp(d^T) is digit j of component c. */
void or_extprod(const or_params* P, const u64* C, const u64* d, u64* out) {
    const int N = P->N, w = P->w, l = P->lg;
    const u64 m = wmask(w);
    u64* dig = (u64*)malloc(sizeof(u64) * 2 * l * N);
    u64* tmp = (u64*)malloc(sizeof(u64) * N);
    u64 digits[64];
    i64 sdigits[64];
    for (int c = 0; c < 2; ++c)
        for (int k = 0; k < N; ++k) {
            if (P->signed_digits) {
                /* a negative digit enters the ring product as its value mod 2^w */
                or_decomp_signed(w, P->log2Bg, l, d[(size_t)c * N + k], sdigits);
                for (int j = 0; j < l; ++j) digits[j] = (u64)sdigits[j] & m;
            } else {
                or_decomp(w, P->log2Bg, l, d[(size_t)c * N + k], digits);
            }
            for (int j = 0; j < l; ++j) dig[((size_t)c * l + j) * N + k] = digits[j];
        }
    memset(out, 0, sizeof(u64) * 2 * N);
    for (int r = 0; r < 2 * l; ++r)
        for (int col = 0; col < 2; ++col) {
            or_poly_mul(w, N, dig + (size_t)r * N, C + ((size_t)r * 2 + col) * N, tmp);
            for (int k = 0; k < N; ++k)
                out[(size_t)col * N + k] = (out[(size_t)col * N + k] + tmp[k]) & m;
        }
    free(tmp);
    free(dig);
}

/* CMux (appendix figure "CMux gate"): extProd(C, g - h) + h. */
void or_cmux(const or_params* P, const u64* C, const u64* g, const u64* h, u64* out) {
    const int N = P->N;
    const u64 m = wmask(P->w);
    u64* d = (u64*)calloc((size_t)2 * N, sizeof(u64));
    for (int k = 0; k < 2 * N; ++k) d[k] = (g[k] - h[k]) & m;
    or_extprod(P, C, d, out);
    for (int k = 0; k < 2 * N; ++k) out[k] = (out[k] + h[k]) & m;
    free(d);
}

/* BlindRotate (appendix figure "Blind Rotation and its setup"), u = {1}:
 * for i = 1..n, acc <- CMux(brK[i], acc * X^{-a[i]}, acc).  ctN holds
 * [b, a_1..a_n] modulo 2N; b is not used here (reading G4).  acc: [2][N],
 * updated in place; bsk: [n][2l][2][N]. */
void or_blind_rotate(const or_params* P, const u64* bsk, u64* acc, const u64* ctN) {
    const int n = P->n, N = P->N, l = P->lg;
    u64* rot = (u64*)malloc(sizeof(u64) * 2 * N);
    u64* nxt = (u64*)malloc(sizeof(u64) * 2 * N);
    for (int i = 0; i < n; ++i) {
        i64 a = (i64)ctN[1 + i];
        or_poly_mul_xk(P->w, N, acc, -a, rot);
        or_poly_mul_xk(P->w, N, acc + N, -a, rot + N);
        or_cmux(P, bsk + (size_t)i * 2 * l * 2 * N, rot, acc, nxt);
        memcpy(acc, nxt, sizeof(u64) * 2 * N);
    }
    free(nxt);
    free(rot);
}

/* SampleExtract (appendix figure "Sample and key extraction") of coefficient
 * kk (0-based; the paper's k = kk + 1): b' = b_kk and
 * a'_i = NSgn(kk - i + 1) * a_{(kk - i) mod N}, with NSgn(x) = 1 iff x > 0
 * (reading G7).  rlwe: [2][N]; out: [N+1] = [b', a'_0 .. a'_{N-1}]. */
void or_sample_extract(int w, int N, const u64* rlwe, int kk, u64* out) {
    const u64 m = wmask(w);
    out[0] = rlwe[kk] & m;
    for (int i = 0; i < N; ++i) {
        int idx = ((kk - i) % N + N) % N;
        u64 v = rlwe[N + idx];
        out[1 + i] = ((kk - i + 1 > 0) ? v : (0 - v)) & m;
    }
}

/* KeySwitch (appendix figure "Key switching algorithm and its setup"):
 * c_out = [b, 0] - sum_{i,j} A[i,j] * key[i][j], A = Decomp(a).  The output
 * is any GLWE shape flattened to out_len words whose first word is the
 * constant coefficient of the b component (LWE: [b, a]; RLWE: [b poly, a
 * poly]).  key: [n_in][ell][out_len]; ct_in: [n_in + 1]. */
void or_keyswitch(int w, int n_in, int log2B, int ell, int out_len, const u64* key,
                  const u64* ct_in, u64* out) {
    const u64 m = wmask(w);
    u64 digits[64];
    for (int k = 0; k < out_len; ++k) out[k] = 0;
    out[0] = ct_in[0] & m;
    for (int i = 0; i < n_in; ++i) {
        or_decomp(w, log2B, ell, ct_in[1 + i], digits);
        for (int j = 0; j < ell; ++j) {
            const u64* kr = key + ((size_t)i * ell + j) * out_len;
            for (int k = 0; k < out_len; ++k) out[k] -= digits[j] * kr[k];
        }
    }
    for (int k = 0; k < out_len; ++k) out[k] &= m;
}

/* ------------------------------------------------------------------------
 * FDFB (Section 3)
 * ---------------------------------------------------------------------- */

/* SetupPolynomial (figure "functional bootstrapping", right): for m in
 * [0, t-1] and e in [-ceil(N/t), ceil(N/t)], y = round(2N/t) m + e mod 2N;
 * y = 0 sets p0[0] = F(m); y in [1, N-1] sets p0[N-y] = -F(m); y = N sets
 * p1[0] = -F(m); y in [N+1, 2N-1] sets p1[2N-y] = F(m).  F = f unscaled
 * (reading G1); loops in the paper's order, later writes win (G8).
 * f: [t]; p0, p1: [N] signed. */
void or_setup_polynomial(int N, int t, const i64* f, i64* p0, i64* p1) {
    const i64 twoN = 2 * (i64)N;
    const i64 E = ((i64)N + t - 1) / t;
    const i64 step = (twoN + t / 2) / t;
    for (int j = 0; j < N; ++j) { p0[j] = 0; p1[j] = 0; }
    for (int mm = 0; mm < t; ++mm)
        for (i64 e = -E; e <= E; ++e) {
            i64 y = ((step * mm + e) % twoN + twoN) % twoN;
            i64 v = f[mm];
            if (y == 0) p0[0] = v;
            if (y >= 1 && y <= N - 1) p0[N - y] = -v;
            if (y == N) p1[0] = -v;
            if (y >= N + 1 && y <= twoN - 1) p1[twoN - y] = v;
        }
}

/* Delta = q / t for q = 2^w and power-of-two t. */
static u64 delta_of(int w, int t) {
    int logt = 0;
    while ((1 << logt) < t) ++logt;
    return (u64)1 << (w - logt);
}

/* PubMux (figure "cmux-accumulator-builder", left) with L_boot = t, one
 * digit (reading G3): p = (p1 - p0) mod t, c_out = [Delta p0, 0] + p * c.
 * c: RLWE [2][N]; p0, p1: signed [N]; out: [2][N]. */
void or_pubmux(int w, int N, int t, const u64* c, const i64* p0, const i64* p1, u64* out) {
    const u64 m = wmask(w);
    const u64 delta = delta_of(w, t);
    u64* p = (u64*)malloc(sizeof(u64) * N);
    u64* tmp = (u64*)malloc(sizeof(u64) * N);
    for (int j = 0; j < N; ++j) {
        i64 d = (p1[j] - p0[j]) % t;
        if (d < 0) d += t;
        p[j] = (u64)d;
    }
    for (int col = 0; col < 2; ++col) {
        or_poly_mul(w, N, p, c + (size_t)col * N, tmp);
        for (int j = 0; j < N; ++j) out[(size_t)col * N + j] = tmp[j];
    }
    for (int j = 0; j < N; ++j) out[j] = (out[j] + delta * (u64)p0[j]) & m;
    free(tmp);
    free(p);
}

/* Intermediates of one bootstrap, any pointer may be NULL:
 *   ctN    [n+1]  ModSwitch(ct, q, 2N)
 *   sgn    [N+1]  SampleExtract of the sign rotation, plus Delta/2
 *   cR     [2N]   KeySwitch(sgn, pK)
 *   accF   [2N]   PubMux output (function accumulator)
 *   accBR  [2N]   function accumulator after the blind rotation
 *   cQ     [N+1]  SampleExtract(accBR) */
typedef struct {
    u64 *ctN, *sgn, *cR, *accF, *accBR, *cQ;
} or_debug;

/* Bootstrap (figure "functional-bootstrapping", left) under readings G1-G4,
 * in two parts.  The sign part depends on the input only: ModSwitch, the sign
 * accumulator, BlindRotate, SampleExtract + Delta/2 and the packing
 * KeySwitch, giving ctN [n+1] and cR [2N].  The function part takes one
 * table's rotation polynomials: PubMux, BlindRotate, SampleExtract and the
 * LWE KeySwitch, giving out [n+1].  Several functions of one input share the
 * sign part (Section "Application of Functional Bootstrapping": the first
 * bootstrap's accumulators are reused for the next function). */
static void or_fdfb_sign_part(const or_params* P, const u64* bsk, const u64* pk, const u64* ct,
                              u64* ctN, u64* cR, const or_debug* dbg) {
    const int n = P->n, N = P->N, w = P->w;
    const u64 m = wmask(w);
    const u64 delta = delta_of(w, out_mod(P));  /* Delta' = q / t' scales the sign LWE */
    int logN = 0;
    while ((1 << logN) < N) ++logN;

    u64* sgnP = (u64*)malloc(sizeof(u64) * N);
    u64* acc = (u64*)malloc(sizeof(u64) * 2 * N);
    u64* lwe = (u64*)malloc(sizeof(u64) * (N + 1));

    /* ct_N = ModSwitch(ct, q, 2N) */
    or_modswitch(w, logN + 1, n, ct, ctN);
    const i64 bN = (i64)ctN[0];
    if (dbg && dbg->ctN) memcpy(dbg->ctN, ctN, sizeof(u64) * (n + 1));

    /* sgnP = 1 - sum_{i=2}^{N} X^{i-1}, scaled by Delta/2, times X^{b_N};
     * acc = [that, 0] (l_boot = 1, L_boot^0 = 1). */
    for (int j = 0; j < N; ++j) sgnP[j] = (j == 0 ? delta / 2 : (0 - delta / 2)) & m;
    or_poly_mul_xk(w, N, sgnP, bN, acc);
    memset(acc + N, 0, sizeof(u64) * N);

    or_blind_rotate(P, bsk, acc, ctN);

    /* acc_c = SampleExtract(acc_BR, 1) + [Delta/2, 0] */
    or_sample_extract(w, N, acc, 0, lwe);
    lwe[0] = (lwe[0] + delta / 2) & m;
    if (dbg && dbg->sgn) memcpy(dbg->sgn, lwe, sizeof(u64) * (N + 1));

    /* BuildAcc, first half: acc_R = KeySwitch(acc_c, pK) */
    or_keyswitch(w, N, P->log2Bpk, P->lpk, 2 * N, pk, lwe, cR);
    if (dbg && dbg->cR) memcpy(dbg->cR, cR, sizeof(u64) * 2 * N);

    free(lwe); free(acc); free(sgnP);
}

static void or_fdfb_function_part(const or_params* P, const u64* bsk, const u64* ksk,
                                  const i64* rotP0, const i64* rotP1, const u64* ctN,
                                  const u64* cR, u64* out, const or_debug* dbg) {
    const int n = P->n, N = P->N, w = P->w, t = out_mod(P);
    const i64 bN = (i64)ctN[0];

    u64* acc = (u64*)malloc(sizeof(u64) * 2 * N);
    u64* lwe = (u64*)malloc(sizeof(u64) * (N + 1));
    i64* r0 = (i64*)malloc(sizeof(i64) * N);
    i64* r1 = (i64*)malloc(sizeof(i64) * N);

    /* BuildAcc, second half: PubMux(acc_R, rotP'_1, rotP'_0), rotP'_j = rotP_j X^{b_N} */
    or_poly_mul_xk_signed(N, rotP0, bN, r0);
    or_poly_mul_xk_signed(N, rotP1, bN, r1);
    or_pubmux(w, N, t, cR, r1, r0, acc);
    if (dbg && dbg->accF) memcpy(dbg->accF, acc, sizeof(u64) * 2 * N);

    /* acc_BR,F = BlindRotate(brK, acc_F, ct_N); c_Q = SampleExtract(., 1) */
    or_blind_rotate(P, bsk, acc, ctN);
    if (dbg && dbg->accBR) memcpy(dbg->accBR, acc, sizeof(u64) * 2 * N);
    or_sample_extract(w, N, acc, 0, lwe);
    if (dbg && dbg->cQ) memcpy(dbg->cQ, lwe, sizeof(u64) * (N + 1));

    /* c_Q,ksK = KeySwitch(c_Q, ksK); q = Q so the final ModSwitch is the identity */
    or_keyswitch(w, N, P->log2Bks, P->lks, n + 1, ksk, lwe, out);

    free(r1); free(r0); free(lwe); free(acc);
}

/* ct: [n+1]; rotP0, rotP1: signed [N] (SetupPolynomial output); out: [n+1]. */
void or_fdfb_bootstrap(const or_params* P, const u64* bsk, const u64* pk, const u64* ksk,
                       const i64* rotP0, const i64* rotP1, const u64* ct, u64* out,
                       const or_debug* dbg) {
    const int n = P->n, N = P->N;
    u64* ctN = (u64*)malloc(sizeof(u64) * (n + 1));
    u64* cR = (u64*)malloc(sizeof(u64) * 2 * N);
    or_fdfb_sign_part(P, bsk, pk, ct, ctN, cR, dbg);
    or_fdfb_function_part(P, bsk, ksk, rotP0, rotP1, ctN, cR, out, dbg);
    free(cR); free(ctN);
}

/* k functions of one input: rotP [k][2][N] signed (p0 then p1 per table);
 * outs [k][n+1]. */
void or_fdfb_bootstrap_multi(const or_params* P, const u64* bsk, const u64* pk, const u64* ksk,
                             const i64* rotP, int k, const u64* ct, u64* outs) {
    const int n = P->n, N = P->N;
    u64* ctN = (u64*)malloc(sizeof(u64) * (n + 1));
    u64* cR = (u64*)malloc(sizeof(u64) * 2 * N);
    or_fdfb_sign_part(P, bsk, pk, ct, ctN, cR, NULL);
    for (int j = 0; j < k; ++j)
        or_fdfb_function_part(P, bsk, ksk, rotP + (size_t)j * 2 * N, rotP + (size_t)j * 2 * N + N,
                              ctN, cR, outs + (size_t)j * (n + 1), NULL);
    free(cR); free(ctN);
}

/* A batch of bootstraps, one thread per ciphertext.  rotP: [n_luts][2][N]
 * signed (p0 then p1); lut_ids: [count]; cts, outs: [count][n+1]. */
void or_fdfb_batch(const or_params* P, const u64* bsk, const u64* pk, const u64* ksk,
                   const i64* rotP, const int32_t* lut_ids, int64_t count, const u64* cts,
                   u64* outs) {
    const int n = P->n, N = P->N;
#pragma omp parallel for num_threads(g_threads) schedule(dynamic, 1) if (g_threads > 1)
    for (int64_t c = 0; c < count; ++c) {
        const i64* rp = rotP + (size_t)lut_ids[c] * 2 * N;
        or_fdfb_bootstrap(P, bsk, pk, ksk, rp, rp + N, cts + (size_t)c * (n + 1),
                          outs + (size_t)c * (n + 1), NULL);
    }
}

/* The batch with k tables per input: lut_ids [count][k]; outs [count][k][n+1]. */
void or_fdfb_batch_multi(const or_params* P, const u64* bsk, const u64* pk, const u64* ksk,
                         const i64* rotP, const int32_t* lut_ids, int k, int64_t count,
                         const u64* cts, u64* outs) {
    const int n = P->n, N = P->N;
#pragma omp parallel for num_threads(g_threads) schedule(dynamic, 1) if (g_threads > 1)
    for (int64_t c = 0; c < count; ++c) {
        i64* sel = (i64*)malloc(sizeof(i64) * (size_t)k * 2 * N);
        for (int j = 0; j < k; ++j)
            memcpy(sel + (size_t)j * 2 * N, rotP + (size_t)lut_ids[c * k + j] * 2 * N,
                   sizeof(i64) * 2 * N);
        or_fdfb_bootstrap_multi(P, bsk, pk, ksk, sel, k, cts + (size_t)c * (n + 1),
                                outs + (size_t)c * k * (n + 1));
        free(sel);
    }
}

/* TFHE bootstrap (figure "TFHE Bootstrapping"): ct [n+1] under s, the
 * pre-rotation polynomial poly [N] (words mod q), out [n+1] under s.
 * ct_N = ModSwitch(ct, q, 2N); acc_F = [poly X^{b_N}, 0];
 * acc_BR = BlindRotate(brK, acc_F, ct_N); c_Q = SampleExtract(acc_BR, 1);
 * out = KeySwitch(c_Q, ksK) (ModSwitch Q -> q is the identity, q = Q). */
void or_tfhe_bootstrap(const or_params* P, const u64* bsk, const u64* ksk, const u64* poly,
                       const u64* ct, u64* out) {
    const int n = P->n, N = P->N, w = P->w;
    int logN = 0;
    while ((1 << logN) < N) ++logN;
    u64* ctN = (u64*)malloc(sizeof(u64) * (n + 1));
    u64* acc = (u64*)malloc(sizeof(u64) * 2 * N);
    u64* lwe = (u64*)malloc(sizeof(u64) * (N + 1));
    or_modswitch(w, logN + 1, n, ct, ctN);
    or_poly_mul_xk(w, N, poly, (i64)ctN[0], acc);
    memset(acc + N, 0, sizeof(u64) * N);
    or_blind_rotate(P, bsk, acc, ctN);
    or_sample_extract(w, N, acc, 0, lwe);
    or_keyswitch(w, N, P->log2Bks, P->lks, n + 1, ksk, lwe, out);
    free(lwe); free(acc); free(ctN);
}

/* A batch of TFHE bootstraps, one thread per ciphertext: polys [n_polys][N],
 * poly_ids [count], cts and outs [count][n+1]. */
void or_tfhe_batch(const or_params* P, const u64* bsk, const u64* ksk, const u64* polys,
                   const int32_t* poly_ids, int64_t count, const u64* cts, u64* outs) {
    const int n = P->n, N = P->N;
#pragma omp parallel for num_threads(g_threads) schedule(dynamic, 1) if (g_threads > 1)
    for (int64_t c = 0; c < count; ++c)
        or_tfhe_bootstrap(P, bsk, ksk, polys + (size_t)poly_ids[c] * N, cts + (size_t)c * (n + 1),
                          outs + (size_t)c * (n + 1));
}

/* LWE linear homomorphism (Lemma "Linear Homomorphism of GLWE samples"):
 * y_j = sum_i W[j][i] * x_i over LWE samples, integer weights.
 * W: [n_out][n_in] signed; x: [n_in][len]; y: [n_out][len]. */
void or_lwe_affine(int w, int len, int n_in, int n_out, const i64* W, const u64* x, u64* y) {
    const u64 m = wmask(w);
    for (int j = 0; j < n_out; ++j)
        for (int k = 0; k < len; ++k) {
            u64 acc = 0;
            for (int i = 0; i < n_in; ++i) acc += (u64)W[(size_t)j * n_in + i] * x[(size_t)i * len + k];
            y[(size_t)j * len + k] = acc & m;
        }
}
