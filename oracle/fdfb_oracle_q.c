/*
 * FDFB oracle, prime-modulus parameter sets -- TEST INFRASTRUCTURE ONLY.
 *
 * The paper's own parameter sets (Table 1) run the bootstrapping side modulo
 * a prime Q (Q_1 = 2^62 - 65535, Q_2 = 2^63 - 278527, Q_3 = 2^48 - 163839,
 * Q_4 = 2^32 - 139263) and the LWE side modulo q = 2N.  This file follows
 * the Bootstrap figure of Section 3 literally for that setting: exact
 * decomposition with l = ceil(log_B Q) digits, l_boot sign blind rotations
 * whose accumulators carry L_boot^(i-1) Delta/2, one packing key switch per
 * sign LWE, PubMux over the l_boot base-L_boot digits of p = p_1 - p_0 in
 * Z_Q, the function rotation, the LWE key switch, and ModSwitch(Q -> q).
 * Like fdfb_oracle.c it is plain and slow on purpose: negacyclic products by
 * the schoolbook definition, every residue reduced with 128-bit integer
 * division.  It shares nothing with the CUDA library.
 *
 * Conventions: values mod Q are uint64_t in [0, Q); signed noise and table
 * entries are int64_t and enter Z_Q by their residue; the LWE side (input
 * and output ciphertexts) lives in Z_q with q = 2N, handled by the
 * power-of-two routines of fdfb_oracle.c (or_lwe_encrypt / or_lwe_decrypt
 * with w = log2 q).
 *
 * Readings of the paper used here (besides G1, G2, G6, G7, G8 of
 * fdfb_oracle.c, which hold unchanged):
 *   G24 Delta_{Q,t} = round(Q / t) and "Delta_{Q,t} / 2" is round(Q / 2t):
 *       with Q prime neither divides exactly (the proofs assume t | Q).
 *   G25 q = 2N for every prime-Q set (Table 1), so the first ModSwitch
 *       (q -> 2N) is the identity; the input words are already in [0, 2N).
 *   G26 Decomposition is the paper's exact one: digits of x in [0, Q),
 *       least significant first, l = ceil(log_B Q), gadget B^(j-1).
 *   G27 The RLWE key is uniform in Z_Q^N (Table 1); the LWE key s is binary;
 *       s_F = Coefs(sk) is therefore a uniform vector mod Q.
 *   G28 PubMux keeps p = p_1 - p_0 in Z_Q (no reduction mod t) and splits it
 *       into l_boot = ceil(log_{L_boot} Q) digits: the literal algorithm.
 *   G29 t need not divide q = 2N (the CRT moduli of Section "Extending the
 *       Arithmetic" are pairwise coprime): inputs carry Delta_{q,t} m with
 *       Delta_{q,t} = round(2N / t), and decryption is round(t phase / q)
 *       mod t.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef uint64_t u64;
typedef int64_t i64;
typedef uint8_t u8;
typedef unsigned __int128 u128;

typedef struct {
    int32_t n, N, t;
    int32_t log2Bg, lg;       /* blind-rotation gadget, lg = ceil(log_Bg Q) */
    int32_t log2Bks, lks;     /* LWE -> LWE key switch */
    int32_t log2Bpk, lpk;     /* LWE -> RLWE packing key switch */
    int32_t log2Lboot, lboot; /* PubMux decomposition of p */
    uint64_t Q;
} orq_params;

/* ------------------------------------------------------------------------
 * Arithmetic in Z_Q
 * ---------------------------------------------------------------------- */

static u64 mq_add(u64 a, u64 b, u64 Q) { u128 s = (u128)a + b; return (u64)(s % Q); }
static u64 mq_sub(u64 a, u64 b, u64 Q) { return a >= b ? a - b : (u64)((u128)a + Q - b); }
static u64 mq_neg(u64 a, u64 Q) { return a == 0 ? 0 : Q - a; }
static u64 mq_mul(u64 a, u64 b, u64 Q) { return (u64)(((u128)a * b) % Q); }
/* residue of a signed integer */
static u64 mq_of(i64 x, u64 Q) {
    if (x >= 0) return (u64)x % Q;
    u64 m = (u64)(-(x + 1)) + 1;  /* |x| without overflow */
    return mq_neg(m % Q, Q);
}

u64 orq_mulmod(u64 a, u64 b, u64 Q) { return mq_mul(a % Q, b % Q, Q); }

/* Delta_{Q,t} = round(Q / t) and round(Q / 2t), round half up (G24, G6) */
u64 orq_delta(u64 Q, int t) { return (u64)(((u128)Q + (u64)(t / 2)) / (u64)t); }
u64 orq_delta_half(u64 Q, int t) { return (u64)(((u128)Q + (u64)t) / (u64)(2 * t)); }

/* B^k mod Q */
static u64 mq_pow2k(int log2B, int k, u64 Q) {
    u64 r = 1 % Q;
    for (int i = 0; i < k; ++i) r = mq_mul(r, ((u64)1 << log2B) % Q, Q);
    return r;
}

/* ------------------------------------------------------------------------
 * Polynomials in Z_Q[X] / (X^N + 1), schoolbook
 * ---------------------------------------------------------------------- */

/* out = a * b (both mod Q); out may not alias a or b */
void orq_poly_mul(int N, u64 Q, const u64* a, const u64* b, u64* out) {
    for (int k = 0; k < N; ++k) out[k] = 0;
    for (int i = 0; i < N; ++i) {
        if (a[i] == 0) continue;
        for (int j = 0; j < N; ++j) {
            u64 p = mq_mul(a[i], b[j], Q);
            int k = i + j;
            if (k < N) out[k] = mq_add(out[k], p, Q);
            else out[k - N] = mq_sub(out[k - N], p, Q);
        }
    }
}

/* out = p * X^k for any integer k (X^N = -1) */
void orq_poly_mul_xk(int N, u64 Q, const u64* p, i64 k, u64* out) {
    i64 kk = ((k % (2 * N)) + 2 * N) % (2 * N);
    for (int j = 0; j < N; ++j) {
        i64 d = j + kk;
        int neg = (int)((d / N) & 1);
        u64 v = p[j];
        out[d % N] = neg ? mq_neg(v, Q) : v;
    }
}

/* ------------------------------------------------------------------------
 * Decomposition (exact, G26)
 * ---------------------------------------------------------------------- */

void orq_decomp(int log2B, int ell, u64 x, u64* out) {
    for (int j = 0; j < ell; ++j)
        out[j] = (j * log2B >= 64) ? 0 : (x >> (j * log2B)) & (((u64)1 << log2B) - 1);
}

/* ------------------------------------------------------------------------
 * Encryption (Definition "Generalized Learning With Errors") mod Q
 * ---------------------------------------------------------------------- */

/* LWE under a key with entries mod Q (binary s, or s_F):
 * out = [b = <a, key> + e + mu, a] */
void orq_lwe_encrypt(int n, u64 Q, const u64* key, const u64* a, i64 e, u64 mu, u64* out) {
    u64 b = 0;
    for (int i = 0; i < n; ++i) b = mq_add(b, mq_mul(a[i], key[i], Q), Q);
    b = mq_add(mq_add(b, mq_of(e, Q), Q), mu % Q, Q);
    out[0] = b;
    for (int i = 0; i < n; ++i) out[1 + i] = a[i];
}

/* b - <a, key> mod Q */
u64 orq_lwe_phase(int n, u64 Q, const u64* key, const u64* ct) {
    u64 ph = ct[0];
    for (int i = 0; i < n; ++i) ph = mq_sub(ph, mq_mul(ct[1 + i], key[i], Q), Q);
    return ph;
}

/* RLWE: out = [b = a * sk + e + mu, a] */
void orq_rlwe_encrypt(int N, u64 Q, const u64* sk, const u64* a, const i64* e, const u64* mu,
                      u64* out) {
    orq_poly_mul(N, Q, a, sk, out);
    for (int j = 0; j < N; ++j) {
        u64 v = mq_add(out[j], mq_of(e[j], Q), Q);
        if (mu) v = mq_add(v, mu[j], Q);
        out[j] = v;
        out[N + j] = a[j];
    }
}

/* b - a * sk */
void orq_rlwe_phase(int N, u64 Q, const u64* sk, const u64* ct, u64* out) {
    orq_poly_mul(N, Q, ct + N, sk, out);
    for (int j = 0; j < N; ++j) out[j] = mq_sub(ct[j], out[j], Q);
}

/* ------------------------------------------------------------------------
 * Key generation (figures "Blind Rotation and its setup", "Key switching
 * algorithm and its setup"), exact gadget B^(j-1)
 * ---------------------------------------------------------------------- */

/* bsk[i][r] = GLWE_sk(0) + s_i B^(j-1) on component c, r = c lg + (j-1).
 * bsk_a, bsk_e: [n][2 lg][N];  out: [n][2 lg][2][N] */
void orq_keygen_bsk(const orq_params* P, const u8* s, const u64* sk, const u64* bsk_a,
                    const i64* bsk_e, u64* out) {
    const int n = P->n, N = P->N, l = P->lg;
    const u64 Q = P->Q;
    for (int i = 0; i < n; ++i)
        for (int r = 0; r < 2 * l; ++r) {
            size_t row = (size_t)i * 2 * l + r;
            u64* o = out + row * 2 * N;
            orq_rlwe_encrypt(N, Q, sk, bsk_a + row * N, bsk_e + row * N, NULL, o);
            int c = r / l, j = r % l;
            if (s[i]) o[(size_t)c * N] = mq_add(o[(size_t)c * N], mq_pow2k(P->log2Bg, j, Q), Q);
        }
}

/* pK[i][j] = RLWE_sk(s_F[i] B_pk^(j-1)), constant message polynomial.
 * pk_a, pk_e: [N][lpk][N];  out: [N][lpk][2][N] */
void orq_keygen_pk(const orq_params* P, const u64* sk, const u64* pk_a, const i64* pk_e, u64* out) {
    const int N = P->N, l = P->lpk;
    const u64 Q = P->Q;
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < l; ++j) {
            size_t row = (size_t)i * l + j;
            u64* o = out + row * 2 * N;
            orq_rlwe_encrypt(N, Q, sk, pk_a + row * N, pk_e + row * N, NULL, o);
            o[0] = mq_add(o[0], mq_mul(sk[i], mq_pow2k(P->log2Bpk, j, Q), Q), Q);
        }
}

/* ksK[i][j] = LWE_s(s_F[i] B_ks^(j-1)).  ksk_a: [N][lks][n]; ksk_e: [N][lks];
 * out: [N][lks][n+1] */
void orq_keygen_ksk(const orq_params* P, const u64* sk, const u8* s, const u64* ksk_a,
                    const i64* ksk_e, u64* out) {
    const int n = P->n, N = P->N, l = P->lks;
    const u64 Q = P->Q;
    u64* sw = (u64*)malloc((size_t)n * sizeof(u64));
    for (int i = 0; i < n; ++i) sw[i] = s[i];
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < l; ++j) {
            size_t row = (size_t)i * l + j;
            u64 mu = mq_mul(sk[i], mq_pow2k(P->log2Bks, j, Q), Q);
            orq_lwe_encrypt(n, Q, sw, ksk_a + row * n, ksk_e[row], mu, out + row * (n + 1));
        }
    free(sw);
}

/* ------------------------------------------------------------------------
 * Homomorphic primitives
 * ---------------------------------------------------------------------- */

/* External product (Definition "External Product"): out = sum_r D_r * C[r]
 * with D = Decomp(d) component major (row r = c lg + j: digit j of component
 * c of d).  C: [2 lg][2][N], d: [2][N], out: [2][N]. */
void orq_extprod(const orq_params* P, const u64* C, const u64* d, u64* out) {
    const int N = P->N, l = P->lg;
    const u64 Q = P->Q;
    u64* D = (u64*)malloc((size_t)2 * l * N * sizeof(u64));
    u64* tmp = (u64*)malloc((size_t)N * sizeof(u64));
    u64 dig[64];
    for (int c = 0; c < 2; ++c)
        for (int k = 0; k < N; ++k) {
            orq_decomp(P->log2Bg, l, d[(size_t)c * N + k], dig);
            for (int j = 0; j < l; ++j) D[((size_t)c * l + j) * N + k] = dig[j];
        }
    for (int k = 0; k < 2 * N; ++k) out[k] = 0;
    for (int r = 0; r < 2 * l; ++r)
        for (int col = 0; col < 2; ++col) {
            orq_poly_mul(N, Q, D + (size_t)r * N, C + ((size_t)r * 2 + col) * N, tmp);
            for (int k = 0; k < N; ++k) out[(size_t)col * N + k] = mq_add(out[(size_t)col * N + k], tmp[k], Q);
        }
    free(tmp);
    free(D);
}

/* BlindRotate (appendix figure "Blind Rotation and its setup", u = {1}):
 * for i = 1..n: acc <- acc + extProd(bsk[i], acc X^{-a_i} - acc).
 * acc: [2][N] in place; ctN: [n+1] values in [0, 2N). */
void orq_blind_rotate(const orq_params* P, const u64* bsk, u64* acc, const u64* ctN) {
    const int n = P->n, N = P->N, l = P->lg;
    const u64 Q = P->Q;
    u64* rot = (u64*)malloc((size_t)2 * N * sizeof(u64));
    u64* prod = (u64*)malloc((size_t)2 * N * sizeof(u64));
    for (int i = 0; i < n; ++i) {
        i64 a = (i64)ctN[1 + i];
        if (a == 0) continue;  /* d = 0 and Decomp(0) = 0: the step adds nothing */
        for (int c = 0; c < 2; ++c) {
            orq_poly_mul_xk(N, Q, acc + (size_t)c * N, -a, rot + (size_t)c * N);
            for (int k = 0; k < N; ++k) rot[(size_t)c * N + k] = mq_sub(rot[(size_t)c * N + k], acc[(size_t)c * N + k], Q);
        }
        orq_extprod(P, bsk + (size_t)i * 2 * l * 2 * N, rot, prod);
        for (int k = 0; k < 2 * N; ++k) acc[k] = mq_add(acc[k], prod[k], Q);
    }
    free(prod);
    free(rot);
}

/* SampleExtract of coefficient 0 (k = 1): b' = b_0, a'_0 = a_0,
 * a'_j = -a_{N-j} (NSgn(x) = 1 iff x > 0, G7). */
void orq_sample_extract(int N, u64 Q, const u64* rlwe, u64* out) {
    out[0] = rlwe[0];
    out[1] = rlwe[N];
    for (int j = 1; j < N; ++j) out[1 + j] = mq_neg(rlwe[N + (N - j)], Q);
}

/* KeySwitch (appendix figure "Key switching algorithm and its setup"):
 * out = [b, 0, .., 0] - sum_{i, j} Decomp(a_i)_j key[i][j]; key rows of
 * out_len words ([N][l][out_len]), ct = [b, a_1 .. a_{n_in}]. */
void orq_keyswitch(int n_in, u64 Q, int log2B, int ell, int out_len, const u64* key, const u64* ct,
                   u64* out) {
    u64 dig[64];
    for (int k = 0; k < out_len; ++k) out[k] = 0;
    out[0] = ct[0];
    for (int i = 0; i < n_in; ++i) {
        orq_decomp(log2B, ell, ct[1 + i], dig);
        for (int j = 0; j < ell; ++j) {
            if (dig[j] == 0) continue;
            const u64* row = key + ((size_t)i * ell + j) * out_len;
            for (int k = 0; k < out_len; ++k) out[k] = mq_sub(out[k], mq_mul(dig[j], row[k], Q), Q);
        }
    }
}

/* Decryption on the LWE side, q = 2^logq, any plaintext modulus t (the
 * pairwise coprime moduli of the CRT representation, Section "Extending the
 * Arithmetic"): round(t (b - <a, s>) / q) mod t, round half up (G6, G29). */
u64 orq_decrypt_q2n(int n, int logq, int t, const u8* s, const u64* ct) {
    const u64 q = (u64)1 << logq;
    u64 ph = ct[0];
    for (int i = 0; i < n; ++i) ph -= ct[1 + i] * (u64)s[i];
    ph &= q - 1;
    return (u64)((((u128)ph * (u64)t + q / 2) >> logq) % (u64)t);
}

/* ModSwitch (appendix figure "Modulus switching algorithm") from Q to
 * q = 2^logq: x -> round(q x / Q) mod q, round half up (G6). */
void orq_modswitch(u64 Q, int logq, int len, const u64* ct, u64* out) {
    const u64 q = (u64)1 << logq;
    for (int i = 0; i < len; ++i) {
        u128 num = (u128)2 * q * ct[i] + Q;
        out[i] = (u64)(num / ((u128)2 * Q)) & (q - 1);
    }
}

/* PubMux (figure "cmux-accumulator-builder", left) over l_boot RLWE samples
 * c_i = RLWE(m L^(i-1)):  p = p_1 - p_0 in Z_Q, its base-L_boot digits
 * p[i] (G28), out = [Delta p_0, 0] + sum_i p[i] * c_i.
 * c: [lboot][2][N]; p0, p1: signed polynomials; out: [2][N]. */
void orq_pubmux(const orq_params* P, const u64* c, const i64* p0, const i64* p1, u64* out) {
    const int N = P->N, lb = P->lboot;
    const u64 Q = P->Q;
    const u64 delta = orq_delta(Q, P->t);
    u64* dig = (u64*)malloc((size_t)lb * N * sizeof(u64));
    u64* tmp = (u64*)malloc((size_t)N * sizeof(u64));
    u64 dd[64];
    for (int k = 0; k < N; ++k) {
        u64 p = mq_sub(mq_of(p1[k], Q), mq_of(p0[k], Q), Q);
        orq_decomp(P->log2Lboot, lb, p, dd);
        for (int i = 0; i < lb; ++i) dig[(size_t)i * N + k] = dd[i];
    }
    for (int k = 0; k < N; ++k) {
        out[k] = mq_mul(delta, mq_of(p0[k], Q), Q);
        out[N + k] = 0;
    }
    for (int i = 0; i < lb; ++i)
        for (int col = 0; col < 2; ++col) {
            orq_poly_mul(N, Q, dig + (size_t)i * N, c + ((size_t)i * 2 + col) * N, tmp);
            for (int k = 0; k < N; ++k) out[(size_t)col * N + k] = mq_add(out[(size_t)col * N + k], tmp[k], Q);
        }
    free(tmp);
    free(dig);
}

/* Intermediates (each may be NULL): sgn [lboot][N+1], cR [lboot][2N],
 * accF [2N], cQ [N+1], cKS [n+1] (mod Q, before the final ModSwitch). */
typedef struct {
    u64* sgn;
    u64* cR;
    u64* accF;
    u64* cQ;
    u64* cKS;
} orq_debug;

/* Bootstrap (figure "functional-bootstrapping", left) on one LWE sample
 * ct [n+1] mod q = 2N; rotation polynomials rp0, rp1 from SetupPolynomial;
 * out [n+1] mod q. */
void orq_fdfb_bootstrap(const orq_params* P, const u64* bsk, const u64* pk, const u64* ksk,
                        const i64* rp0, const i64* rp1, const u64* ct, u64* out, const orq_debug* dbg) {
    const int n = P->n, N = P->N, lb = P->lboot;
    const u64 Q = P->Q;
    int logq = 0;
    while ((1 << logq) < 2 * N) ++logq;
    /* ModSwitch(ct, q, 2N) with q = 2N is the identity (G25) */
    u64* ctN = (u64*)malloc((size_t)(n + 1) * sizeof(u64));
    for (int i = 0; i <= n; ++i) ctN[i] = ct[i] & (u64)(2 * N - 1);
    const i64 bN = (i64)ctN[0];
    const u64 h = orq_delta_half(Q, P->t);
    /* sgnP = 1 - sum_{i>=2} X^{i-1}, sgnP_b = sgnP X^{b_N} */
    u64* sg = (u64*)malloc((size_t)N * sizeof(u64));
    u64* sgb = (u64*)malloc((size_t)N * sizeof(u64));
    for (int j = 0; j < N; ++j) sg[j] = j == 0 ? 1 : Q - 1;
    orq_poly_mul_xk(N, Q, sg, bN, sgb);
    u64* acc = (u64*)malloc((size_t)2 * N * sizeof(u64));
    u64* sgn = (u64*)malloc((size_t)lb * (N + 1) * sizeof(u64));
    for (int i = 0; i < lb; ++i) {
        const u64 sc = mq_mul(mq_pow2k(P->log2Lboot, i, Q), h, Q);  /* L_boot^(i-1) Delta/2 */
        for (int j = 0; j < N; ++j) {
            acc[j] = mq_mul(sc, sgb[j], Q);
            acc[N + j] = 0;
        }
        orq_blind_rotate(P, bsk, acc, ctN);
        u64* s_i = sgn + (size_t)i * (N + 1);
        orq_sample_extract(N, Q, acc, s_i);
        s_i[0] = mq_add(s_i[0], sc, Q);
    }
    /* rotP'_j = rotP_j X^{b_N} (signed, entries in (-t, t)) */
    i64* r0 = (i64*)malloc((size_t)N * sizeof(i64));
    i64* r1 = (i64*)malloc((size_t)N * sizeof(i64));
    for (int j = 0; j < N; ++j) {
        i64 d = j + bN;
        int neg = (int)((d / N) & 1);
        r0[d % N] = neg ? -rp0[j] : rp0[j];
        r1[d % N] = neg ? -rp1[j] : rp1[j];
    }
    /* BuildAcc: key switch every sign LWE to RLWE, then PubMux with
     * (p_0, p_1) := (rotP'_1, rotP'_0) (G2) */
    u64* cR = (u64*)malloc((size_t)lb * 2 * N * sizeof(u64));
    for (int i = 0; i < lb; ++i)
        orq_keyswitch(N, Q, P->log2Bpk, P->lpk, 2 * N, pk, sgn + (size_t)i * (N + 1), cR + (size_t)i * 2 * N);
    orq_pubmux(P, cR, r1, r0, acc);
    if (dbg && dbg->accF) memcpy(dbg->accF, acc, (size_t)2 * N * sizeof(u64));
    orq_blind_rotate(P, bsk, acc, ctN);
    u64* cQ = (u64*)malloc((size_t)(N + 1) * sizeof(u64));
    orq_sample_extract(N, Q, acc, cQ);
    u64* cKS = (u64*)malloc((size_t)(n + 1) * sizeof(u64));
    orq_keyswitch(N, Q, P->log2Bks, P->lks, n + 1, ksk, cQ, cKS);
    orq_modswitch(Q, logq, n + 1, cKS, out);
    if (dbg) {
        if (dbg->sgn) memcpy(dbg->sgn, sgn, (size_t)lb * (N + 1) * sizeof(u64));
        if (dbg->cR) memcpy(dbg->cR, cR, (size_t)lb * 2 * N * sizeof(u64));
        if (dbg->cQ) memcpy(dbg->cQ, cQ, (size_t)(N + 1) * sizeof(u64));
        if (dbg->cKS) memcpy(dbg->cKS, cKS, (size_t)(n + 1) * sizeof(u64));
    }
    free(cKS);
    free(cQ);
    free(cR);
    free(r1);
    free(r0);
    free(sgn);
    free(acc);
    free(sgb);
    free(sg);
    free(ctN);
}

/* Batch: item b uses tables (rp0, rp1)[lut_ids[b]] ([n_luts][N] each). */
void orq_fdfb_batch(const orq_params* P, const u64* bsk, const u64* pk, const u64* ksk,
                    const i64* rp0, const i64* rp1, const int32_t* lut_ids, int64_t batch,
                    const u64* ct, u64* out, int threads) {
    const int n = P->n, N = P->N;
#pragma omp parallel for num_threads(threads > 0 ? threads : 1) schedule(dynamic, 1) if (threads > 1)
    for (int64_t b = 0; b < batch; ++b) {
        const int id = lut_ids[b];
        orq_fdfb_bootstrap(P, bsk, pk, ksk, rp0 + (size_t)id * N, rp1 + (size_t)id * N,
                           ct + (size_t)b * (n + 1), out + (size_t)b * (n + 1), NULL);
    }
}

/* TFHE bootstrap (figure "TFHE Bootstrapping") on a prime-modulus set:
 * ctN = ct (q = 2N, G25); acc = [poly X^{b_N}, 0]; BlindRotate;
 * SampleExtract; KeySwitch(ksK); ModSwitch(Q -> q).  poly: [N] mod Q. */
void orq_tfhe_bootstrap(const orq_params* P, const u64* bsk, const u64* ksk, const u64* poly,
                        const u64* ct, u64* out) {
    const int n = P->n, N = P->N;
    const u64 Q = P->Q;
    int logq = 0;
    while ((1 << logq) < 2 * N) ++logq;
    u64* ctN = (u64*)malloc((size_t)(n + 1) * sizeof(u64));
    for (int i = 0; i <= n; ++i) ctN[i] = ct[i] & (u64)(2 * N - 1);
    u64* acc = (u64*)malloc((size_t)2 * N * sizeof(u64));
    orq_poly_mul_xk(N, Q, poly, (i64)ctN[0], acc);
    for (int j = 0; j < N; ++j) acc[N + j] = 0;
    orq_blind_rotate(P, bsk, acc, ctN);
    u64* cQ = (u64*)malloc((size_t)(N + 1) * sizeof(u64));
    orq_sample_extract(N, Q, acc, cQ);
    u64* cKS = (u64*)malloc((size_t)(n + 1) * sizeof(u64));
    orq_keyswitch(N, Q, P->log2Bks, P->lks, n + 1, ksk, cQ, cKS);
    orq_modswitch(Q, logq, n + 1, cKS, out);
    free(cKS);
    free(cQ);
    free(acc);
    free(ctN);
}

/* Batch: item b uses polys[poly_ids[b]] ([n_polys][N]). */
void orq_tfhe_batch(const orq_params* P, const u64* bsk, const u64* ksk, const u64* polys,
                    const int32_t* poly_ids, int64_t batch, const u64* ct, u64* out, int threads) {
    const int n = P->n, N = P->N;
#pragma omp parallel for num_threads(threads > 0 ? threads : 1) schedule(dynamic, 1) if (threads > 1)
    for (int64_t b = 0; b < batch; ++b)
        orq_tfhe_bootstrap(P, bsk, ksk, polys + (size_t)poly_ids[b] * N, ct + (size_t)b * (n + 1),
                           out + (size_t)b * (n + 1));
}
