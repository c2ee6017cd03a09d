/* Runs both oracles end to end (oracle/fdfb_oracle.c and fdfb_oracle_q.c)
 * on small noiseless parameter sets, for building under AddressSanitizer
 * and UndefinedBehaviorSanitizer: key generation, encryption, the full-domain
 * bootstrap of every message (power-of-two modulus with unsigned and
 * balanced digits and an output modulus t' = 8; prime modulus Q_1 with the
 * literal l_boot sign rotations), and decryption to f(m).  The random masks
 * come from a SplitMix64 counter (test data only).  Prints "ok" and exits 0
 * when every output decrypts to f(m). */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef uint64_t u64;
typedef int64_t i64;
typedef uint8_t u8;

/* the oracles' parameter structs (same layout as in their sources) */
typedef struct {
    int32_t n, N, w, t;
    int32_t log2Bg, lg, log2Bks, lks, log2Bpk, lpk;
    int32_t signed_digits, t_out;
} or_params;
typedef struct {
    int32_t n, N, t, log2Bg, lg, log2Bks, lks, log2Bpk, lpk, log2Lboot, lboot;
    uint64_t Q;
} orq_params;

void or_keygen_bsk(const or_params*, const u8*, const u8*, const u64*, const i64*, u64*);
void or_keygen_pk(const or_params*, const u8*, const u64*, const i64*, u64*);
void or_keygen_ksk(const or_params*, const u8*, const u8*, const u64*, const i64*, u64*);
void or_lwe_encrypt(int, int, const u8*, const u64*, i64, u64, u64*);
u64 or_lwe_decrypt(int, int, int, const u8*, const u64*);
void or_setup_polynomial(int, int, const i64*, i64*, i64*);
void or_fdfb_bootstrap(const or_params*, const u64*, const u64*, const u64*, const i64*, const i64*,
                       const u64*, u64*, const void*);
void orq_keygen_bsk(const orq_params*, const u8*, const u64*, const u64*, const i64*, u64*);
void orq_keygen_pk(const orq_params*, const u64*, const u64*, const i64*, u64*);
void orq_keygen_ksk(const orq_params*, const u64*, const u8*, const u64*, const i64*, u64*);
void orq_fdfb_bootstrap(const orq_params*, const u64*, const u64*, const u64*, const i64*, const i64*,
                        const u64*, u64*, const void*);
u64 orq_decrypt_q2n(int, int, int, const u8*, const u64*);

static u64 g_state = 2109;
static u64 next(void) {
    u64 z = (g_state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static u64* words(size_t count, u64 mod) {  /* mod 0: full 64-bit words */
    u64* a = (u64*)malloc(count * sizeof(u64));
    for (size_t i = 0; i < count; ++i) a[i] = mod ? next() % mod : next();
    return a;
}
static u8* bits(size_t count) {
    u8* b = (u8*)malloc(count);
    for (size_t i = 0; i < count; ++i) b[i] = (u8)(next() >> 63);
    return b;
}

/* power-of-two modulus, noiseless, exact decomposition */
static int run_pow2(int signed_digits, int t_out) {
    or_params P = {16, 256, 32, 4, 8, 4, 4, 8, 8, 4, signed_digits, t_out};
    const int n = P.n, N = P.N, to = t_out ? t_out : P.t;
    u8* s = bits(n);
    u8* sk = bits(N);
    u64* bsk_a = words((size_t)n * 2 * P.lg * N, 0);
    i64* bsk_e = (i64*)calloc((size_t)n * 2 * P.lg * N, sizeof(i64));
    u64* pk_a = words((size_t)N * P.lpk * N, 0);
    i64* pk_e = (i64*)calloc((size_t)N * P.lpk * N, sizeof(i64));
    u64* ksk_a = words((size_t)N * P.lks * n, 0);
    i64* ksk_e = (i64*)calloc((size_t)N * P.lks, sizeof(i64));
    u64* bsk = (u64*)malloc((size_t)n * 2 * P.lg * 2 * N * sizeof(u64));
    u64* pk = (u64*)malloc((size_t)N * P.lpk * 2 * N * sizeof(u64));
    u64* ksk = (u64*)malloc((size_t)N * P.lks * (n + 1) * sizeof(u64));
    or_keygen_bsk(&P, s, sk, bsk_a, bsk_e, bsk);
    or_keygen_pk(&P, sk, pk_a, pk_e, pk);
    or_keygen_ksk(&P, sk, s, ksk_a, ksk_e, ksk);
    i64 f[4] = {3 % to, 1 % to, 7 % to, 2 % to};
    i64 p0[256], p1[256];
    or_setup_polynomial(N, P.t, f, p0, p1);
    int bad = 0;
    for (int m = 0; m < P.t; ++m) {
        u64* a = words((size_t)n, 0);
        u64 ct[17], out[17];
        or_lwe_encrypt(P.w, n, s, a, 0, ((u64)m << (P.w - 2)), ct);
        or_fdfb_bootstrap(&P, bsk, pk, ksk, p0, p1, ct, out, NULL);
        if ((i64)or_lwe_decrypt(P.w, n, to, s, out) != f[m]) ++bad;
        free(a);
    }
    free(s); free(sk); free(bsk_a); free(bsk_e); free(pk_a); free(pk_e); free(ksk_a); free(ksk_e);
    free(bsk); free(pk); free(ksk);
    return bad;
}

/* prime modulus Q_1 = 2^62 - 65535, noiseless, q = 2N */
static int run_prime(void) {
    const u64 Q = (1ull << 62) - 65535;
    orq_params P = {8, 64, 4, 11, 6, 6, 11, 13, 5, 11, 6, Q};
    const int n = P.n, N = P.N, logq = 7;
    u8* s = bits(n);
    u64* s64 = (u64*)malloc((size_t)n * sizeof(u64));
    for (int i = 0; i < n; ++i) s64[i] = s[i];
    u64* sk = words((size_t)N, Q);
    u64* bsk_a = words((size_t)n * 2 * P.lg * N, Q);
    i64* bsk_e = (i64*)calloc((size_t)n * 2 * P.lg * N, sizeof(i64));
    u64* pk_a = words((size_t)N * P.lpk * N, Q);
    i64* pk_e = (i64*)calloc((size_t)N * P.lpk * N, sizeof(i64));
    u64* ksk_a = words((size_t)N * P.lks * n, Q);
    i64* ksk_e = (i64*)calloc((size_t)N * P.lks, sizeof(i64));
    u64* bsk = (u64*)malloc((size_t)n * 2 * P.lg * 2 * N * sizeof(u64));
    u64* pk = (u64*)malloc((size_t)N * P.lpk * 2 * N * sizeof(u64));
    u64* ksk = (u64*)malloc((size_t)N * P.lks * (n + 1) * sizeof(u64));
    orq_keygen_bsk(&P, s, sk, bsk_a, bsk_e, bsk);
    orq_keygen_pk(&P, sk, pk_a, pk_e, pk);
    orq_keygen_ksk(&P, sk, s, ksk_a, ksk_e, ksk);
    i64 f[4] = {2, 0, 3, 1};
    i64 p0[64], p1[64];
    or_setup_polynomial(N, P.t, f, p0, p1);
    int bad = 0;
    for (int m = 0; m < P.t; ++m) {
        u64 ct[9], out[9];
        u64 b = (u64)m * (2 * (u64)N / (u64)P.t);
        for (int i = 0; i < n; ++i) {
            ct[1 + i] = next() % (2 * (u64)N);
            b += ct[1 + i] * s64[i];
        }
        ct[0] = b % (2 * (u64)N);
        orq_fdfb_bootstrap(&P, bsk, pk, ksk, p0, p1, ct, out, NULL);
        if ((i64)orq_decrypt_q2n(n, logq, P.t, s, out) != f[m]) ++bad;
    }
    free(s); free(s64); free(sk); free(bsk_a); free(bsk_e); free(pk_a); free(pk_e); free(ksk_a);
    free(ksk_e); free(bsk); free(pk); free(ksk);
    return bad;
}

int main(void) {
    int bad = run_pow2(0, 0) + run_pow2(1, 0) + run_pow2(0, 8) + run_prime();
    if (bad) {
        printf("%d wrong outputs\n", bad);
        return 1;
    }
    printf("ok\n");
    return 0;
}
