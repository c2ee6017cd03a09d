/*
 * fdfb.h -- C ABI of the GB300 library for full-domain functional
 * bootstrapping (FDFB, Kluczniak and Schild, arXiv 2109.02731).
 *
 * The library evaluates an arbitrary lookup table f: Z_t -> Z_t on LWE
 * ciphertexts, on the whole plaintext domain including its negacyclic half
 * (Section 3, figure "functional-bootstrapping").  One bootstrap is
 *   ModSwitch(q -> 2N); sign BlindRotate; SampleExtract + Delta/2;
 *   BuildAcc = KeySwitch(LWE -> RLWE, pK) then PubMux of the two rotation
 *   polynomials; function BlindRotate; SampleExtract; KeySwitch(ksK).
 * All arithmetic is exact integer arithmetic modulo q = 2^w (w = 32 or 64):
 * results are bit-for-bit those of the paper's algorithm under the readings
 * stated with each call.
 *
 * Conventions (all calls):
 *   - Words are little-endian uint32_t (log2q = 32) or uint64_t (log2q = 64)
 *     holding residues mod q.  An LWE ciphertext is [b, a_1 .. a_n] with
 *     b = <a, s> + e + m (Definition "Generalized Learning With Errors"); an
 *     RLWE ciphertext is the two polynomials [b, a] of N words each, every
 *     polynomial in ascending powers of X (Coefs()).
 *   - k = 1 (RLWE) and u = {1} (binary LWE key): the paper's Table 1 setting.
 *   - Gadget decomposition is unsigned and truncated: with r = max(0, w -
 *     l*log2B), a word x is rounded to x~ = ((x + 2^(r-1)) mod q) >> r and
 *     split into l base-B digits, least significant first, against the gadget
 *     values B^(j-1) 2^r (Definitions "Gadget Matrix" and "Decomposition").
 *     With l*log2B >= w this is the paper's exact decomposition.
 *   - Pointers documented as "device" must be device memory of the context's
 *     GPU; "host" pointers are ordinary host memory.  The caller owns every
 *     buffer it passes; the library owns keys, lookup tables and its scratch.
 *   - Every call that takes a stream (a cudaStream_t passed as void*, NULL =
 *     legacy default stream) is asynchronous and stream ordered.  Argument
 *     errors are returned synchronously; device-side errors are latched and
 *     reported by fdfb_sync().
 *   - Return value: FDFB_OK (0) or a negative FDFB_E* code (fdfb_strerror).
 *   - There is no CPU fallback: without a usable GPU, fdfb_create fails.
 */
#ifndef FDFB_H
#define FDFB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  FDFB_OK = 0,
  FDFB_EINVAL = -1,    /* bad argument, unsupported parameters or sizes */
  FDFB_ENOMEM = -2,    /* device allocation failed */
  FDFB_ECUDA = -3,     /* a CUDA runtime call failed */
  FDFB_ETIMEOUT = -4,  /* a bounded device-side wait expired */
  FDFB_ENOKEYS = -5,   /* keys of the parameter set were never installed */
  FDFB_EBADLUT = -6    /* unknown lookup-table id, or table entry outside Z_t */
};

typedef struct fdfb_ctx fdfb_ctx;

/* One parameter set (paper notation, Table 1).  k must be 1; log2q is 32 or
 * 64.  With Q = 0 (power-of-two sets) q = Q = 2^log2q: the final ModSwitch
 * Q -> q of the Bootstrap figure is the identity, t is a power of two with
 * 2 <= t <= N, and log2Lboot / lboot, which describe the PubMux
 * decomposition of Bootstrap step "l_boot", must be log2 t and 1 (L_boot =
 * t, l_boot = 1: one sign blind rotation, the PubMux selector (p_1 - p_0)
 * mod t one digit).  With Q != 0 the rules of the Q field below apply. */
typedef struct {
  uint32_t n, N, k, log2q, t;
  uint32_t log2Bg, lg;     /* bootstrapping-key gadget: base 2^log2Bg, lg digits (lg <= 4) */
  uint32_t log2Bks, lks;   /* LWE->LWE key-switching gadget */
  uint32_t log2Bpk, lpk;   /* LWE->RLWE packing-key gadget */
  uint32_t log2Lboot, lboot;
  /* 1: the blind rotation decomposes into balanced digits in [-B/2, B/2)
   * (the same rounded value, carried upward; the carry out of the top digit
   * vanishes mod q), a quarter of the digit variance of [0, B); 0: digits
   * in [0, B).  The key switches always use [0, B). */
  uint32_t signed_digits;
  /* Output plaintext modulus t' of f: Z_t -> Z_t' (Section 1.1, footnote:
   * the same method with a different message scaling); 0 means t' = t.  A
   * power of two, 2 <= t' <= 2^15.  The sign LWE is scaled by Delta'/2 and
   * PubMux by Delta' = q / t', table entries lie in Z_t', and the bootstrap's
   * outputs encrypt Delta' f(m). */
  uint32_t t_out;
  /* Prime-modulus parameter sets (Table 1); 0 selects q = Q = 2^log2q
   * (everything above).  Q = 2^k - c with 32 <= k <= 63 and odd c < 2^20
   * (the paper's Q_1 = 2^62 - 65535, Q_2 = 2^63 - 278527, Q_3 = 2^48 -
   * 163839, Q_4 = 2^32 - 139263) runs the paper's Bootstrap
   * figure literally:
   *   - the RLWE side (keys, accumulators, the extracted and key-switched
   *     LWE samples) lives mod Q in 64-bit words (log2q = 64);
   *   - the LWE side lives mod q = 2N: input and output ciphertexts are
   *     [n+1] 64-bit words in [0, 2N), Delta_q = round(2N / t), so the first
   *     ModSwitch (q -> 2N) is the identity and the last is ModSwitch(Q -> q),
   *     round(q x / Q) round half up;
   *   - every gadget decomposition is exact: lg, lks, lpk must equal
   *     ceil(k / log2B) for their bases (digits of x in [0, Q), least
   *     significant first, gadget B^(j-1));
   *   - lboot = ceil(k / log2Lboot) <= 8 sign blind rotations per input, the
   *     i-th starting from L_boot^(i-1) round(Q / 2t) sgnP X^{b_N} and adding
   *     the same constant after SampleExtract; each sign LWE is key switched
   *     to RLWE; PubMux splits p = rotP'_0 - rotP'_1 in Z_Q into lboot
   *     base-L_boot digits and returns [round(Q/t) rotP'_1, 0] + sum_i p[i]
   *     c_R,i; the function rotation, SampleExtract and KeySwitch(ksK) follow,
   *     then ModSwitch(Q -> q);
   *   - t is any integer in [2, N] (the pairwise coprime moduli of a CRT
   *     representation, Section "Extending the Arithmetic", need not divide
   *     2N): Delta_q = round(2N / t), and fdfb_lwe_decrypt returns
   *     round(t (b - <a, s>) / 2N) mod t;
   *   - N is 256, 1024, 2048, 4096 or 8192 (Table 1's FDFB:80:8 and
   *     FDFB:100:8; at N = 8192 the blind rotation keeps the accumulator in
   *     shared memory and needs n <= 1536); signed_digits and t_out must be 0;
   *     fdfb_bootstrap_multi (k > 1) and fdfb_lwe_affine are not available
   *     (FDFB_EINVAL);
   *   - the TFHE bootstrap takes polynomials of residues mod Q and, like the
   *     full-domain one, inputs mod 2N (ModSwitch the identity), returning
   *     ModSwitch(Q -> 2N) of the key-switched sample.
   * Keys are uploaded in the canonical layouts as residues mod Q; the RLWE
   * key of fdfb_keys_generate is uniform in Z_Q^N (fdfb_keygen_inputs.sk_q). */
  uint64_t Q;
} fdfb_params;

/* Concurrency.  Every call is stream-ordered.  A parameter set owns one
 * scratch area for its pipeline intermediates, so bootstrap calls on the
 * same set must be ordered on the GPU (one stream, or events between
 * streams); calls on different sets may run concurrently.  Registration,
 * key installation and table setup take the context's lock and synchronise
 * the device where they replace device buffers; issue them before the calls
 * that use them.  A call that grows scratch (a larger batch than before)
 * allocates, so make it once outside any stream capture. */

/* Creates a context on CUDA device `device`.  *out receives the handle. */
int fdfb_create(fdfb_ctx** out, int device);

/* Destroys the context and frees every device buffer it owns.  The caller
 * must make sure no work of the context is still running. */
int fdfb_destroy(fdfb_ctx* ctx);

/* Registers a parameter set; *set_id_out receives its id.  Fails with
 * FDFB_EINVAL for unsupported shapes (prime-modulus sets: the rules given
 * with fdfb_params.Q, lg <= 7, N up to 8192): N not in {256, 512, 1024, 2048, 4096},
 * n > 4096, lg > 4, signed_digits > 1, or a negacyclic product whose exact
 * value could exceed what the 30-bit primes lift exactly (2l N (B-1) q/2 for
 * the blind rotation, N (t-1) q for PubMux).  Registration also builds the
 * set's blind-rotation variants (fdfb_autotune): the layouts whose shared
 * memory fits the device, whose digit width holds B, that are built with
 * balanced digits if the set asks for them, and -- for the lazy 28-bit prime
 * family and the split-key layouts of q = 2^64 -- whose own primes lift the
 * products exactly. */
int fdfb_params_register(fdfb_ctx* ctx, const fdfb_params* prm, int* set_id_out);

/* Size in words of each key in its canonical layout (what keys_upload reads):
 *   which = 0: bsk, n * (2 lg) * 2 * N   (GGSW rows of BRKeyGen, figure
 *              "Blind Rotation and its setup")
 *   which = 1: pK,  N * lpk * 2 * N      (KeySwitchSetup, LWE dim N -> RLWE)
 *   which = 2: ksK, N * lks * (n + 1)    (KeySwitchSetup, LWE dim N -> dim n) */
int fdfb_key_words(const fdfb_params* prm, int which, uint64_t* words_out);

/* Installs keys given in canonical layout (host pointers, may be freed on
 * return; the call synchronises the stream before returning):
 *   bsk [n][2 lg][2][N]: bsk[i][r] = GGSW row r of RGSW(s_i), row
 *        r = c*lg + (j-1) adding s_i * g_j to component c (0 = b, 1 = a);
 *   pk  [N][lpk][2][N]:  RLWE_sk(s_F[i] * g_j), constant message polynomial;
 *   ksk [N][lks][n+1]:   LWE_s(s_F[i] * g_j).
 * The bootstrapping key is converted to the NTT domain on the device. */
int fdfb_keys_upload(fdfb_ctx* ctx, int set_id, const void* bsk, const void* pk,
                     const void* ksk, void* cuda_stream);

/* Randomness of key generation (host pointers; words are w-bit residues,
 * noise is signed):  s[n], sk[N] binary keys (s_F = Coefs(sk));
 * bsk_a/bsk_e [n][2 lg][N]; pk_a/pk_e [N][lpk][N]; ksk_a [N][lks][n];
 * ksk_e [N][lks].  Prime-modulus sets: the masks are 64-bit residues mod Q,
 * sk is unused and sk_q [N] (uint64 residues mod Q) is the RLWE key. */
typedef struct {
  const uint8_t* s;
  const uint8_t* sk;
  const void* bsk_a;
  const int64_t* bsk_e;
  const void* pk_a;
  const int64_t* pk_e;
  const void* ksk_a;
  const int64_t* ksk_e;
  const uint64_t* sk_q;
} fdfb_keygen_inputs;

/* Generates the keys on the GPU from the given randomness -- BRKeyGen and
 * KeySwitchSetup (figures "Blind Rotation and its setup" and "Key switching
 * algorithm and its setup"), every GLWE sample b = a*sk + e + m computed
 * exactly -- and installs them, as fdfb_keys_upload would.  Synchronises the
 * stream before returning. */
int fdfb_keys_generate(fdfb_ctx* ctx, int set_id, const fdfb_keygen_inputs* in, void* cuda_stream);

/* Copies the installed keys back in canonical layout (host pointers, each
 * may be NULL).  Synchronises the stream. */
int fdfb_keys_download(fdfb_ctx* ctx, int set_id, void* bsk, void* pk, void* ksk, void* cuda_stream);

/* Installs a lookup table f: Z_t -> Z_t (host, t entries; BootsMap[m+1] =
 * f(m), unscaled) and builds its rotation polynomials with SetupPolynomial
 * (figure "functional-bootstrapping", right: m ascending, e ascending, later
 * writes win).  *lut_id_out receives the id, dense from 0 per parameter set.
 * FDFB_EBADLUT if an entry is >= t' (the output modulus, = t by default). */
int fdfb_lut_setup(fdfb_ctx* ctx, int set_id, const uint32_t* f, int* lut_id_out);

/* Reads back the rotation polynomials of a table: p0, p1 host int32[N]. */
int fdfb_lut_polys(fdfb_ctx* ctx, int set_id, int lut_id, int32_t* p0, int32_t* p1);

/* Full-domain functional bootstrap of a batch (figure "functional-
 * bootstrapping", left):
 *   ct_in   device, [batch][n+1] words, LWE_s(Delta m), Delta = q/t;
 *   lut_ids device, int32[batch], ids from fdfb_lut_setup;
 *   ct_out  device, [batch][n+1] words, LWE_s(Delta f(m)); may not alias ct_in.
 * batch may be 0.  The library keeps scratch for the largest batch seen
 * (allocated on first use, outside any stream capture). */
int fdfb_bootstrap(fdfb_ctx* ctx, int set_id, const void* ct_in, const int32_t* lut_ids,
                   int64_t batch, void* ct_out, void* cuda_stream);

/* TFHE bootstrap (figure "TFHE Bootstrapping"): one blind rotation of a
 * caller-given pre-rotation polynomial, for negacyclic functions (f(m + t/2)
 * = -f(m)); the paper's comparison point for the full-domain bootstrap.
 *   ct_N = ModSwitch(ct, q, 2N); acc = [poly X^{b_N}, 0];
 *   acc = BlindRotate(brK, acc, ct_N); c = SampleExtract(acc, 1);
 *   ct_out = KeySwitch(c, ksK) (the final ModSwitch Q -> q is the identity).
 * fdfb_tfhe_poly_setup installs a polynomial (host, N words mod q) and
 * returns its id, dense from 0 per parameter set.  fdfb_tfhe_bootstrap:
 * ct_in device [batch][n+1] words; poly_ids device int32[batch]; ct_out
 * device [batch][n+1].  FDFB_ENOKEYS without keys, FDFB_EBADLUT without a
 * polynomial; an id out of range is latched as FDFB_EBADLUT (reported by
 * fdfb_sync) and polynomial 0 used. */
int fdfb_tfhe_poly_setup(fdfb_ctx* ctx, int set_id, const void* poly, int* poly_id_out);
int fdfb_tfhe_bootstrap(fdfb_ctx* ctx, int set_id, const void* ct_in, const int32_t* poly_ids,
                        int64_t batch, void* ct_out, void* cuda_stream);

/* Several functions of one input (Section "Application of Functional
 * Bootstrapping", multiple univariate functions with the same input: the
 * accumulators of the first bootstrap are reused for the next function).
 * The sign rotation, its SampleExtract and the packing key switch run once
 * per input; PubMux, the function rotation, SampleExtract and the LWE key
 * switch run once per (input, table):
 *   ct_in   device, [batch][n+1] words;
 *   lut_ids device, int32[batch][k], table ids from fdfb_lut_setup;
 *   ct_out  device, [batch][k][n+1] words; ct_out[b][j] is bit for bit what
 *           fdfb_bootstrap returns for ct_in[b] with table lut_ids[b][j].
 * k >= 1 and batch * k < 2^31, else FDFB_EINVAL.  Scratch grows as for
 * fdfb_bootstrap (for batch inputs and batch * k outputs). */
int fdfb_bootstrap_multi(fdfb_ctx* ctx, int set_id, const void* ct_in, const int32_t* lut_ids,
                         int64_t batch, int k, void* ct_out, void* cuda_stream);

/* Intermediates of fdfb_bootstrap for checking (device pointers, each may
 * be NULL; [batch] x ...):
 *   ctN  uint32 [n+1]  ModSwitch(ct, q, 2N)
 *   sgn  words [N+1]   SampleExtract of the sign rotation + [Delta/2, 0]
 *   cR   words [2N]    KeySwitch(sgn, pK)
 *   accF words [2N]    PubMux(cR, rotP'_1, rotP'_0)
 *   cQ   words [N+1]   SampleExtract of the function rotation
 *   cKS  words [n+1]   (prime-modulus sets) KeySwitch(cQ, ksK) mod Q, before
 *                      ModSwitch(Q -> q)
 * Prime-modulus sets hold lboot sign LWEs and packed RLWEs per input (sgn
 * [lboot][N+1], cR [lboot][2N]) and produce no ctN (the input is already
 * modulo 2N). */
typedef struct {
  void* ctN;
  void* sgn;
  void* cR;
  void* accF;
  void* cQ;
  void* cKS;
} fdfb_debug_bufs;

int fdfb_bootstrap_debug(fdfb_ctx* ctx, int set_id, const void* ct_in, const int32_t* lut_ids,
                         int64_t batch, void* ct_out, const fdfb_debug_bufs* dbg,
                         void* cuda_stream);

/* fdfb_bootstrap for callers that cannot allocate GPU memory at call time
 * and so cannot let fdfb_bootstrap grow its scratch on first use: code in a
 * host callback enqueued on a stream (CUDA calls are not allowed there),
 * services whose device memory is all handed to a caching allocator up front
 * or capped by a budget, and latency-bound loops that cannot afford the
 * device-wide synchronisation cudaMalloc and cudaFree may imply.  The paper
 * has no counterpart; this is a library convenience.
 *
 * Same arguments, results and errors as fdfb_bootstrap, bit for bit.  The
 * intermediates live in one fixed 32 MiB device array compiled into the
 * library (every GPU that loads the library holds it until the process
 * exits); this call performs no cudaMalloc, cudaFree or other allocation.
 *   - batch may be at most fdfb_noalloc_max_batch(ctx, set_id), which is
 *     32 MiB divided by the intermediates of one input:
 *       power-of-two sets: (6N + 2) words, e.g. 1364 ciphertexts at N = 1024,
 *       q = 2^32 and 170 at N = 4096, q = 2^64;
 *       prime-modulus sets: l_boot (7N + 1) + 3N + 1 + 2(n + 1) 64-bit
 *       words, e.g. 44 ciphertexts for FDFB-80-6 (n = 700, N = 2048,
 *       l_boot = 6); at N = 8192 also l_boot x 98,304 32-bit words of
 *       blind-rotation scratch, e.g. 4 ciphertexts for FDFB-80-8.
 *     Larger batches return FDFB_EINVAL.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - All calls, from any context on the device, share the one array: calls
 *     that can overlap on the GPU (different streams, no ordering) race and
 *     corrupt each other's results.  Every intermediate is fully rewritten by
 *     each call (sums that accumulate are zeroed first), so nothing left by
 *     an earlier call is read.
 *   - Keys and tables must be installed beforehand (those calls allocate). */
int fdfb_bootstrap_noalloc(fdfb_ctx* ctx, int set_id, const void* ct_in, const int32_t* lut_ids,
                           int64_t batch, void* ct_out, void* cuda_stream);

/* Largest batch fdfb_bootstrap_noalloc accepts for the parameter set. */
int fdfb_noalloc_max_batch(fdfb_ctx* ctx, int set_id, int64_t* max_batch);

/* One group of a mixed batch: a parameter set and its ciphertexts. */
typedef struct {
  int set_id;
  const void* ct_in;       /* device [batch][n+1] */
  const int32_t* lut_ids;  /* device [batch] */
  int64_t batch;
  void* ct_out;            /* device [batch][n+1] */
} fdfb_group;

/* Bootstraps several groups, possibly under different parameter sets, as
 * fdfb_bootstrap would for each.  Groups of distinct parameter sets run
 * concurrently on library-owned side streams forked from and joined back to
 * cuda_stream with events (so the call can be captured into a CUDA graph
 * once every set's scratch exists); groups of one set run in order.  The
 * first call may create the side streams and grow scratch. */
int fdfb_bootstrap_mixed(fdfb_ctx* ctx, int n_groups, const fdfb_group* groups, void* cuda_stream);

/* LWE key switching with the installed ksK (figure "Key switching algorithm
 * and its setup"): ct_in device [batch][N+1] words under s_F, ct_out device
 * [batch][n+1] words under s (prime-modulus sets: both mod Q; there the call
 * allocates a temporary buffer for the exact half sums and synchronises the
 * stream before returning). */
int fdfb_keyswitch(fdfb_ctx* ctx, int set_id, const void* ct_in, int64_t batch, void* ct_out,
                   void* cuda_stream);

/* LWE encryption b = <a, s> + e + Delta m (device pointers):  s uint8[n];
 * a [count][n] words; e int64[count]; m int64[count] (in Z_t);
 * ct_out [count][n+1] words.  Prime-modulus sets: mod q = 2N, Delta = 2N/t. */
int fdfb_lwe_encrypt(fdfb_ctx* ctx, int set_id, const uint8_t* s, const void* a, const int64_t* e,
                     const int64_t* m, int64_t count, void* ct_out, void* cuda_stream);

/* LWE decryption round(t' * (b - <a, s>) / q) mod t', round half up, in the
 * bootstrap's output space Z_t' (t' = t unless the set's t_out says
 * otherwise) (device pointers): s uint8[n]; ct [count][n+1]; m_out
 * int32[count]. */
int fdfb_lwe_decrypt(fdfb_ctx* ctx, int set_id, const uint8_t* s, const void* ct, int64_t count,
                     int32_t* m_out, void* cuda_stream);

/* LWE affine layer without bootstrapping (Lemma "Linear Homomorphism of
 * GLWE samples"; Section 3.4 "Computing in Z_t"):
 *   y[b][o] = sum_i W[o][i] * x[b][i]  (mod q), every LWE component;
 *   W device int32 [n_out][n_in]; x device [batch][n_in][len] words;
 *   y device [batch][n_out][len] words; len = n+1 of the set. */
int fdfb_lwe_affine(fdfb_ctx* ctx, int set_id, const int32_t* W, int n_in, int n_out,
                    const void* x, int64_t batch, void* y, void* cuda_stream);

/* Autotuner; the paper has no counterpart.  The blind rotation is compiled
 * in several register layouts ("variants": coefficients of one transform per
 * thread, which sets the threads per prime, the shared-memory exchanges per
 * transform and the resident CTAs per SM).  fdfb_autotune times one blind
 * rotation of every variant on `batch` trial ciphertexts with the installed
 * keys and keeps the fastest for the parameter set (*variant_out, its time
 * in *ms_out, and the time of variant i in ms_each[i] for i < ms_each_len;
 * any of them may be NULL).  Results never depend on the variant:
 * every variant computes the same exact products.  It then chooses the
 * set's chunk count (fdfb_set_chunks) by timing whole bootstrap calls.  Needs
 * keys (FDFB_ENOKEYS), may grow the set's scratch, creates the chunk side
 * streams, and synchronises the stream.
 * fdfb_set_variant selects a variant by index; fdfb_variant_info reports the
 * current index, the number of variants and the current coefficients per
 * thread (any output pointer may be NULL). */
int fdfb_autotune(fdfb_ctx* ctx, int set_id, int64_t batch, void* cuda_stream, int* variant_out,
                  double* ms_out, double* ms_each, int ms_each_len);
int fdfb_set_variant(fdfb_ctx* ctx, int set_id, int variant);

/* How many consecutive slices fdfb_bootstrap and fdfb_bootstrap_multi split
 * a batch into, each slice's pipeline on a library side stream forked from
 * and joined back to the caller's stream (the paper has no counterpart: the
 * launches of the slices overlap on the GPU, filling the last partial wave of
 * one blind-rotation launch with the next).  Results do not depend on it.
 * 1 to 8; 1 (one pipeline on the caller's stream) until fdfb_autotune times
 * the whole pipeline with 1, 2, 3, 4, 6 and 8 slices for batches below 8
 * waves of the blind rotation.  A call with more than one slice creates the side streams on
 * first use; make it outside any stream capture.  The debug, no-allocation
 * and mixed entry points always run one pipeline per group. */
int fdfb_set_chunks(fdfb_ctx* ctx, int set_id, int chunks);
int fdfb_get_chunks(fdfb_ctx* ctx, int set_id, int* chunks);
int fdfb_variant_info(fdfb_ctx* ctx, int set_id, int* current, int* count, int* coeffs_per_thread);

/* Measurement hook; the paper has no counterpart.  While enabled, every
 * launch of the bootstrap pipeline is bracketed by a CUDA event pair recorded
 * on the caller's stream, and the device time is accumulated per stage:
 *   0 sign blind rotation, 1 packing key switch, 2 PubMux (or the TFHE
 *   bootstrap's accumulator),
 *   3 function blind rotation, 4 LWE key switch,
 *   5 all blind rotations: the length of the union of the intervals of the
 *     stage 0 and 3 launches (launches of the chunks of one call, on
 *     different streams, overlap; stages 0-4 add their durations up).
 * fdfb_profile_read synchronises on the recorded events and returns the
 * accumulated milliseconds and launch count of `stage` since the last
 * enable.  Disabled by default. */
int fdfb_profile_enable(fdfb_ctx* ctx, int enable);
int fdfb_profile_read(fdfb_ctx* ctx, int stage, double* total_ms, int64_t* launches);

/* Test hook; the paper has no counterpart.  flags = 0 (the default) is
 * normal operation.  Bit 0: the blind rotations of fdfb_bootstrap issue none
 * of the bulk copies that stage key rows in shared memory (the staged-key
 * layout of N = 2048, q = 2^64) and bound the wait for them to 2^12 polls,
 * so the wait expires with no copy in flight: the call then latches
 * FDFB_ETIMEOUT (reported by fdfb_sync), computes garbage for the batch and
 * leaves the context usable.  It exists to exercise that error path without
 * any fault.  Bit 1: every key switch runs as the CUDA-core contraction
 * instead of on the tensor cores (same results; for comparisons).
 * FDFB_EINVAL for unknown bits. */
int fdfb_test_hooks(fdfb_ctx* ctx, int flags);

/* Which contraction the set's key switches use (the paper has no
 * counterpart): *pk_path for the packing key (BuildAcc), *ksk_path for the
 * LWE key switch; 1 = fifth-generation tensor cores, 0 = CUDA cores (either
 * pointer may be NULL).  Key switching (figure "Key switching algorithm and
 * its setup") is the dense contraction out = [b, 0] - D K mod 2^w of the
 * digit matrix D and the key K.  On the tensor cores it is computed exactly:
 * the key words are split into balanced limbs of b bits and the digits are
 * summed in chunks short enough that every fp32 partial sum is an integer
 * below 2^24 in magnitude.  On the prime-modulus sets the tensor cores
 * compute the exact integer sums (key residues as limbs covering 65 bits,
 * digits above 11 bits in two halves), reduced mod Q afterwards.  The limb
 * form is built when keys are installed, for gadget bases up to 2^11 (2^22
 * on the prime-modulus sets); wider digits and fdfb_bootstrap_noalloc use
 * the CUDA cores. */
int fdfb_keyswitch_path(fdfb_ctx* ctx, int set_id, int* pk_path, int* ksk_path);

/* Waits for the stream and reports latched device-side errors (e.g.
 * FDFB_ETIMEOUT) and CUDA errors; clears the latch. */
int fdfb_sync(fdfb_ctx* ctx, void* cuda_stream);

/* Static description of an error code. */
const char* fdfb_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* FDFB_H */
