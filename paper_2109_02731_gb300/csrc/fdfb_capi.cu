// C ABI of the FDFB library: context, parameter registry, key installation,
// lookup tables and the bootstrapping pipeline.  See include/fdfb.h.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <memory>
#include <mutex>
#include <vector>

#include "../../include/fdfb.h"
#include "fdfb_host.hpp"
#include "fdfb_ks_tc.hpp"
#include "fdfb_ops.hpp"

namespace fdfb {
const Ops* ops_n8(int w, int variant);
const Ops* ops_n9(int w, int variant);
const Ops* ops_n10(int w, int variant);
const Ops* ops_n11(int w, int variant);
const Ops* ops_n12(int w, int variant);

const Ops* ops_q_n8(int variant);
const Ops* ops_q_n10(int variant);
const Ops* ops_q_n11(int variant);
const Ops* ops_q_n12(int variant);
const Ops* ops_q_n13(int variant);

const Ops* find_ops_q(int L, int variant) {
  switch (L) {
    case 8: return ops_q_n8(variant);
    case 10: return ops_q_n10(variant);
    case 11: return ops_q_n11(variant);
    case 12: return ops_q_n12(variant);
    case 13: return ops_q_n13(variant);
    default: return nullptr;
  }
}

const Ops* find_ops(int L, int w, int variant) {
  switch (L) {
    case 8: return ops_n8(w, variant);
    case 9: return ops_n9(w, variant);
    case 10: return ops_n10(w, variant);
    case 11: return ops_n11(w, variant);
    case 12: return ops_n12(w, variant);
    default: return nullptr;
  }
}
}  // namespace fdfb

using namespace fdfb;

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  int ensure(size_t want) {
    if (want <= bytes) return FDFB_OK;
    release();
    if (want == 0) return FDFB_OK;
    if (cudaMalloc(&p, want) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return FDFB_ENOMEM;
    }
    bytes = want;
    return FDFB_OK;
  }
};

// One register-layout variant of the transforms: its twiddle tables and the
// bootstrapping key transformed for it.
struct Variant {
  const Ops* ops = nullptr;
  PrimeSet S{};
  DevBuf tw;        // [2][P][N] uint2
  DevBuf bsk_ntt;   // [n][P][2 lg][2][N] uint32
  size_t br_smem = 0;
  uint32_t br_r1 = 0, br_ex = 0;
};

struct SetState {
  fdfb_params prm{};
  int w = 0, L = 0, logt = 0, tout = 0, logtout = 0;  // tout: output plaintext modulus t'
  std::vector<std::unique_ptr<Variant>> var;  // var[0] also serves key generation and PubMux
  int cur = 0;                                // variant used by the blind rotations
  DevBuf bsk;       // canonical [n][2 lg][2][N] words
  DevBuf pk;        // canonical [N][lpk][2][N] words
  DevBuf ksk;       // canonical [N][lks][n+1] words
  bool keys = false;
  std::vector<int16_t> luts_host;  // [n_luts][2][N]
  DevBuf luts;
  int n_luts = 0;
  std::vector<uint64_t> tpolys_host;  // [n_tpolys][N] words (TFHE bootstrap polynomials)
  DevBuf tpolys;
  int n_tpolys = 0;
  DevBuf scratch;   // sgn | cR | accF | cQ for the largest batch seen
  int chunks = 1;  // pieces fdfb_bootstrap splits a large batch into (set by fdfb_autotune)
  // prime-modulus sets (prm.Q != 0)
  ModQ mq{};                 // mq.Q == 0 for the power-of-two sets
  int lboot = 1;             // sign rotations per input
  uint64_t sgn_scale[8] = {0};  // L_boot^i round(Q / 2t) mod Q
  uint64_t delta_q = 0;      // round(Q / t)
  DevBuf pk_split, ksk_split;  // key-switch layouts: 32-bit halves as columns
  // power-of-two sets: the key-switching keys in tensor-core limb form, and
  // the f16 digit matrices of the key switches (rows of the largest batch)
  TcKsKey tc_pk, tc_ksk;
  DevBuf tc_digits;
  ~SetState() {
    tc_ks_release(tc_pk);
    tc_ks_release(tc_ksk);
  }
  size_t wbytes() const { return (size_t)w / 8; }
  Variant& base() { return *var[0]; }
  Variant& br() { return *var[cur]; }
};

}  // namespace

constexpr int kStages = 6;  // 5: union of all blind-rotation launches (computed when read)

struct fdfb_ctx {
  int device = 0;
  int sms = 0;  // streaming multiprocessors of the device
  std::vector<std::unique_ptr<SetState>> sets;
  int* d_err = nullptr;
  std::mutex mu;
  // measurement hook
  bool prof = false;
  struct Mark { int stage; cudaEvent_t a, b; };
  std::vector<Mark> marks;
  double prof_ms[kStages] = {0, 0, 0, 0, 0, 0};
  int64_t prof_n[kStages] = {0, 0, 0, 0, 0, 0};
  // side streams and fork/join events of fdfb_bootstrap_mixed
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> events;
  // side streams and fork/join events of the chunked single-set pipeline
  std::vector<cudaStream_t> chunk_side;
  std::vector<cudaEvent_t> chunk_events;
  // fdfb_test_hooks flags (0 in normal use)
  int test_flags = 0;
};

namespace {

int cuda_err(cudaError_t e) {
  if (e == cudaSuccess) return FDFB_OK;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? FDFB_ENOMEM : FDFB_ECUDA;
}

#define FD_TRY(x)                    \
  do {                               \
    int _rc = (x);                   \
    if (_rc != FDFB_OK) return _rc;  \
  } while (0)
#define FD_CUDA(x) FD_TRY(cuda_err(x))

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

bool is_pow2(uint32_t x) { return x && !(x & (x - 1)); }
int ilog2(uint32_t x) {
  int r = 0;
  while ((1u << r) < x) ++r;
  return r;
}
int trunc_bits(int w, int log2B, int ell) {
  int r = w - ell * log2B;
  return r > 0 ? r : 0;
}
uint64_t gadget(int w, int log2B, int ell, int j) {
  int sh = trunc_bits(w, log2B, ell) + log2B * j;
  if (sh >= w) return 0;
  return (uint64_t)1 << sh;
}

SetState* get_set(fdfb_ctx* ctx, int id) {
  if (!ctx || id < 0 || id >= (int)ctx->sets.size()) return nullptr;
  return ctx->sets[id].get();
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// SetupPolynomial (figure "functional-bootstrapping", right) on unscaled
// table entries: for m = 0..t-1, e = -ceil(N/t)..ceil(N/t),
// y = round(2N/t) m + e mod 2N writes rotP_0[0] = f(m) (y = 0),
// rotP_0[N-y] = -f(m) (0 < y < N), rotP_1[0] = -f(m) (y = N),
// rotP_1[2N-y] = f(m) (N < y < 2N); later writes replace earlier ones.
void setup_polynomial(int N, int t, const uint32_t* f, int16_t* p0, int16_t* p1) {
  for (int j = 0; j < N; ++j) p0[j] = p1[j] = 0;
  const int64_t twoN = 2 * (int64_t)N;
  const int64_t E = ((int64_t)N + t - 1) / t;
  const int64_t step = (twoN + t / 2) / t;
  for (int m = 0; m < t; ++m)
    for (int64_t e = -E; e <= E; ++e) {
      int64_t y = ((step * m + e) % twoN + twoN) % twoN;
      const int16_t v = (int16_t)f[m];
      if (y == 0) p0[0] = v;
      else if (y < N) p0[N - y] = (int16_t)-v;
      else if (y == N) p1[0] = (int16_t)-v;
      else p1[twoN - y] = v;
    }
}

int install_bsk_ntt(SetState& st, cudaStream_t s) {
  const fdfb_params& P = st.prm;
  const size_t N = P.N;
  for (auto& v : st.var) {
    FD_TRY(v->bsk_ntt.ensure((size_t)P.n * v->ops->P * 2 * P.lg * 2 * v->ops->key_halves * N * 4));
    FD_CUDA(v->ops->bsk_ntt(v->S, st.bsk.p, (int64_t)P.n * 2 * P.lg, 2 * (int)P.lg,
                            (uint32_t*)v->bsk_ntt.p, st.mq.Q, s));
  }
  return FDFB_OK;
}

// Prime-modulus sets: the key-switching keys as 32-bit halves in separate
// columns (what keyswitch_kernel<uint64_t, uint32_t> reads).
int install_split_keys(SetState& st, cudaStream_t s) {
  const fdfb_params& P = st.prm;
  const int64_t N = P.N, n = P.n;
  FD_TRY(st.pk_split.ensure((size_t)N * P.lpk * 2 * N * 2 * 4));
  FD_TRY(st.ksk_split.ensure((size_t)N * P.lks * (n + 1) * 2 * 4));
  split_halves_kernel<<<1024, 256, 0, s>>>((const uint64_t*)st.pk.p, N * P.lpk, (int)(2 * N),
                                          (uint32_t*)st.pk_split.p);
  split_halves_kernel<<<1024, 256, 0, s>>>((const uint64_t*)st.ksk.p, N * P.lks, (int)(n + 1),
                                          (uint32_t*)st.ksk_split.p);
  return cuda_err(cudaGetLastError());
}

// Power-of-two sets: both key-switching keys in the tensor-core form (limbs
// of f16, see fdfb_ks_tc.hpp).  A key whose digits are too wide for f16
// (log2 B > 11) keeps the CUDA-core contraction.
int install_tc_keys(SetState& st, cudaStream_t s) {
  const fdfb_params& P = st.prm;
  const int N = (int)P.N;
  const bool exact = st.mq.Q != 0;  // prime-modulus sets: exact integer sums, reduced mod Q afterwards
  int rc = tc_ks_prepare(st.tc_pk, st.pk.p, st.w, N, (int)P.lpk, (int)P.log2Bpk, 2 * N, s, exact);
  if (rc != FDFB_OK && rc != FDFB_EINVAL) return rc;
  rc = tc_ks_prepare(st.tc_ksk, st.ksk.p, st.w, N, (int)P.lks, (int)P.log2Bks, (int)P.n + 1, s, exact);
  if (rc != FDFB_OK && rc != FDFB_EINVAL) return rc;
  return FDFB_OK;
}

// Bytes of the key switches' digit matrices per input of a pipeline (0
// without a tensor-core key): the packing key switch reads l_boot sign LWEs
// per input on the prime-modulus sets, one on the others.
size_t tc_digit_row_bytes(const SetState& st) {
  size_t r = 0;
  if (st.tc_pk.ready) r = std::max(r, (size_t)st.lboot * tc_ks_digits_bytes(st.tc_pk, 1));
  if (st.tc_ksk.ready) r = std::max(r, tc_ks_digits_bytes(st.tc_ksk, 1));
  return r;
}

int ensure_tc_digits(SetState& st, int64_t rows) {
  const size_t rb = tc_digit_row_bytes(st);
  if (rb == 0) return FDFB_OK;
  return st.tc_digits.ensure((size_t)rows * rb);
}

// Pipeline intermediates for `batch` inputs with k tables each: per input the
// sign LWE [N+1] and the packed RLWE [2N], per (input, table) the function
// accumulator [2N] and the extracted LWE [N+1].
// Prime-modulus sets (k = 1): per input lboot sign LWEs [N+1], their raw
// packing key-switch sums [4N] and packed RLWEs [2N], then accF [2N], cQ
// [N+1] and the raw LWE key-switch sums [2(n+1)], all 64-bit words; at N =
// 2^13 then per sign item the blind rotation's half results (n13_half_words).
size_t mq_scratch_words(const SetState& st, int64_t batch) {
  const size_t N = st.prm.N, lb = st.lboot, n = st.prm.n;
  return (size_t)batch * (lb * ((N + 1) + 4 * N + 2 * N) + 2 * N + (N + 1) + 2 * (n + 1));
}
// 32-bit words of one item's BRParams::half_y at N = 2^13 (half results
// [P][2][2][KH][4096] and the accumulator [2][8192] words, the largest over
// the set's variants), else 0.
size_t n13_half_words(const SetState& st) {
  if (st.L != 13) return 0;
  int pk = 0;
  for (const auto& v : st.var) pk = std::max(pk, v->ops->P * v->ops->key_halves);
  return (size_t)pk * 4 * 4096 + 4 * 8192;
}
// The half-result region of a prime-modulus scratch area laid out for `batch`
// inputs (after the 64-bit words above), or nullptr below N = 2^13.
uint32_t* n13_half_region(const SetState& st, void* base, int64_t batch) {
  if (!n13_half_words(st)) return nullptr;
  return (uint32_t*)((unsigned char*)base + mq_scratch_words(st, batch) * 8);
}
size_t scratch_bytes(const SetState& st, int64_t batch, int k) {
  const size_t N = st.prm.N;
  if (st.mq.Q) return mq_scratch_words(st, batch) * 8 + (size_t)batch * st.lboot * n13_half_words(st) * 4;
  return ((size_t)batch * ((N + 1) + 2 * N) + (size_t)batch * k * (2 * N + (N + 1))) * st.wbytes();
}

int ensure_scratch(SetState& st, int64_t batch, int k = 1) {
  FD_TRY(st.scratch.ensure(scratch_bytes(st, batch, k) + 256));
  return FDFB_OK;
}

// Key switching out[m] = (b_m, 0..) - sum_{i,j} Decomp(a_{m,i})_j key[i][j]
// of `batch` LWE samples of dimension n_in (figure "Key switching algorithm
// and its setup").  The reduction is split over enough CTAs to give every SM
// two when the output tiles alone would leave SMs idle; the split parts are
// added atomically into a zeroed output.
int launch_keyswitch(const fdfb_ctx* ctx, int w, const void* in, int64_t batch, int n_in,
                     const void* key, int ell, int log2B, int rt, int out_len, void* out,
                     cudaStream_t s, const TcKsKey* tk = nullptr, void* digits = nullptr) {
  if (batch <= 0) return FDFB_OK;
  // the tensor-core contraction when the key has a limb form and the caller
  // gave digit scratch (fdfb_test_hooks bit 1 forces the CUDA cores)
  if (tk && tk->ready && digits && !(ctx->test_flags & 2))
    return tc_keyswitch(*tk, in, batch, rt, out, digits, ctx->d_err, s);
  const int64_t tiles = (int64_t)((out_len + KS_BN - 1) / KS_BN) * ((batch + KS_BM - 1) / KS_BM);
  const int kt = (n_in * ell + KS_BK - 1) / KS_BK;
  int64_t split = (2 * (int64_t)ctx->sms + tiles - 1) / tiles;
  if (split > kt / 4) split = kt / 4;  // keep at least four reduction steps per slice
  if (split > 64) split = 64;
  if (split < 1) split = 1;
  dim3 grid((unsigned)((batch + KS_BM - 1) / KS_BM), (unsigned)((out_len + KS_BN - 1) / KS_BN),
            (unsigned)split);
  const size_t wb = (size_t)w / 8;
  if (split > 1) FD_CUDA(cudaMemsetAsync(out, 0, (size_t)batch * out_len * wb, s));
  if (w == 32)
    keyswitch_kernel<uint32_t><<<grid, KS_THREADS, 0, s>>>((const uint32_t*)in, batch, n_in,
                                                          (const uint32_t*)key, ell, log2B, rt, out_len,
                                                          (uint32_t*)out, (int)split);
  else
    keyswitch_kernel<uint64_t><<<grid, KS_THREADS, 0, s>>>((const uint64_t*)in, batch, n_in,
                                                          (const uint64_t*)key, ell, log2B, rt, out_len,
                                                          (uint64_t*)out, (int)split);
  return cuda_err(cudaGetLastError());
}

// Prime-modulus key switching: the exact sums of the two key halves
// (keyswitch_kernel<uint64_t, uint32_t>, raw), then ks_finalize_q_kernel:
// out = ([b, 0..] - sums) mod Q, and with logq > 0 ModSwitch(Q -> 2^logq).
int launch_keyswitch_q(const fdfb_ctx* ctx, const SetState& st, const uint64_t* in, int64_t batch,
                       int n_in, const uint32_t* key_split, int ell, int log2B, int out_len,
                       uint64_t* sums, int logq, uint64_t* out, cudaStream_t s, const TcKsKey* tk = nullptr,
                       void* digits = nullptr) {
  if (batch <= 0) return FDFB_OK;
  if (tk && tk->ready && digits && !(ctx->test_flags & 2)) {
    // the exact sums on the tensor cores, in the layout the reduction reads
    FD_TRY(tc_keyswitch(*tk, in, batch, 0, sums, digits, ctx->d_err, s));
    const int64_t total = batch * out_len;
    const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 8 * (int64_t)ctx->sms);
    ks_finalize_q_kernel<<<blocks, 256, 0, s>>>(in, n_in, batch, sums, out_len, st.mq, logq, out);
    return cuda_err(cudaGetLastError());
  }
  const int cols = 2 * out_len;
  const int64_t tiles = (int64_t)((cols + KS_BN - 1) / KS_BN) * ((batch + KS_BM - 1) / KS_BM);
  const int kt = (n_in * ell + KS_BK - 1) / KS_BK;
  int64_t split = (2 * (int64_t)ctx->sms + tiles - 1) / tiles;
  if (split > kt / 4) split = kt / 4;
  if (split > 64) split = 64;
  if (split < 1) split = 1;
  dim3 grid((unsigned)((batch + KS_BM - 1) / KS_BM), (unsigned)((cols + KS_BN - 1) / KS_BN), (unsigned)split);
  if (split > 1) FD_CUDA(cudaMemsetAsync(sums, 0, (size_t)batch * cols * 8, s));
  keyswitch_kernel<uint64_t, uint32_t><<<grid, KS_THREADS, 0, s>>>(in, batch, n_in, key_split, ell, log2B, 0,
                                                                   cols, sums, (int)split, 1);
  FD_CUDA(cudaGetLastError());
  const int64_t total = batch * out_len;
  const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 8 * (int64_t)ctx->sms);
  ks_finalize_q_kernel<<<blocks, 256, 0, s>>>(in, n_in, batch, sums, out_len, st.mq, logq, out);
  return cuda_err(cudaGetLastError());
}

void fill_br_q(BRParams& br, const SetState& st) {
  br.mq = st.mq;
  for (int i = 0; i < 8; ++i) br.sgn_scale[i] = st.sgn_scale[i];
  br.rtrunc = 0;
}

// Pipeline stages as NVTX ranges (shown by external profilers on the host
// timeline, with the launches they enqueue).
const char* const kStageNames[kStages] = {
    "fdfb: sign blind rotation", "fdfb: packing key switch", "fdfb: PubMux / TFHE accumulator",
    "fdfb: function blind rotation", "fdfb: LWE key switch", "fdfb: blind rotations"};

// Brackets one launch with an NVTX range, and with an event pair when the
// measurement hook is on (the no-allocation path passes ctx = nullptr: no
// events are created there; the NVTX range needs no runtime object).
struct StageTimer {
  fdfb_ctx* ctx;
  int stage;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  StageTimer(fdfb_ctx* c, int st, cudaStream_t str) : ctx(c), stage(st), s(str) {
    nvtxRangePushA(kStageNames[stage]);
    if (ctx && ctx->prof && cudaEventCreate(&a) == cudaSuccess) cudaEventRecord(a, s);
  }
  ~StageTimer() {
    nvtxRangePop();
    if (!a) return;
    cudaEvent_t b;
    if (cudaEventCreate(&b) == cudaSuccess) {
      cudaEventRecord(b, s);
      ctx->marks.push_back({stage, a, b});
    } else {
      cudaEventDestroy(a);
    }
  }
};

// The Bootstrap figure for a prime-modulus set (one table per input):
// lboot sign rotations per input (item i of input b starts from L_boot^i
// Delta/2 sgnP X^{b_N}), SampleExtract + the same constant, the packing key
// switch of every sign LWE, PubMux over the lboot digits of p, the function
// rotation, SampleExtract, KeySwitch(ksK) and ModSwitch(Q -> q = 2N).
int run_pipeline_q(fdfb_ctx* ctx, SetState& st, const void* ct_in, const int32_t* lut_ids,
                   int64_t batch, int k, void* ct_out, const fdfb_debug_bufs* dbg, cudaStream_t s,
                   void* fixed_scratch, bool timed, void* dig) {
  if (k != 1) return FDFB_EINVAL;
  const fdfb_params& P = st.prm;
  const size_t N = P.N, n = P.n, lb = st.lboot;
  if (batch * (int64_t)lb > 0x7fffffff) return FDFB_EINVAL;
  if (!fixed_scratch) FD_TRY(ensure_scratch(st, batch, 1));
  unsigned char* base = fixed_scratch ? (unsigned char*)fixed_scratch : (unsigned char*)st.scratch.p;
  fdfb_ctx* tctx = timed ? ctx : nullptr;
  uint64_t* sgn = (uint64_t*)base;
  uint64_t* sums_pk = sgn + (size_t)batch * lb * (N + 1);
  uint64_t* cR = sums_pk + (size_t)batch * lb * 4 * N;
  uint64_t* accF = cR + (size_t)batch * lb * 2 * N;
  uint64_t* cQ = accF + (size_t)batch * 2 * N;
  uint64_t* sums_ks = cQ + (size_t)batch * (N + 1);
  if (dbg) {
    if (dbg->sgn) sgn = (uint64_t*)dbg->sgn;
    if (dbg->cR) cR = (uint64_t*)dbg->cR;
    if (dbg->accF) accF = (uint64_t*)dbg->accF;
    if (dbg->cQ) cQ = (uint64_t*)dbg->cQ;
  }
  const int64_t items = batch * (int64_t)lb;
  Variant& bv = st.br();
  BRParams br{};
  br.S = bv.S;
  br.bsk = (const uint32_t*)bv.bsk_ntt.p;
  br.ct = ct_in;
  br.acc0 = nullptr;
  br.lwe_out = sgn;
  br.ctN_out = nullptr;
  br.n = P.n;
  br.lg = P.lg;
  br.log2Bg = P.log2Bg;
  br.batch = items;
  br.sign_mode = 1;
  br.smem_r1 = bv.br_r1;
  br.smem_exch = bv.br_ex;
  br.rep = (int)lb;
  br.signed_digits = 0;
  br.err = ctx->d_err;
  fill_br_q(br, st);
  br.half_y = n13_half_region(st, base, batch);
  {
    StageTimer tm(tctx, 0, s);
    FD_CUDA(bv.ops->br(br, items, bv.br_smem, s));
  }
  {
    StageTimer tm(tctx, 1, s);
    FD_TRY(launch_keyswitch_q(ctx, st, sgn, items, (int)N, (const uint32_t*)st.pk_split.p, P.lpk,
                              P.log2Bpk, (int)(2 * N), sums_pk, 0, cR, s, &st.tc_pk, dig));
  }
  PubMuxQParams pm{};
  pm.S = st.base().S;
  pm.mq = st.mq;
  pm.cR = cR;
  pm.ct = (const uint64_t*)ct_in;
  pm.rep = 1;
  pm.lut_ids = lut_ids;
  pm.luts = (const int16_t*)st.luts.p;
  pm.n_luts = st.n_luts;
  pm.accF = accF;
  pm.n = P.n;
  pm.lboot = (int)lb;
  pm.log2Lboot = (int)P.log2Lboot;
  pm.delta = st.delta_q;
  pm.err = ctx->d_err;
  {
    StageTimer tm(tctx, 2, s);
    FD_CUDA(st.base().ops->pubmux_q(pm, batch, s));
  }
  br.acc0 = accF;
  br.lwe_out = cQ;
  br.sign_mode = 0;
  br.batch = batch;
  br.rep = 1;
  {
    StageTimer tm(tctx, 3, s);
    FD_CUDA(bv.ops->br(br, batch, bv.br_smem, s));
  }
  {
    StageTimer tm(tctx, 4, s);
    FD_TRY(launch_keyswitch_q(ctx, st, cQ, batch, (int)N, (const uint32_t*)st.ksk_split.p, P.lks,
                              P.log2Bks, (int)n + 1, sums_ks, (int)st.L + 1, (uint64_t*)ct_out, s, &st.tc_ksk,
                              dig));
    if (dbg && dbg->cKS) {
      const int64_t total = batch * (int64_t)(n + 1);
      const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 8 * (int64_t)ctx->sms);
      ks_finalize_q_kernel<<<blocks, 256, 0, s>>>(cQ, (int)N, batch, sums_ks, (int)n + 1, st.mq, 0,
                                                 (uint64_t*)dbg->cKS);
      FD_CUDA(cudaGetLastError());
    }
  }
  return FDFB_OK;
}

// One bootstrap pipeline on one parameter set (figure "functional-
// bootstrapping", left), steps 1-14, for `batch` inputs and k tables per
// input: steps 1-10 (sign rotation, packing key switch) once per input, steps
// 11-14 (PubMux, function rotation, key switch) once per (input, table) --
// the reuse of the sign accumulators for further functions of one input
// (Section "Application of Functional Bootstrapping", multiple univariate
// functions with the same input).  lut_ids and ct_out are [batch][k].
int run_pipeline(fdfb_ctx* ctx, SetState& st, const void* ct_in, const int32_t* lut_ids,
                 int64_t batch, int k, void* ct_out, const fdfb_debug_bufs* dbg, cudaStream_t s,
                 void* fixed_scratch = nullptr, bool timed = true, unsigned char* tc_digits = nullptr,
                 bool use_tc = true) {
  if (batch < 0 || k < 1) return FDFB_EINVAL;
  if (batch == 0) return FDFB_OK;
  if (!ct_in || !lut_ids || !ct_out) return FDFB_EINVAL;
  if (!st.keys) return FDFB_ENOKEYS;
  if (st.n_luts == 0) return FDFB_EBADLUT;
  if (batch * (int64_t)k > 0x7fffffff) return FDFB_EINVAL;
  // Digit matrices of the tensor-core key switches (a slice given by a
  // chunked caller, else the set's buffer grown to this call's inputs).
  void* dig = nullptr;
  if (use_tc && tc_digit_row_bytes(st) && !(ctx->test_flags & 2)) {
    if (!tc_digits) {
      FD_TRY(ensure_tc_digits(st, batch * k));
      tc_digits = (unsigned char*)st.tc_digits.p;
    }
    dig = tc_digits;
  }
  if (st.mq.Q) return run_pipeline_q(ctx, st, ct_in, lut_ids, batch, k, ct_out, dbg, s, fixed_scratch, timed, dig);
  const fdfb_params& P = st.prm;
  const size_t N = P.N, wb = st.wbytes();
  const int64_t items = batch * k;
  if (!fixed_scratch) FD_TRY(ensure_scratch(st, batch, k));
  unsigned char* base = fixed_scratch ? (unsigned char*)fixed_scratch : (unsigned char*)st.scratch.p;
  // The measurement hook creates CUDA events; the no-allocation path stays
  // free of any runtime object creation.
  fdfb_ctx* tctx = timed ? ctx : nullptr;
  void* sgn = base;
  void* cR = base + (size_t)batch * (N + 1) * wb;
  void* accF = (unsigned char*)cR + (size_t)batch * 2 * N * wb;
  void* cQ = (unsigned char*)accF + (size_t)items * 2 * N * wb;
  if (dbg) {
    if (dbg->sgn) sgn = dbg->sgn;
    if (dbg->cR) cR = dbg->cR;
    if (dbg->accF) accF = dbg->accF;
    if (dbg->cQ) cQ = dbg->cQ;
  }
  const uint64_t delta = (uint64_t)1 << (st.w - st.logtout);  // Delta' = q / t'

  // Steps 1-8: ModSwitch, sign accumulator, BlindRotate, SampleExtract + Delta/2.
  Variant& bv = st.br();
  BRParams br{};
  br.S = bv.S;
  br.bsk = (const uint32_t*)bv.bsk_ntt.p;
  br.ct = ct_in;
  br.acc0 = nullptr;
  br.lwe_out = sgn;
  br.ctN_out = dbg ? (uint32_t*)dbg->ctN : nullptr;
  br.n = P.n;
  br.lg = P.lg;
  br.log2Bg = P.log2Bg;
  br.rtrunc = trunc_bits(st.w, P.log2Bg, P.lg);
  br.batch = batch;
  br.delta_half = delta / 2;
  br.sign_mode = 1;
  br.smem_r1 = bv.br_r1;
  br.smem_exch = bv.br_ex;
  br.rep = 1;
  br.signed_digits = (int)P.signed_digits;
  br.err = ctx->d_err;
  if (ctx->test_flags & 1) {  // fdfb_test_hooks: no staged-key copies, a short bounded wait
    br.test_skip_key_copy = 1;
    br.key_wait_polls = 1u << 12;
  }
  {
    StageTimer tm(tctx, 0, s);
    FD_CUDA(bv.ops->br(br, batch, bv.br_smem, s));
  }

  // Steps 9-11, BuildAcc: KeySwitch to RLWE with pK, then PubMux.
  {
    StageTimer tm(tctx, 1, s);
    FD_TRY(launch_keyswitch(ctx, st.w, sgn, batch, (int)N, st.pk.p, P.lpk, P.log2Bpk,
                            trunc_bits(st.w, P.log2Bpk, P.lpk), (int)(2 * N), cR, s, &st.tc_pk, dig));
  }
  PubMuxParams pm{};
  pm.S = st.base().S;
  pm.cR = cR;
  pm.ct = ct_in;
  pm.rep = k;
  pm.lut_ids = lut_ids;
  pm.luts = (const int16_t*)st.luts.p;
  pm.n_luts = st.n_luts;
  pm.accF = accF;
  pm.n = P.n;
  pm.t = st.tout;
  pm.delta = delta;
  pm.err = ctx->d_err;
  {
    StageTimer tm(tctx, 2, s);
    FD_CUDA(st.base().ops->pubmux(pm, items, s));
  }

  // Steps 12-13: function BlindRotate, SampleExtract.
  br.acc0 = accF;
  br.lwe_out = cQ;
  br.ctN_out = nullptr;
  br.sign_mode = 0;
  br.batch = items;
  br.rep = k;
  {
    StageTimer tm(tctx, 3, s);
    FD_CUDA(bv.ops->br(br, items, bv.br_smem, s));
  }

  // Step 14: KeySwitch with ksK (ModSwitch Q -> q is the identity, q = Q;
  // the prime-modulus sets take run_pipeline_q).
  {
    StageTimer tm(tctx, 4, s);
    FD_TRY(launch_keyswitch(ctx, st.w, cQ, items, (int)N, st.ksk.p, P.lks, P.log2Bks,
                            trunc_bits(st.w, P.log2Bks, P.lks), (int)P.n + 1, ct_out, s, &st.tc_ksk, dig));
  }
  return FDFB_OK;
}

constexpr int kMaxChunks = 8;

// Library side streams (and count + 1 fork/join events) for chunked calls.
int ensure_chunk_streams(fdfb_ctx* ctx, int count) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  while ((int)ctx->chunk_side.size() < count) {
    cudaStream_t ns;
    FD_CUDA(cudaStreamCreateWithFlags(&ns, cudaStreamNonBlocking));
    ctx->chunk_side.push_back(ns);
  }
  while ((int)ctx->chunk_events.size() < count + 1) {
    cudaEvent_t e;
    FD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ctx->chunk_events.push_back(e);
  }
  return FDFB_OK;
}

// The pipeline on `chunks` consecutive slices of the inputs, each on its own
// library side stream forked from and joined back to s, each slice on its
// own part of the set's scratch.  The launches of different slices overlap on
// the GPU, so the last wave of one blind-rotation launch shares the SMs with
// the next launch instead of leaving them idle.  Results are those of one
// pipeline over the whole batch (every ciphertext is independent).
int run_chunked(fdfb_ctx* ctx, SetState& st, const void* ct_in, const int32_t* lut_ids,
                int64_t batch, int k, void* ct_out, cudaStream_t s, int chunks) {
  if (chunks <= 1 || batch < 2 * (int64_t)chunks)
    return run_pipeline(ctx, st, ct_in, lut_ids, batch, k, ct_out, nullptr, s);
  if (k < 1 || !ct_in || !lut_ids || !ct_out) return FDFB_EINVAL;
  if (!st.keys) return FDFB_ENOKEYS;
  if (st.n_luts == 0) return FDFB_EBADLUT;
  if (batch * (int64_t)k > 0x7fffffff) return FDFB_EINVAL;
  FD_TRY(ensure_scratch(st, batch, k));
  FD_TRY(ensure_chunk_streams(ctx, chunks));
  const bool tc = tc_digit_row_bytes(st) && !(ctx->test_flags & 2);
  if (tc) FD_TRY(ensure_tc_digits(st, batch * k));
  const size_t drow = tc_digit_row_bytes(st);
  const size_t wb = st.wbytes(), row = (size_t)(st.prm.n + 1) * wb;
  unsigned char* base = (unsigned char*)st.scratch.p;
  FD_CUDA(cudaEventRecord(ctx->chunk_events[0], s));
  for (int c = 0; c < chunks; ++c) FD_CUDA(cudaStreamWaitEvent(ctx->chunk_side[c], ctx->chunk_events[0], 0));
  int rc = FDFB_OK;
  for (int c = 0; c < chunks && rc == FDFB_OK; ++c) {
    const int64_t b0 = batch * c / chunks, b1 = batch * (c + 1) / chunks;
    rc = run_pipeline(ctx, st, (const unsigned char*)ct_in + b0 * row, lut_ids + b0 * k, b1 - b0, k,
                      (unsigned char*)ct_out + b0 * k * row, nullptr, ctx->chunk_side[c],
                      base + scratch_bytes(st, b0, k), true,
                      tc ? (unsigned char*)st.tc_digits.p + (size_t)b0 * k * drow : nullptr, tc);
  }
  // Join even after an error, so the caller's stream never runs ahead of
  // work already queued on the side streams.
  for (int c = 0; c < chunks; ++c) {
    FD_CUDA(cudaEventRecord(ctx->chunk_events[1 + c], ctx->chunk_side[c]));
    FD_CUDA(cudaStreamWaitEvent(s, ctx->chunk_events[1 + c], 0));
  }
  return rc;
}

// Scratch of fdfb_bootstrap_noalloc: a file-scope device array, so that the
// entry point itself never allocates.  Every GPU that loads the library
// holds it until the process exits.
constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch per device (the host-side symbol is only
// a stand-in and must never be handed to a kernel).
std::mutex g_noalloc_mu;
void* g_noalloc_addr[64] = {nullptr};

int noalloc_scratch(int device, void** out) {
  if (device < 0 || device >= 64) return FDFB_EINVAL;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[device]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
      cudaGetLastError();
      return FDFB_ECUDA;
    }
    g_noalloc_addr[device] = ptr;
  }
  *out = g_noalloc_addr[device];
  return FDFB_OK;
}

// Chooses how many chunks fdfb_bootstrap splits a batch of `batch` into: the
// whole pipeline on zero trial ciphertexts (table 0) is timed with 1, 2, 3,
// 4, 6 and 8 chunks.  Only batches below 8 waves of the blind rotation are
// tried (beyond that the last partial wave costs little) and only when a
// table is installed; otherwise one chunk.
int tune_chunks(fdfb_ctx* ctx, SetState& st, int64_t batch, cudaStream_t s) {
  int dev_sms = 0;
  FD_CUDA(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, ctx->device));
  const int per_sm = st.br().ops->br_blocks_per_sm(st.br().br_smem);
  const int64_t slots = (int64_t)dev_sms * (per_sm > 0 ? per_sm : 1);
  int best = 1;
  if (st.n_luts > 0 && batch >= 2 && batch < 8 * slots) {
    const size_t row = (size_t)(st.prm.n + 1) * st.wbytes();
    DevBuf in, out, ids;
    FD_TRY(in.ensure(batch * row));
    FD_TRY(out.ensure(batch * row));
    FD_TRY(ids.ensure(batch * sizeof(int32_t)));
    FD_CUDA(cudaMemsetAsync(in.p, 0, batch * row, s));
    FD_CUDA(cudaMemsetAsync(ids.p, 0, batch * sizeof(int32_t), s));
    FD_TRY(ensure_scratch(st, batch, 1));
    FD_TRY(ensure_chunk_streams(ctx, kMaxChunks));
    cudaEvent_t a, b;
    FD_CUDA(cudaEventCreate(&a));
    FD_CUDA(cudaEventCreate(&b));
    float best_ms = 1e30f;
    int rc = FDFB_OK;
    for (int c : {1, 2, 3, 4, 6, 8}) {
      if (rc != FDFB_OK || c > kMaxChunks) break;
      float ms_c = 1e30f;
      for (int rep = 0; rep < 2 && rc == FDFB_OK; ++rep) {
        cudaEventRecord(a, s);
        rc = run_chunked(ctx, st, in.p, (const int32_t*)ids.p, batch, 1, out.p, s, c);
        cudaEventRecord(b, s);
        if (cudaEventSynchronize(b) != cudaSuccess) rc = cuda_err(cudaGetLastError());
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        if (rep > 0 && ms < ms_c) ms_c = ms;  // the first run warms caches
      }
      if (ms_c < best_ms) {
        best_ms = ms_c;
        best = c;
      }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    FD_CUDA(cudaStreamSynchronize(s));
    if (rc != FDFB_OK) return rc;
  }
  std::lock_guard<std::mutex> lk(ctx->mu);
  st.chunks = best;
  return FDFB_OK;
}

// Registration of a prime-modulus set (fdfb_params.Q != 0): checks the
// shape (Q = 2^k - c, exact decompositions, l_boot <= 8), the exactness of
// every lift with the primes of each variant, and builds the variants.
int register_q(fdfb_ctx* ctx, const fdfb_params& P, int* set_id_out) {
  if (P.k != 1 || P.log2q != 64) return FDFB_EINVAL;
  if (P.N != 256 && P.N != 1024 && P.N != 2048 && P.N != 4096 && P.N != 8192) return FDFB_EINVAL;
  if (P.n < 1 || P.n > 4096) return FDFB_EINVAL;
  if (P.t < 2 || P.t > P.N) return FDFB_EINVAL;  // any t: CRT moduli need not divide q = 2N
  if (P.signed_digits || P.t_out) return FDFB_EINVAL;
  const uint64_t Q = P.Q;
  int kbits = 64;
  while (kbits > 0 && !((Q >> (kbits - 1)) & 1)) --kbits;
  if (kbits < 32 || kbits > 63) return FDFB_EINVAL;
  const uint64_t c = ((uint64_t)1 << kbits) - Q;
  if (!(Q & 1) || c == 0 || c >= ((uint64_t)1 << 20)) return FDFB_EINVAL;
  auto exact_l = [&](uint32_t log2B, uint32_t l) {
    return log2B >= 1 && log2B <= 16 && l == (uint32_t)((kbits + (int)log2B - 1) / (int)log2B);
  };
  if (!exact_l(P.log2Bg, P.lg) || !exact_l(P.log2Bks, P.lks) || !exact_l(P.log2Bpk, P.lpk)) return FDFB_EINVAL;
  if (P.log2Lboot < 1 || P.log2Lboot > 63 ||
      P.lboot != (uint32_t)((kbits + (int)P.log2Lboot - 1) / (int)P.log2Lboot) || P.lboot > 8)
    return FDFB_EINVAL;
  if (P.lg > 7) return FDFB_EINVAL;
  const int L = ilog2(P.N);
  const Ops* ops0 = find_ops_q(L, 0);
  if (!ops0 || ops0->P != 3) return FDFB_EINVAL;
  const long double B = ldexpl(1.0L, (int)P.log2Bg), Qh = (long double)Q / 2;
  const long double br_max = 2.0L * P.lg * P.N * (B - 1) * Qh;
  const long double pm_max = (long double)P.lboot * P.N * (ldexpl(1.0L, (int)std::min<uint32_t>(P.log2Lboot, 62)) - 1) * Qh;
  const long double enc_max = (long double)P.N * ldexpl(1.0L, kSkLimbBits - 1) * Qh;
  if (!host::lift_is_exact(3, br_max) || !host::lift_is_exact(3, pm_max) || !host::lift_is_exact(3, enc_max))
    return FDFB_EINVAL;

  std::lock_guard<std::mutex> lk(ctx->mu);
  DeviceGuard g(ctx->device);
  auto st = std::make_unique<SetState>();
  st->prm = P;
  st->w = 64;
  st->L = L;
  st->logt = ilog2(P.t);
  st->tout = (int)P.t;
  st->logtout = st->logt;
  st->mq = ModQ{Q, c, kbits, modq_folds(Q, c, kbits), modq_folds64(Q, c, kbits)};
  st->lboot = (int)P.lboot;
  const uint64_t h = (uint64_t)(((unsigned __int128)Q + P.t) / (2 * (uint64_t)P.t));  // round(Q / 2t)
  st->delta_q = (uint64_t)(((unsigned __int128)Q + P.t / 2) / P.t);                // round(Q / t)
  uint64_t Lpow = 1;
  for (int i = 0; i < st->lboot; ++i) {
    st->sgn_scale[i] = host::mulmod(Lpow, h, Q);
    Lpow = host::mulmod(Lpow, P.log2Lboot >= 64 ? 0 : (((uint64_t)1 << P.log2Lboot) % Q), Q);
  }
  int max_smem = 0;
  FD_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
  for (int vi = 0;; ++vi) {
    const Ops* ops = find_ops_q(L, vi);
    if (!ops) break;
    if ((int)P.log2Bg > ops->max_log2B) continue;
    if (ops->key_halves == 2 && !host::lift_is_exact(ops->P, 2.0L * P.lg * P.N * (B - 1) * ldexpl(1.0L, 31)))
      continue;
    if (ops->key_halves == 1 && !host::lift_is_exact(ops->P, br_max)) continue;
    // two primes with whole key words reduce their lift in 64 bits (k <= 60)
    if (ops->P == 2 && ops->key_halves == 1 && kbits > 60) continue;
    auto v = std::make_unique<Variant>();
    v->ops = ops;
    v->br_smem = ops->br_smem((int)P.n, (int)P.lg, &v->br_r1, &v->br_ex);
    if (v->br_smem > (size_t)max_smem) continue;
    FD_CUDA(ops->br_prepare(v->br_smem));
    std::vector<uint2> fwd, inv;
    if (L == 13)
      host::make_prime_set_n13(ops->P, ops->EL, v->S, fwd, inv);
    else
      host::make_prime_set(ops->P, L, ops->EL, v->S, fwd, inv, ops->family);
    FD_TRY(v->tw.ensure((fwd.size() + inv.size()) * sizeof(uint2)));
    FD_CUDA(cudaMemcpy(v->tw.p, fwd.data(), fwd.size() * sizeof(uint2), cudaMemcpyHostToDevice));
    FD_CUDA(cudaMemcpy((uint2*)v->tw.p + fwd.size(), inv.data(), inv.size() * sizeof(uint2),
                       cudaMemcpyHostToDevice));
    v->S.tw_fwd = (const uint2*)v->tw.p;
    v->S.tw_inv = (const uint2*)v->tw.p + fwd.size();
    st->var.push_back(std::move(v));
  }
  if (st->var.empty() || st->var[0]->ops != ops0) return FDFB_EINVAL;
  ctx->sets.push_back(std::move(st));
  *set_id_out = (int)ctx->sets.size() - 1;
  return FDFB_OK;
}

// Key generation of a prime-modulus set: GLWE samples with the uniform key
// sk_q (rlwe_encrypt_q_kernel over its 13-bit limbs) and LWE samples mod Q.
int keys_generate_q(fdfb_ctx* ctx, SetState* st, const fdfb_keygen_inputs* in, cudaStream_t s) {
  if (!in->sk_q) return FDFB_EINVAL;
  const fdfb_params& P = st->prm;
  const size_t n = P.n, N = P.N;
  const uint64_t Q = st->mq.Q;
  for (size_t j = 0; j < N; ++j)
    if (in->sk_q[j] >= Q) return FDFB_EINVAL;
  uint64_t wb_, wp_, wk_;
  fdfb_key_words(&P, 0, &wb_);
  fdfb_key_words(&P, 1, &wp_);
  fdfb_key_words(&P, 2, &wk_);
  FD_TRY(st->bsk.ensure(wb_ * 8));
  FD_TRY(st->pk.ensure(wp_ * 8));
  FD_TRY(st->ksk.ensure(wk_ * 8));
  Variant& v0 = st->base();
  DevBuf d_sk, d_limbs, d_skl, d_s, d_a, d_e, d_mu, d_comp;
  FD_TRY(d_sk.ensure(N * 8));
  FD_TRY(d_limbs.ensure((size_t)kSkLimbs * 2 * N * 8));
  FD_TRY(d_skl.ensure((size_t)kSkLimbs * v0.ops->P * 2 * N * 4));
  FD_TRY(d_s.ensure(n));
  FD_CUDA(cudaMemcpyAsync(d_sk.p, in->sk_q, N * 8, cudaMemcpyHostToDevice, s));
  FD_CUDA(cudaMemcpyAsync(d_s.p, in->s, n, cudaMemcpyHostToDevice, s));
  sk_limbs_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>((const uint64_t*)d_sk.p, (int)N, st->mq,
                                                             (uint64_t*)d_limbs.p);
  FD_CUDA(cudaGetLastError());
  FD_CUDA(v0.ops->bsk_ntt(v0.S, d_limbs.p, kSkLimbs, 1, (uint32_t*)d_skl.p, Q, s));
  auto glwe = [&](size_t rows, const void* a, const int64_t* e, const std::vector<uint64_t>& mu,
                  const std::vector<uint8_t>& comp, void* out) -> int {
    FD_TRY(d_a.ensure(rows * N * 8));
    FD_TRY(d_e.ensure(rows * N * 8));
    FD_TRY(d_mu.ensure(rows * 8));
    FD_TRY(d_comp.ensure(rows));
    FD_CUDA(cudaMemcpyAsync(d_a.p, a, rows * N * 8, cudaMemcpyHostToDevice, s));
    FD_CUDA(cudaMemcpyAsync(d_e.p, e, rows * N * 8, cudaMemcpyHostToDevice, s));
    FD_CUDA(cudaMemcpyAsync(d_mu.p, mu.data(), rows * 8, cudaMemcpyHostToDevice, s));
    FD_CUDA(cudaMemcpyAsync(d_comp.p, comp.data(), rows, cudaMemcpyHostToDevice, s));
    RlweEncQParams rp{v0.S, st->mq, (const uint32_t*)d_skl.p, (const uint64_t*)d_a.p, (const int64_t*)d_e.p,
                      (const uint64_t*)d_mu.p, (const uint8_t*)d_comp.p, (uint64_t*)out};
    FD_CUDA(v0.ops->rlwe_enc_q(rp, (int64_t)rows, s));
    FD_CUDA(cudaStreamSynchronize(s));
    return FDFB_OK;
  };
  auto gpow = [&](uint32_t log2B, int j) {  // B^j mod Q
    uint64_t r = 1;
    for (int i = 0; i < j; ++i) r = host::mulmod(r, ((uint64_t)1 << log2B) % Q, Q);
    return r;
  };
  {  // BRKeyGen: row r = c lg + j adds s_i B^j to component c
    const size_t rows = n * 2 * P.lg;
    std::vector<uint64_t> mu(rows);
    std::vector<uint8_t> comp(rows);
    for (size_t i = 0; i < n; ++i)
      for (size_t r = 0; r < 2 * P.lg; ++r) {
        mu[i * 2 * P.lg + r] = in->s[i] ? gpow(P.log2Bg, (int)(r % P.lg)) : 0;
        comp[i * 2 * P.lg + r] = (uint8_t)(r / P.lg);
      }
    FD_TRY(glwe(rows, in->bsk_a, in->bsk_e, mu, comp, st->bsk.p));
  }
  {  // pK: RLWE(s_F[i] B_pk^j), s_F = Coefs(sk_q)
    const size_t rows = N * P.lpk;
    std::vector<uint64_t> mu(rows);
    std::vector<uint8_t> comp(rows, 0);
    for (size_t i = 0; i < N; ++i)
      for (size_t j = 0; j < P.lpk; ++j) mu[i * P.lpk + j] = host::mulmod(in->sk_q[i], gpow(P.log2Bpk, (int)j), Q);
    FD_TRY(glwe(rows, in->pk_a, in->pk_e, mu, comp, st->pk.p));
  }
  {  // ksK: LWE_s(s_F[i] B_ks^j)
    const size_t rows = N * P.lks;
    std::vector<uint64_t> mu(rows);
    for (size_t i = 0; i < N; ++i)
      for (size_t j = 0; j < P.lks; ++j) mu[i * P.lks + j] = host::mulmod(in->sk_q[i], gpow(P.log2Bks, (int)j), Q);
    FD_TRY(d_a.ensure(rows * n * 8));
    FD_TRY(d_e.ensure(rows * 8));
    FD_TRY(d_mu.ensure(rows * 8));
    FD_CUDA(cudaMemcpyAsync(d_a.p, in->ksk_a, rows * n * 8, cudaMemcpyHostToDevice, s));
    FD_CUDA(cudaMemcpyAsync(d_e.p, in->ksk_e, rows * 8, cudaMemcpyHostToDevice, s));
    FD_CUDA(cudaMemcpyAsync(d_mu.p, mu.data(), rows * 8, cudaMemcpyHostToDevice, s));
    lwe_encrypt_q_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, s>>>(
        (const uint8_t*)d_s.p, (const uint64_t*)d_a.p, (const int64_t*)d_e.p, (const uint64_t*)d_mu.p,
        (int64_t)rows, (int)n, st->mq, (uint64_t*)st->ksk.p);
    FD_CUDA(cudaGetLastError());
    FD_CUDA(cudaStreamSynchronize(s));
  }
  FD_TRY(install_bsk_ntt(*st, s));
  FD_TRY(install_split_keys(*st, s));
  FD_TRY(install_tc_keys(*st, s));
  FD_CUDA(cudaStreamSynchronize(s));
  st->keys = true;
  return FDFB_OK;
}

// The TFHE bootstrap's accumulator kernel for ring degree 2^L.
template <typename W>
cudaError_t launch_tfhe_acc(int L, int64_t batch, cudaStream_t s, const W* ct, int n, const int32_t* ids,
                            const W* polys, int n_polys, W* acc, int* err, uint64_t Q) {
  switch (L) {
    case 8: tfhe_acc_kernel<W, 8><<<(unsigned)batch, 256, 0, s>>>(ct, n, ids, polys, n_polys, acc, err, Q); break;
    case 9: tfhe_acc_kernel<W, 9><<<(unsigned)batch, 256, 0, s>>>(ct, n, ids, polys, n_polys, acc, err, Q); break;
    case 10: tfhe_acc_kernel<W, 10><<<(unsigned)batch, 256, 0, s>>>(ct, n, ids, polys, n_polys, acc, err, Q); break;
    case 11: tfhe_acc_kernel<W, 11><<<(unsigned)batch, 256, 0, s>>>(ct, n, ids, polys, n_polys, acc, err, Q); break;
    case 12: tfhe_acc_kernel<W, 12><<<(unsigned)batch, 256, 0, s>>>(ct, n, ids, polys, n_polys, acc, err, Q); break;
    case 13: tfhe_acc_kernel<W, 13><<<(unsigned)batch, 256, 0, s>>>(ct, n, ids, polys, n_polys, acc, err, Q); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
}  // namespace

extern "C" {

const char* fdfb_strerror(int code) {
  switch (code) {
    case FDFB_OK: return "ok";
    case FDFB_EINVAL: return "invalid argument or unsupported parameters";
    case FDFB_ENOMEM: return "device allocation failed";
    case FDFB_ECUDA: return "CUDA runtime error";
    case FDFB_ETIMEOUT: return "device-side wait timed out";
    case FDFB_ENOKEYS: return "keys not installed for this parameter set";
    case FDFB_EBADLUT: return "bad lookup table id or entry";
    default: return "unknown error";
  }
}

int fdfb_create(fdfb_ctx** out, int device) {
  if (!out) return FDFB_EINVAL;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return FDFB_ECUDA;
  }
  DeviceGuard g(device);
  auto* ctx = new fdfb_ctx();
  ctx->device = device;
  if (cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    cudaGetLastError();
    ctx->sms = 1;
  }
  if (cudaMalloc(&ctx->d_err, sizeof(int)) != cudaSuccess ||
      cudaMemset(ctx->d_err, 0, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return FDFB_ENOMEM;
  }
  *out = ctx;
  return FDFB_OK;
}

int fdfb_destroy(fdfb_ctx* ctx) {
  if (!ctx) return FDFB_EINVAL;
  {
    DeviceGuard g(ctx->device);
    for (cudaStream_t st : ctx->side) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
    for (cudaEvent_t e : ctx->events) cudaEventDestroy(e);
    for (cudaStream_t st : ctx->chunk_side) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
    for (cudaEvent_t e : ctx->chunk_events) cudaEventDestroy(e);
    ctx->sets.clear();
    if (ctx->d_err) cudaFree(ctx->d_err);
  }
  delete ctx;
  return FDFB_OK;
}

int fdfb_key_words(const fdfb_params* p, int which, uint64_t* words_out) {
  if (!p || !words_out) return FDFB_EINVAL;
  const uint64_t n = p->n, N = p->N;
  switch (which) {
    case 0: *words_out = n * 2 * p->lg * 2 * N; return FDFB_OK;
    case 1: *words_out = N * p->lpk * 2 * N; return FDFB_OK;
    case 2: *words_out = N * p->lks * (n + 1); return FDFB_OK;
    default: return FDFB_EINVAL;
  }
}

int fdfb_params_register(fdfb_ctx* ctx, const fdfb_params* prm, int* set_id_out) {
  if (!ctx || !prm || !set_id_out) return FDFB_EINVAL;
  const fdfb_params& P = *prm;
  if (P.Q) return register_q(ctx, P, set_id_out);
  if (P.k != 1 || (P.log2q != 32 && P.log2q != 64)) return FDFB_EINVAL;
  if (!is_pow2(P.N) || P.N < 256 || P.N > 4096) return FDFB_EINVAL;
  if (P.n < 1 || P.n > 4096) return FDFB_EINVAL;
  if (!is_pow2(P.t) || P.t < 2 || P.t > P.N) return FDFB_EINVAL;
  if (P.lg < 1 || P.lg > 4 || P.log2Bg < 1 || P.log2Bg > 16) return FDFB_EINVAL;
  if (P.lks < 1 || P.lks > 64 || P.log2Bks < 1 || P.log2Bks > 16) return FDFB_EINVAL;
  if (P.lpk < 1 || P.lpk > 64 || P.log2Bpk < 1 || P.log2Bpk > 16) return FDFB_EINVAL;
  if (P.lboot != 1 || P.log2Lboot != (uint32_t)ilog2(P.t)) return FDFB_EINVAL;
  if (P.signed_digits > 1) return FDFB_EINVAL;
  if (P.t_out && (!is_pow2(P.t_out) || P.t_out < 2 || P.t_out > (1u << 15))) return FDFB_EINVAL;
  const int w = (int)P.log2q, L = ilog2(P.N);
  const Ops* ops0 = find_ops(L, w, 0);
  if (!ops0) return FDFB_EINVAL;
  // Exactness of the lifted negacyclic products with the 30-bit primes of
  // variant 0 (which also serves PubMux and key generation); variants of the
  // lazy prime family are kept below only where the blind rotation stays exact.
  const long double q = ldexpl(1.0L, w);
  const long double br_max = 2.0L * P.lg * P.N * (ldexpl(1.0L, P.log2Bg) - 1) * (q / 2);
  const long double pm_max = (long double)P.N * ((P.t_out ? P.t_out : P.t) - 1) * q;
  const long double enc_max = (long double)P.N * q;
  if (!host::lift_is_exact(ops0->P, br_max) || !host::lift_is_exact(ops0->P, pm_max) ||
      !host::lift_is_exact(ops0->P, enc_max))
    return FDFB_EINVAL;

  std::lock_guard<std::mutex> lk(ctx->mu);
  DeviceGuard g(ctx->device);
  auto st = std::make_unique<SetState>();
  st->prm = P;
  st->w = w;
  st->L = L;
  st->logt = ilog2(P.t);
  st->tout = P.t_out ? (int)P.t_out : (int)P.t;
  st->logtout = ilog2((uint32_t)st->tout);
  int max_smem = 0;
  FD_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
  for (int vi = 0;; ++vi) {
    const Ops* ops = find_ops(L, w, vi);
    if (!ops) break;
    auto v = std::make_unique<Variant>();
    v->ops = ops;
    if ((int)P.log2Bg > ops->max_log2B) continue;  // digits too wide for this variant
    if (P.signed_digits && !ops->has_signed) continue;  // not built with balanced digits
    if (ops->family && !host::lift_is_exact(ops->P, br_max, ops->family)) continue;
    if (ops->key_halves == 2 &&
        !host::lift_is_exact(ops->P, 2.0L * P.lg * P.N * (ldexpl(1.0L, P.log2Bg) - 1) * ldexpl(1.0L, 31),
                             ops->family))
      continue;  // each key half's products must lift exactly
    v->br_smem = ops->br_smem((int)P.n, (int)P.lg, &v->br_r1, &v->br_ex);
    if (v->br_smem > (size_t)max_smem) {
      continue;
    }
    FD_CUDA(ops->br_prepare(v->br_smem));
    std::vector<uint2> fwd, inv;
    host::make_prime_set(ops->P, L, ops->EL, v->S, fwd, inv, ops->family);
    FD_TRY(v->tw.ensure((fwd.size() + inv.size()) * sizeof(uint2)));
    FD_CUDA(cudaMemcpy(v->tw.p, fwd.data(), fwd.size() * sizeof(uint2), cudaMemcpyHostToDevice));
    FD_CUDA(cudaMemcpy((uint2*)v->tw.p + fwd.size(), inv.data(), inv.size() * sizeof(uint2),
                       cudaMemcpyHostToDevice));
    v->S.tw_fwd = (const uint2*)v->tw.p;
    v->S.tw_inv = (const uint2*)v->tw.p + fwd.size();
    st->var.push_back(std::move(v));
  }
  if (st->var.empty() || st->var[0]->ops != ops0) return FDFB_EINVAL;
  ctx->sets.push_back(std::move(st));
  *set_id_out = (int)ctx->sets.size() - 1;
  return FDFB_OK;
}

int fdfb_keys_upload(fdfb_ctx* ctx, int set_id, const void* bsk, const void* pk, const void* ksk,
                     void* cuda_stream) {
  SetState* st = get_set(ctx, set_id);
  if (!st || !bsk || !pk || !ksk) return FDFB_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  DeviceGuard g(ctx->device);
  cudaStream_t s = as_stream(cuda_stream);
  uint64_t wb_, wp_, wk_;
  fdfb_key_words(&st->prm, 0, &wb_);
  fdfb_key_words(&st->prm, 1, &wp_);
  fdfb_key_words(&st->prm, 2, &wk_);
  const size_t wb = st->wbytes();
  FD_TRY(st->bsk.ensure(wb_ * wb));
  FD_TRY(st->pk.ensure(wp_ * wb));
  FD_TRY(st->ksk.ensure(wk_ * wb));
  FD_CUDA(cudaMemcpyAsync(st->bsk.p, bsk, wb_ * wb, cudaMemcpyHostToDevice, s));
  FD_CUDA(cudaMemcpyAsync(st->pk.p, pk, wp_ * wb, cudaMemcpyHostToDevice, s));
  FD_CUDA(cudaMemcpyAsync(st->ksk.p, ksk, wk_ * wb, cudaMemcpyHostToDevice, s));
  FD_TRY(install_bsk_ntt(*st, s));
  if (st->mq.Q) FD_TRY(install_split_keys(*st, s));
  FD_TRY(install_tc_keys(*st, s));
  FD_CUDA(cudaStreamSynchronize(s));
  st->keys = true;
  return FDFB_OK;
}

int fdfb_keys_generate(fdfb_ctx* ctx, int set_id, const fdfb_keygen_inputs* in, void* cuda_stream) {
  SetState* st = get_set(ctx, set_id);
  if (!st || !in || !in->s || !in->sk || !in->bsk_a || !in->bsk_e || !in->pk_a || !in->pk_e ||
      !in->ksk_a || !in->ksk_e)
    return FDFB_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  DeviceGuard g(ctx->device);
  cudaStream_t s = as_stream(cuda_stream);
  if (st->mq.Q) return keys_generate_q(ctx, st, in, s);
  const fdfb_params& P = st->prm;
  const size_t n = P.n, N = P.N, wb = st->wbytes();
  const int w = st->w;
  uint64_t wb_, wp_, wk_;
  fdfb_key_words(&P, 0, &wb_);
  fdfb_key_words(&P, 1, &wp_);
  fdfb_key_words(&P, 2, &wk_);
  FD_TRY(st->bsk.ensure(wb_ * wb));
  FD_TRY(st->pk.ensure(wp_ * wb));
  FD_TRY(st->ksk.ensure(wk_ * wb));

  DevBuf d_sk, d_s, d_a, d_e, d_mu, d_comp, d_m;
  FD_TRY(d_sk.ensure(N));
  FD_TRY(d_s.ensure(n));
  FD_CUDA(cudaMemcpyAsync(d_sk.p, in->sk, N, cudaMemcpyHostToDevice, s));
  FD_CUDA(cudaMemcpyAsync(d_s.p, in->s, n, cudaMemcpyHostToDevice, s));

  // BRKeyGen: rows r = c*lg + j of RGSW(s_i) add s_i * g_j to component c.
  {
    const size_t rows = n * 2 * P.lg;
    std::vector<uint64_t> mu(rows);
    std::vector<uint8_t> comp(rows);
    for (size_t i = 0; i < n; ++i)
      for (size_t r = 0; r < 2 * P.lg; ++r) {
        const int c = (int)(r / P.lg), j = (int)(r % P.lg);
        mu[i * 2 * P.lg + r] = in->s[i] ? gadget(w, P.log2Bg, P.lg, j) : 0;
        comp[i * 2 * P.lg + r] = (uint8_t)c;
      }
    FD_TRY(d_a.ensure(rows * N * wb));
    FD_TRY(d_e.ensure(rows * N * 8));
    FD_TRY(d_mu.ensure(rows * 8));
    FD_TRY(d_comp.ensure(rows));
    FD_CUDA(cudaMemcpyAsync(d_a.p, in->bsk_a, rows * N * wb, cudaMemcpyHostToDevice, s));
    FD_CUDA(cudaMemcpyAsync(d_e.p, in->bsk_e, rows * N * 8, cudaMemcpyHostToDevice, s));
    FD_CUDA(cudaMemcpyAsync(d_mu.p, mu.data(), rows * 8, cudaMemcpyHostToDevice, s));
    FD_CUDA(cudaMemcpyAsync(d_comp.p, comp.data(), rows, cudaMemcpyHostToDevice, s));
    RlweEncParams rp{st->base().S, (const uint8_t*)d_sk.p, d_a.p, (const int64_t*)d_e.p,
                     (const uint64_t*)d_mu.p, (const uint8_t*)d_comp.p, st->bsk.p};
    FD_CUDA(st->base().ops->rlwe_enc(rp, (int64_t)rows, s));
    FD_CUDA(cudaStreamSynchronize(s));
  }
  // KeySwitchSetup for pK: RLWE_sk(s_F[i] g_j), constant message polynomial.
  {
    const size_t rows = N * P.lpk;
    std::vector<uint64_t> mu(rows);
    std::vector<uint8_t> comp(rows, 0);
    for (size_t i = 0; i < N; ++i)
      for (size_t j = 0; j < P.lpk; ++j)
        mu[i * P.lpk + j] = in->sk[i] ? gadget(w, P.log2Bpk, P.lpk, (int)j) : 0;
    FD_TRY(d_a.ensure(rows * N * wb));
    FD_TRY(d_e.ensure(rows * N * 8));
    FD_TRY(d_mu.ensure(rows * 8));
    FD_TRY(d_comp.ensure(rows));
    FD_CUDA(cudaMemcpyAsync(d_a.p, in->pk_a, rows * N * wb, cudaMemcpyHostToDevice, s));
    FD_CUDA(cudaMemcpyAsync(d_e.p, in->pk_e, rows * N * 8, cudaMemcpyHostToDevice, s));
    FD_CUDA(cudaMemcpyAsync(d_mu.p, mu.data(), rows * 8, cudaMemcpyHostToDevice, s));
    FD_CUDA(cudaMemcpyAsync(d_comp.p, comp.data(), rows, cudaMemcpyHostToDevice, s));
    RlweEncParams rp{st->base().S, (const uint8_t*)d_sk.p, d_a.p, (const int64_t*)d_e.p,
                     (const uint64_t*)d_mu.p, (const uint8_t*)d_comp.p, st->pk.p};
    FD_CUDA(st->base().ops->rlwe_enc(rp, (int64_t)rows, s));
    FD_CUDA(cudaStreamSynchronize(s));
  }
  // KeySwitchSetup for ksK: LWE_s(s_F[i] g_j).
  {
    const size_t rows = N * P.lks;
    std::vector<int64_t> m(rows);
    for (size_t i = 0; i < N; ++i)
      for (size_t j = 0; j < P.lks; ++j)
        m[i * P.lks + j] = in->sk[i] ? (int64_t)gadget(w, P.log2Bks, P.lks, (int)j) : 0;
    FD_TRY(d_a.ensure(rows * n * wb));
    FD_TRY(d_e.ensure(rows * 8));
    FD_TRY(d_m.ensure(rows * 8));
    FD_CUDA(cudaMemcpyAsync(d_a.p, in->ksk_a, rows * n * wb, cudaMemcpyHostToDevice, s));
    FD_CUDA(cudaMemcpyAsync(d_e.p, in->ksk_e, rows * 8, cudaMemcpyHostToDevice, s));
    FD_CUDA(cudaMemcpyAsync(d_m.p, m.data(), rows * 8, cudaMemcpyHostToDevice, s));
    const unsigned blocks = (unsigned)((rows + 7) / 8);
    if (w == 32)
      lwe_encrypt_kernel<uint32_t><<<blocks, 256, 0, s>>>((const uint8_t*)d_s.p, (const uint32_t*)d_a.p,
                                                          (const int64_t*)d_e.p, (const int64_t*)d_m.p,
                                                          (int64_t)rows, (int)n, 1, (uint32_t*)st->ksk.p, 32);
    else
      lwe_encrypt_kernel<uint64_t><<<blocks, 256, 0, s>>>((const uint8_t*)d_s.p, (const uint64_t*)d_a.p,
                                                          (const int64_t*)d_e.p, (const int64_t*)d_m.p,
                                                          (int64_t)rows, (int)n, 1, (uint64_t*)st->ksk.p, 64);
    FD_CUDA(cudaGetLastError());
  }
  FD_TRY(install_bsk_ntt(*st, s));
  FD_TRY(install_tc_keys(*st, s));
  FD_CUDA(cudaStreamSynchronize(s));
  st->keys = true;
  return FDFB_OK;
}

int fdfb_keys_download(fdfb_ctx* ctx, int set_id, void* bsk, void* pk, void* ksk, void* cuda_stream) {
  SetState* st = get_set(ctx, set_id);
  if (!st) return FDFB_EINVAL;
  if (!st->keys) return FDFB_ENOKEYS;
  std::lock_guard<std::mutex> lk(ctx->mu);
  DeviceGuard g(ctx->device);
  cudaStream_t s = as_stream(cuda_stream);
  uint64_t wb_, wp_, wk_;
  fdfb_key_words(&st->prm, 0, &wb_);
  fdfb_key_words(&st->prm, 1, &wp_);
  fdfb_key_words(&st->prm, 2, &wk_);
  const size_t wb = st->wbytes();
  if (bsk) FD_CUDA(cudaMemcpyAsync(bsk, st->bsk.p, wb_ * wb, cudaMemcpyDeviceToHost, s));
  if (pk) FD_CUDA(cudaMemcpyAsync(pk, st->pk.p, wp_ * wb, cudaMemcpyDeviceToHost, s));
  if (ksk) FD_CUDA(cudaMemcpyAsync(ksk, st->ksk.p, wk_ * wb, cudaMemcpyDeviceToHost, s));
  FD_CUDA(cudaStreamSynchronize(s));
  return FDFB_OK;
}

int fdfb_lut_setup(fdfb_ctx* ctx, int set_id, const uint32_t* f, int* lut_id_out) {
  SetState* st = get_set(ctx, set_id);
  if (!st || !f || !lut_id_out) return FDFB_EINVAL;
  const int N = (int)st->prm.N, t = (int)st->prm.t;
  for (int m = 0; m < t; ++m)
    if (f[m] >= (uint32_t)st->tout) return FDFB_EBADLUT;  // entries lie in the output space Z_t'
  std::lock_guard<std::mutex> lk(ctx->mu);
  DeviceGuard g(ctx->device);
  const size_t off = st->luts_host.size();
  st->luts_host.resize(off + 2 * (size_t)N);
  setup_polynomial(N, t, f, st->luts_host.data() + off, st->luts_host.data() + off + N);
  // Tables are few and small: re-upload all of them after a device sync, so
  // no launch in flight still reads a buffer that is being replaced.
  FD_CUDA(cudaDeviceSynchronize());
  FD_TRY(st->luts.ensure(st->luts_host.size() * sizeof(int16_t)));
  FD_CUDA(cudaMemcpy(st->luts.p, st->luts_host.data(), st->luts_host.size() * sizeof(int16_t),
                     cudaMemcpyHostToDevice));
  *lut_id_out = st->n_luts++;
  return FDFB_OK;
}

int fdfb_tfhe_poly_setup(fdfb_ctx* ctx, int set_id, const void* poly, int* poly_id_out) {
  SetState* st = get_set(ctx, set_id);
  if (!st || !poly || !poly_id_out) return FDFB_EINVAL;
  const size_t N = st->prm.N;
  if (st->mq.Q)
    for (size_t j = 0; j < N; ++j)
      if (((const uint64_t*)poly)[j] >= st->mq.Q) return FDFB_EINVAL;  // residues mod Q
  std::lock_guard<std::mutex> lk(ctx->mu);
  DeviceGuard g(ctx->device);
  const size_t off = st->tpolys_host.size();
  st->tpolys_host.resize(off + N);
  for (size_t j = 0; j < N; ++j)
    st->tpolys_host[off + j] = st->w == 32 ? ((const uint32_t*)poly)[j] : ((const uint64_t*)poly)[j];
  // re-upload all polynomials after a device sync (no launch still reads the old buffer)
  FD_CUDA(cudaDeviceSynchronize());
  const size_t wb = st->wbytes(), count = st->tpolys_host.size();
  FD_TRY(st->tpolys.ensure(count * wb));
  if (st->w == 32) {
    std::vector<uint32_t> narrow(st->tpolys_host.begin(), st->tpolys_host.end());
    FD_CUDA(cudaMemcpy(st->tpolys.p, narrow.data(), count * wb, cudaMemcpyHostToDevice));
  } else {
    FD_CUDA(cudaMemcpy(st->tpolys.p, st->tpolys_host.data(), count * wb, cudaMemcpyHostToDevice));
  }
  *poly_id_out = st->n_tpolys++;
  return FDFB_OK;
}

int fdfb_tfhe_bootstrap(fdfb_ctx* ctx, int set_id, const void* ct_in, const int32_t* poly_ids,
                        int64_t batch, void* ct_out, void* cuda_stream) {
  SetState* st = get_set(ctx, set_id);
  if (!st || batch < 0 || batch > 0x7fffffff) return FDFB_EINVAL;
  if (batch == 0) return FDFB_OK;
  if (!ct_in || !poly_ids || !ct_out) return FDFB_EINVAL;
  if (!st->keys) return FDFB_ENOKEYS;
  if (st->n_tpolys == 0) return FDFB_EBADLUT;
  DeviceGuard g(ctx->device);
  cudaStream_t s = as_stream(cuda_stream);
  const fdfb_params& P = st->prm;
  const size_t N = P.N, wb = st->wbytes();
  FD_TRY(ensure_scratch(*st, batch, 1));
  unsigned char* base = (unsigned char*)st->scratch.p;
  void* accF = base + (size_t)batch * ((N + 1) + 2 * N) * wb;
  void* cQ = (unsigned char*)accF + (size_t)batch * 2 * N * wb;
  {
    StageTimer tm(ctx, 2, s);
    if (st->w == 32)
      FD_CUDA(launch_tfhe_acc<uint32_t>(st->L, batch, s, (const uint32_t*)ct_in, (int)P.n, poly_ids,
                                        (const uint32_t*)st->tpolys.p, st->n_tpolys, (uint32_t*)accF,
                                        ctx->d_err, 0));
    else
      FD_CUDA(launch_tfhe_acc<uint64_t>(st->L, batch, s, (const uint64_t*)ct_in, (int)P.n, poly_ids,
                                        (const uint64_t*)st->tpolys.p, st->n_tpolys, (uint64_t*)accF,
                                        ctx->d_err, st->mq.Q));
  }
  Variant& bv = st->br();
  BRParams br{};
  br.S = bv.S;
  br.bsk = (const uint32_t*)bv.bsk_ntt.p;
  br.ct = ct_in;
  br.acc0 = accF;
  br.lwe_out = cQ;
  br.n = P.n;
  br.lg = P.lg;
  br.log2Bg = P.log2Bg;
  br.rtrunc = trunc_bits(st->w, P.log2Bg, P.lg);
  br.batch = batch;
  br.sign_mode = 0;
  br.smem_r1 = bv.br_r1;
  br.smem_exch = bv.br_ex;
  br.rep = 1;
  br.signed_digits = (int)P.signed_digits;
  br.err = ctx->d_err;
  if (st->mq.Q) {
    fill_br_q(br, *st);
    br.half_y = n13_half_region(*st, base, batch);
  }
  {
    StageTimer tm(ctx, 3, s);
    FD_CUDA(bv.ops->br(br, batch, bv.br_smem, s));
  }
  {
    StageTimer tm(ctx, 4, s);
    if (st->mq.Q) {
      // exact half sums after cQ, then mod Q and ModSwitch(Q -> 2N)
      uint64_t* sums = (uint64_t*)((unsigned char*)cQ + (size_t)batch * (N + 1) * wb);
      void* dig = nullptr;
      if (tc_digit_row_bytes(*st) && !(ctx->test_flags & 2)) {
        FD_TRY(ensure_tc_digits(*st, batch));
        dig = st->tc_digits.p;
      }
      FD_TRY(launch_keyswitch_q(ctx, *st, (const uint64_t*)cQ, batch, (int)N,
                                (const uint32_t*)st->ksk_split.p, P.lks, P.log2Bks, (int)P.n + 1, sums,
                                st->L + 1, (uint64_t*)ct_out, s, &st->tc_ksk, dig));
    } else {
      void* dig = nullptr;
      if (tc_digit_row_bytes(*st) && !(ctx->test_flags & 2)) {
        FD_TRY(ensure_tc_digits(*st, batch));
        dig = st->tc_digits.p;
      }
      FD_TRY(launch_keyswitch(ctx, st->w, cQ, batch, (int)N, st->ksk.p, P.lks, P.log2Bks,
                              trunc_bits(st->w, P.log2Bks, P.lks), (int)P.n + 1, ct_out, s, &st->tc_ksk, dig));
    }
  }
  return FDFB_OK;
}

int fdfb_lut_polys(fdfb_ctx* ctx, int set_id, int lut_id, int32_t* p0, int32_t* p1) {
  SetState* st = get_set(ctx, set_id);
  if (!st || !p0 || !p1) return FDFB_EINVAL;
  if (lut_id < 0 || lut_id >= st->n_luts) return FDFB_EBADLUT;
  const int N = (int)st->prm.N;
  const int16_t* src = st->luts_host.data() + (size_t)lut_id * 2 * N;
  for (int j = 0; j < N; ++j) {
    p0[j] = src[j];
    p1[j] = src[N + j];
  }
  return FDFB_OK;
}

int fdfb_bootstrap(fdfb_ctx* ctx, int set_id, const void* ct_in, const int32_t* lut_ids,
                   int64_t batch, void* ct_out, void* cuda_stream) {
  SetState* st = get_set(ctx, set_id);
  if (!st) return FDFB_EINVAL;
  DeviceGuard g(ctx->device);
  return run_chunked(ctx, *st, ct_in, lut_ids, batch, 1, ct_out, as_stream(cuda_stream), st->chunks);
}

int fdfb_bootstrap_multi(fdfb_ctx* ctx, int set_id, const void* ct_in, const int32_t* lut_ids,
                         int64_t batch, int k, void* ct_out, void* cuda_stream) {
  SetState* st = get_set(ctx, set_id);
  if (!st) return FDFB_EINVAL;
  DeviceGuard g(ctx->device);
  return run_chunked(ctx, *st, ct_in, lut_ids, batch, k, ct_out, as_stream(cuda_stream), st->chunks);
}

int fdfb_noalloc_max_batch(fdfb_ctx* ctx, int set_id, int64_t* max_batch) {
  SetState* st = get_set(ctx, set_id);
  if (!st || !max_batch) return FDFB_EINVAL;
  *max_batch = (int64_t)(kNoAllocScratchBytes / scratch_bytes(*st, 1, 1));
  return FDFB_OK;
}

int fdfb_bootstrap_noalloc(fdfb_ctx* ctx, int set_id, const void* ct_in, const int32_t* lut_ids,
                           int64_t batch, void* ct_out, void* cuda_stream) {
  SetState* st = get_set(ctx, set_id);
  if (!st) return FDFB_EINVAL;
  int64_t cap = 0;
  FD_TRY(fdfb_noalloc_max_batch(ctx, set_id, &cap));
  if (batch > cap) return FDFB_EINVAL;  // beyond the fixed scratch
  DeviceGuard g(ctx->device);
  void* scratch = nullptr;
  FD_TRY(noalloc_scratch(ctx->device, &scratch));
  return run_pipeline(ctx, *st, ct_in, lut_ids, batch, 1, ct_out, nullptr, as_stream(cuda_stream),
                      scratch, false, nullptr, false);
}

int fdfb_bootstrap_debug(fdfb_ctx* ctx, int set_id, const void* ct_in, const int32_t* lut_ids,
                         int64_t batch, void* ct_out, const fdfb_debug_bufs* dbg, void* cuda_stream) {
  SetState* st = get_set(ctx, set_id);
  if (!st || !dbg) return FDFB_EINVAL;
  DeviceGuard g(ctx->device);
  return run_pipeline(ctx, *st, ct_in, lut_ids, batch, 1, ct_out, dbg, as_stream(cuda_stream));
}

int fdfb_bootstrap_mixed(fdfb_ctx* ctx, int n_groups, const fdfb_group* groups, void* cuda_stream) {
  if (!ctx || n_groups < 0 || (n_groups > 0 && !groups)) return FDFB_EINVAL;
  if (n_groups == 0) return FDFB_OK;
  DeviceGuard g(ctx->device);
  cudaStream_t s = as_stream(cuda_stream);
  // Groups of the same parameter set share that set's scratch, so they run
  // one after another on one side stream; distinct sets run concurrently.
  std::vector<int> sets;
  std::vector<int> lane(n_groups);
  for (int i = 0; i < n_groups; ++i) {
    SetState* st = get_set(ctx, groups[i].set_id);
    if (!st || groups[i].batch < 0) return FDFB_EINVAL;
    int k = 0;
    while (k < (int)sets.size() && sets[k] != groups[i].set_id) ++k;
    if (k == (int)sets.size()) sets.push_back(groups[i].set_id);
    lane[i] = k;
  }
  // Grow every set's scratch before forking, so the forked work allocates nothing.
  for (int k = 0; k < (int)sets.size(); ++k) {
    int64_t mx = 0;
    for (int i = 0; i < n_groups; ++i)
      if (lane[i] == k && groups[i].batch > mx) mx = groups[i].batch;
    FD_TRY(ensure_scratch(*get_set(ctx, sets[k]), mx));
    FD_TRY(ensure_tc_digits(*get_set(ctx, sets[k]), mx));
  }
  if (sets.size() == 1) {
    for (int i = 0; i < n_groups; ++i)
      FD_TRY(run_pipeline(ctx, *get_set(ctx, groups[i].set_id), groups[i].ct_in, groups[i].lut_ids,
                          groups[i].batch, 1, groups[i].ct_out, nullptr, s));
    return FDFB_OK;
  }
  std::lock_guard<std::mutex> lk(ctx->mu);
  while (ctx->side.size() < sets.size()) {
    cudaStream_t ns;
    FD_CUDA(cudaStreamCreateWithFlags(&ns, cudaStreamNonBlocking));
    ctx->side.push_back(ns);
  }
  while (ctx->events.size() < sets.size() + 1) {
    cudaEvent_t e;
    FD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ctx->events.push_back(e);
  }
  FD_CUDA(cudaEventRecord(ctx->events[0], s));
  for (size_t k = 0; k < sets.size(); ++k) FD_CUDA(cudaStreamWaitEvent(ctx->side[k], ctx->events[0], 0));
  int rc = FDFB_OK;
  for (int i = 0; i < n_groups && rc == FDFB_OK; ++i)
    rc = run_pipeline(ctx, *get_set(ctx, groups[i].set_id), groups[i].ct_in, groups[i].lut_ids,
                      groups[i].batch, 1, groups[i].ct_out, nullptr, ctx->side[lane[i]]);
  // Join even after an error, so the caller's stream never runs ahead of
  // work already queued on the side streams.
  for (size_t k = 0; k < sets.size(); ++k) {
    FD_CUDA(cudaEventRecord(ctx->events[1 + k], ctx->side[k]));
    FD_CUDA(cudaStreamWaitEvent(s, ctx->events[1 + k], 0));
  }
  return rc;
}

int fdfb_keyswitch(fdfb_ctx* ctx, int set_id, const void* ct_in, int64_t batch, void* ct_out,
                   void* cuda_stream) {
  SetState* st = get_set(ctx, set_id);
  if (!st || batch < 0 || batch > 0x7fffffffLL) return FDFB_EINVAL;
  if (batch == 0) return FDFB_OK;
  if (!ct_in || !ct_out) return FDFB_EINVAL;
  if (!st->keys) return FDFB_ENOKEYS;
  DeviceGuard g(ctx->device);
  cudaStream_t s = as_stream(cuda_stream);
  const fdfb_params& P = st->prm;
  if (st->mq.Q) {
    DevBuf sums;
    FD_TRY(sums.ensure((size_t)batch * 2 * (P.n + 1) * 8));
    void* dig = nullptr;
    if (tc_digit_row_bytes(*st) && !(ctx->test_flags & 2)) {
      FD_TRY(ensure_tc_digits(*st, batch));
      dig = st->tc_digits.p;
    }
    FD_TRY(launch_keyswitch_q(ctx, *st, (const uint64_t*)ct_in, batch, (int)P.N,
                              (const uint32_t*)st->ksk_split.p, P.lks, P.log2Bks, (int)P.n + 1,
                              (uint64_t*)sums.p, 0, (uint64_t*)ct_out, s, &st->tc_ksk, dig));
    FD_CUDA(cudaStreamSynchronize(s));  // the sums buffer is released on return
    return FDFB_OK;
  }
  void* dig = nullptr;
  if (tc_digit_row_bytes(*st) && !(ctx->test_flags & 2)) {
    FD_TRY(ensure_tc_digits(*st, batch));
    dig = st->tc_digits.p;
  }
  return launch_keyswitch(ctx, st->w, ct_in, batch, (int)P.N, st->ksk.p, P.lks, P.log2Bks,
                          trunc_bits(st->w, P.log2Bks, P.lks), (int)P.n + 1, ct_out, s, &st->tc_ksk, dig);
}

int fdfb_keyswitch_path(fdfb_ctx* ctx, int set_id, int* pk_path, int* ksk_path) {
  SetState* st = get_set(ctx, set_id);
  if (!st) return FDFB_EINVAL;
  const bool on = !(ctx->test_flags & 2);
  if (pk_path) *pk_path = (on && st->tc_pk.ready) ? 1 : 0;
  if (ksk_path) *ksk_path = (on && st->tc_ksk.ready) ? 1 : 0;
  return FDFB_OK;
}

int fdfb_lwe_encrypt(fdfb_ctx* ctx, int set_id, const uint8_t* s, const void* a, const int64_t* e,
                     const int64_t* m, int64_t count, void* ct_out, void* cuda_stream) {
  SetState* st = get_set(ctx, set_id);
  if (!st || count < 0) return FDFB_EINVAL;
  if (count == 0) return FDFB_OK;
  if (!s || !a || !e || !m || !ct_out) return FDFB_EINVAL;
  DeviceGuard g(ctx->device);
  // prime-modulus sets encrypt mod q = 2N with Delta = round(2N / t)
  const int logq = st->mq.Q ? st->L + 1 : st->w;
  const uint64_t delta = st->mq.Q ? ((2ull << st->L) + st->prm.t / 2) / st->prm.t
                                  : (uint64_t)1 << (logq - st->logt);
  const unsigned blocks = (unsigned)((count + 7) / 8);
  cudaStream_t cs = as_stream(cuda_stream);
  if (st->w == 32)
    lwe_encrypt_kernel<uint32_t><<<blocks, 256, 0, cs>>>(s, (const uint32_t*)a, e, m, count,
                                                         (int)st->prm.n, delta, (uint32_t*)ct_out, logq);
  else
    lwe_encrypt_kernel<uint64_t><<<blocks, 256, 0, cs>>>(s, (const uint64_t*)a, e, m, count,
                                                         (int)st->prm.n, delta, (uint64_t*)ct_out, logq);
  return cuda_err(cudaGetLastError());
}

int fdfb_lwe_decrypt(fdfb_ctx* ctx, int set_id, const uint8_t* s, const void* ct, int64_t count,
                     int32_t* m_out, void* cuda_stream) {
  SetState* st = get_set(ctx, set_id);
  if (!st || count < 0) return FDFB_EINVAL;
  if (count == 0) return FDFB_OK;
  if (!s || !ct || !m_out) return FDFB_EINVAL;
  DeviceGuard g(ctx->device);
  const int logq = st->mq.Q ? st->L + 1 : st->w;
  const unsigned blocks = (unsigned)((count + 7) / 8);
  cudaStream_t cs = as_stream(cuda_stream);
  if (st->w == 32)
    lwe_decrypt_kernel<uint32_t><<<blocks, 256, 0, cs>>>(s, (const uint32_t*)ct, count,
                                                         (int)st->prm.n, st->logtout, m_out, logq, 0);
  else
    lwe_decrypt_kernel<uint64_t><<<blocks, 256, 0, cs>>>(s, (const uint64_t*)ct, count,
                                                         (int)st->prm.n, st->logtout, m_out, logq,
                                                         st->mq.Q ? (int)st->prm.t : 0);
  return cuda_err(cudaGetLastError());
}

int fdfb_lwe_affine(fdfb_ctx* ctx, int set_id, const int32_t* W, int n_in, int n_out, const void* x,
                    int64_t batch, void* y, void* cuda_stream) {
  SetState* st = get_set(ctx, set_id);
  if (!st || n_in < 1 || n_out < 1 || batch < 0 || batch > 65535 || st->mq.Q) return FDFB_EINVAL;
  if (batch == 0) return FDFB_OK;
  if (!W || !x || !y) return FDFB_EINVAL;
  DeviceGuard g(ctx->device);
  const int len = (int)st->prm.n + 1;
  dim3 grid((unsigned)((len + AFF_TK - 1) / AFF_TK), (unsigned)((n_out + AFF_TO - 1) / AFF_TO),
            (unsigned)batch);
  cudaStream_t cs = as_stream(cuda_stream);
  if (st->w == 32)
    lwe_affine_kernel<uint32_t><<<grid, AFF_TK, 0, cs>>>(W, n_in, n_out, (const uint32_t*)x, len,
                                                        (uint32_t*)y);
  else
    lwe_affine_kernel<uint64_t><<<grid, AFF_TK, 0, cs>>>(W, n_in, n_out, (const uint64_t*)x, len,
                                                        (uint64_t*)y);
  return cuda_err(cudaGetLastError());
}

int fdfb_variant_info(fdfb_ctx* ctx, int set_id, int* current, int* count, int* coeffs_per_thread) {
  SetState* st = get_set(ctx, set_id);
  if (!st) return FDFB_EINVAL;
  if (current) *current = st->cur;
  if (count) *count = (int)st->var.size();
  if (coeffs_per_thread) *coeffs_per_thread = 1 << st->br().ops->EL;
  return FDFB_OK;
}

int fdfb_set_variant(fdfb_ctx* ctx, int set_id, int variant) {
  SetState* st = get_set(ctx, set_id);
  if (!st || variant < 0 || variant >= (int)st->var.size()) return FDFB_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  st->cur = variant;
  return FDFB_OK;
}

int fdfb_autotune(fdfb_ctx* ctx, int set_id, int64_t batch, void* cuda_stream, int* variant_out,
                  double* ms_out, double* ms_each, int ms_each_len) {
  SetState* st = get_set(ctx, set_id);
  if (!st || batch < 1 || batch > 0x7fffffff) return FDFB_EINVAL;
  if (!st->keys) return FDFB_ENOKEYS;
  if (st->prm.n > st->prm.N) return FDFB_EINVAL;  // the trial ciphertexts live in scratch
  DeviceGuard g(ctx->device);
  cudaStream_t s = as_stream(cuda_stream);
  FD_TRY(ensure_scratch(*st, batch));
  const size_t N = st->prm.N, wb = st->wbytes();
  unsigned char* base = (unsigned char*)st->scratch.p;
  void* trial_ct = base + (size_t)batch * ((N + 1) + 4 * N) * wb;  // the cQ region
  void* trial_out = base;                                           // the sgn region
  FD_CUDA(cudaMemsetAsync(trial_ct, 0, (size_t)batch * (st->prm.n + 1) * wb, s));
  cudaEvent_t a, b;
  FD_CUDA(cudaEventCreate(&a));
  FD_CUDA(cudaEventCreate(&b));
  int best = st->cur;
  float best_ms = 1e30f;
  for (int vi = 0; vi < (int)st->var.size(); ++vi) {
    Variant& v = *st->var[vi];
    BRParams br{};
    br.S = v.S;
    br.bsk = (const uint32_t*)v.bsk_ntt.p;
    br.ct = trial_ct;
    br.lwe_out = trial_out;
    br.n = st->prm.n;
    br.lg = st->prm.lg;
    br.log2Bg = st->prm.log2Bg;
    br.rtrunc = trunc_bits(st->w, st->prm.log2Bg, st->prm.lg);
    br.batch = batch;
    br.delta_half = ((uint64_t)1 << (st->w - st->logtout)) / 2;
    br.sign_mode = 1;
    br.smem_r1 = v.br_r1;
    br.smem_exch = v.br_ex;
    br.rep = 1;
    br.signed_digits = (int)st->prm.signed_digits;
    br.err = ctx->d_err;
    if (st->mq.Q) {
      fill_br_q(br, *st);
      br.half_y = n13_half_region(*st, base, batch);
    }
    float ms_v = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(a, s);
      cudaError_t e = v.ops->br(br, batch, v.br_smem, s);
      cudaEventRecord(b, s);
      if (e != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess) {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        return cuda_err(e != cudaSuccess ? e : cudaGetLastError());
      }
      float ms = 0;
      cudaEventElapsedTime(&ms, a, b);
      if (rep > 0 && ms < ms_v) ms_v = ms;  // the first run warms caches
    }
    if (ms_each && vi < ms_each_len) ms_each[vi] = ms_v;
    if (ms_v < best_ms) {
      best_ms = ms_v;
      best = vi;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    st->cur = best;
  }
  if (variant_out) *variant_out = best;
  if (ms_out) *ms_out = best_ms;
  return tune_chunks(ctx, *st, batch, s);
}

int fdfb_set_chunks(fdfb_ctx* ctx, int set_id, int chunks) {
  SetState* st = get_set(ctx, set_id);
  if (!st || chunks < 1 || chunks > kMaxChunks) return FDFB_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  st->chunks = chunks;
  return FDFB_OK;
}

int fdfb_get_chunks(fdfb_ctx* ctx, int set_id, int* chunks) {
  SetState* st = get_set(ctx, set_id);
  if (!st || !chunks) return FDFB_EINVAL;
  *chunks = st->chunks;
  return FDFB_OK;
}

int fdfb_profile_enable(fdfb_ctx* ctx, int enable) {
  if (!ctx) return FDFB_EINVAL;
  DeviceGuard g(ctx->device);
  for (auto& m : ctx->marks) {
    cudaEventSynchronize(m.b);
    cudaEventDestroy(m.a);
    cudaEventDestroy(m.b);
  }
  ctx->marks.clear();
  for (int i = 0; i < kStages; ++i) {
    ctx->prof_ms[i] = 0;
    ctx->prof_n[i] = 0;
  }
  ctx->prof = enable != 0;
  return FDFB_OK;
}

int fdfb_profile_read(fdfb_ctx* ctx, int stage, double* total_ms, int64_t* launches) {
  if (!ctx || stage < 0 || stage >= kStages || !total_ms || !launches) return FDFB_EINVAL;
  DeviceGuard g(ctx->device);
  // Blind-rotation launches of different chunks overlap: stage 5 is the
  // length of the union of their [start, end] intervals.
  std::vector<std::pair<double, double>> br;
  for (auto& m : ctx->marks) {
    float ms = 0, t0 = 0;
    FD_CUDA(cudaEventSynchronize(m.b));
    FD_CUDA(cudaEventElapsedTime(&ms, m.a, m.b));
    ctx->prof_ms[m.stage] += ms;
    ctx->prof_n[m.stage] += 1;
    // start relative to the first mark (negative when it ran earlier on
    // another stream)
    if ((m.stage == 0 || m.stage == 3) && cudaEventElapsedTime(&t0, ctx->marks[0].a, m.a) == cudaSuccess)
      br.push_back({(double)t0, (double)t0 + ms});
  }
  std::sort(br.begin(), br.end());
  double lo = 0, hi = -1e300;
  for (auto& iv : br) {
    if (iv.first > hi) {
      if (hi > lo) ctx->prof_ms[5] += hi - lo;
      lo = iv.first;
      hi = iv.second;
    } else if (iv.second > hi) {
      hi = iv.second;
    }
  }
  if (!br.empty() && hi > lo) ctx->prof_ms[5] += hi - lo;
  ctx->prof_n[5] += (int64_t)br.size();
  for (auto& m : ctx->marks) {
    cudaEventDestroy(m.a);
    cudaEventDestroy(m.b);
  }
  ctx->marks.clear();
  *total_ms = ctx->prof_ms[stage];
  *launches = ctx->prof_n[stage];
  return FDFB_OK;
}

int fdfb_test_hooks(fdfb_ctx* ctx, int flags) {
  if (!ctx || (flags & ~3)) return FDFB_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->test_flags = flags;
  return FDFB_OK;
}

int fdfb_sync(fdfb_ctx* ctx, void* cuda_stream) {
  if (!ctx) return FDFB_EINVAL;
  DeviceGuard g(ctx->device);
  FD_CUDA(cudaStreamSynchronize(as_stream(cuda_stream)));
  int h = 0;
  FD_CUDA(cudaMemcpy(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h != 0) {
    FD_CUDA(cudaMemset(ctx->d_err, 0, sizeof(int)));
    return h;
  }
  return cuda_err(cudaGetLastError());
}

}  // extern "C"
