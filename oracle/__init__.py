"""FDFB oracle (test infrastructure only).

Plain CPU implementation of the paper's method in `fdfb_oracle.c`, wrapped
with ctypes.  Only the tests, `__graft_entry__.smoke()` and the CPU-baseline
leg of `bench.py` may use it; the CUDA library never does.  Every array is
handed to C as uint64 words (w-bit values, w <= 64) or int64 for signed
quantities.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fdfb_oracle.c")
_SRC_Q = os.path.join(_HERE, "fdfb_oracle_q.c")  # prime-modulus parameter sets
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()


class or_params(C.Structure):
    _fields_ = [(k, C.c_int32) for k in
                ("n", "N", "w", "t", "log2Bg", "lg", "log2Bks", "lks", "log2Bpk", "lpk", "signed_digits",
                 "t_out")]


class or_debug(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("ctN", "sgn", "cR", "accF", "accBR", "cQ")]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, OpenMP for threads over items)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_Q))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, _SRC_Q])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            vp, i32, i64 = C.c_void_p, C.c_int, C.c_int64
            sig = {
                "or_set_threads": ([i32], None),
                "or_max_threads": ([], i32),
                "or_poly_mul": ([i32, i32, vp, vp, vp], None),
                "or_poly_mul_xk": ([i32, i32, vp, i64, vp], None),
                "or_poly_mul_xk_signed": ([i32, vp, i64, vp], None),
                "or_decomp_round": ([i32, i32, i32, C.c_uint64], C.c_uint64),
                "or_decomp": ([i32, i32, i32, C.c_uint64, vp], None),
                "or_decomp_signed": ([i32, i32, i32, C.c_uint64, vp], None),
                "or_gadget": ([i32, i32, i32, i32], C.c_uint64),
                "or_lwe_encrypt": ([i32, i32, vp, vp, i64, C.c_uint64, vp], None),
                "or_lwe_phase": ([i32, i32, vp, vp], C.c_uint64),
                "or_lwe_decrypt": ([i32, i32, i32, vp, vp], C.c_uint64),
                "or_rlwe_encrypt": ([i32, i32, vp, vp, vp, vp, vp], None),
                "or_rlwe_phase": ([i32, i32, vp, vp, vp], None),
                "or_keygen_bsk": ([vp, vp, vp, vp, vp, vp], None),
                "or_keygen_pk": ([vp, vp, vp, vp, vp], None),
                "or_keygen_bsk_row": ([vp, vp, vp, vp, vp, i32, i32, vp], None),
                "or_keygen_pk_row": ([vp, vp, vp, vp, i32, i32, vp], None),
                "or_keygen_ksk": ([vp, vp, vp, vp, vp, vp], None),
                "or_modswitch": ([i32, i32, i32, vp, vp], None),
                "or_extprod": ([vp, vp, vp, vp], None),
                "or_cmux": ([vp, vp, vp, vp, vp], None),
                "or_blind_rotate": ([vp, vp, vp, vp], None),
                "or_sample_extract": ([i32, i32, vp, i32, vp], None),
                "or_keyswitch": ([i32, i32, i32, i32, i32, vp, vp, vp], None),
                "or_setup_polynomial": ([i32, i32, vp, vp, vp], None),
                "or_pubmux": ([i32, i32, i32, vp, vp, vp, vp], None),
                "or_fdfb_bootstrap": ([vp, vp, vp, vp, vp, vp, vp, vp, vp], None),
                "or_fdfb_batch": ([vp, vp, vp, vp, vp, vp, i64, vp, vp], None),
                "or_fdfb_bootstrap_multi": ([vp, vp, vp, vp, vp, i32, vp, vp], None),
                "or_tfhe_bootstrap": ([vp, vp, vp, vp, vp, vp], None),
                "or_tfhe_batch": ([vp, vp, vp, vp, vp, i64, vp, vp], None),
                "or_fdfb_batch_multi": ([vp, vp, vp, vp, vp, vp, i32, i64, vp, vp], None),
                "or_lwe_affine": ([i32, i32, i32, i32, vp, vp, vp], None),
                # prime-modulus sets (fdfb_oracle_q.c; wrapped in oracle/prime_q.py)
                "orq_mulmod": ([C.c_uint64, C.c_uint64, C.c_uint64], C.c_uint64),
                "orq_delta": ([C.c_uint64, i32], C.c_uint64),
                "orq_delta_half": ([C.c_uint64, i32], C.c_uint64),
                "orq_poly_mul": ([i32, C.c_uint64, vp, vp, vp], None),
                "orq_poly_mul_xk": ([i32, C.c_uint64, vp, i64, vp], None),
                "orq_decomp": ([i32, i32, C.c_uint64, vp], None),
                "orq_lwe_encrypt": ([i32, C.c_uint64, vp, vp, i64, C.c_uint64, vp], None),
                "orq_lwe_phase": ([i32, C.c_uint64, vp, vp], C.c_uint64),
                "orq_rlwe_encrypt": ([i32, C.c_uint64, vp, vp, vp, vp, vp], None),
                "orq_rlwe_phase": ([i32, C.c_uint64, vp, vp, vp], None),
                "orq_keygen_bsk": ([vp, vp, vp, vp, vp, vp], None),
                "orq_keygen_pk": ([vp, vp, vp, vp, vp], None),
                "orq_keygen_ksk": ([vp, vp, vp, vp, vp, vp], None),
                "orq_extprod": ([vp, vp, vp, vp], None),
                "orq_blind_rotate": ([vp, vp, vp, vp], None),
                "orq_sample_extract": ([i32, C.c_uint64, vp, vp], None),
                "orq_keyswitch": ([i32, C.c_uint64, i32, i32, i32, vp, vp, vp], None),
                "orq_modswitch": ([C.c_uint64, i32, i32, vp, vp], None),
                "orq_decrypt_q2n": ([i32, i32, i32, vp, vp], C.c_uint64),
                "orq_tfhe_bootstrap": ([vp, vp, vp, vp, vp, vp], None),
                "orq_tfhe_batch": ([vp, vp, vp, vp, vp, i64, vp, vp, i32], None),
                "orq_pubmux": ([vp, vp, vp, vp, vp], None),
                "orq_fdfb_bootstrap": ([vp, vp, vp, vp, vp, vp, vp, vp, vp], None),
                "orq_fdfb_batch": ([vp, vp, vp, vp, vp, vp, vp, i64, vp, vp, i32], None),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def _u64(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x).astype(np.uint64, copy=False))


def _i64(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x).astype(np.int64, copy=False))


def _u8(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x).astype(np.uint8, copy=False))


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


def max_threads() -> int:
    return int(lib().or_max_threads())


def params(ps) -> or_params:
    return or_params(ps.n, ps.N, ps.w, ps.t, ps.log2Bg, ps.lg, ps.log2Bks, ps.lks,
                     ps.log2Bpk, ps.lpk, 1 if ps.signed_digits else 0, ps.t_out)


# --------------------------------------------------------------------------
# ring arithmetic
# --------------------------------------------------------------------------

def poly_mul(w: int, a, b) -> np.ndarray:
    a, b = _u64(a), _u64(b)
    N = a.shape[-1]
    out = np.zeros(N, dtype=np.uint64)
    lib().or_poly_mul(w, N, _p(a), _p(b), _p(out))
    return out


def poly_mul_xk(w: int, p, k: int) -> np.ndarray:
    p = _u64(p)
    out = np.zeros_like(p)
    lib().or_poly_mul_xk(w, p.shape[-1], _p(p), int(k), _p(out))
    return out


def poly_mul_xk_signed(p, k: int) -> np.ndarray:
    p = _i64(p)
    out = np.zeros_like(p)
    lib().or_poly_mul_xk_signed(p.shape[-1], _p(p), int(k), _p(out))
    return out


def decomp(w: int, log2B: int, ell: int, x: int) -> np.ndarray:
    out = np.zeros(ell, dtype=np.uint64)
    lib().or_decomp(w, log2B, ell, int(x), _p(out))
    return out


def decomp_signed(w: int, log2B: int, ell: int, x: int) -> np.ndarray:
    out = np.zeros(ell, dtype=np.int64)
    lib().or_decomp_signed(w, log2B, ell, int(x), _p(out))
    return out


def decomp_round(w: int, log2B: int, ell: int, x: int) -> int:
    return int(lib().or_decomp_round(w, log2B, ell, int(x)))


def gadget(w: int, log2B: int, ell: int, j: int) -> int:
    return int(lib().or_gadget(w, log2B, ell, j))


# --------------------------------------------------------------------------
# encryption
# --------------------------------------------------------------------------

def lwe_encrypt(w: int, s, a, e: int, mu: int) -> np.ndarray:
    s, a = _u8(s), _u64(a)
    out = np.zeros(len(s) + 1, dtype=np.uint64)
    lib().or_lwe_encrypt(w, len(s), _p(s), _p(a), int(e), int(mu) & ((1 << 64) - 1), _p(out))
    return out


def lwe_phase(w: int, s, ct) -> int:
    s, ct = _u8(s), _u64(ct)
    return int(lib().or_lwe_phase(w, len(s), _p(s), _p(ct)))


def lwe_decrypt(w: int, t: int, s, ct) -> int:
    s, ct = _u8(s), _u64(ct)
    return int(lib().or_lwe_decrypt(w, len(s), t, _p(s), _p(ct)))


def rlwe_encrypt(w: int, sk, a, e, mu=None) -> np.ndarray:
    sk, a, e = _u8(sk), _u64(a), _i64(e)
    N = len(sk)
    out = np.zeros(2 * N, dtype=np.uint64)
    mu_p = None
    if mu is not None:
        mu = _u64(mu)
        mu_p = _p(mu)
    lib().or_rlwe_encrypt(w, N, _p(sk), _p(a), _p(e), mu_p, _p(out))
    return out


def rlwe_phase(w: int, sk, ct) -> np.ndarray:
    sk, ct = _u8(sk), _u64(ct)
    N = len(sk)
    out = np.zeros(N, dtype=np.uint64)
    lib().or_rlwe_phase(w, N, _p(sk), _p(ct), _p(out))
    return out


class Keys:
    """Oracle key material in canonical layouts (uint64 words)."""

    def __init__(self, ps, kr):
        P = params(ps)
        self.ps = ps
        self.s = _u8(kr.s)
        self.sk = _u8(kr.sk)
        n, N = ps.n, ps.N
        self.bsk = np.zeros((n, 2 * ps.lg, 2, N), dtype=np.uint64)
        self.pk = np.zeros((N, ps.lpk, 2, N), dtype=np.uint64)
        self.ksk = np.zeros((N, ps.lks, n + 1), dtype=np.uint64)
        ba, be = _u64(kr.bsk_a), _i64(kr.bsk_e)
        lib().or_keygen_bsk(C.byref(P), _p(self.s), _p(self.sk), _p(ba), _p(be), _p(self.bsk))
        pa, pe = _u64(kr.pk_a), _i64(kr.pk_e)
        lib().or_keygen_pk(C.byref(P), _p(self.sk), _p(pa), _p(pe), _p(self.pk))
        ka, ke = _u64(kr.ksk_a), _i64(kr.ksk_e)
        lib().or_keygen_ksk(C.byref(P), _p(self.sk), _p(self.s), _p(ka), _p(ke), _p(self.ksk))


def keygen_bsk_row(ps, kr, i: int, r: int) -> np.ndarray:
    """GGSW row r of RGSW(s_i) (one row of BRKeyGen), [2][N]."""
    P = params(ps)
    a, e = _u64(kr.bsk_a[i, r]), _i64(kr.bsk_e[i, r])
    s, sk = _u8(kr.s), _u8(kr.sk)
    out = np.zeros(2 * ps.N, dtype=np.uint64)
    lib().or_keygen_bsk_row(C.byref(P), _p(s), _p(sk), _p(a), _p(e), i, r, _p(out))
    return out.reshape(2, ps.N)


def keygen_pk_row(ps, kr, i: int, j: int) -> np.ndarray:
    """Packing-key sample pK[i][j] = RLWE_sk(s_F[i] g_j), [2][N]."""
    P = params(ps)
    a, e = _u64(kr.pk_a[i, j]), _i64(kr.pk_e[i, j])
    sk = _u8(kr.sk)
    out = np.zeros(2 * ps.N, dtype=np.uint64)
    lib().or_keygen_pk_row(C.byref(P), _p(sk), _p(a), _p(e), i, j, _p(out))
    return out.reshape(2, ps.N)


def delta(w: int, t: int) -> int:
    """Delta_{q,t} = round(q / t) (Section 2, notation) for q = 2^w and a
    power-of-two t, where the quotient is exact."""
    return (1 << w) // t


def t_out(ps) -> int:
    """Output plaintext modulus t' of f: Z_t -> Z_t' (Section 1.1, footnote);
    a set with t_out = 0 maps into Z_t."""
    return ps.t_out or ps.t


def delta_out(ps) -> int:
    """Delta_{q,t'}: the scale of the bootstrap's outputs."""
    return delta(ps.w, t_out(ps))


def encrypt_messages(ps, s, mr) -> np.ndarray:
    """Fresh LWE ciphertexts [count][n+1] of Delta*m with the given randomness."""
    count = len(mr.m)
    out = np.zeros((count, ps.n + 1), dtype=np.uint64)
    D = delta(ps.w, ps.t)
    for i in range(count):
        out[i] = lwe_encrypt(ps.w, s, mr.a[i], int(mr.e[i]), (D * int(mr.m[i])) % (1 << ps.w))
    return out


# --------------------------------------------------------------------------
# homomorphic primitives
# --------------------------------------------------------------------------

def modswitch(w: int, k: int, ct) -> np.ndarray:
    ct = _u64(ct)
    out = np.zeros_like(ct)
    lib().or_modswitch(w, k, len(ct) - 1, _p(ct), _p(out))
    return out


def extprod(ps, C_row, d) -> np.ndarray:
    P = params(ps)
    C_row, d = _u64(C_row), _u64(d)
    out = np.zeros(2 * ps.N, dtype=np.uint64)
    lib().or_extprod(C.byref(P), _p(C_row), _p(d), _p(out))
    return out


def cmux(ps, C_row, g, h) -> np.ndarray:
    P = params(ps)
    C_row, g, h = _u64(C_row), _u64(g), _u64(h)
    out = np.zeros(2 * ps.N, dtype=np.uint64)
    lib().or_cmux(C.byref(P), _p(C_row), _p(g), _p(h), _p(out))
    return out


def blind_rotate(ps, bsk, acc, ctN) -> np.ndarray:
    P = params(ps)
    bsk, ctN = _u64(bsk), _u64(ctN)
    acc = _u64(acc).copy()
    lib().or_blind_rotate(C.byref(P), _p(bsk), _p(acc), _p(ctN))
    return acc


def sample_extract(w: int, rlwe, k: int = 0) -> np.ndarray:
    rlwe = _u64(rlwe)
    N = len(rlwe) // 2
    out = np.zeros(N + 1, dtype=np.uint64)
    lib().or_sample_extract(w, N, _p(rlwe), k, _p(out))
    return out


def keyswitch(w: int, log2B: int, ell: int, key, ct) -> np.ndarray:
    key, ct = _u64(key), _u64(ct)
    n_in = len(ct) - 1
    out_len = key.size // (n_in * ell)
    out = np.zeros(out_len, dtype=np.uint64)
    lib().or_keyswitch(w, n_in, log2B, ell, out_len, _p(key), _p(ct), _p(out))
    return out


def setup_polynomial(N: int, t: int, f):
    f = _i64(f)
    p0 = np.zeros(N, dtype=np.int64)
    p1 = np.zeros(N, dtype=np.int64)
    lib().or_setup_polynomial(N, t, _p(f), _p(p0), _p(p1))
    return p0, p1


def pubmux(w: int, t: int, c, p0, p1) -> np.ndarray:
    c, p0, p1 = _u64(c), _i64(p0), _i64(p1)
    N = len(p0)
    out = np.zeros(2 * N, dtype=np.uint64)
    lib().or_pubmux(w, N, t, _p(c), _p(p0), _p(p1), _p(out))
    return out


def fdfb_bootstrap(ps, keys: Keys, p0, p1, ct, debug: bool = False):
    P = params(ps)
    p0, p1, ct = _i64(p0), _i64(p1), _u64(ct)
    out = np.zeros(ps.n + 1, dtype=np.uint64)
    dbg = None
    d = None
    if debug:
        N = ps.N
        d = {"ctN": np.zeros(ps.n + 1, np.uint64), "sgn": np.zeros(N + 1, np.uint64),
             "cR": np.zeros(2 * N, np.uint64), "accF": np.zeros(2 * N, np.uint64),
             "accBR": np.zeros(2 * N, np.uint64), "cQ": np.zeros(N + 1, np.uint64)}
        dbg = or_debug(*[d[k].ctypes.data for k in ("ctN", "sgn", "cR", "accF", "accBR", "cQ")])
    lib().or_fdfb_bootstrap(C.byref(P), _p(keys.bsk), _p(keys.pk), _p(keys.ksk), _p(p0), _p(p1),
                            _p(ct), _p(out), C.byref(dbg) if dbg is not None else None)
    return (out, d) if debug else out


def fdfb_batch(ps, keys: Keys, rotP, lut_ids, cts, threads: int | None = None) -> np.ndarray:
    """rotP: int64[n_luts][2][N]; lut_ids: int32[count]; cts: [count][n+1]."""
    P = params(ps)
    rotP, cts = _i64(rotP), _u64(cts)
    ids = np.ascontiguousarray(np.asarray(lut_ids, dtype=np.int32))
    out = np.zeros_like(cts)
    if threads is not None:
        set_threads(threads)
    lib().or_fdfb_batch(C.byref(P), _p(keys.bsk), _p(keys.pk), _p(keys.ksk), _p(rotP), _p(ids),
                        len(ids), _p(cts), _p(out))
    return out


def fdfb_bootstrap_multi(ps, keys: Keys, rots, ct) -> np.ndarray:
    """k functions of one input, sharing the sign part.  rots: int64[k][2][N]
    (p0, p1 per table); returns [k][n+1]."""
    P = params(ps)
    rots, ct = _i64(rots), _u64(ct)
    k = rots.shape[0]
    out = np.zeros((k, ps.n + 1), dtype=np.uint64)
    lib().or_fdfb_bootstrap_multi(C.byref(P), _p(keys.bsk), _p(keys.pk), _p(keys.ksk), _p(rots), k,
                                  _p(ct), _p(out))
    return out


def fdfb_batch_multi(ps, keys: Keys, rotP, lut_ids, cts, threads: int | None = None) -> np.ndarray:
    """rotP: int64[n_luts][2][N]; lut_ids: int32[count][k]; cts: [count][n+1];
    returns [count][k][n+1]."""
    P = params(ps)
    rotP, cts = _i64(rotP), _u64(cts)
    ids = np.ascontiguousarray(np.asarray(lut_ids, dtype=np.int32))
    count, k = ids.shape
    out = np.zeros((count, k, ps.n + 1), dtype=np.uint64)
    if threads is not None:
        set_threads(threads)
    lib().or_fdfb_batch_multi(C.byref(P), _p(keys.bsk), _p(keys.pk), _p(keys.ksk), _p(rotP), _p(ids),
                              k, count, _p(cts), _p(out))
    return out


def tfhe_bootstrap(ps, keys: Keys, poly, ct) -> np.ndarray:
    """TFHE bootstrap of one ciphertext with the pre-rotation polynomial poly
    (N words mod q)."""
    P = params(ps)
    poly, ct = _u64(poly), _u64(ct)
    out = np.zeros(ps.n + 1, dtype=np.uint64)
    lib().or_tfhe_bootstrap(C.byref(P), _p(keys.bsk), _p(keys.ksk), _p(poly), _p(ct), _p(out))
    return out


def tfhe_batch(ps, keys: Keys, polys, poly_ids, cts, threads: int | None = None) -> np.ndarray:
    """polys: [n_polys][N] words; poly_ids: int32[count]; cts: [count][n+1]."""
    P = params(ps)
    polys, cts = _u64(polys), _u64(cts)
    ids = np.ascontiguousarray(np.asarray(poly_ids, dtype=np.int32))
    out = np.zeros_like(cts)
    if threads is not None:
        set_threads(threads)
    lib().or_tfhe_batch(C.byref(P), _p(keys.bsk), _p(keys.ksk), _p(polys), _p(ids), len(ids), _p(cts),
                        _p(out))
    return out


def tfhe_test_polynomial(ps, f_half) -> np.ndarray:
    """A pre-rotation polynomial for the TFHE bootstrap that maps m in
    [0, t/2) to Delta f_half[m] (and m + t/2 to -Delta f_half[m], the
    negacyclic half): coefficient 0 of poly X^y must be Delta f(m) for every
    y within N/t of the ModSwitched phase 2N m / t, y in [0, N), and y rounding
    to t/2 must give -Delta f(0).  Coefficient 0 of poly X^y is poly[0] for
    y = 0 and -poly[N - y] for 0 < y < N (and minus that for y in [N, 2N))."""
    N, t = ps.N, ps.t
    mask = (1 << ps.w) - 1
    poly = np.zeros(N, dtype=np.uint64)
    step = 2 * N // t
    D = delta(ps.w, t)
    for y in range(N):
        m = (y + step // 2) // step               # nearest message, 0 .. t/2
        v = D * int(f_half[m]) if m < t // 2 else -D * int(f_half[0])
        if y == 0:
            poly[0] = v & mask
        else:
            poly[N - y] = (-v) & mask
    return poly


def lwe_affine(w: int, W, x) -> np.ndarray:
    W, x = _i64(W), _u64(x)
    n_out, n_in = W.shape
    length = x.shape[1]
    y = np.zeros((n_out, length), dtype=np.uint64)
    lib().or_lwe_affine(w, length, n_in, n_out, _p(W), _p(x), _p(y))
    return y
