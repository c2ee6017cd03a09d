"""FDFB oracle for the prime-modulus parameter sets (test infrastructure only).

ctypes wrappers of `fdfb_oracle_q.c`: the Bootstrap figure of Section 3 run
literally with the RLWE side modulo a prime Q and the LWE side modulo
q = 2N (Table 1).  Values mod Q travel as uint64; the LWE side reuses the
power-of-two routines of the main oracle with w = log2 q.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _i64, _p, _u8, _u64, lib, lwe_encrypt, setup_polynomial


class orq_params(C.Structure):
    _fields_ = [(k, C.c_int32) for k in
                ("n", "N", "t", "log2Bg", "lg", "log2Bks", "lks", "log2Bpk", "lpk",
                 "log2Lboot", "lboot")] + [("Q", C.c_uint64)]


class orq_debug(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("sgn", "cR", "accF", "cQ", "cKS")]


def params(ps) -> orq_params:
    return orq_params(ps.n, ps.N, ps.t, ps.log2Bg, ps.lg, ps.log2Bks, ps.lks, ps.log2Bpk, ps.lpk,
                      ps.log2Lboot, ps.lboot, ps.Q)


def mulmod(a: int, b: int, Q: int) -> int:
    return int(lib().orq_mulmod(a % (1 << 64), b % (1 << 64), Q))


def delta(Q: int, t: int) -> int:
    return int(lib().orq_delta(Q, t))


def delta_half(Q: int, t: int) -> int:
    return int(lib().orq_delta_half(Q, t))


def poly_mul(Q: int, a, b) -> np.ndarray:
    a, b = _u64(a), _u64(b)
    N = a.shape[-1]
    out = np.zeros(N, dtype=np.uint64)
    lib().orq_poly_mul(N, Q, _p(a), _p(b), _p(out))
    return out


def poly_mul_xk(Q: int, p, k: int) -> np.ndarray:
    p = _u64(p)
    out = np.zeros(len(p), dtype=np.uint64)
    lib().orq_poly_mul_xk(len(p), Q, _p(p), int(k), _p(out))
    return out


def decomp(log2B: int, ell: int, x: int) -> np.ndarray:
    out = np.zeros(ell, dtype=np.uint64)
    lib().orq_decomp(log2B, ell, int(x), _p(out))
    return out


def lwe_encrypt_q(Q: int, key, a, e: int, mu: int) -> np.ndarray:
    key, a = _u64(key), _u64(a)
    out = np.zeros(len(a) + 1, dtype=np.uint64)
    lib().orq_lwe_encrypt(len(a), Q, _p(key), _p(a), int(e), int(mu) % Q, _p(out))
    return out


def lwe_phase_q(Q: int, key, ct) -> int:
    key, ct = _u64(key), _u64(ct)
    return int(lib().orq_lwe_phase(len(key), Q, _p(key), _p(ct)))


def rlwe_encrypt(Q: int, sk, a, e, mu=None) -> np.ndarray:
    sk, a, e = _u64(sk), _u64(a), _i64(e)
    N = len(sk)
    out = np.zeros(2 * N, dtype=np.uint64)
    mu_p = None
    if mu is not None:
        mu = _u64(mu)
        mu_p = _p(mu)
    lib().orq_rlwe_encrypt(N, Q, _p(sk), _p(a), _p(e), mu_p, _p(out))
    return out.reshape(2, N)


def rlwe_phase(Q: int, sk, ct) -> np.ndarray:
    sk, ct = _u64(sk), _u64(ct)
    N = len(sk)
    out = np.zeros(N, dtype=np.uint64)
    lib().orq_rlwe_phase(N, Q, _p(sk), _p(ct), _p(out))
    return out


class QKeys:
    """Oracle key material of a prime-Q set in canonical layouts (uint64 mod Q)."""

    def __init__(self, ps, kr):
        P = params(ps)
        self.ps = ps
        self.s = _u8(kr.s)
        self.sk = _u64(kr.sk)
        n, N = ps.n, ps.N
        self.bsk = np.zeros((n, 2 * ps.lg, 2, N), dtype=np.uint64)
        self.pk = np.zeros((N, ps.lpk, 2, N), dtype=np.uint64)
        self.ksk = np.zeros((N, ps.lks, n + 1), dtype=np.uint64)
        ba, be = _u64(kr.bsk_a), _i64(kr.bsk_e)
        lib().orq_keygen_bsk(C.byref(P), _p(self.s), _p(self.sk), _p(ba), _p(be), _p(self.bsk))
        pa, pe = _u64(kr.pk_a), _i64(kr.pk_e)
        lib().orq_keygen_pk(C.byref(P), _p(self.sk), _p(pa), _p(pe), _p(self.pk))
        ka, ke = _u64(kr.ksk_a), _i64(kr.ksk_e)
        lib().orq_keygen_ksk(C.byref(P), _p(self.sk), _p(self.s), _p(ka), _p(ke), _p(self.ksk))


def exact_digits(Q: int, log2B: int) -> int:
    """Digits of the exact decomposition of Z_Q in base B = 2^log2B
    (Definition "Decomposition": l = ceil(log_B Q)); for 2^(k-1) < Q < 2^k
    that is ceil(k / log2B).  Also l_boot = ceil(log_{L_boot} Q) (Bootstrap
    figure, step "for i in [l_boot]")."""
    k = int(Q).bit_length()
    return -(-k // log2B)


def delta_in(ps) -> int:
    """Delta_{q,t} = round(q / t), round half up, on the LWE side q = 2N
    (Section 2's rounding; G29's reading for t not dividing 2N)."""
    return (ps.q + ps.t // 2) // ps.t


def encrypt_messages(ps, s, mr) -> np.ndarray:
    """Fresh LWE ciphertexts mod q = 2N of Delta_q m, [count][n+1] uint64."""
    out = np.zeros((len(mr.m), ps.n + 1), dtype=np.uint64)
    D = delta_in(ps)
    for i in range(len(mr.m)):
        out[i] = lwe_encrypt(ps.logq, s, mr.a[i], int(mr.e[i]), (D * int(mr.m[i])) % ps.q)
    return out


def decrypt(ps, s, ct) -> int:
    """round(t (b - <a, s>) / q) mod t on the LWE side (q = 2N, any t)."""
    s, ct = _u8(s), _u64(ct)
    return int(lib().orq_decrypt_q2n(len(s), ps.logq, ps.t, _p(s), _p(ct)))


def extprod(ps, C_row, d) -> np.ndarray:
    P = params(ps)
    C_row, d = _u64(C_row), _u64(d)
    out = np.zeros(2 * ps.N, dtype=np.uint64)
    lib().orq_extprod(C.byref(P), _p(C_row), _p(d), _p(out))
    return out.reshape(2, ps.N)


def blind_rotate(ps, bsk, acc, ctN) -> np.ndarray:
    P = params(ps)
    bsk, ctN = _u64(bsk), _u64(ctN)
    acc = _u64(acc).copy()
    lib().orq_blind_rotate(C.byref(P), _p(bsk), _p(acc), _p(ctN))
    return acc.reshape(2, ps.N)


def sample_extract(Q: int, rlwe) -> np.ndarray:
    rlwe = _u64(rlwe)
    N = rlwe.size // 2
    out = np.zeros(N + 1, dtype=np.uint64)
    lib().orq_sample_extract(N, Q, _p(rlwe), _p(out))
    return out


def keyswitch(Q: int, log2B: int, ell: int, key, ct) -> np.ndarray:
    key, ct = _u64(key), _u64(ct)
    n_in = len(ct) - 1
    out_len = key.size // (n_in * ell)
    out = np.zeros(out_len, dtype=np.uint64)
    lib().orq_keyswitch(n_in, Q, log2B, ell, out_len, _p(key), _p(ct), _p(out))
    return out


def modswitch(Q: int, logq: int, ct) -> np.ndarray:
    ct = _u64(ct)
    out = np.zeros(len(ct), dtype=np.uint64)
    lib().orq_modswitch(Q, logq, len(ct), _p(ct), _p(out))
    return out


def pubmux(ps, c, p0, p1) -> np.ndarray:
    P = params(ps)
    c, p0, p1 = _u64(c), _i64(p0), _i64(p1)
    out = np.zeros(2 * ps.N, dtype=np.uint64)
    lib().orq_pubmux(C.byref(P), _p(c), _p(p0), _p(p1), _p(out))
    return out.reshape(2, ps.N)


def fdfb_bootstrap(ps, keys: QKeys, p0, p1, ct, debug: bool = False):
    """One bootstrap of ct (mod q = 2N) with rotation polynomials (p0, p1)
    from SetupPolynomial; returns the output [n+1] mod q and, with debug,
    the intermediates (sgn, cR, accF, cQ, cKS)."""
    P = params(ps)
    N, n, lb = ps.N, ps.n, ps.lboot
    p0, p1, ct = _i64(p0), _i64(p1), _u64(ct)
    out = np.zeros(n + 1, dtype=np.uint64)
    bufs = {"sgn": np.zeros((lb, N + 1), np.uint64), "cR": np.zeros((lb, 2, N), np.uint64),
            "accF": np.zeros((2, N), np.uint64), "cQ": np.zeros(N + 1, np.uint64),
            "cKS": np.zeros(n + 1, np.uint64)}
    dbg = orq_debug(*[_p(bufs[k]).value for k in ("sgn", "cR", "accF", "cQ", "cKS")]) if debug else None
    lib().orq_fdfb_bootstrap(C.byref(P), _p(keys.bsk), _p(keys.pk), _p(keys.ksk), _p(p0), _p(p1),
                             _p(ct), _p(out), C.byref(dbg) if debug else None)
    return (out, bufs) if debug else out


def fdfb_batch(ps, keys: QKeys, rotP, lut_ids, cts, threads: int = 1) -> np.ndarray:
    """rotP: [n_luts][2][N] signed rotation polynomials."""
    P = params(ps)
    rotP = _i64(rotP)
    rp0 = np.ascontiguousarray(rotP[:, 0])
    rp1 = np.ascontiguousarray(rotP[:, 1])
    ids = np.ascontiguousarray(np.asarray(lut_ids, dtype=np.int32))
    cts = _u64(cts)
    out = np.zeros_like(cts)
    lib().orq_fdfb_batch(C.byref(P), _p(keys.bsk), _p(keys.pk), _p(keys.ksk), _p(rp0), _p(rp1),
                         _p(ids), len(ids), _p(cts), _p(out), int(threads))
    return out


def rotation_polys(ps, tables) -> np.ndarray:
    """SetupPolynomial of every table: [count][2][N] int64."""
    out = []
    for f in tables:
        p0, p1 = setup_polynomial(ps.N, ps.t, f)
        out.append(np.stack([p0, p1]))
    return np.stack(out).astype(np.int64)


def tfhe_bootstrap(ps, keys: QKeys, poly, ct) -> np.ndarray:
    """The TFHE bootstrap of ct (mod q = 2N) with pre-rotation polynomial
    poly ([N] mod Q); returns [n+1] mod q."""
    P = params(ps)
    poly, ct = _u64(poly), _u64(ct)
    out = np.zeros(ps.n + 1, dtype=np.uint64)
    lib().orq_tfhe_bootstrap(C.byref(P), _p(keys.bsk), _p(keys.ksk), _p(poly), _p(ct), _p(out))
    return out


def tfhe_batch(ps, keys: QKeys, polys, poly_ids, cts, threads: int = 1) -> np.ndarray:
    P = params(ps)
    polys, cts = _u64(polys), _u64(cts)
    ids = np.ascontiguousarray(np.asarray(poly_ids, dtype=np.int32))
    out = np.zeros_like(cts)
    lib().orq_tfhe_batch(C.byref(P), _p(keys.bsk), _p(keys.ksk), _p(polys), _p(ids), len(ids),
                         _p(cts), _p(out), int(threads))
    return out


def tfhe_test_polynomial(ps, f_half) -> np.ndarray:
    """A pre-rotation polynomial mod Q mapping m in [0, t/2) to
    Delta_Q f_half[m] and m + t/2 to -Delta_Q f_half[m] (the negacyclic
    half): coefficient 0 of poly X^y must be Delta_Q f(m) for y within N/t of
    round(2N/t) m in [0, N), and y rounding to t/2 gives -Delta_Q f(0).
    Coefficient 0 of poly X^y is poly[0] for y = 0 and -poly[N - y] for
    0 < y < N.  Test-side construction (the library takes any polynomial)."""
    N, t, Q = ps.N, ps.t, ps.Q
    D = delta(Q, t)
    poly = np.zeros(N, dtype=np.uint64)
    step = delta_in(ps)
    for y in range(N):
        m = (y + step // 2) // step
        v = D * int(f_half[m]) if m < t // 2 else -D * int(f_half[0])
        if y == 0:
            poly[0] = v % Q
        else:
            poly[N - y] = (-v) % Q
    return poly
