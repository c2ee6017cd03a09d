"""Pins for the CPU oracle: each test checks an oracle function against
something other than itself -- a closed form, an invariant the paper states,
an independent exact method, brute force on tiny inputs, or the paper's own
correctness theorems -- chosen so that a dropped term, a wrong sign or index
or a transposed operand fails at least one of them.  No GPU needed.
"""
import itertools

import numpy as np
import pytest

from paper_2109_02731_gb300 import synth as S

W32, W64 = 32, 64


def rng(seed):
    return np.random.default_rng(seed)


def rand_words(r, w, size):
    if w == 64:
        return r.integers(0, 1 << 63, size=size, dtype=np.uint64) * np.uint64(2) + \
            r.integers(0, 2, size=size, dtype=np.uint64)
    return r.integers(0, 1 << w, size=size, dtype=np.uint64)


def kronecker_negacyclic(a, b, w):
    """Independent exact product in Z_{2^w}[X]/(X^N+1): pack both operands
    into big integers (Kronecker substitution), multiply with Python's
    arbitrary-precision integers, unpack the 2N-1 coefficients of the plain
    product and fold the upper half back with X^N = -1."""
    N = len(a)
    slot = 2 * w + N.bit_length() + 2
    A = 0
    B = 0
    for i in reversed(range(N)):
        A = (A << slot) | int(a[i])
        B = (B << slot) | int(b[i])
    Cp = A * B
    mask = (1 << slot) - 1
    c = [(Cp >> (slot * k)) & mask for k in range(2 * N)]
    return np.array([(c[k] - c[k + N]) % (1 << w) for k in range(N)], dtype=np.uint64)


def monomial(N, k, w):
    """X^k as a coefficient vector from the closed form X^N = -1, X^{2N} = 1."""
    k %= 2 * N
    v = np.zeros(N, dtype=np.uint64)
    if k < N:
        v[k] = 1
    else:
        v[k - N] = (1 << w) - 1
    return v


# ---------------------------------------------------------------- ring ------

@pytest.mark.parametrize("w", [W32, W64])
def test_xn_is_minus_one(oracle, w):
    N = 64
    x = monomial(N, 1, w)
    xn1 = monomial(N, N - 1, w)
    prod = oracle.poly_mul(w, xn1, x)
    expect = np.zeros(N, np.uint64)
    expect[0] = (1 << w) - 1
    assert np.array_equal(prod, expect)
    one = np.zeros(N, np.uint64)
    one[0] = 1
    assert np.array_equal(oracle.poly_mul_xk(w, one, 2 * N), one)
    assert np.array_equal(oracle.poly_mul_xk(w, one, N), expect)


@pytest.mark.parametrize("w,N", [(W32, 16), (W32, 256), (W64, 64), (W64, 256), (12, 32)])
def test_poly_mul_matches_kronecker(oracle, w, N):
    r = rng(N + w)
    for _ in range(3):
        a = rand_words(r, w, N)
        b = rand_words(r, w, N)
        assert np.array_equal(oracle.poly_mul(w, a, b), kronecker_negacyclic(a, b, w))


@pytest.mark.parametrize("w", [W32, W64])
def test_monomial_rotation_group(oracle, w):
    N = 32
    r = rng(5)
    p = rand_words(r, w, N)
    for k in list(range(-2 * N - 3, 3 * N + 3, 7)) + [0, N, 2 * N, -N]:
        via_mul = oracle.poly_mul(w, p, monomial(N, k, w))
        assert np.array_equal(oracle.poly_mul_xk(w, p, k), via_mul), k
    for a, b in [(3, 5), (N - 1, N + 2), (2 * N - 1, 2 * N - 1), (-7, 11)]:
        lhs = oracle.poly_mul_xk(w, oracle.poly_mul_xk(w, p, a), b)
        assert np.array_equal(lhs, oracle.poly_mul_xk(w, p, a + b))
    mask = np.uint64((1 << w) - 1)
    ps = np.arange(N, dtype=np.int64) - 10
    for k in (0, 1, N - 1, N, N + 3, 2 * N - 1, -5):
        got = oracle.poly_mul_xk_signed(ps, k)
        ref = oracle.poly_mul_xk(w, ps.astype(np.uint64) & mask, k)
        assert np.array_equal(got.astype(np.uint64) & mask, ref)


def test_poly_mul_ring_axioms(oracle):
    w, N = W64, 128
    r = rng(9)
    a, b, c = (rand_words(r, w, N) for _ in range(3))
    assert np.array_equal(oracle.poly_mul(w, a, b), oracle.poly_mul(w, b, a))
    lhs = oracle.poly_mul(w, a, (b + c))
    rhs = oracle.poly_mul(w, a, b) + oracle.poly_mul(w, a, c)
    assert np.array_equal(lhs, rhs)


# ----------------------------------------------------------- decomposition --

def test_decomp_closed_form_exact(oracle):
    # exact base-256 digits of a 32-bit word, least significant first
    d = oracle.decomp(32, 8, 4, 0x12345678)
    assert list(d) == [0x78, 0x56, 0x34, 0x12]
    assert [oracle.gadget(32, 8, 4, j) for j in range(4)] == [1, 1 << 8, 1 << 16, 1 << 24]
    # truncated: l*beta = 24 < 32 keeps the top 24 bits, rounded half up
    assert list(oracle.decomp(32, 8, 3, 0x12345678)) == [0x56, 0x34, 0x12]
    assert list(oracle.decomp(32, 8, 3, 0x12345680)) == [0x57, 0x34, 0x12]
    assert list(oracle.decomp(32, 8, 3, 0xFFFFFF80)) == [0, 0, 0]  # wraps to 0
    assert [oracle.gadget(32, 8, 3, j) for j in range(3)] == [1 << 8, 1 << 16, 1 << 24]


@pytest.mark.parametrize("log2B,ell", [(3, 2), (2, 3), (4, 3), (3, 4), (5, 2), (4, 2), (1, 7)])
def test_decomp_recomposition_exhaustive_w12(oracle, log2B, ell):
    w = 12
    q = 1 << w
    r = max(0, w - ell * log2B)
    g = [oracle.gadget(w, log2B, ell, j) for j in range(ell)]
    for x in range(q):
        d = oracle.decomp(w, log2B, ell, x)
        assert all(0 <= int(v) < (1 << log2B) for v in d)
        rec = sum(int(v) * gj for v, gj in zip(d, g)) % q
        eps = (x - rec) % q
        if eps >= q // 2:
            eps -= q
        if r == 0:
            assert eps == 0
        else:
            assert -(1 << (r - 1)) <= eps < (1 << (r - 1)), (x, eps)


@pytest.mark.parametrize("w,log2B,ell", [(32, 7, 3), (32, 8, 3), (32, 2, 8), (64, 10, 4), (64, 3, 10),
                                         (32, 8, 4), (64, 16, 4)])
def test_decomp_recomposition_random(oracle, w, log2B, ell):
    q = 1 << w
    r = max(0, w - ell * log2B)
    g = [oracle.gadget(w, log2B, ell, j) for j in range(ell)]
    for x in rand_words(rng(w * ell), w, 300):
        d = oracle.decomp(w, log2B, ell, int(x))
        rec = sum(int(v) * gj for v, gj in zip(d, g)) % q
        eps = (int(x) - rec) % q
        if eps >= q // 2:
            eps -= q
        bound = (1 << (r - 1)) if r else 0
        assert -bound <= eps <= max(0, bound - 1)


# ------------------------------------------------------------- encryption ---

@pytest.mark.parametrize("w", [W32, W64])
def test_lwe_rlwe_phase_is_message_plus_error(oracle, w):
    r = rng(1)
    n, N = 40, 64
    s = r.integers(0, 2, n).astype(np.uint8)
    a = rand_words(r, w, n)
    ct = oracle.lwe_encrypt(w, s, a, -37, 12345)
    assert oracle.lwe_phase(w, s, ct) == (12345 - 37) % (1 << w)
    sk = r.integers(0, 2, N).astype(np.uint8)
    a = rand_words(r, w, N)
    e = r.integers(-100, 100, N)
    mu = rand_words(r, w, N)
    c = oracle.rlwe_encrypt(w, sk, a, e, mu)
    ph = oracle.rlwe_phase(w, sk, c)
    assert np.array_equal(ph, (mu + e.astype(np.uint64)) & np.uint64((1 << w) - 1))
    # b = a*sk + e + mu against the independent product
    b = (kronecker_negacyclic(a, sk.astype(np.uint64), w) + e.astype(np.uint64) + mu)
    if w < 64:
        b &= np.uint64((1 << w) - 1)
    assert np.array_equal(c[:N], b)


# -------------------------------------------------------- sample extract ----

@pytest.mark.parametrize("w", [W32, W64])
def test_sample_extract_phase_identity(oracle, w):
    """Lemma 'Correctness of Sample Extraction' is an exact identity: the
    extracted LWE phase under Coefs(sk) is coefficient k of the RLWE phase."""
    r = rng(2)
    N = 64
    sk = r.integers(0, 2, N).astype(np.uint8)
    for trial in range(3):
        c = rand_words(r, w, 2 * N)
        ph = oracle.rlwe_phase(w, sk, c)
        for k in range(N):
            lwe = oracle.sample_extract(w, c, k)
            assert oracle.lwe_phase(w, sk, lwe) == int(ph[k])


# ----------------------------------------------------------- key switching --

def _tiny_keys(oracle, ps, seed=0):
    return oracle.Keys(ps, S.key_randomness(ps, seed))


def test_keyswitch_exact_phase_noiseless(oracle):
    """Noiseless keys and exact decomposition: KeySwitch preserves the phase
    exactly (proof of Lemma 'Correctness of Key Switching')."""
    ps = S.PARAM_SETS["Z"]
    k = _tiny_keys(oracle, ps)
    r = rng(3)
    sF = k.sk
    for _ in range(5):
        ct = rand_words(r, ps.w, ps.N + 1)
        ph = oracle.lwe_phase(ps.w, sF, ct)
        out = oracle.keyswitch(ps.w, ps.log2Bks, ps.lks, k.ksk, ct)
        assert oracle.lwe_phase(ps.w, k.s, out) == ph
        outR = oracle.keyswitch(ps.w, ps.log2Bpk, ps.lpk, k.pk, ct)
        phR = oracle.rlwe_phase(ps.w, k.sk, outR)
        assert int(phR[0]) == ph and not phR[1:].any()


def test_keyswitch_noise_within_lemma(oracle):
    """Lemma 'Correctness of Key Switching': error variance <= B_c +
    (1/3) n l B^2 B_ksK, plus the truncation term n * 4^r / 12 * E[s]."""
    ps = S.PARAM_SETS["A"]
    k = _tiny_keys(oracle, ps, 1)
    r = rng(4)
    errs = []
    for _ in range(60):
        mu = int(r.integers(0, ps.t)) * oracle.delta(ps.w, ps.t)
        ct = oracle.lwe_encrypt(ps.w, k.sk, rand_words(r, ps.w, ps.N), 0, mu)
        out = oracle.keyswitch(ps.w, ps.log2Bks, ps.lks, k.ksk, ct)
        e = (oracle.lwe_phase(ps.w, k.s, out) - mu) % (1 << ps.w)
        if e >= 1 << (ps.w - 1):
            e -= 1 << ps.w
        errs.append(e)
    var = np.var(np.array(errs, dtype=np.float64)) + np.mean(np.array(errs, dtype=np.float64)) ** 2
    rbits = ps.w - ps.lks * ps.log2Bks
    bound = (1 / 3) * ps.N * ps.lks * (1 << ps.log2Bks) ** 2 * ps.sigma_lwe ** 2 \
        + ps.N * (4.0 ** rbits) / 12 * 0.5
    assert var <= 1.5 * bound
    assert var >= bound / 16


# ------------------------------------------------- external product / CMux --

def _rgsw_noiseless(oracle, ps, sk, mbit, r):
    """RGSW(m) with sigma = 0 (Definition 'Generalized-GSW Sample')."""
    N, l = ps.N, ps.lg
    rows = np.zeros((2 * l, 2, N), dtype=np.uint64)
    for row in range(2 * l):
        c = oracle.rlwe_encrypt(ps.w, sk, rand_words(r, ps.w, N), np.zeros(N, np.int64))
        c = c.reshape(2, N)
        cc, j = row // l, row % l
        c[cc, 0] = (int(c[cc, 0]) + mbit * oracle.gadget(ps.w, ps.log2Bg, l, j)) % (1 << ps.w)
        rows[row] = c
    return rows


def test_cmux_selects_exactly_noiseless(oracle):
    ps = S.PARAM_SETS["Z"]
    r = rng(6)
    sk = r.integers(0, 2, ps.N).astype(np.uint8)
    for mbit in (0, 1):
        C = _rgsw_noiseless(oracle, ps, sk, mbit, r)
        g = rand_words(r, ps.w, 2 * ps.N)
        h = rand_words(r, ps.w, 2 * ps.N)
        out = oracle.cmux(ps, C, g, h)
        want = g if mbit else h
        assert np.array_equal(oracle.rlwe_phase(ps.w, sk, out), oracle.rlwe_phase(ps.w, sk, want))


def test_blind_rotate_noiseless_is_monomial_rotation(oracle):
    """Noiseless BR of a trivial accumulator (v, 0) by ct_N gives an RLWE of
    v * X^{-<a, s>} exactly (Lemma 'Correctness of TFHE-Style Blind-Rotation'
    under reading G4)."""
    ps = S.PARAM_SETS["Z"]
    k = _tiny_keys(oracle, ps, 3)
    r = rng(7)
    N = ps.N
    for _ in range(2):
        v = rand_words(r, ps.w, N)
        acc = np.concatenate([v, np.zeros(N, np.uint64)])
        ctN = r.integers(0, 2 * N, ps.n + 1).astype(np.uint64)
        out = oracle.blind_rotate(ps, k.bsk, acc, ctN)
        rot = -int(np.dot(ctN[1:].astype(np.int64), k.s.astype(np.int64)))
        assert np.array_equal(oracle.rlwe_phase(ps.w, k.sk, out), oracle.poly_mul_xk(ps.w, v, rot))


def test_blind_rotate_noise_within_lemma(oracle):
    """Error variance of BR vs Lemma 'Correctness of TFHE-Style Blind-Rotation'
    (2/3 n N l B^2 B_brK) plus the truncation term of our decomposition."""
    ps = S.PARAM_SETS["A"]
    k = _tiny_keys(oracle, ps, 4)
    r = rng(8)
    N = ps.N
    errs = []
    for _ in range(4):
        v = rand_words(r, ps.w, N)
        acc = np.concatenate([v, np.zeros(N, np.uint64)])
        ctN = r.integers(0, 2 * N, ps.n + 1).astype(np.uint64)
        out = oracle.blind_rotate(ps, k.bsk, acc, ctN)
        rot = -int(np.dot(ctN[1:].astype(np.int64), k.s.astype(np.int64)))
        e = (oracle.rlwe_phase(ps.w, k.sk, out) - oracle.poly_mul_xk(ps.w, v, rot)).astype(np.int64)
        errs.append(e.astype(np.int32).astype(np.float64))   # centred in 32 bits
    var = float(np.mean(np.concatenate(errs) ** 2))
    rb = ps.w - ps.lg * ps.log2Bg
    B2 = (1 << ps.log2Bg) ** 2
    bound = (2 / 3) * ps.n * N * ps.lg * B2 * ps.sigma_glwe ** 2 \
        + ps.n * (N * 0.5 + 1) * (4.0 ** rb) / 12 * 2
    assert var <= 1.5 * bound
    assert var >= bound / 64


@pytest.mark.parametrize("log2B,ell", [(2, 3), (3, 4), (4, 3), (3, 2), (6, 2)])
def test_decomp_signed_recomposition_exhaustive_w12(oracle, log2B, ell):
    """Balanced digits (reading G21): every digit in [-B/2, B/2), and for all
    x in Z_{2^12} the digits recompose (mod 2^12) to the same rounded value
    x~ 2^r as the unsigned decomposition, within 2^{r-1} of x."""
    w = 12
    B = 1 << log2B
    r = max(0, w - ell * log2B)
    g = [oracle.gadget(w, log2B, ell, j) for j in range(ell)]
    for x in range(1 << w):
        d = oracle.decomp_signed(w, log2B, ell, x)
        assert all(-B // 2 <= int(v) < B // 2 for v in d), (x, d)
        rec = sum(int(v) * gj for v, gj in zip(d, g)) % (1 << w)
        assert rec == (oracle.decomp_round(w, log2B, ell, x) << r) % (1 << w)
        err = (x - rec) % (1 << w)
        err = err - (1 << w) if err >= (1 << (w - 1)) else err
        assert abs(err) <= (1 << (r - 1) if r else 0)


def test_decomp_signed_is_the_unique_balanced_form(oracle):
    """Brute force at w = 6, B = 4, l = 3 (exact): the 64 digit vectors in
    [-2, 2)^3 hit every residue of Z_64 once, and the oracle returns that
    vector for each x."""
    w, log2B, ell = 6, 2, 3
    table = {}
    for d in itertools.product(range(-2, 2), repeat=ell):
        table[sum(v * 4 ** j for j, v in enumerate(d)) % 64] = d
    assert len(table) == 64
    for x in range(64):
        assert tuple(int(v) for v in oracle.decomp_signed(w, log2B, ell, x)) == table[x]


def test_blind_rotate_signed_noiseless_is_monomial_rotation(oracle):
    """With balanced digits the noiseless BR still multiplies by X^{-<a, s>}
    exactly (the digits recompose to the same value)."""
    import dataclasses
    ps = dataclasses.replace(S.PARAM_SETS["Z"], signed_digits=True)
    k = _tiny_keys(oracle, ps, 3)
    r = rng(17)
    N = ps.N
    for _ in range(2):
        v = rand_words(r, ps.w, N)
        acc = np.concatenate([v, np.zeros(N, np.uint64)])
        ctN = r.integers(0, 2 * N, ps.n + 1).astype(np.uint64)
        out = oracle.blind_rotate(ps, k.bsk, acc, ctN)
        rot = -int(np.dot(ctN[1:].astype(np.int64), k.s.astype(np.int64)))
        assert np.array_equal(oracle.rlwe_phase(ps.w, k.sk, out), oracle.poly_mul_xk(ps.w, v, rot))


def test_blind_rotate_signed_digits_quarter_noise(oracle):
    """Balanced digits have E[d^2] = B^2/12 against B^2/3 for digits uniform in
    [0, B): on set A, where the key noise dominates, the BR error variance
    drops about fourfold, and stays within a quarter of the lemma's bound."""
    import dataclasses
    base = S.PARAM_SETS["A"]
    k = _tiny_keys(oracle, base, 4)
    N = base.N
    var = {}
    for sgn in (False, True):
        ps = dataclasses.replace(base, signed_digits=sgn)
        r = rng(8)
        errs = []
        for _ in range(4):
            v = rand_words(r, ps.w, N)
            acc = np.concatenate([v, np.zeros(N, np.uint64)])
            ctN = r.integers(0, 2 * N, ps.n + 1).astype(np.uint64)
            out = oracle.blind_rotate(ps, k.bsk, acc, ctN)
            rot = -int(np.dot(ctN[1:].astype(np.int64), k.s.astype(np.int64)))
            e = (oracle.rlwe_phase(ps.w, k.sk, out) - oracle.poly_mul_xk(ps.w, v, rot)).astype(np.int64)
            errs.append(e.astype(np.int32).astype(np.float64))
        var[sgn] = float(np.mean(np.concatenate(errs) ** 2))
    assert 2.5 < var[False] / var[True] < 6.0
    B2 = (1 << base.log2Bg) ** 2
    rb = base.w - base.lg * base.log2Bg
    bound = (2 / 3) * base.n * N * base.lg * B2 * base.sigma_glwe ** 2 / 4 \
        + base.n * (N * 0.5 + 1) * (4.0 ** rb) / 12 * 2
    assert var[True] <= 1.5 * bound


# ------------------------------------------------------------- mod switch ---

def test_modswitch_rounding_and_error(oracle):
    w, k = 32, 9
    # round half up at the exact midpoint, and wrap-around at the top
    half = 1 << (w - k - 1)
    assert list(oracle.modswitch(w, k, [half - 1, half, (1 << w) - 1])) == [0, 1, 0]
    r = rng(10)
    n = 50
    s = r.integers(0, 2, n).astype(np.uint8)
    for _ in range(50):
        ph_target = int(r.integers(0, 1 << w))
        ct = oracle.lwe_encrypt(w, s, rand_words(r, w, n), 0, ph_target)
        ctN = oracle.modswitch(w, k, ct)
        phN = (int(ctN[0]) - int(np.dot(ctN[1:].astype(np.int64), s.astype(np.int64)))) % (1 << k)
        err = (phN - ph_target * (1 << k) / (1 << w)) % (1 << k)
        if err > (1 << (k - 1)):
            err -= 1 << k
        assert abs(err) <= (1 + int(s.sum())) / 2


# ------------------------------------------------------ SetupPolynomial -----

@pytest.mark.parametrize("N,t", [(256, 4), (64, 8), (1024, 16), (128, 32), (64, 64)])
def test_setup_polynomial_theorem_bruteforce(oracle, N, t):
    """Theorem 'rotation-polynomial-correctness': for every m and every e with
    |e| < N/t, coefficient 0 of rotP_0 * X^y (y in [0,N)) or rotP_1 * X^y
    (y in [N,2N)) equals f(m)."""
    r = rng(N * t)
    for trial in range(3):
        f = r.integers(0, t, t)
        p0, p1 = oracle.setup_polynomial(N, t, f)
        step = 2 * N // t
        E = N // t
        for m in range(t):
            for e in range(-E + 1, E):
                y = (step * m + e) % (2 * N)
                p = p0 if y < N else p1
                assert oracle.poly_mul_xk_signed(p, y)[0] == f[m], (m, e)


def test_setup_polynomial_tie_rules(oracle):
    """Reading G8: windows overlap at y = step*m + N/t; the later write (m+1)
    wins inside, and m = t-1 wins at the wrap y = 2N - N/t."""
    N, t = 64, 8
    f = np.array([11, 12, 13, 14, 15, 16, 17, 18])
    p0, p1 = oracle.setup_polynomial(N, t, f)
    step, E = 2 * N // t, N // t
    for m in range(t - 1):
        y = step * m + E
        p = p0 if y < N else p1
        assert oracle.poly_mul_xk_signed(p, y)[0] == f[m + 1]
    y = 2 * N - E
    assert oracle.poly_mul_xk_signed(p1, y)[0] == f[t - 1]
    # every slot is written, and by the sign pattern of the construction
    assert (p0[1:] <= 0).all() and p0[0] >= 0 and (p1[1:] >= 0).all() and p1[0] <= 0


# -------------------------------------------------------------- whole FDFB --

def test_fdfb_noiseless_exhaustive(oracle):
    """Theorem 'Correctness of the Bootstrapping' at sigma = 0 with exact
    decompositions: for all m in Z_4 (both halves of the torus) and all 256
    functions f: Z_4 -> Z_4 the output phase is exactly Delta * f(m)."""
    ps = S.PARAM_SETS["Z"]
    k = _tiny_keys(oracle, ps, 0)
    t = ps.t
    fs = np.array(list(itertools.product(range(t), repeat=t)), dtype=np.int64)   # 256 x 4
    rot = np.zeros((len(fs), 2, ps.N), dtype=np.int64)
    for i, f in enumerate(fs):
        rot[i, 0], rot[i, 1] = oracle.setup_polynomial(ps.N, t, f)
    ms = np.tile(np.arange(t), len(fs))
    ids = np.repeat(np.arange(len(fs)), t).astype(np.int32)
    mr = S.message_randomness(ps, 0, len(ms), m=ms)
    cts = oracle.encrypt_messages(ps, k.s, mr)
    outs = oracle.fdfb_batch(ps, k, rot, ids, cts)
    for c in range(len(ms)):
        want = (oracle.delta(ps.w, ps.t) * int(fs[ids[c], ms[c]])) % (1 << ps.w)
        assert oracle.lwe_phase(ps.w, k.s, outs[c]) == want, (ids[c], ms[c])


def test_fdfb_signed_digits_noiseless(oracle):
    """The whole FDFB with balanced blind-rotation digits, sigma = 0 and
    exact decompositions: for all m in Z_4 and 32 functions f: Z_4 -> Z_4
    the output phase is exactly Delta f(m)."""
    import dataclasses
    ps = dataclasses.replace(S.PARAM_SETS["Z"], signed_digits=True)
    k = _tiny_keys(oracle, ps, 0)
    t = ps.t
    fs = np.array(list(itertools.product(range(t), repeat=t)), dtype=np.int64)[::8]
    rot = np.zeros((len(fs), 2, ps.N), dtype=np.int64)
    for i, f in enumerate(fs):
        rot[i, 0], rot[i, 1] = oracle.setup_polynomial(ps.N, t, f)
    ms = np.tile(np.arange(t), len(fs))
    ids = np.repeat(np.arange(len(fs)), t).astype(np.int32)
    mr = S.message_randomness(ps, 0, len(ms), m=ms)
    cts = oracle.encrypt_messages(ps, k.s, mr)
    outs = oracle.fdfb_batch(ps, k, rot, ids, cts)
    for c in range(len(ms)):
        want = (oracle.delta(ps.w, ps.t) * int(fs[ids[c], ms[c]])) % (1 << ps.w)
        assert oracle.lwe_phase(ps.w, k.s, outs[c]) == want, (ids[c], ms[c])


@pytest.mark.parametrize("t_out", [2, 8, 16])
def test_fdfb_other_output_modulus_noiseless(oracle, t_out):
    """f: Z_t -> Z_t' with t' != t (Section 1.1, footnote: a different message
    scaling): sigma = 0, exact decompositions, t = 4; for all m in Z_4 and
    every function (t' = 2: all 16) or 48 seeded ones (t' = 8, 16), the output
    phase is exactly Delta' f(m) with Delta' = q / t'."""
    import dataclasses
    ps = dataclasses.replace(S.PARAM_SETS["Z"], t_out=t_out)
    k = _tiny_keys(oracle, ps, 0)
    t = ps.t
    if t_out ** t <= 64:
        fs = np.array(list(itertools.product(range(t_out), repeat=t)), dtype=np.int64)
    else:
        fs = np.random.default_rng(t_out).integers(0, t_out, size=(48, t))
    rot = np.zeros((len(fs), 2, ps.N), dtype=np.int64)
    for i, f in enumerate(fs):
        rot[i, 0], rot[i, 1] = oracle.setup_polynomial(ps.N, t, f)
    ms = np.tile(np.arange(t), len(fs))
    ids = np.repeat(np.arange(len(fs)), t).astype(np.int32)
    mr = S.message_randomness(ps, 0, len(ms), m=ms)
    cts = oracle.encrypt_messages(ps, k.s, mr)
    outs = oracle.fdfb_batch(ps, k, rot, ids, cts)
    for c in range(len(ms)):
        want = (oracle.delta_out(ps) * int(fs[ids[c], ms[c]])) % (1 << ps.w)
        assert oracle.lwe_phase(ps.w, k.s, outs[c]) == want, (ids[c], ms[c])


def test_fdfb_multi_noiseless_exhaustive(oracle):
    """Several functions of one input (Section 'Application of Functional
    Bootstrapping': the sign accumulators are reused): at sigma = 0 with exact
    decompositions, one call per message m in Z_4 evaluates all 256 functions
    f: Z_4 -> Z_4, and every output phase is exactly Delta * f(m)."""
    ps = S.PARAM_SETS["Z"]
    k = _tiny_keys(oracle, ps, 0)
    t = ps.t
    fs = np.array(list(itertools.product(range(t), repeat=t)), dtype=np.int64)
    rot = np.zeros((len(fs), 2, ps.N), dtype=np.int64)
    for i, f in enumerate(fs):
        rot[i, 0], rot[i, 1] = oracle.setup_polynomial(ps.N, t, f)
    ms = np.arange(t)
    ids = np.tile(np.arange(len(fs), dtype=np.int32), (t, 1))     # [4][256]
    mr = S.message_randomness(ps, 1, t, m=ms)
    cts = oracle.encrypt_messages(ps, k.s, mr)
    outs = oracle.fdfb_batch_multi(ps, k, rot, ids, cts)
    assert outs.shape == (t, len(fs), ps.n + 1)
    for m in range(t):
        for i in range(len(fs)):
            want = (oracle.delta(ps.w, ps.t) * int(fs[i, m])) % (1 << ps.w)
            assert oracle.lwe_phase(ps.w, k.s, outs[m, i]) == want, (m, i)


def test_fdfb_multi_equals_single(oracle):
    """The sign part of the bootstrap does not depend on the table, so the
    multi-table form returns, for every (input, table), the bits of the
    single-table bootstrap (set A with noise, 5 inputs x 3 tables)."""
    ps = S.PARAM_SETS["A"]
    k = _tiny_keys(oracle, ps, 4)
    fs = S.lut_tables(ps, 4, 4)
    rot = np.stack([np.stack(oracle.setup_polynomial(ps.N, ps.t, f)) for f in fs])
    ids = np.array([[0, 1, 2], [3, 3, 0], [1, 2, 3], [2, 0, 1], [0, 0, 0]], dtype=np.int32)
    mr = S.message_randomness(ps, 4, len(ids))
    cts = oracle.encrypt_messages(ps, k.s, mr)
    multi = oracle.fdfb_batch_multi(ps, k, rot, ids, cts)
    single = oracle.fdfb_batch(ps, k, rot, ids.reshape(-1), np.repeat(cts, ids.shape[1], axis=0))
    assert np.array_equal(multi.reshape(-1, ps.n + 1), single)
    one = oracle.fdfb_bootstrap_multi(ps, k, rot[ids[1]], cts[1])
    assert np.array_equal(one, multi[1])


def test_tfhe_bootstrap_noiseless_closed_form(oracle):
    """TFHE bootstrap (figure 'TFHE Bootstrapping') with noiseless keys and
    exact decompositions: BlindRotate multiplies by X^{-<a_N, s>} exactly, so
    the output phase is coefficient 0 of poly X^{b_N - <a_N, s>}, computed
    here from the definition of the negacyclic ring (X^N = -1) for arbitrary
    input words and a random polynomial."""
    ps = S.PARAM_SETS["Z"]
    k = _tiny_keys(oracle, ps, 2)
    rng = np.random.default_rng(21)
    N, w = ps.N, ps.w
    logN = N.bit_length() - 1
    for trial in range(6):
        poly = rng.integers(0, 1 << w, size=N, dtype=np.uint64)
        ct = rng.integers(0, 1 << w, size=ps.n + 1, dtype=np.uint64)
        out = oracle.tfhe_bootstrap(ps, k, poly, ct)
        # ModSwitch to 2N with rounding half up, then the rotation exponent
        msw = [((int(x) + (1 << (w - logN - 2))) >> (w - logN - 1)) % (2 * N) for x in ct]
        e = (msw[0] - sum(msw[1 + i] * int(k.s[i]) for i in range(ps.n))) % (2 * N)
        # the coefficient of X^0 in poly X^e comes from poly[j], j + e = 0 mod 2N,
        # negated when j lies in [N, 2N) (X^N = -1)
        j = (2 * N - e) % (2 * N)
        want = int(poly[j]) if j < N else (-int(poly[j - N])) % (1 << w)
        assert oracle.lwe_phase(w, k.s, out) == want, trial


def test_tfhe_bootstrap_toy_decrypts(oracle):
    """Set A: the TFHE bootstrap with a test polynomial for a random f on the
    first half of Z_t maps every m < t/2 to f(m) and m >= t/2 to -f(m - t/2)
    (negacyclic), after decryption."""
    ps = S.PARAM_SETS["A"]
    k = _tiny_keys(oracle, ps, 3)
    f_half = np.random.default_rng(22).integers(0, ps.t, size=ps.t // 2)
    poly = oracle.tfhe_test_polynomial(ps, f_half)
    mr = S.message_randomness(ps, 3, 24)
    cts = oracle.encrypt_messages(ps, k.s, mr)
    outs = oracle.tfhe_batch(ps, k, poly[None, :], np.zeros(len(cts), np.int32), cts)
    got = [oracle.lwe_decrypt(ps.w, ps.t, k.s, o) for o in outs]
    want = [int(f_half[m]) if m < ps.t // 2 else (-int(f_half[m - ps.t // 2])) % ps.t for m in mr.m]
    assert got == want


def test_fdfb_toy_decrypts(oracle):
    """Toy workload (set A, seed 0): every output decrypts to f(m)."""
    wl = S.WORKLOADS["toy"]
    g = wl.groups[0]
    ps = S.PARAM_SETS[g.set_name]
    k = _tiny_keys(oracle, ps, wl.seed)
    fs = S.lut_tables(ps, wl.seed, g.n_luts)
    rot = np.stack([np.stack(oracle.setup_polynomial(ps.N, ps.t, f)) for f in fs])
    ids = S.lut_assignment(wl.seed, g.batch, g.n_luts, g.lut_assign)
    mr = S.message_randomness(ps, wl.seed, g.batch)
    cts = oracle.encrypt_messages(ps, k.s, mr)
    outs = oracle.fdfb_batch(ps, k, rot, ids, cts)
    got = [oracle.lwe_decrypt(ps.w, ps.t, k.s, o) for o in outs]
    want = [int(fs[i][m]) for i, m in zip(ids, mr.m)]
    assert got == want


# ------------------------------------------------------- LWE affine layer ---

@pytest.mark.parametrize("w", [W32, W64])
def test_lwe_affine_matches_big_integer_sum(oracle, w):
    """The affine layer (Lemma 'Linear Homomorphism of GLWE samples'):
    y[j][k] = sum_i W[j][i] x[i][k] mod 2^w, recomputed with Python's exact
    integers.  Non-square weights (a transposed W cannot even be applied),
    weights of both signs including the int32 extremes, and every LWE
    component k, so a dropped sign, a swapped index or a truncated product
    fails."""
    r = rng(40 + w)
    n_in, n_out, length = 7, 5, 11
    W = r.integers(-8, 8, size=(n_out, n_in), dtype=np.int64)
    W[0, 0], W[1, 2], W[4, 6] = -(1 << 31), (1 << 31) - 1, -1
    x = rand_words(r, w, (n_in, length))
    y = oracle.lwe_affine(w, W, x)
    assert y.shape == (n_out, length)
    for j in range(n_out):
        for k in range(length):
            want = sum(int(W[j, i]) * int(x[i, k]) for i in range(n_in)) % (1 << w)
            assert int(y[j, k]) == want, (j, k)


@pytest.mark.parametrize("name", ["A", "D"])
def test_lwe_affine_is_homomorphic(oracle, name):
    """The linear homomorphism itself: for noiseless LWE samples of Delta m_i
    under one key, row j of the layer's output has phase exactly
    Delta * sum_i W[j][i] m_i mod q, so it decrypts to sum_i W[j][i] m_i
    mod t; with fresh noise it still decrypts to that sum mod t while the
    accumulated noise sum_i W[j][i] e_i stays below Delta/2."""
    ps = S.PARAM_SETS[name]
    w, t, n = ps.w, ps.t, ps.n
    D = oracle.delta(w, t)
    r = rng(50)
    s = r.integers(0, 2, size=n, dtype=np.uint8)
    n_in, n_out = 9, 4
    m = r.integers(0, t, size=n_in)
    W = r.integers(-8, 8, size=(n_out, n_in), dtype=np.int64)
    for sigma in (0.0, 2.0 ** (w - 20)):
        x = np.stack([oracle.lwe_encrypt(w, s, rand_words(r, w, n), int(round(sigma * r.standard_normal())),
                                         (D * int(m[i])) % (1 << w)) for i in range(n_in)])
        y = oracle.lwe_affine(w, W, x)
        for j in range(n_out):
            want = sum(int(W[j, i]) * int(m[i]) for i in range(n_in)) % t
            if sigma == 0.0:
                assert oracle.lwe_phase(w, s, y[j]) == (D * want) % (1 << w)
            assert oracle.lwe_decrypt(w, t, s, y[j]) == want


def test_prime_set_digit_counts(oracle):
    """Every prime-modulus set states l_g, l_ks, l_pk and l_boot equal to the
    exact decomposition's digit count ceil(log_B Q) (Definition
    'Decomposition'; Bootstrap figure, l_boot = ceil(log_{L_boot} Q)), and
    that count is the smallest l with B^l > Q -- checked here with exact
    integers, independently of the oracle's helper."""
    import oracle.prime_q as OQ
    for ps in S.Q_PARAM_SETS.values():
        for log2B, ell in ((ps.log2Bg, ps.lg), (ps.log2Bks, ps.lks), (ps.log2Bpk, ps.lpk),
                           (ps.log2Lboot, ps.lboot)):
            assert OQ.exact_digits(ps.Q, log2B) == ell, (ps.name, log2B)
            assert (1 << (log2B * ell)) > ps.Q and (1 << (log2B * (ell - 1))) <= ps.Q, (ps.name, log2B)
