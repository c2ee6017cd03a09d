"""Pins of the prime-modulus oracle (`oracle/fdfb_oracle_q.c`) against what
the paper and the mathematics fix: brute-force ring products with Python
integers, exact recomposition of the gadget digits, exact rounding with
fractions, the GLWE phase identities, the noise bounds of the external
product, blind rotation and key switching, PubMux on noiseless inputs (an
exact identity), and the bootstrap's decryption on every message."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import oracle.prime_q as OQ
from paper_2109_02731_gb300 import synth as S

PS = S.Q_PARAM_SETS["QZ"]
Q = PS.Q


@pytest.fixture(scope="module")
def keys():
    kr = S.q_key_randomness(PS, 11)
    return kr, OQ.QKeys(PS, kr)


def centred(x: int) -> int:
    x %= Q
    return x - Q if x > Q // 2 else x


def negacyclic(a, b, N):
    """Brute force: sum_{i,j} a_i b_j X^{i+j} with X^N = -1, Python integers."""
    out = [0] * N
    for i in range(N):
        for j in range(N):
            k = i + j
            if k < N:
                out[k] += int(a[i]) * int(b[j])
            else:
                out[k - N] -= int(a[i]) * int(b[j])
    return [v % Q for v in out]


def test_moduli_of_table_1():
    # Table 1's caption: Q_1 = 2^62 - 65535, ..., Q_4 = 2^32 - 139263;
    # every set's q is 2N and l = ceil(log_B Q)
    assert (S.Q1, S.Q2, S.Q3, S.Q4) == (2 ** 62 - 65535, 2 ** 63 - 278527, 2 ** 48 - 163839,
                                        2 ** 32 - 139263)
    for ps in S.Q_PARAM_SETS.values():
        assert ps.q == 2 * ps.N
        for log2B, ell in ((ps.log2Bg, ps.lg), (ps.log2Bks, ps.lks), (ps.log2Bpk, ps.lpk),
                           (ps.log2Lboot, ps.lboot)):
            assert 2 ** (log2B * ell) > ps.Q >= 2 ** (log2B * (ell - 1))
    p = S.Q_PARAM_SETS["FDFB-80-6"]
    assert (p.lg, p.lks, p.lpk, p.lboot) == (6, 11, 5, 6)


def test_poly_mul_brute_force():
    rng = np.random.default_rng(1)
    for N in (1, 2, 8):
        a = [int(x) for x in rng.integers(0, 2 ** 62, N, dtype=np.uint64) % np.uint64(Q)]
        b = [int(x) for x in rng.integers(0, 2 ** 62, N, dtype=np.uint64) % np.uint64(Q)]
        a[0] = Q - 1
        got = [int(x) for x in OQ.poly_mul(Q, a, b)]
        assert got == negacyclic(a, b, N)


def test_poly_mul_xk_is_monomial_product():
    rng = np.random.default_rng(2)
    N = 8
    p = [int(x) for x in rng.integers(0, 2 ** 62, N, dtype=np.uint64) % np.uint64(Q)]
    for k in (-17, -1, 0, 3, 8, 15, 16, 21):
        mono = [0] * N
        kk = k % (2 * N)
        mono[kk % N] = 1 if kk < N else Q - 1
        assert [int(x) for x in OQ.poly_mul_xk(Q, p, k)] == negacyclic(p, mono, N)


@pytest.mark.parametrize("log2B", [1, 6, 11, 13])
def test_exact_decomposition_recomposes(log2B):
    ell = -(-62 // log2B)
    rng = np.random.default_rng(log2B)
    xs = [0, 1, Q - 1, Q // 2] + [int(x) % Q for x in rng.integers(0, 2 ** 63, 50, dtype=np.uint64)]
    for x in xs:
        d = [int(v) for v in OQ.decomp(log2B, ell, x)]
        assert all(0 <= v < 2 ** log2B for v in d)
        assert sum(v << (log2B * j) for j, v in enumerate(d)) == x


def test_deltas_and_modswitch_round_exactly():
    for t in (2, 8, 64, 128):
        assert OQ.delta(Q, t) == int(Fraction(Q, t) + Fraction(1, 2))
        assert OQ.delta_half(Q, t) == int(Fraction(Q, 2 * t) + Fraction(1, 2))
    rng = np.random.default_rng(3)
    xs = [0, 1, Q - 1, Q // 2, (Q + 1) // 2] + [int(x) % Q for x in rng.integers(0, 2 ** 63, 200, dtype=np.uint64)]
    for logq in (9, 12, 13):
        got = OQ.modswitch(Q, logq, xs)
        want = [int(Fraction(2 ** logq * x, Q) + Fraction(1, 2)) % 2 ** logq for x in xs]
        assert [int(v) for v in got] == want


def test_rlwe_phase_is_message_plus_noise(keys):
    kr, _ = keys
    N = PS.N
    rng = np.random.default_rng(4)
    a = kr.pk_a[0, 0]
    e = rng.integers(-50, 50, N)
    mu = rng.integers(0, 2 ** 62, N, dtype=np.uint64) % np.uint64(Q)
    ct = OQ.rlwe_encrypt(Q, kr.sk, a, e, mu)
    ph = [int(x) for x in OQ.rlwe_phase(Q, kr.sk, ct)]
    assert ph == [(int(m) + int(x)) % Q for m, x in zip(mu, e)]
    # b = a * sk + e + mu by brute force on the first coefficients
    full = negacyclic([int(x) for x in a], [int(x) for x in kr.sk], N)
    assert [int(x) for x in ct[0][:4]] == [(full[k] + int(e[k]) + int(mu[k])) % Q for k in range(4)]


def test_key_rows_carry_the_gadget(keys):
    kr, K = keys
    N, lg = PS.N, PS.lg
    for i in (0, 5):
        for r in range(2 * lg):
            c, j = divmod(r, lg)
            row = K.bsk[i, r]
            g = int(kr.s[i]) * (1 << (PS.log2Bg * j)) % Q
            if c == 0:
                ph = OQ.rlwe_phase(Q, kr.sk, row)
                want = [(int(e) + (g if k == 0 else 0)) % Q for k, e in enumerate(kr.bsk_e[i, r])]
            else:
                # component 1 carries s_i g_j: phase = e - s_i g_j sk
                ph = OQ.rlwe_phase(Q, kr.sk, row)
                want = [(int(e) - g * int(kr.sk[k])) % Q for k, e in enumerate(kr.bsk_e[i, r])]
            assert [int(x) for x in ph] == want
    # ksK[i][j] = LWE_s(s_F[i] B^(j-1))
    for i in (0, 100):
        for j in (0, PS.lks - 1):
            ph = OQ.lwe_phase_q(Q, kr.s.astype(np.uint64), K.ksk[i, j])
            assert ph == (int(kr.sk[i]) * (1 << (PS.log2Bks * j)) + int(kr.ksk_e[i, j])) % Q


def test_external_product_message_and_noise(keys):
    kr, K = keys
    N = PS.N
    rng = np.random.default_rng(5)
    i = int(np.flatnonzero(kr.s)[0])  # RGSW(1)
    mu = rng.integers(0, 2 ** 62, N, dtype=np.uint64) % np.uint64(Q)
    d = OQ.rlwe_encrypt(Q, kr.sk, kr.pk_a[1, 0], np.zeros(N, np.int64), mu)
    out = OQ.extprod(PS, K.bsk[i], d)
    ph = OQ.rlwe_phase(Q, kr.sk, out)
    # phase = 1 * mu + sum_r D_r e_r: |noise| <= 2 lg N (B - 1) max|e|
    bound = 2 * PS.lg * N * (2 ** PS.log2Bg - 1) * int(np.abs(kr.bsk_e[i]).max())
    noise = [centred(int(p) - int(m)) for p, m in zip(ph, mu)]
    assert max(abs(v) for v in noise) <= bound
    assert max(abs(v) for v in noise) > 0


def test_blind_rotation_rotates_by_the_phase(keys):
    kr, K = keys
    N, n = PS.N, PS.n
    rng = np.random.default_rng(6)
    ctN = np.concatenate([[0], rng.integers(0, 2 * N, n)]).astype(np.uint64)
    h = OQ.delta_half(Q, PS.t)
    acc0 = np.zeros((2, N), dtype=np.uint64)
    acc0[0, 0] = h
    acc = OQ.blind_rotate(PS, K.bsk, acc0, ctN)
    # message h X^{-sum a_i s_i}
    rot = -int(sum(int(a) * int(s) for a, s in zip(ctN[1:], kr.s)))
    want = OQ.poly_mul_xk(Q, acc0[0], rot)
    ph = OQ.rlwe_phase(Q, kr.sk, acc)
    noise = [centred(int(p) - int(w)) for p, w in zip(ph, want)]
    bound = n * 2 * PS.lg * N * (2 ** PS.log2Bg - 1) * int(np.abs(kr.bsk_e).max())
    assert max(abs(v) for v in noise) <= bound
    assert max(abs(v) for v in noise) < h // 1000


def test_sample_extract_is_coefficient_zero(keys):
    kr, K = keys
    rng = np.random.default_rng(7)
    N = PS.N
    mu = rng.integers(0, 2 ** 62, N, dtype=np.uint64) % np.uint64(Q)
    ct = OQ.rlwe_encrypt(Q, kr.sk, kr.pk_a[2, 0], np.zeros(N, np.int64), mu)
    lwe = OQ.sample_extract(Q, ct)
    assert OQ.lwe_phase_q(Q, kr.sk, lwe) == int(mu[0])


def test_keyswitch_preserves_phase(keys):
    kr, K = keys
    N, n = PS.N, PS.n
    rng = np.random.default_rng(8)
    a = rng.integers(0, 2 ** 62, N, dtype=np.uint64) % np.uint64(Q)
    m = 123456789123
    ct = OQ.lwe_encrypt_q(Q, kr.sk, a, 0, m)
    out = OQ.keyswitch(Q, PS.log2Bks, PS.lks, K.ksk, ct)
    ph = OQ.lwe_phase_q(Q, kr.s.astype(np.uint64), out)
    bound = N * PS.lks * (2 ** PS.log2Bks - 1) * int(np.abs(kr.ksk_e).max())
    assert abs(centred(ph - m)) <= bound
    # packing key: LWE dim N -> RLWE, constant term keeps the phase
    rl = OQ.keyswitch(Q, PS.log2Bpk, PS.lpk, K.pk, ct).reshape(2, N)
    rph = OQ.rlwe_phase(Q, kr.sk, rl)
    bound = N * PS.lpk * (2 ** PS.log2Bpk - 1) * int(np.abs(kr.pk_e).max()) * 1
    assert abs(centred(int(rph[0]) - m)) <= bound
    assert all(abs(centred(int(v))) <= bound for v in rph[1:])


def test_pubmux_is_exact_on_noiseless_inputs():
    # c_i = [m L^(i-1), 0] (trivial RLWE samples): out = [Delta p_0 + m p, 0]
    # exactly, so m = 0 gives Delta p_0 and m = Delta gives Delta p_1
    N = PS.N
    rng = np.random.default_rng(9)
    p0 = rng.integers(-PS.t + 1, PS.t, N)
    p1 = rng.integers(-PS.t + 1, PS.t, N)
    D = OQ.delta(Q, PS.t)
    for m, pick in ((0, p0), (D, p1)):
        c = np.zeros((PS.lboot, 2, N), dtype=np.uint64)
        for i in range(PS.lboot):
            c[i, 0, 0] = m * (1 << (PS.log2Lboot * i)) % Q
        out = OQ.pubmux(PS, c, p0, p1)
        want = [D * int(v) % Q for v in pick]
        assert [int(x) for x in out[0]] == want
        assert not out[1].any()


def test_bootstrap_every_message(keys):
    kr, K = keys
    tables = S.q_lut_tables(PS, 11, 2)
    rot = OQ.rotation_polys(PS, tables)
    for li, f in enumerate(tables):
        mr = S.q_message_randomness(PS, 11, PS.t, group=li, m=np.arange(PS.t))
        cts = OQ.encrypt_messages(PS, kr.s, mr)
        out = OQ.fdfb_batch(PS, K, rot, np.full(PS.t, li, np.int32), cts, threads=oracle.max_threads())
        assert [OQ.decrypt(PS, kr.s, o) for o in out] == [int(v) for v in f]


def test_bootstrap_intermediates(keys):
    kr, K = keys
    f = S.q_lut_tables(PS, 11, 1)[0]
    rot = OQ.rotation_polys(PS, [f])[0]
    for m in (0, PS.t - 1):
        mr = S.q_message_randomness(PS, 12, 1, m=np.array([m]))
        ct = OQ.encrypt_messages(PS, kr.s, mr)[0]
        out, dbg = OQ.fdfb_bootstrap(PS, K, rot[0], rot[1], ct, debug=True)
        # sign LWE i encrypts L^(i-1) * 2 round(Q/2t) * beta, beta = [phase_N in [0, N)]
        phN = (int(ct[0]) - sum(int(a) * int(s) for a, s in zip(ct[1:], kr.s))) % PS.q
        beta = 1 if phN < PS.N else 0
        h = OQ.delta_half(Q, PS.t)
        for i in range(PS.lboot):
            ph = OQ.lwe_phase_q(Q, kr.sk, dbg["sgn"][i])
            want = (1 << (PS.log2Lboot * i)) * 2 * h * beta % Q
            assert abs(centred(ph - want)) < h // 1000
        # cKS decrypts under s to Delta_Q f(m); out is its ModSwitch to q
        ph = OQ.lwe_phase_q(Q, kr.s.astype(np.uint64), dbg["cKS"])
        assert abs(centred(ph - OQ.delta(Q, PS.t) * int(f[m]))) < OQ.delta(Q, PS.t) // 8
        assert np.array_equal(out, OQ.modswitch(Q, PS.logq, dbg["cKS"]))


def test_single_digit_pubmux_decrypts_alike(keys):
    # l_boot = 1 (L_boot >= Q): one sign rotation, the selector one digit
    # of 62 bits; the outputs differ in their noise but decrypt alike
    import dataclasses
    kr, K = keys
    ps1 = dataclasses.replace(PS, log2Lboot=62, lboot=1)
    assert ps1.lboot == 1
    f = S.q_lut_tables(PS, 11, 1)[0]
    rot = OQ.rotation_polys(PS, [f])
    mr = S.q_message_randomness(PS, 13, PS.t, m=np.arange(PS.t))
    cts = OQ.encrypt_messages(PS, kr.s, mr)
    out = OQ.fdfb_batch(ps1, K, rot, np.zeros(PS.t, np.int32), cts, threads=oracle.max_threads())
    assert [OQ.decrypt(PS, kr.s, o) for o in out] == [int(v) for v in f]


# ------------------------------------------------- CRT plaintexts (G29) -----

def crt_combine(residues, moduli):
    """The x in Z_t (t = prod moduli) with x = r_i mod t_i (brute force)."""
    t = int(np.prod(moduli))
    for x in range(t):
        if all(x % m == r for r, m in zip(residues, moduli)):
            return x
    raise AssertionError("no CRT solution")


def test_general_t_decryption_rounds_exactly():
    import dataclasses
    rng = np.random.default_rng(31)
    s = rng.integers(0, 2, PS.n).astype(np.uint8)
    for t in (3, 5, 7, 9, 64):
        ps = dataclasses.replace(PS, t=t)
        for _ in range(40):
            ct = rng.integers(0, PS.q, PS.n + 1).astype(np.uint64)
            ph = (int(ct[0]) - sum(int(a) * int(b) for a, b in zip(ct[1:], s))) % PS.q
            want = int(Fraction(t * ph, PS.q) + Fraction(1, 2)) % t
            assert OQ.decrypt(ps, s, ct) == want
    assert OQ.delta_in(S.crt_sets("QZ", [7])[0]) == round(PS.q / 7)


def test_crt_polynomial_on_every_residue():
    """Section "Extending the Arithmetic": Z_105 = Z_3 x Z_5 x Z_7; the
    polynomial P(x) = x^2 + 5x + 3 acts residue-wise, so each residue's
    bootstrap maps x_i to P(x_i) mod t_i.  Every residue of every modulus is
    bootstrapped; recombining the decrypted outputs gives P(x) mod 105 for
    every x in Z_105."""
    moduli = (3, 5, 7)
    sets = S.crt_sets("QZ", moduli)
    kr = S.q_key_randomness(PS, 41)
    K = OQ.QKeys(PS, kr)  # the keys do not depend on t
    P = lambda x: x * x + 5 * x + 3
    dec = []
    for ps in sets:
        table = np.array([P(m) % ps.t for m in range(ps.t)])
        rot = OQ.rotation_polys(ps, [table])
        mr = S.q_message_randomness(ps, 42, ps.t, m=np.arange(ps.t))
        cts = OQ.encrypt_messages(ps, kr.s, mr)
        out = OQ.fdfb_batch(ps, K, rot, np.zeros(ps.t, np.int32), cts, threads=oracle.max_threads())
        got = [OQ.decrypt(ps, kr.s, o) for o in out]
        assert got == [int(v) for v in table]
        dec.append(got)
    t = int(np.prod(moduli))
    for x in range(t):
        y = crt_combine([dec[i][x % m] for i, m in enumerate(moduli)], moduli)
        assert y == P(x) % t


def test_crt_addition_wraps_before_bootstrapping():
    """With t = 7 not dividing q = 2N, the sum of two encryptions still
    decrypts (after an identity bootstrap) to (a + b) mod 7, wrap included:
    Delta t = q + eps with |eps| < t/2 only adds eps to the noise (G29)."""
    ps = S.crt_sets("QZ", [7])[0]
    kr = S.q_key_randomness(PS, 43)
    K = OQ.QKeys(PS, kr)
    rot = OQ.rotation_polys(ps, [np.arange(7)])
    pairs = [(3, 5), (6, 6), (4, 3), (0, 6), (2, 1)]
    m = np.array([p for ab in pairs for p in ab])
    mr = S.q_message_randomness(ps, 44, len(m), m=m)
    cts = OQ.encrypt_messages(ps, kr.s, mr)
    sums = np.array([(cts[2 * i].astype(object) + cts[2 * i + 1].astype(object)) % ps.q
                     for i in range(len(pairs))], dtype=np.uint64)
    out = OQ.fdfb_batch(ps, K, rot, np.zeros(len(pairs), np.int32), sums, threads=oracle.max_threads())
    assert [OQ.decrypt(ps, kr.s, o) for o in out] == [(a + b) % 7 for a, b in pairs]


# ------------------------------- TFHE bootstrap, Q_4 (k = 32) ---------------

@pytest.mark.parametrize("name", ["QZ", "QT"])
def test_tfhe_bootstrap_decrypts_the_negacyclic_function(name):
    """Figure "TFHE Bootstrapping" on a prime modulus: with the test
    polynomial of f_half, m in [0, t/2) decrypts to f_half[m] and m + t/2 to
    -f_half[m] mod t, for every m."""
    ps = S.Q_PARAM_SETS[name]
    kr = S.q_key_randomness(ps, 61)
    K = OQ.QKeys(ps, kr)
    f_half = np.array([(3 * m + 1) % ps.t for m in range(ps.t // 2)])
    poly = OQ.tfhe_test_polynomial(ps, f_half)
    mr = S.q_message_randomness(ps, 62, ps.t, m=np.arange(ps.t))
    cts = OQ.encrypt_messages(ps, kr.s, mr)
    out = OQ.tfhe_batch(ps, K, poly[None, :], np.zeros(ps.t, np.int32), cts, threads=oracle.max_threads())
    want = [int(f_half[m]) if m < ps.t // 2 else (-int(f_half[m - ps.t // 2])) % ps.t for m in range(ps.t)]
    assert [OQ.decrypt(ps, kr.s, o) for o in out] == want
    # one rotation: coefficient 0 of the key-switched sample before ModSwitch
    # is Delta_Q f within the key switch's noise, so the output is exactly the
    # ModSwitch of a value near Delta_Q f (checked through decryption above)


def test_fdfb_on_q4_every_message():
    """The full-domain bootstrap's arithmetic on Q_4 = 2^32 - 139263 (k = 32),
    noiseless: with Delta_Q / 2 ~ 2^29 the literal PubMux over l_boot digits
    of p in Z_Q multiplies the packed samples' noise by digits up to 2^11
    (about 2^33 at these gadgets), which is why Table 1 uses Q_4 only for the
    TFHE bootstrap."""
    import dataclasses
    ps = dataclasses.replace(S.Q_PARAM_SETS["QT"], sigma_lwe=0.0, sigma_glwe=0.0, sigma_in=0.0)
    kr = S.q_key_randomness(ps, 63)
    K = OQ.QKeys(ps, kr)
    f = np.array([3, 0, 2, 1])
    rot = OQ.rotation_polys(ps, [f])
    mr = S.q_message_randomness(ps, 64, 2 * ps.t, m=np.tile(np.arange(ps.t), 2))
    cts = OQ.encrypt_messages(ps, kr.s, mr)
    out = OQ.fdfb_batch(ps, K, rot, np.zeros(len(cts), np.int32), cts, threads=oracle.max_threads())
    assert [OQ.decrypt(ps, kr.s, o) for o in out] == [int(f[m]) for m in mr.m]


def test_external_product_noise_matches_its_expectation(keys):
    """The external product's noise (Definition "External Product", exact
    decomposition) in closed form, conditional on the key: extProd(RGSW(s_i),
    d) has phase s_i mu + sum_r D_r * e_r with e_r row r's key error and D_r
    the digit polynomials of a uniform d.  Digits are independent with mean
    mu_r and variance v_r ((B-1)/2 and (B^2-1)/12 for the l-1 full digits;
    the exact distribution of floor(x / B^(l-1)) for the top digit of x
    uniform mod Q), so coefficient j's mean square is
        sum_r v_r ||e_r||^2 + (sum_r mu_r S_r(j))^2,
    S_r(j) = sum_{m <= j} e_r[m] - sum_{m > j} e_r[m] (the negacyclic signs).
    Averaged over 64 random d and all j, the oracle must be within 6 %."""
    kr, K = keys
    N, l = PS.N, PS.lg
    B = 1 << PS.log2Bg
    G = B ** (l - 1)
    T = -(-Q // G)
    probs = np.array([(min(Q, (v + 1) * G) - v * G) / Q for v in range(T)])
    vals = np.arange(T, dtype=np.float64)
    mu_T = float(probs @ vals)
    var_T = float(probs @ vals ** 2) - mu_T ** 2
    mus = [(B - 1) / 2] * (l - 1) + [mu_T]
    vrs = [(B * B - 1) / 12] * (l - 1) + [var_T]
    i = int(np.flatnonzero(kr.s)[0])
    want_var = 0.0
    mean_part = np.zeros(N)
    for r in range(2 * l):
        e = kr.bsk_e[i, r].astype(np.float64)
        jd = r % l
        want_var += vrs[jd] * float(e @ e)
        pre = np.cumsum(e)
        S_r = pre - (pre[-1] - pre)          # sum_{m<=j} e - sum_{m>j} e
        mean_part += mus[jd] * S_r
    want = want_var + float(np.mean(mean_part ** 2))
    rng = np.random.default_rng(92)
    acc = []
    for _ in range(64):
        mu = rng.integers(0, 2 ** 62, N, dtype=np.uint64) % np.uint64(Q)
        a = rng.integers(0, 2 ** 62, N, dtype=np.uint64) % np.uint64(Q)
        d = OQ.rlwe_encrypt(Q, kr.sk, a, np.zeros(N, np.int64), mu)
        ph = OQ.rlwe_phase(Q, kr.sk, OQ.extprod(PS, K.bsk[i], d))
        acc.append(np.array([centred(int(p) - int(m)) for p, m in zip(ph, mu)], dtype=np.float64))
    got = float(np.mean(np.concatenate(acc) ** 2))
    assert 0.94 * want <= got <= 1.06 * want, (got, want)


def _noiseless(ps):
    import dataclasses
    return dataclasses.replace(ps, sigma_lwe=0.0, sigma_glwe=0.0, sigma_in=0.0)


def test_tfhe_noiseless_phase_is_the_rotated_coefficient():
    """Figure "TFHE Bootstrapping" at sigma = 0 with the exact decomposition:
    the extracted sample's phase (under s_F) is exactly coefficient 0 of
    poly X^{b_N - <a_N, s>}, the key switch keeps it exactly (under s), and
    the bootstrap's output is the ModSwitch of that sample."""
    ps = _noiseless(PS)
    kr = S.q_key_randomness(ps, 93)
    K = OQ.QKeys(ps, kr)
    rng = np.random.default_rng(94)
    N, n = ps.N, ps.n
    for _ in range(3):
        poly = rng.integers(0, 2 ** 62, N, dtype=np.uint64) % np.uint64(Q)
        ct = rng.integers(0, 2 * N, n + 1).astype(np.uint64)
        acc = np.zeros((2, N), dtype=np.uint64)
        acc[0] = OQ.poly_mul_xk(Q, poly, int(ct[0]))
        acc = OQ.blind_rotate(ps, K.bsk, acc, ct)
        cQ = OQ.sample_extract(Q, acc)
        k = int(ct[0]) - sum(int(a) * int(s) for a, s in zip(ct[1:], kr.s))
        want = int(OQ.poly_mul_xk(Q, poly, k)[0])
        assert OQ.lwe_phase_q(Q, kr.sk, cQ) == want
        cks = OQ.keyswitch(Q, ps.log2Bks, ps.lks, K.ksk, cQ)
        assert OQ.lwe_phase_q(Q, kr.s.astype(np.uint64), cks) == want
        out = OQ.tfhe_bootstrap(ps, K, poly, ct)
        assert np.array_equal(out, OQ.modswitch(Q, ps.logq, cks))


def test_fdfb_noiseless_phase_within_the_rounding_of_delta():
    """The full-domain bootstrap at sigma = 0 (inputs noiseless too): the key
    switched sample's phase is Delta_Q f(m) up to the mismatch of G24 -- the
    sign samples carry 2 round(Q/2t) where PubMux uses round(Q/t), which
    differ by at most 1, times p_1 - p_0 (|.| < 2t) -- for every m and two
    tables; where the two roundings agree (Q_1, t = 8) the phase is exactly
    Delta_Q f(m)."""
    ps = _noiseless(PS)
    kr = S.q_key_randomness(ps, 95)
    K = OQ.QKeys(ps, kr)
    D = OQ.delta(Q, ps.t)
    for f in S.q_lut_tables(ps, 95, 2):
        rot = OQ.rotation_polys(ps, [f])[0]
        mr = S.q_message_randomness(ps, 96, ps.t, m=np.arange(ps.t))
        for m, ct in zip(range(ps.t), OQ.encrypt_messages(ps, kr.s, mr)):
            out, dbg = OQ.fdfb_bootstrap(ps, K, rot[0], rot[1], ct, debug=True)
            ph = OQ.lwe_phase_q(Q, kr.s.astype(np.uint64), dbg["cKS"])
            dev = centred(ph - D * int(f[m]))
            if 2 * OQ.delta_half(Q, ps.t) == D:
                assert dev == 0      # Q_1 with t = 8: the two roundings agree
            else:
                assert abs(dev) <= 2 * ps.t
            assert OQ.decrypt(ps, kr.s, out) == int(f[m])


def test_poly_mul_by_a_monomial_at_n_8192():
    """At Table 1's largest ring degree (FDFB:80:8, 100:8) the oracle's
    schoolbook product by +-X^k equals multiplication by X^k in
    Z_Q[X]/(X^N + 1): coefficient j receives p[j - k], negated where j - k
    wraps below 0 (X^N = -1)."""
    N = 8192
    rng = np.random.default_rng(3)
    p = rng.integers(0, 2 ** 62, N, dtype=np.uint64) % np.uint64(Q)
    for k, sgn in ((0, 1), (1, 1), (4095, Q - 1), (4096, 1), (8191, Q - 1)):
        mono = np.zeros(N, dtype=np.uint64)
        mono[k] = sgn
        got = [int(x) for x in OQ.poly_mul(Q, mono, p)]
        want = [(sgn * (int(p[j - k]) if j >= k else Q - int(p[j - k + N]))) % Q for j in range(N)]
        assert got == want, k
