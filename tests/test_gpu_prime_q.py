"""GPU parity for the prime-modulus parameter sets (Table 1): the CUDA
library, through its C ABI, against the prime-Q oracle on the same seeded
inputs.  Everything is exact integer arithmetic (mod Q on the RLWE side,
mod q = 2N on the LWE side), so every comparison is bit-exact."""
from __future__ import annotations

import dataclasses

import numpy as np
import pytest

from paper_2109_02731_gb300 import synth as S

pytestmark = pytest.mark.gpu

QZ = S.Q_PARAM_SETS["QZ"]


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("these tests need a CUDA GPU")
    return torch


@pytest.fixture(scope="module")
def F(torch_cuda):
    from paper_2109_02731_gb300 import fdfb
    return fdfb


@pytest.fixture(scope="module")
def ctx(F):
    c = F.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def OQ(oracle):
    import oracle.prime_q as m
    return m


@pytest.fixture(scope="module")
def qz(ctx, OQ):
    """QZ registered with the oracle's keys and two tables."""
    kr = S.q_key_randomness(QZ, 21)
    K = OQ.QKeys(QZ, kr)
    sid = ctx.register(QZ)
    ctx.keys_upload(sid, K.bsk, K.pk, K.ksk)
    tables = S.q_lut_tables(QZ, 21, 2)
    assert [ctx.lut_setup(sid, f) for f in tables] == [0, 1]
    rot = OQ.rotation_polys(QZ, tables)
    return sid, kr, K, tables, rot


def run_q(F, torch, ctx, sid, ps, cts, ids, debug=True):
    ct_d = F.to_device_words(ps, cts)
    ids_d = torch.tensor(np.asarray(ids, dtype=np.int32), device="cuda")
    out_d = torch.empty_like(ct_d)
    b, N, lb = len(cts), ps.N, ps.lboot
    if debug:
        e = lambda *shape: torch.empty(shape, dtype=torch.int64, device="cuda")
        dbg = dict(sgn=e(b, lb, N + 1), cR=e(b, lb, 2 * N), accF=e(b, 2 * N), cQ=e(b, N + 1),
                   cKS=e(b, ps.n + 1))
        ctx.bootstrap_debug(sid, ct_d, ids_d, out_d, dbg)
    else:
        ctx.bootstrap(sid, ct_d, ids_d, out_d)
    ctx.sync()
    out = F.to_host_words(ps, out_d).astype(np.uint64)
    if not debug:
        return out, None
    return out, {k: F.to_host_words(ps, v).astype(np.uint64) for k, v in dbg.items()}


def test_every_variant_matches_the_oracle(F, torch_cuda, ctx, OQ, qz):
    """Every message of Z_t under both tables plus a ragged tail: outputs and
    every intermediate bit for bit equal to the oracle, for every layout."""
    sid, kr, K, tables, rot = qz
    m = np.concatenate([np.arange(QZ.t), np.arange(QZ.t), [0, QZ.t - 1, 3]])
    ids = np.concatenate([np.zeros(QZ.t), np.ones(QZ.t), [1, 0, 1]]).astype(np.int32)
    mr = S.q_message_randomness(QZ, 22, len(m), m=m)
    cts = OQ.encrypt_messages(QZ, kr.s, mr)
    refs = [OQ.fdfb_bootstrap(QZ, K, rot[i][0], rot[i][1], c, debug=True) for c, i in zip(cts, ids)]
    cur, count, _ = ctx.variant_info(sid)
    assert count == 4
    for v in range(count):
        ctx.set_variant(sid, v)
        out, dbg = run_q(F, torch_cuda, ctx, sid, QZ, cts, ids)
        for c, (o, d) in enumerate(refs):
            for key in ("sgn", "cR", "accF", "cQ", "cKS"):
                assert np.array_equal(dbg[key][c].reshape(d[key].shape), d[key]), f"{key}, variant {v}, ct {c}"
            assert np.array_equal(out[c], o), f"output, variant {v}, ct {c}"
        dec = [OQ.decrypt(QZ, kr.s, o) for o in out]
        assert dec == [int(tables[i][mm]) for mm, i in zip(m, ids)]
    ctx.set_variant(sid, cur)


def test_plain_call_and_autotune_match(F, torch_cuda, ctx, OQ, qz):
    sid, kr, K, tables, rot = qz
    mr = S.q_message_randomness(QZ, 23, 40)
    cts = OQ.encrypt_messages(QZ, kr.s, mr)
    ids = S.lut_assignment(23, 40, 2, "uniform")
    ref = OQ.fdfb_batch(QZ, K, rot, ids, cts, threads=8)
    out, _ = run_q(F, torch_cuda, ctx, sid, QZ, cts, ids, debug=False)
    assert np.array_equal(out, ref)
    best, ms = ctx.autotune(sid, 40)
    assert ms > 0
    out2, _ = run_q(F, torch_cuda, ctx, sid, QZ, cts, ids, debug=False)
    assert np.array_equal(out2, ref)


def test_keygen_matches_the_oracle(ctx, OQ):
    kr = S.q_key_randomness(QZ, 24)
    sid = ctx.register(QZ)
    ctx.keys_generate(sid, kr)
    bsk, pk, ksk = ctx.keys_download(sid)
    K = OQ.QKeys(QZ, kr)
    assert np.array_equal(bsk.astype(np.uint64), K.bsk)
    assert np.array_equal(pk.astype(np.uint64), K.pk)
    assert np.array_equal(ksk.astype(np.uint64), K.ksk)


def test_lwe_side_and_keyswitch(F, torch_cuda, ctx, OQ, oracle, qz):
    sid, kr, K, tables, rot = qz
    torch = torch_cuda
    mr = S.q_message_randomness(QZ, 25, 33)
    s_d = torch.tensor(kr.s.astype(np.uint8), device="cuda")
    a_d = F.to_device_words(QZ, mr.a)
    ct_d = torch.empty((33, QZ.n + 1), dtype=torch.int64, device="cuda")
    ctx.lwe_encrypt(sid, s_d, a_d, torch.tensor(mr.e, device="cuda"), torch.tensor(mr.m, device="cuda"), ct_d)
    m_d = torch.empty(33, dtype=torch.int32, device="cuda")
    ctx.lwe_decrypt(sid, s_d, ct_d, m_d)
    ctx.sync()
    assert np.array_equal(F.to_host_words(QZ, ct_d).astype(np.uint64), OQ.encrypt_messages(QZ, kr.s, mr))
    assert np.array_equal(m_d.cpu().numpy(), mr.m)
    # standalone key switch mod Q: LWE under s_F (dimension N) -> under s
    rng = np.random.default_rng(5)
    x = (rng.integers(0, 2 ** 63, (7, QZ.N + 1), dtype=np.uint64) % np.uint64(QZ.Q))
    x_d = F.to_device_words(QZ, x)
    y_d = torch.empty((7, QZ.n + 1), dtype=torch.int64, device="cuda")
    ctx.keyswitch(sid, x_d, y_d)
    ctx.sync()
    y = F.to_host_words(QZ, y_d).astype(np.uint64)
    for i in range(7):
        assert np.array_equal(y[i], OQ.keyswitch(QZ.Q, QZ.log2Bks, QZ.lks, K.ksk, x[i]))


def test_registration_rules(F, ctx):
    def reg(ps):
        return ctx.register(ps)
    with pytest.raises(F.FDFBError):
        reg(dataclasses.replace(QZ, N=512))               # no layout at N = 512
    with pytest.raises(F.FDFBError):
        reg(dataclasses.replace(QZ, Q=S.Q1 + 1))          # even modulus
    with pytest.raises(F.FDFBError):
        reg(dataclasses.replace(QZ, Q=(1 << 31) - 1))     # k = 31 < 32
    with pytest.raises(F.FDFBError):
        reg(dataclasses.replace(QZ, log2Lboot=7, lboot=9))  # l_boot = 9 > 8
    # a caller-given l that is not ceil(k / log2 B)
    from paper_2109_02731_gb300.fdfb import fdfb_params
    import ctypes as C
    p = F.params_struct(QZ)
    p.lg = p.lg + 1
    sid = C.c_int()
    assert ctx.L.fdfb_params_register(ctx.h, C.byref(p), C.byref(sid)) == -1


def test_unavailable_calls_refuse(F, torch_cuda, ctx, qz):
    sid = qz[0]
    torch = torch_cuda
    ct = torch.zeros((2, QZ.n + 1), dtype=torch.int64, device="cuda")
    ids = torch.zeros((2, 2), dtype=torch.int32, device="cuda")
    out = torch.empty((2, 2, QZ.n + 1), dtype=torch.int64, device="cuda")
    with pytest.raises(F.FDFBError):
        ctx.bootstrap_multi(sid, ct, ids, out)
    with pytest.raises(F.FDFBError):  # a coefficient not below Q
        ctx.tfhe_poly_setup(sid, np.full(QZ.N, QZ.Q, np.uint64))


@pytest.mark.parametrize("name", ["FDFB-80-6", "FDFB-80-7"])
def test_full_size_decrypts_and_variants_agree(F, torch_cuda, ctx, OQ, name):
    """The paper's parameter sets at full size, keys generated on the GPU:
    every output decrypts to f(m), and every layout variant (and the
    autotuned, chunked call) returns the same bits."""
    ps = S.Q_PARAM_SETS[name]
    kr = S.q_key_randomness(ps, 31)
    sid = ctx.register(ps)
    ctx.keys_generate(sid, kr)
    tables = S.q_lut_tables(ps, 31, 3)
    for f in tables:
        ctx.lut_setup(sid, f)
    batch = 300
    mr = S.q_message_randomness(ps, 32, batch)
    cts = OQ.encrypt_messages(ps, kr.s, mr)
    ids = S.lut_assignment(32, batch, 3, "uniform")
    cur, count, _ = ctx.variant_info(sid)
    outs = []
    for v in range(count):
        ctx.set_variant(sid, v)
        out, _ = run_q(F, torch_cuda, ctx, sid, ps, cts, ids, debug=False)
        outs.append(out)
    for v in range(1, count):
        assert np.array_equal(outs[v], outs[0]), f"variant {v}"
    dec = [OQ.decrypt(ps, kr.s, o) for o in outs[0]]
    assert dec == [int(tables[i][m]) for m, i in zip(mr.m, ids)]
    ctx.autotune(sid, batch)
    out, _ = run_q(F, torch_cuda, ctx, sid, ps, cts, ids, debug=False)
    assert np.array_equal(out, outs[0])


# ------------------------------------------------- CRT plaintexts -----------

def test_crt_residue_set_matches_the_oracle(F, torch_cuda, ctx, OQ):
    """An odd plaintext modulus (t = 7, not dividing q = 2N): bootstraps bit
    for bit equal to the oracle's, and the library's encryption and general-t
    decryption equal the oracle's."""
    torch = torch_cuda
    ps = S.crt_sets("QZ", [7])[0]
    kr = S.q_key_randomness(QZ, 51)
    K = OQ.QKeys(QZ, kr)
    sid = ctx.register(ps)
    ctx.keys_upload(sid, K.bsk, K.pk, K.ksk)
    table = np.array([(m * m + 5 * m + 3) % 7 for m in range(7)])
    ctx.lut_setup(sid, table)
    rot = OQ.rotation_polys(ps, [table])
    m = np.concatenate([np.arange(7), np.arange(7)])
    mr = S.q_message_randomness(ps, 52, len(m), m=m)
    cts = OQ.encrypt_messages(ps, kr.s, mr)
    s_d = torch.tensor(kr.s.astype(np.uint8), device="cuda")
    ct_d = torch.empty((len(m), ps.n + 1), dtype=torch.int64, device="cuda")
    ctx.lwe_encrypt(sid, s_d, F.to_device_words(ps, mr.a), torch.tensor(mr.e, device="cuda"),
                    torch.tensor(mr.m, device="cuda"), ct_d)
    ctx.sync()
    assert np.array_equal(F.to_host_words(ps, ct_d).astype(np.uint64), cts)
    ids = np.zeros(len(m), np.int32)
    ref = OQ.fdfb_batch(ps, K, rot, ids, cts, threads=8)
    for v in range(ctx.variant_info(sid)[1]):
        ctx.set_variant(sid, v)
        out, _ = run_q(F, torch, ctx, sid, ps, cts, ids, debug=False)
        assert np.array_equal(out, ref), f"variant {v}"
    m_d = torch.empty(len(m), dtype=torch.int32, device="cuda")
    ctx.lwe_decrypt(sid, s_d, F.to_device_words(ps, out), m_d)
    ctx.sync()
    got = m_d.cpu().numpy()
    assert list(got) == [OQ.decrypt(ps, kr.s, o) for o in out] == [int(table[x]) for x in m]


def test_crt_polynomial_full_size(F, torch_cuda, ctx, OQ):
    """Z_9009 = Z_7 x Z_9 x Z_11 x Z_13 on FDFB-80-6's geometry: P(x) =
    x^2 + 5x + 3 for 300 random x, one bootstrap per residue (the four sets
    in one fdfb_bootstrap_mixed call), recombined by the CRT after
    decryption."""
    torch = torch_cuda
    moduli = (7, 9, 11, 13)
    t = int(np.prod(moduli))
    sets = S.crt_sets("FDFB-80-6", moduli)
    kr = S.q_key_randomness(S.Q_PARAM_SETS["FDFB-80-6"], 53)  # one secret for every residue
    rng = np.random.default_rng(54)
    x = rng.integers(0, t, 300)
    P = lambda v: (v * v + 5 * v + 3)
    s_d = torch.tensor(kr.s.astype(np.uint8), device="cuda")
    groups, dec = [], []
    for gi, ps in enumerate(sets):
        sid = ctx.register(ps)
        ctx.keys_generate(sid, kr)
        ctx.lut_setup(sid, [P(m) % ps.t for m in range(ps.t)])
        mr = S.q_message_randomness(ps, 55, len(x), m=x % ps.t)
        ct = torch.empty((len(x), ps.n + 1), dtype=torch.int64, device="cuda")
        ctx.lwe_encrypt(sid, s_d, F.to_device_words(ps, mr.a), torch.tensor(mr.e, device="cuda"),
                        torch.tensor(mr.m, device="cuda"), ct)
        ids = torch.zeros(len(x), dtype=torch.int32, device="cuda")
        groups.append((sid, ct, ids, torch.empty_like(ct)))
    ctx.bootstrap_mixed(groups)
    ctx.sync()
    for (sid, _, _, out), ps in zip(groups, sets):
        m_d = torch.empty(len(x), dtype=torch.int32, device="cuda")
        ctx.lwe_decrypt(sid, s_d, out, m_d)
        ctx.sync()
        got = m_d.cpu().numpy()
        assert np.array_equal(got, P(x) % ps.t), f"modulus {ps.t}"
        dec.append(got)
    # CRT recombination: y = sum r_i M_i (M_i^-1 mod t_i) mod t
    y = np.zeros(len(x), dtype=object)
    for r, mi in zip(dec, moduli):
        Mi = t // mi
        y = y + r.astype(object) * Mi * pow(Mi, -1, mi)
    assert [int(v) % t for v in y] == [int(P(int(v)) % t) for v in x]


# ----------------------------------- TFHE bootstrap and Q_4 (k = 32) --------

@pytest.mark.parametrize("name", ["QZ", "QT"])
def test_tfhe_matches_the_oracle(F, torch_cuda, ctx, OQ, name):
    """The TFHE bootstrap on a prime modulus, every layout, bit for bit equal
    to the oracle; outputs decrypt to the negacyclic function."""
    torch = torch_cuda
    ps = S.Q_PARAM_SETS[name]
    kr = S.q_key_randomness(ps, 71)
    K = OQ.QKeys(ps, kr)
    sid = ctx.register(ps)
    ctx.keys_upload(sid, K.bsk, K.pk, K.ksk)
    f_half = np.array([(3 * m + 1) % ps.t for m in range(ps.t // 2)])
    polys = np.stack([OQ.tfhe_test_polynomial(ps, f_half),
                      S.q_tfhe_polynomials(ps, 72, 1)[0]])
    assert [ctx.tfhe_poly_setup(sid, p) for p in polys] == [0, 1]
    m = np.concatenate([np.arange(ps.t), np.arange(ps.t), [1]])
    ids = np.concatenate([np.zeros(ps.t), np.ones(ps.t), [0]]).astype(np.int32)
    mr = S.q_message_randomness(ps, 73, len(m), m=m)
    cts = OQ.encrypt_messages(ps, kr.s, mr)
    ref = OQ.tfhe_batch(ps, K, polys, ids, cts, threads=8)
    for v in range(ctx.variant_info(sid)[1]):
        ctx.set_variant(sid, v)
        ct_d = F.to_device_words(ps, cts)
        out_d = torch.empty_like(ct_d)
        ctx.tfhe_bootstrap(sid, ct_d, torch.tensor(ids, device="cuda"), out_d)
        ctx.sync()
        out = F.to_host_words(ps, out_d).astype(np.uint64)
        assert np.array_equal(out, ref), f"variant {v}"
    want = [int(f_half[x]) if x < ps.t // 2 else (-int(f_half[x - ps.t // 2])) % ps.t for x in m[:ps.t]]
    assert [OQ.decrypt(ps, kr.s, o) for o in ref[:ps.t]] == want


def test_fdfb_on_q4_matches_the_oracle(F, torch_cuda, ctx, OQ):
    """The full-domain bootstrap's mod-Q arithmetic at k = 32 (noiseless, see
    the oracle pin), every layout bit for bit equal to the oracle."""
    ps = dataclasses.replace(S.Q_PARAM_SETS["QT"], sigma_lwe=0.0, sigma_glwe=0.0, sigma_in=0.0)
    kr = S.q_key_randomness(ps, 74)
    K = OQ.QKeys(ps, kr)
    sid = ctx.register(ps)
    ctx.keys_upload(sid, K.bsk, K.pk, K.ksk)
    f = np.array([3, 0, 2, 1])
    ctx.lut_setup(sid, f)
    rot = OQ.rotation_polys(ps, [f])
    m = np.tile(np.arange(ps.t), 3)
    mr = S.q_message_randomness(ps, 75, len(m), m=m)
    cts = OQ.encrypt_messages(ps, kr.s, mr)
    ids = np.zeros(len(m), np.int32)
    refs = [OQ.fdfb_bootstrap(ps, K, rot[0][0], rot[0][1], c, debug=True) for c in cts]
    for v in range(ctx.variant_info(sid)[1]):
        ctx.set_variant(sid, v)
        out, dbg = run_q(F, torch_cuda, ctx, sid, ps, cts, ids)
        for c, (o, d) in enumerate(refs):
            for key in ("sgn", "cR", "accF", "cQ", "cKS"):
                assert np.array_equal(dbg[key][c].reshape(d[key].shape), d[key]), f"{key}, variant {v}, ct {c}"
            assert np.array_equal(out[c], o), f"variant {v}, ct {c}"
    assert [OQ.decrypt(ps, kr.s, o) for o in out] == [int(f[x]) for x in m]


def test_tfhe_80_2_full_size(F, torch_cuda, ctx, OQ):
    """Table 1's TFHE:80:2 (n = 424, N = 1024, Q_4) at full size, keys
    generated on the GPU: every output decrypts to the negacyclic function,
    every layout returns the same bits."""
    torch = torch_cuda
    ps = S.Q_PARAM_SETS["TFHE-80-2"]
    kr = S.q_key_randomness(ps, 76)
    sid = ctx.register(ps)
    ctx.keys_generate(sid, kr)
    f_half = np.array([1, 3])
    ctx.tfhe_poly_setup(sid, OQ.tfhe_test_polynomial(ps, f_half))
    batch = 512
    mr = S.q_message_randomness(ps, 77, batch)
    s_d = torch.tensor(kr.s.astype(np.uint8), device="cuda")
    ct = torch.empty((batch, ps.n + 1), dtype=torch.int64, device="cuda")
    ctx.lwe_encrypt(sid, s_d, F.to_device_words(ps, mr.a), torch.tensor(mr.e, device="cuda"),
                    torch.tensor(mr.m, device="cuda"), ct)
    ids = torch.zeros(batch, dtype=torch.int32, device="cuda")
    outs = []
    for v in range(ctx.variant_info(sid)[1]):
        ctx.set_variant(sid, v)
        out = torch.empty_like(ct)
        ctx.tfhe_bootstrap(sid, ct, ids, out)
        ctx.sync()
        outs.append(F.to_host_words(ps, out).astype(np.uint64))
    for v in range(1, len(outs)):
        assert np.array_equal(outs[v], outs[0]), f"variant {v}"
    m_d = torch.empty(batch, dtype=torch.int32, device="cuda")
    ctx.lwe_decrypt(sid, s_d, F.to_device_words(ps, outs[0]), m_d)
    ctx.sync()
    want = [int(f_half[x]) if x < 2 else (-int(f_half[x - 2])) % 4 for x in mr.m]
    assert list(m_d.cpu().numpy()) == want


def test_fdfb_100_6_and_noalloc(F, torch_cuda, ctx, OQ):
    """FDFB:100:6 (n = 1050, B_ks = 2: 62 key-switch digits per word) decrypts
    correctly, and the no-allocation entry point returns the same bits as
    fdfb_bootstrap on a prime-modulus set."""
    torch = torch_cuda
    ps = S.Q_PARAM_SETS["FDFB-100-6"]
    kr = S.q_key_randomness(ps, 81)
    sid = ctx.register(ps)
    ctx.keys_generate(sid, kr)
    f = S.q_lut_tables(ps, 81, 1)[0]
    ctx.lut_setup(sid, f)
    batch = 64
    mr = S.q_message_randomness(ps, 82, batch)
    s_d = torch.tensor(kr.s.astype(np.uint8), device="cuda")
    ct = torch.empty((batch, ps.n + 1), dtype=torch.int64, device="cuda")
    ctx.lwe_encrypt(sid, s_d, F.to_device_words(ps, mr.a), torch.tensor(mr.e, device="cuda"),
                    torch.tensor(mr.m, device="cuda"), ct)
    ids = torch.zeros(batch, dtype=torch.int32, device="cuda")
    out = torch.empty_like(ct)
    ctx.bootstrap(sid, ct, ids, out)
    m_d = torch.empty(batch, dtype=torch.int32, device="cuda")
    ctx.lwe_decrypt(sid, s_d, out, m_d)
    ctx.sync()
    assert list(m_d.cpu().numpy()) == [int(f[m]) for m in mr.m]
    cap = ctx.noalloc_max_batch(sid)
    assert cap >= 1
    k = min(cap, 8)
    out2 = torch.empty_like(ct[:k])
    ctx.bootstrap_noalloc(sid, ct[:k].contiguous(), ids[:k].contiguous(), out2)
    ctx.sync()
    assert torch.equal(out2, out[:k])


def test_tfhe_100_7_full_size(F, torch_cuda, ctx, OQ):
    """Table 1's TFHE:100:7 (n = 1500, N = 4096, Q_3 = 2^48 - 163839, 16-bit
    blind-rotation digits, 48 key-switch digits): outputs decrypt to the
    negacyclic function."""
    torch = torch_cuda
    ps = S.Q_PARAM_SETS["TFHE-100-7"]
    kr = S.q_key_randomness(ps, 83)
    sid = ctx.register(ps)
    ctx.keys_generate(sid, kr)
    f_half = np.array([(5 * m + 2) % ps.t for m in range(ps.t // 2)])
    ctx.tfhe_poly_setup(sid, OQ.tfhe_test_polynomial(ps, f_half))
    batch = 64
    mr = S.q_message_randomness(ps, 84, batch)
    s_d = torch.tensor(kr.s.astype(np.uint8), device="cuda")
    ct = torch.empty((batch, ps.n + 1), dtype=torch.int64, device="cuda")
    ctx.lwe_encrypt(sid, s_d, F.to_device_words(ps, mr.a), torch.tensor(mr.e, device="cuda"),
                    torch.tensor(mr.m, device="cuda"), ct)
    out = torch.empty_like(ct)
    ctx.tfhe_bootstrap(sid, ct, torch.zeros(batch, dtype=torch.int32, device="cuda"), out)
    m_d = torch.empty(batch, dtype=torch.int32, device="cuda")
    ctx.lwe_decrypt(sid, s_d, out, m_d)
    ctx.sync()
    h = ps.t // 2
    want = [int(f_half[x]) if x < h else (-int(f_half[x - h])) % ps.t for x in mr.m]
    assert list(m_d.cpu().numpy()) == want


def test_fdfb_100_7_and_tfhe_100_2(F, torch_cuda, ctx, OQ):
    """The remaining Table 1 columns with N <= 4096: FDFB:100:7 (n = 1100,
    N = 4096, Q_2, 63 key-switch digits) decrypts to f(m); TFHE:100:2 (n =
    525, N = 1024, Q_4) decrypts to the negacyclic function."""
    torch = torch_cuda
    for name in ("FDFB-100-7", "TFHE-100-2"):
        ps = S.Q_PARAM_SETS[name]
        kr = S.q_key_randomness(ps, 85)
        sid = ctx.register(ps)
        ctx.keys_generate(sid, kr)
        batch = 32
        mr = S.q_message_randomness(ps, 86, batch)
        s_d = torch.tensor(kr.s.astype(np.uint8), device="cuda")
        ct = torch.empty((batch, ps.n + 1), dtype=torch.int64, device="cuda")
        ctx.lwe_encrypt(sid, s_d, F.to_device_words(ps, mr.a), torch.tensor(mr.e, device="cuda"),
                        torch.tensor(mr.m, device="cuda"), ct)
        ids = torch.zeros(batch, dtype=torch.int32, device="cuda")
        out = torch.empty_like(ct)
        if name.startswith("FDFB"):
            f = S.q_lut_tables(ps, 85, 1)[0]
            ctx.lut_setup(sid, f)
            ctx.bootstrap(sid, ct, ids, out)
            want = [int(f[m]) for m in mr.m]
        else:
            f_half = np.array([1, 2])
            ctx.tfhe_poly_setup(sid, OQ.tfhe_test_polynomial(ps, f_half))
            ctx.tfhe_bootstrap(sid, ct, ids, out)
            want = [int(f_half[x]) if x < 2 else (-int(f_half[x - 2])) % 4 for x in mr.m]
        m_d = torch.empty(batch, dtype=torch.int32, device="cuda")
        ctx.lwe_decrypt(sid, s_d, out, m_d)
        ctx.sync()
        assert list(m_d.cpu().numpy()) == want, name


class _Words:
    """Key material for the oracle given as words (no key generation)."""

    def __init__(self, bsk, pk, ksk):
        self.bsk, self.pk, self.ksk = bsk, pk, ksk


@pytest.mark.slow
@pytest.mark.parametrize("base,n,count", [("FDFB-80-6", 3, 2), ("FDFB-80-7", 3, 1)])
def test_full_geometry_matches_the_oracle(F, torch_cuda, ctx, OQ, base, n, count):
    """The paper's sets at their full ring degree and digit counts (N = 2048,
    l_g = 6 and N = 4096, l_g = 7 with its 14-row sums; l_pk = 5, l_boot = 6
    sign rotations), with n reduced to 3 so that the schoolbook oracle finishes
    in about a minute, and key words drawn uniformly mod Q (the algorithm is
    defined for any words; the outputs do not decrypt).  Every layout variant
    must give every intermediate (six sign LWEs, six packed RLWEs, PubMux, the
    function rotation, the key switch mod Q) and the output bit for bit as the
    oracle does."""
    ps = dataclasses.replace(S.Q_PARAM_SETS[base], name=f"{base}-n{n}", n=n)
    bsk, pk, ksk = S.q_uniform_key_words(ps, 31)
    sid = ctx.register(ps)
    ctx.keys_upload(sid, bsk, pk, ksk)
    tables = S.q_lut_tables(ps, 31, 2)
    assert [ctx.lut_setup(sid, f) for f in tables] == [0, 1]
    rot = OQ.rotation_polys(ps, tables)
    s = S.Stream(31, 7).bits(n)
    mr = S.q_message_randomness(ps, 32, count)
    cts = OQ.encrypt_messages(ps, s, mr)
    ids = np.arange(count, dtype=np.int32) % 2
    K = _Words(bsk, pk, ksk)
    refs = [OQ.fdfb_bootstrap(ps, K, rot[i][0], rot[i][1], c, debug=True) for c, i in zip(cts, ids)]
    cur, nvar, _ = ctx.variant_info(sid)
    for v in range(nvar):
        ctx.set_variant(sid, v)
        out, dbg = run_q(F, torch_cuda, ctx, sid, ps, cts, ids)
        for c, (o, d) in enumerate(refs):
            for key in ("sgn", "cR", "accF", "cQ", "cKS"):
                assert np.array_equal(dbg[key][c].reshape(d[key].shape), d[key]), f"{key}, variant {v}, ct {c}"
            assert np.array_equal(out[c], o), f"output, variant {v}, ct {c}"
    ctx.set_variant(sid, cur)
