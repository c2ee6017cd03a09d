"""GPU parity at ring degree N = 2^13, Table 1's FDFB:80:8 and FDFB:100:8
(the split transforms: one Cooley-Tukey stage plus two 4096-point halves),
against the prime-Q oracle on the same seeded inputs, bit for bit.

The schoolbook oracle needs about a minute per blind-rotation step of one
ciphertext at this degree (eight sign rotations and one function rotation,
fourteen products of 8192 x 8192 terms each), so the stage-by-stage checks
keep the full ring degree and digit counts but reduce n; the full-size set
is checked by decryption, by sampled key rows and by agreement between the
layout variants."""
from __future__ import annotations

import dataclasses

import numpy as np
import pytest

from paper_2109_02731_gb300 import synth as S

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

BASE = "FDFB-80-8"


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


class _Words:
    """Key material for the oracle given as words (no key generation)."""

    def __init__(self, bsk, pk, ksk):
        self.bsk, self.pk, self.ksk = bsk, pk, ksk


@pytest.fixture(scope="module")
def reduced(ctx):
    """FDFB-80-8's geometry (N = 8192, l_g = 7, l_pk = 5, l_boot = 8) with
    n = 2 and key words drawn uniformly mod Q: the arithmetic is defined for
    any words, the outputs do not decrypt."""
    ps = dataclasses.replace(S.Q_PARAM_SETS[BASE], name=f"{BASE}-n2", n=2)
    bsk, pk, ksk = S.q_uniform_key_words(ps, 61)
    sid = ctx.register(ps)
    ctx.keys_upload(sid, bsk, pk, ksk)
    return ps, sid, _Words(bsk, pk, ksk)


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


def test_registers_with_the_n13_variants(ctx, reduced):
    ps, sid, _ = reduced
    cur, count, _ = ctx.variant_info(sid)
    assert count == 3 and 0 <= cur < count


def test_full_geometry_matches_the_oracle(F, torch_cuda, ctx, OQ, reduced):
    """Every intermediate of one bootstrap -- eight sign LWEs, eight packed
    RLWEs, PubMux, the function rotation, the key switch mod Q -- and the
    output, for every layout variant, bit for bit equal to the oracle's."""
    ps, sid, K = reduced
    tables = S.q_lut_tables(ps, 62, 2)
    assert [ctx.lut_setup(sid, f) for f in tables] == [0, 1]
    rot = OQ.rotation_polys(ps, tables)
    s = S.Stream(62, 7).bits(ps.n)
    mr = S.q_message_randomness(ps, 63, 1)
    cts = OQ.encrypt_messages(ps, s, mr)
    ids = np.array([1], np.int32)
    assert all(int(a) != 0 for a in cts[0][1:]), "every blind-rotation step must rotate"
    o, d = OQ.fdfb_bootstrap(ps, K, rot[1][0], rot[1][1], cts[0], debug=True)
    cur, nvar, _ = ctx.variant_info(sid)
    for v in range(nvar):
        ctx.set_variant(sid, v)
        out, dbg = run_q(F, torch_cuda, ctx, sid, ps, cts, ids)
        for key in ("sgn", "cR", "accF", "cQ", "cKS"):
            assert np.array_equal(dbg[key][0].reshape(d[key].shape), d[key]), f"{key}, variant {v}"
        assert np.array_equal(out[0], o), f"output, variant {v}"
    ctx.set_variant(sid, cur)


def test_tfhe_bootstrap_matches_the_oracle(F, torch_cuda, ctx, OQ, reduced):
    """The TFHE bootstrap (one blind rotation, key switch, ModSwitch) at N =
    8192 on two ciphertexts with different pre-rotation polynomials, every
    layout, bit for bit equal to the oracle."""
    torch = torch_cuda
    ps, sid, K = reduced
    polys = S.q_tfhe_polynomials(ps, 64, 2)
    base = ctx.variant_info(sid)
    pids = [ctx.tfhe_poly_setup(sid, p) for p in polys]
    s = S.Stream(64, 7).bits(ps.n)
    mr = S.q_message_randomness(ps, 65, 2)
    cts = OQ.encrypt_messages(ps, s, mr)
    ids = np.array(pids, np.int32)
    ref = np.stack([OQ.tfhe_bootstrap(ps, K, polys[k], c) for k, c in enumerate(cts)])
    for v in range(base[1]):
        ctx.set_variant(sid, v)
        ct_d = F.to_device_words(ps, cts)
        out_d = torch.empty_like(ct_d)
        ctx.tfhe_bootstrap(sid, ct_d, torch.tensor(ids, device="cuda"), out_d)
        ctx.sync()
        assert np.array_equal(F.to_host_words(ps, out_d).astype(np.uint64), ref), f"variant {v}"
    ctx.set_variant(sid, base[0])


def test_no_allocation_entry_at_n13(F, torch_cuda, ctx, reduced):
    """fdfb_bootstrap_noalloc at N = 8192 (the blind rotation's per-item
    scratch carved from the fixed array too): its cap is 32 MiB over one
    input's intermediates, and at the cap it returns fdfb_bootstrap's bits on
    two calls in a row."""
    torch = torch_cuda
    ps, sid, _ = reduced
    N, n, lb = ps.N, ps.n, ps.lboot
    per_input = (lb * (7 * N + 1) + 3 * N + 1 + 2 * (n + 1)) * 8 + lb * (4 * 4 * 4096 + 4 * 8192) * 4
    cap = ctx.noalloc_max_batch(sid)
    assert cap == (32 << 20) // per_input
    lid = ctx.lut_setup(sid, (np.arange(ps.t) * 5 + 1) % ps.t)
    rng = np.random.default_rng(70)
    for call in range(2):
        cts = rng.integers(0, ps.q, (cap, n + 1), dtype=np.int64).astype(np.uint64)
        ids = torch.full((cap,), lid, dtype=torch.int32, device="cuda")
        ct_d = F.to_device_words(ps, cts)
        ref = torch.empty_like(ct_d)
        got = torch.empty_like(ct_d)
        ctx.bootstrap(sid, ct_d, ids, ref)
        ctx.bootstrap_noalloc(sid, ct_d, ids, got)
        ctx.sync()
        assert torch.equal(ref, got), f"call {call}"
    ct_d = torch.zeros((cap + 1, n + 1), dtype=torch.int64, device="cuda")
    with pytest.raises(F.FDFBError):
        ctx.bootstrap_noalloc(sid, ct_d, torch.full((cap + 1,), lid, dtype=torch.int32, device="cuda"),
                              torch.empty_like(ct_d))


def test_mixed_call_with_an_n13_group(F, torch_cuda, OQ, ctx, reduced):
    """fdfb_bootstrap_mixed with an N = 8192 group beside a small prime set
    (their pipelines run concurrently on the library's side streams, each in
    its own scratch): every group returns the bits of its own
    fdfb_bootstrap call."""
    torch = torch_cuda
    ps, sid, _ = reduced
    qz = S.Q_PARAM_SETS["QZ"]
    kr = S.q_key_randomness(qz, 81)
    K = OQ.QKeys(qz, kr)
    sq = ctx.register(qz)
    ctx.keys_upload(sq, K.bsk, K.pk, K.ksk)
    lq = ctx.lut_setup(sq, np.arange(qz.t)[::-1] % qz.t)
    l8 = ctx.lut_setup(sid, (np.arange(ps.t) * 3 + 2) % ps.t)
    rng = np.random.default_rng(82)
    groups, refs = [], []
    for s_id, pset, lid, count in ((sid, ps, l8, 3), (sq, qz, lq, 40)):
        cts = rng.integers(0, pset.q, (count, pset.n + 1), dtype=np.int64).astype(np.uint64)
        ct_d = F.to_device_words(pset, cts)
        ids = torch.full((count,), lid, dtype=torch.int32, device="cuda")
        ref = torch.empty_like(ct_d)
        ctx.bootstrap(s_id, ct_d, ids, ref)
        ctx.sync()
        refs.append(ref)
        groups.append((s_id, ct_d, ids, torch.empty_like(ct_d)))
    ctx.bootstrap_mixed(groups)
    ctx.sync()
    for (s_id, _, _, out), ref in zip(groups, refs):
        assert torch.equal(out, ref), f"set {s_id}"


def test_shared_memory_bounds_n(F, ctx):
    """At N = 8192 the accumulator stays in shared memory: n = 1536 registers,
    n = 1537 leaves no layout that fits and is refused."""
    ps = S.Q_PARAM_SETS[BASE]
    ctx.register(dataclasses.replace(ps, name="n1536", n=1536))
    with pytest.raises(F.FDFBError):
        ctx.register(dataclasses.replace(ps, name="n1537", n=1537))


def test_full_size_keygen_and_decryption(F, torch_cuda, ctx, OQ):
    """FDFB:80:8 at full size with keys generated on the GPU: sampled rows of
    the bootstrapping and packing keys equal the oracle's RLWE encryptions of
    the same randomness, every output decrypts to f(m), and the layout
    variants and the autotuned call return the same bits."""
    ps = S.Q_PARAM_SETS[BASE]
    kr = S.q_key_randomness(ps, 66)
    sid = ctx.register(ps)
    ctx.keys_generate(sid, kr)
    bsk, pk, _ = ctx.keys_download(sid)
    N, Q, lg = ps.N, ps.Q, ps.lg
    for i, r in ((0, 0), (ps.n - 1, 2 * lg - 1), (ps.n // 2, lg)):
        want = OQ.rlwe_encrypt(Q, kr.sk, kr.bsk_a[i][r], kr.bsk_e[i][r])
        if kr.s[i]:  # s_i B_g^j on coefficient 0 of component r // lg
            c, j = divmod(r, lg)
            want[c][0] = (int(want[c][0]) + pow(2, ps.log2Bg * j, Q)) % Q
        assert np.array_equal(bsk[i][r].astype(np.uint64), want), f"bsk row ({i}, {r})"
    for i, j in ((0, 0), (N - 1, ps.lpk - 1), (N // 3, 2)):
        mu = np.zeros(N, dtype=np.uint64)
        mu[0] = int(kr.sk[i]) * pow(2, ps.log2Bpk * j, Q) % Q  # s_F[i] B_pk^j
        want = OQ.rlwe_encrypt(Q, kr.sk, kr.pk_a[i][j], kr.pk_e[i][j], mu)
        assert np.array_equal(pk[i][j].astype(np.uint64), want), f"pK row ({i}, {j})"
    del bsk, pk
    tables = S.q_lut_tables(ps, 66, 3)
    for f in tables:
        ctx.lut_setup(sid, f)
    batch = 40
    mr = S.q_message_randomness(ps, 67, batch)
    cts = OQ.encrypt_messages(ps, kr.s, mr)
    ids = S.lut_assignment(67, batch, 3, "uniform")
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


def test_fdfb_100_8_full_size_decrypts(F, torch_cuda, ctx, OQ):
    """FDFB:100:8 at full size (n = 1100, l_ks = 63 binary key-switch digits,
    keys generated on the GPU): every output decrypts to f(m)."""
    ps = S.Q_PARAM_SETS["FDFB-100-8"]
    kr = S.q_key_randomness(ps, 68)
    sid = ctx.register(ps)
    ctx.keys_generate(sid, kr)
    tables = S.q_lut_tables(ps, 68, 2)
    for f in tables:
        ctx.lut_setup(sid, f)
    batch = 16
    mr = S.q_message_randomness(ps, 69, batch)
    cts = OQ.encrypt_messages(ps, kr.s, mr)
    ids = S.lut_assignment(69, batch, 2, "uniform")
    out, _ = run_q(F, torch_cuda, ctx, sid, ps, cts, ids, debug=False)
    dec = [OQ.decrypt(ps, kr.s, o) for o in out]
    assert dec == [int(tables[i][m]) for m, i in zip(mr.m, ids)]
