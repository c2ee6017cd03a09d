"""GPU parity: the CUDA library, called through its C ABI, against the CPU
oracle on the same seeded inputs.  Ciphertext arithmetic is exact integer
arithmetic mod 2^w, so every comparison is bit-exact (tolerance 0)."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2109_02731_gb300 import synth as S

from _fdfb_cases import fresh_cts, luts, oracle_keys

pytestmark = pytest.mark.gpu


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


_installed = {}


def install(ctx, oracle, name, seed, luts_count=1, group=0, generate=False):
    """Registers set `name`, installs the oracle's keys (or generates them on
    the GPU from the same randomness) and the lookup tables."""
    key = (id(ctx), name, seed, luts_count, group, generate)
    if key in _installed:
        return _installed[key]
    ps = S.PARAM_SETS[name]
    sid = ctx.register(ps)
    if generate:
        ctx.keys_generate(sid, S.key_randomness(ps, seed))
    else:
        K = oracle_keys(name, seed)
        ctx.keys_upload(sid, K.bsk, K.pk, K.ksk)
    fs, _ = luts(name, seed, luts_count, group)
    ids = [ctx.lut_setup(sid, f) for f in fs]
    assert ids == list(range(luts_count))
    _installed[key] = sid
    return sid


def run_gpu(F, torch, ctx, sid, ps, cts, lut_ids, debug=True):
    dev = "cuda"
    b = len(cts)
    ct_d = F.to_device_words(ps, cts)
    ids_d = torch.tensor(np.asarray(lut_ids, dtype=np.int32), device=dev)
    out_d = torch.empty_like(ct_d)
    wt = F.word_torch(ps)
    dbg = None
    if debug:
        dbg = dict(ctN=torch.empty((b, ps.n + 1), dtype=torch.int32, device=dev),
                   sgn=torch.empty((b, ps.N + 1), dtype=wt, device=dev),
                   cR=torch.empty((b, 2 * ps.N), dtype=wt, device=dev),
                   accF=torch.empty((b, 2 * ps.N), dtype=wt, device=dev),
                   cQ=torch.empty((b, ps.N + 1), dtype=wt, device=dev))
        ctx.bootstrap_debug(sid, ct_d, ids_d, out_d, dbg)
    else:
        ctx.bootstrap(sid, ct_d, ids_d, out_d)
    ctx.sync()
    out = F.to_host_words(ps, out_d).astype(np.uint64)
    if not debug:
        return out, None
    host = {k: (v.cpu().numpy().view(np.uint32) if k == "ctN" else F.to_host_words(ps, v)).astype(np.uint64)
            for k, v in dbg.items()}
    return out, host


def check_against_oracle(oracle, ps, K, rot, cts, lut_ids, out, dbg, idx):
    for c in idx:
        o, d = oracle.fdfb_bootstrap(ps, K, rot[lut_ids[c]][0], rot[lut_ids[c]][1], cts[c], debug=True)
        assert np.array_equal(dbg["ctN"][c], d["ctN"]), f"ModSwitch differs, ct {c}"
        assert np.array_equal(dbg["sgn"][c], d["sgn"]), f"sign LWE differs, ct {c}"
        assert np.array_equal(dbg["cR"][c], d["cR"]), f"packing key switch differs, ct {c}"
        assert np.array_equal(dbg["accF"][c], d["accF"]), f"PubMux differs, ct {c}"
        assert np.array_equal(dbg["cQ"][c], d["cQ"]), f"function rotation differs, ct {c}"
        assert np.array_equal(out[c], o), f"output differs, ct {c}"


# ------------------------------------------------------------------ keygen --

@pytest.mark.parametrize("name", ["Z", "A", "B"])
def test_keygen_parity_full(ctx, oracle, name):
    """GPU key generation (exact NTT products) equals the oracle's schoolbook
    keys word for word."""
    ps = S.PARAM_SETS[name]
    sid = ctx.register(ps)
    kr = S.key_randomness(ps, 11)
    ctx.keys_generate(sid, kr)
    bsk, pk, ksk = ctx.keys_download(sid)
    K = oracle.Keys(ps, kr)
    assert np.array_equal(bsk.astype(np.uint64), K.bsk)
    assert np.array_equal(pk.astype(np.uint64), K.pk)
    assert np.array_equal(ksk.astype(np.uint64), K.ksk)


@pytest.mark.parametrize("name", ["D", "C"])
def test_keygen_parity_sampled(ctx, oracle, name):
    """Full-size key generation on the GPU; sampled rows recomputed by the oracle."""
    ps = S.PARAM_SETS[name]
    sid = ctx.register(ps)
    kr = S.key_randomness(ps, 12)
    ctx.keys_generate(sid, kr)
    bsk, pk, ksk = ctx.keys_download(sid)
    rng = np.random.default_rng(0)
    for i, r in [(0, 0), (ps.n - 1, 2 * ps.lg - 1)] + [(int(rng.integers(ps.n)), int(rng.integers(2 * ps.lg)))
                                                      for _ in range(3)]:
        assert np.array_equal(bsk[i, r].astype(np.uint64), oracle.keygen_bsk_row(ps, kr, i, r)), (i, r)
    for i, j in [(0, 0), (ps.N - 1, ps.lpk - 1), (int(rng.integers(ps.N)), int(rng.integers(ps.lpk)))]:
        assert np.array_equal(pk[i, j].astype(np.uint64), oracle.keygen_pk_row(ps, kr, i, j)), (i, j)
    for i, j in [(0, 0), (ps.N - 1, ps.lks - 1), (7, 3)]:
        mu = int(kr.sk[i]) * oracle.gadget(ps.w, ps.log2Bks, ps.lks, j)
        ref = oracle.lwe_encrypt(ps.w, kr.s, kr.ksk_a[i, j], int(kr.ksk_e[i, j]), mu)
        assert np.array_equal(ksk[i, j].astype(np.uint64), ref)


# -------------------------------------------------------------- bootstrap --

def test_fdfb_noiseless_all_functions(F, torch_cuda, ctx, oracle):
    """Set Z (sigma = 0, exact gadgets): every m in Z_4 and a spread of the
    256 functions Z_4 -> Z_4; bit-exact with the oracle at every stage, and
    the output phase is exactly Delta f(m)."""
    import itertools
    ps = S.PARAM_SETS["Z"]
    K = oracle_keys("Z", 0)
    sid = ctx.register(ps)
    ctx.keys_upload(sid, K.bsk, K.pk, K.ksk)
    fs = np.array(list(itertools.product(range(4), repeat=4)))[::5]
    rot = np.stack([np.stack(oracle.setup_polynomial(ps.N, ps.t, f)) for f in fs])
    for f in fs:
        ctx.lut_setup(sid, f)
    ms = np.tile(np.arange(4), len(fs))
    ids = np.repeat(np.arange(len(fs)), 4).astype(np.int32)
    mr, cts = fresh_cts("Z", 0, len(ms), K, m=ms)
    out, dbg = run_gpu(F, torch_cuda, ctx, sid, ps, cts, ids)
    check_against_oracle(oracle, ps, K, rot, cts, ids, out, dbg, range(0, len(ms), 7))
    for c in range(len(ms)):
        assert oracle.lwe_phase(ps.w, K.s, out[c]) == oracle.delta(ps.w, ps.t) * int(fs[ids[c], ms[c]])


def test_lut_polys_match_oracle(ctx, oracle):
    """SetupPolynomial on the library side (host code of the C ABI) equals the
    oracle's, ties included."""
    for name in ("A", "B", "D"):
        ps = S.PARAM_SETS[name]
        sid = ctx.register(ps)
        fs = S.lut_tables(ps, 5, 3)
        for f in fs:
            lid = ctx.lut_setup(sid, f)
            p0, p1 = ctx.lut_polys(sid, lid)
            q0, q1 = oracle.setup_polynomial(ps.N, ps.t, f)
            assert np.array_equal(p0, q0) and np.array_equal(p1, q1)


def test_fdfb_toy_workload(F, torch_cuda, ctx, oracle):
    """The toy workload (set A, 16 ciphertexts, seed 0): all outputs and
    intermediates bit-exact, and every output decrypts to f(m)."""
    wl = S.WORKLOADS["toy"]
    g = wl.groups[0]
    ps = S.PARAM_SETS[g.set_name]
    K = oracle_keys(g.set_name, wl.seed)
    sid = install(ctx, oracle, g.set_name, wl.seed, g.n_luts)
    fs, rot = luts(g.set_name, wl.seed, g.n_luts)
    ids = S.lut_assignment(wl.seed, g.batch, g.n_luts, g.lut_assign)
    mr, cts = fresh_cts(g.set_name, wl.seed, g.batch, K)
    out, dbg = run_gpu(F, torch_cuda, ctx, sid, ps, cts, ids)
    check_against_oracle(oracle, ps, K, rot, cts, ids, out, dbg, range(g.batch))
    got = [oracle.lwe_decrypt(ps.w, ps.t, K.s, o) for o in out]
    assert got == [int(fs[i][m]) for i, m in zip(ids, mr.m)]


@pytest.mark.parametrize("batch", [1, 33, 37, 70])
def test_fdfb_ragged_batches(F, torch_cuda, ctx, oracle, batch):
    """Batches that leave partial tiles in the key-switching GEMM."""
    ps = S.PARAM_SETS["A"]
    K = oracle_keys("A", 3)
    sid = install(ctx, oracle, "A", 3, 3)
    fs, rot = luts("A", 3, 3)
    ids = (np.arange(batch) % 3).astype(np.int32)
    mr, cts = fresh_cts("A", 3, batch, K, group=batch)
    out, dbg = run_gpu(F, torch_cuda, ctx, sid, ps, cts, ids)
    check_against_oracle(oracle, ps, K, rot, cts, ids, out, dbg, sorted({0, batch // 2, batch - 1}))
    ref = oracle.fdfb_batch(ps, K, rot, ids, cts)
    assert np.array_equal(out, ref)


def test_fdfb_tfhe_scale_sampled(F, torch_cuda, ctx, oracle):
    """The TFHE-scale workload (set B) at its full size, 1024 ciphertexts in
    one call with four tables round robin; sampled ciphertexts recomputed by
    the oracle, all stages bit-exact."""
    wl = S.WORKLOADS["tfhe_scale"]
    g = wl.groups[0]
    ps = S.PARAM_SETS[g.set_name]
    K = oracle_keys(g.set_name, wl.seed)
    sid = install(ctx, oracle, g.set_name, wl.seed, g.n_luts)
    fs, rot = luts(g.set_name, wl.seed, g.n_luts)
    ids = S.lut_assignment(wl.seed, g.batch, g.n_luts, g.lut_assign)
    mr, cts = fresh_cts(g.set_name, wl.seed, g.batch, K)
    # the launch configuration the benchmark times: the autotuned layout
    ctx.autotune(sid, g.batch)
    out, dbg = run_gpu(F, torch_cuda, ctx, sid, ps, cts, ids)
    check_against_oracle(oracle, ps, K, rot, cts, ids, out, dbg, [0, 1, 2, 3, 517, g.batch - 1])


def _big_workload(F, torch_cuda, ctx, oracle, name, batch, n_luts, seed, sample):
    ps = S.PARAM_SETS[name]
    K = oracle_keys(name, seed)
    sid = install(ctx, oracle, name, seed, n_luts)
    fs, rot = luts(name, seed, n_luts)
    ids = S.lut_assignment(seed, batch, n_luts, "uniform")
    mr, cts = fresh_cts(name, seed, batch, K)
    # the configuration the benchmark times: autotuned layout and chunk count
    ctx.autotune(sid, batch)
    out_dbg, dbg = run_gpu(F, torch_cuda, ctx, sid, ps, cts, ids)
    check_against_oracle(oracle, ps, K, rot, cts, ids, out_dbg, dbg, sample)
    out, _ = run_gpu(F, torch_cuda, ctx, sid, ps, cts, ids, debug=False)
    assert np.array_equal(out, out_dbg)
    # every output decrypts to f(m): decryption on the GPU, checked on the host
    dev_s = torch_cuda.tensor(K.s, device="cuda")
    out_d = F.to_device_words(ps, out)
    m_d = torch_cuda.empty(batch, dtype=torch_cuda.int32, device="cuda")
    ctx.lwe_decrypt(sid, dev_s, out_d, m_d)
    ctx.sync()
    got = m_d.cpu().numpy()
    want = np.array([fs[i][m] for i, m in zip(ids, mr.m)])
    assert np.array_equal(got, want), f"{int((got != want).sum())} wrong decryptions"


@pytest.mark.slow
def test_fdfb_set_D_full_batch(F, torch_cuda, ctx, oracle):
    """Set D (N = 2048, q = 2^64, t = 32) at the mixed workload's batch of
    1000, in the autotuned layout and chunking the benchmark times: sampled
    bit-exact parity of every stage, chunked call = single pipeline, every
    output decrypts correctly."""
    # eight ciphertexts: both ends, across the seven waves of 152 CTAs, every table
    _big_workload(F, torch_cuda, ctx, oracle, "D", 1000, 4, 3, [0, 151, 152, 333, 500, 761, 998, 999])


@pytest.mark.slow
def test_fdfb_large_t_full_batch(F, torch_cuda, ctx, oracle):
    """The large-plaintext workload (set C, N = 4096, t = 64) at its full
    4096 ciphertexts and 16 tables: one ciphertext recomputed by the oracle,
    every output decrypts correctly."""
    wl = S.WORKLOADS["large_t"]
    g = wl.groups[0]
    # four ciphertexts: first, last and two from inner waves
    _big_workload(F, torch_cuda, ctx, oracle, "C", g.batch, g.n_luts, wl.seed, [0, 1517, 3040, g.batch - 1])


def test_keygen_then_bootstrap_matches_upload(F, torch_cuda, ctx, oracle):
    """Keys generated on the GPU give the same bootstrap as the oracle's keys."""
    ps = S.PARAM_SETS["A"]
    K = oracle_keys("A", 4)
    sid_u = install(ctx, oracle, "A", 4, 2)
    sid_g = install(ctx, oracle, "A", 4, 2, generate=True)
    ids = np.array([0, 1, 1, 0, 1], np.int32)
    mr, cts = fresh_cts("A", 4, len(ids), K)
    out_u, _ = run_gpu(F, torch_cuda, ctx, sid_u, ps, cts, ids, debug=False)
    out_g, _ = run_gpu(F, torch_cuda, ctx, sid_g, ps, cts, ids, debug=False)
    assert np.array_equal(out_u, out_g)


# ------------------------------------------------------ other entry points --

@pytest.mark.parametrize("name", ["A", "D"])
def test_keyswitch_entry(F, torch_cuda, ctx, oracle, name):
    ps = S.PARAM_SETS[name]
    K = oracle_keys(name, 5)
    sid = install(ctx, oracle, name, 5, 1)
    rng = np.random.default_rng(1)
    cts = rng.integers(0, 1 << 62, size=(45, ps.N + 1), dtype=np.uint64) * np.uint64(4) + \
        rng.integers(0, 4, size=(45, ps.N + 1), dtype=np.uint64)
    cts &= np.uint64((1 << ps.w) - 1)
    ci = F.to_device_words(ps, cts)
    co = torch_cuda.empty((45, ps.n + 1), dtype=F.word_torch(ps), device="cuda")
    ctx.keyswitch(sid, ci, co)
    ctx.sync()
    got = F.to_host_words(ps, co).astype(np.uint64)
    for c in range(45):
        assert np.array_equal(got[c], oracle.keyswitch(ps.w, ps.log2Bks, ps.lks, K.ksk, cts[c]))


@pytest.mark.parametrize("name", ["B", "D"])
def test_lwe_encrypt_decrypt_entries(F, torch_cuda, ctx, oracle, name):
    ps = S.PARAM_SETS[name]
    sid = ctx.register(ps)
    s = S.key_randomness(ps, 6).s
    mr = S.message_randomness(ps, 6, 300)
    d = "cuda"
    ct = torch_cuda.empty((300, ps.n + 1), dtype=F.word_torch(ps), device=d)
    ctx.lwe_encrypt(sid, torch_cuda.tensor(s, device=d), F.to_device_words(ps, mr.a),
                    torch_cuda.tensor(mr.e, device=d), torch_cuda.tensor(mr.m, device=d), ct)
    m = torch_cuda.empty(300, dtype=torch_cuda.int32, device=d)
    ctx.lwe_decrypt(sid, torch_cuda.tensor(s, device=d), ct, m)
    ctx.sync()
    ref = oracle.encrypt_messages(ps, s, mr)
    assert np.array_equal(F.to_host_words(ps, ct).astype(np.uint64), ref)
    assert np.array_equal(m.cpu().numpy(), [oracle.lwe_decrypt(ps.w, ps.t, s, r) for r in ref])


def test_lwe_affine_entry(F, torch_cuda, ctx, oracle):
    ps = S.PARAM_SETS["D"]
    sid = ctx.register(ps)
    rng = np.random.default_rng(2)
    batch, n_in, n_out = 3, 70, 11
    W = rng.integers(-8, 8, size=(n_out, n_in)).astype(np.int32)
    x = rng.integers(0, 1 << 63, size=(batch, n_in, ps.n + 1), dtype=np.uint64)
    y = torch_cuda.empty((batch, n_out, ps.n + 1), dtype=torch_cuda.int64, device="cuda")
    ctx.lwe_affine(sid, torch_cuda.tensor(W, device="cuda"), F.to_device_words(ps, x), y)
    ctx.sync()
    got = F.to_host_words(ps, y)
    for b in range(batch):
        assert np.array_equal(got[b], oracle.lwe_affine(ps.w, W, x[b]))


def test_errors_and_edge_cases(F, torch_cuda, ctx, oracle):
    ps = S.PARAM_SETS["A"]
    K = oracle_keys("A", 0)
    sid = install(ctx, oracle, "A", 0, 1)
    d = "cuda"
    ct = torch_cuda.zeros((2, ps.n + 1), dtype=torch_cuda.int32, device=d)
    out = torch_cuda.zeros_like(ct)
    # empty batch is a no-op
    ctx.bootstrap(sid, ct[:0], torch_cuda.zeros(0, dtype=torch_cuda.int32, device=d), out[:0])
    ctx.sync()
    # unknown table id is latched and reported by fdfb_sync
    ctx.bootstrap(sid, ct, torch_cuda.tensor([0, 7], dtype=torch_cuda.int32, device=d), out)
    with pytest.raises(F.FDFBError) as e:
        ctx.sync()
    assert e.value.code == -6
    ctx.sync()  # latch cleared
    # an impossible scratch allocation (2^30 ciphertexts: terabytes) fails with
    # FDFB_ENOMEM before any launch, and the context keeps working
    ids1 = torch_cuda.zeros(2, dtype=torch_cuda.int32, device=d)
    with pytest.raises(F.FDFBError) as e:
        ctx.bootstrap(sid, ct, ids1, out, batch=1 << 30)
    assert e.value.code == -2
    ctx.sync()
    ctx.bootstrap(sid, ct, ids1, out)
    ctx.sync()
    # keys missing
    sid2 = ctx.register(ps)
    ctx.lut_setup(sid2, [0, 1, 2, 3])
    with pytest.raises(F.FDFBError) as e:
        ctx.bootstrap(sid2, ct, torch_cuda.zeros(2, dtype=torch_cuda.int32, device=d), out)
    assert e.value.code == -5
    # bad table entry, unsupported parameters
    with pytest.raises(F.FDFBError):
        ctx.lut_setup(sid, [0, 1, 2, 4])
    import dataclasses
    with pytest.raises(F.FDFBError):
        ctx.register(dataclasses.replace(ps, N=128))
    with pytest.raises(F.FDFBError):
        ctx.register(dataclasses.replace(ps, lg=5))


# ------------------------------------------------------------ mixed groups --

def test_mixed_groups_match_separate_calls(F, torch_cuda, ctx, oracle):
    """Three parameter sets (and a repeated set) in one fdfb_bootstrap_mixed
    call give exactly the outputs of separate fdfb_bootstrap calls; the q = 2^64
    groups decrypt to f(m)."""
    spec = [("B", 1, 4, 37), ("D", 3, 4, 64), ("C", 2, 16, 12), ("B", 1, 4, 5)]
    groups, refs, checks = [], [], []
    for gi, (name, seed, nl, batch) in enumerate(spec):
        ps = S.PARAM_SETS[name]
        K = oracle_keys(name, seed)
        sid = install(ctx, oracle, name, seed, nl)
        fs, _ = luts(name, seed, nl)
        ids = S.lut_assignment(seed, batch, nl, "uniform", group=10 + gi)
        mr, cts = fresh_cts(name, seed, batch, K, group=10 + gi)
        ref, _ = run_gpu(F, torch_cuda, ctx, sid, ps, cts, ids, debug=False)
        ct_d = F.to_device_words(ps, cts)
        out_d = torch_cuda.empty_like(ct_d)
        groups.append((sid, ct_d, torch_cuda.tensor(ids, device="cuda"), out_d))
        refs.append(ref)
        checks.append((ps, K, fs, ids, mr))
    ctx.bootstrap_mixed(groups)
    ctx.sync()
    for (sid, _, _, out_d), ref, (ps, K, fs, ids, mr) in zip(groups, refs, checks):
        got = F.to_host_words(ps, out_d).astype(np.uint64)
        assert np.array_equal(got, ref), ps.name
        if ps.w == 64:
            dec = [oracle.lwe_decrypt(ps.w, ps.t, K.s, c) for c in got]
            assert dec == [int(fs[i][m]) for i, m in zip(ids, mr.m)]


@pytest.mark.slow
def test_mixed_workload_full_size_matches_oracle(F, torch_cuda, ctx, oracle):
    """The mixed workload's shape in one fdfb_bootstrap_mixed call: set B x 37,
    set D x 1000 and set C x 2900 with uniform table choices, each set's
    autotuned layout and chunking as the benchmark uses them.  Sampled
    outputs of every group equal the oracle's bit for bit, and every output of
    the q = 2^64 groups decrypts to f(m)."""
    spec = [("B", 1, 4, 37, [0, 18, 36]), ("D", 3, 4, 1000, [7, 999]), ("C", 2, 16, 2900, [0, 2899])]
    groups, checks = [], []
    for gi, (name, seed, nl, batch, sample) in enumerate(spec):
        ps = S.PARAM_SETS[name]
        K = oracle_keys(name, seed)
        sid = install(ctx, oracle, name, seed, nl)
        ctx.autotune(sid, batch)
        fs, rot = luts(name, seed, nl)
        ids = S.lut_assignment(seed, batch, nl, "uniform", group=30 + gi)
        mr, cts = fresh_cts(name, seed, batch, K, group=30 + gi)
        ct_d = F.to_device_words(ps, cts)
        out_d = torch_cuda.empty_like(ct_d)
        groups.append((sid, ct_d, torch_cuda.tensor(ids, device="cuda"), out_d))
        checks.append((ps, K, fs, rot, ids, mr, cts, sample))
    ctx.bootstrap_mixed(groups)
    ctx.sync()
    for (sid, _, _, out_d), (ps, K, fs, rot, ids, mr, cts, sample) in zip(groups, checks):
        got = F.to_host_words(ps, out_d).astype(np.uint64)
        for c in sample:
            ref = oracle.fdfb_bootstrap(ps, K, rot[ids[c]][0], rot[ids[c]][1], cts[c])
            assert np.array_equal(got[c], ref), f"set {ps.name}, ct {c}"
        if ps.w == 64:
            dev_s = torch_cuda.tensor(K.s, device="cuda")
            m_d = torch_cuda.empty(len(cts), dtype=torch_cuda.int32, device="cuda")
            ctx.lwe_decrypt(sid, dev_s, out_d, m_d)
            ctx.sync()
            want = np.array([fs[i][m] for i, m in zip(ids, mr.m)])
            assert np.array_equal(m_d.cpu().numpy(), want), ps.name


# ------------------------------------------------------------- MLP layers --

def test_mlp_small_network_matches_oracle(F, torch_cuda, ctx, oracle):
    """A small dense network (set A, t = 4) on the GPU -- affine launch, then
    one batched bootstrap per layer -- against the oracle doing the same
    affine maps and bootstraps, bit for bit, and against the plaintext
    network mod t."""
    from paper_2109_02731_gb300 import mlp
    ps = S.PARAM_SETS["A"]
    K = oracle_keys("A", 7)
    sid = ctx.register(ps)
    ctx.keys_upload(sid, K.bsk, K.pk, K.ksk)
    rng = np.random.default_rng(5)
    layers = [9, 6, 3]
    Ws = [rng.integers(-1, 2, size=(layers[i + 1], layers[i])) for i in range(len(layers) - 1)]
    net = mlp.EncryptedMLP(ctx, sid, Ws)
    n_inputs = 2
    xs = rng.integers(0, ps.t, size=(n_inputs, layers[0]))
    mr = S.message_randomness(ps, 7, n_inputs * layers[0], m=xs.reshape(-1))
    cts = oracle.encrypt_messages(ps, K.s, mr).reshape(n_inputs, layers[0], ps.n + 1)
    out = F.to_host_words(ps, net.forward(F.to_device_words(ps, cts))).astype(np.uint64)
    ctx.sync()
    rot = {lid: np.stack(oracle.setup_polynomial(ps.N, ps.t, f))
           for lid, f in ((net.relu_id, mlp.relu_table(ps.t)), (net.sign_id, mlp.sign_table(ps.t)))}
    h = cts
    for li, W in enumerate(Ws):
        lid = net.sign_id if li == len(Ws) - 1 else net.relu_id
        y = np.stack([oracle.lwe_affine(ps.w, W, h[b]) for b in range(n_inputs)])
        h = np.stack([[oracle.fdfb_bootstrap(ps, K, rot[lid][0], rot[lid][1], y[b, j])
                       for j in range(W.shape[0])] for b in range(n_inputs)])
    assert np.array_equal(out, h)
    dec = np.array([[oracle.lwe_decrypt(ps.w, ps.t, K.s, c) for c in row] for row in out])
    assert np.array_equal(dec, mlp.plain_forward(xs, Ws, ps.t))


@pytest.mark.slow
def test_mlp_workload_full_size_decrypts(F, torch_cuda, ctx, oracle):
    """The MLP workload at full size (set D, 784 -> 128 -> 64 -> 10, 64 inputs,
    weights in [-8, 7], pixels in Z_16): every output decrypts to the
    plaintext network's value mod t."""
    from paper_2109_02731_gb300 import mlp
    wl = S.WORKLOADS["mlp"]
    ps = S.PARAM_SETS["D"]
    sid = ctx.register(ps)
    kr = S.key_randomness(ps, wl.seed)
    ctx.keys_generate(sid, kr)
    x, Ws = S.mlp_inputs_and_weights(wl.seed, wl.mlp_layers, wl.mlp_inputs)
    net = mlp.EncryptedMLP(ctx, sid, Ws)
    ctx.autotune(sid, wl.mlp_inputs * wl.mlp_layers[1])  # as the benchmark does
    mr = S.message_randomness(ps, wl.seed, x.size, m=x.reshape(-1))
    d = "cuda"
    ct = torch_cuda.empty((x.size, ps.n + 1), dtype=torch_cuda.int64, device=d)
    ctx.lwe_encrypt(sid, torch_cuda.tensor(kr.s, device=d), F.to_device_words(ps, mr.a),
                    torch_cuda.tensor(mr.e, device=d), torch_cuda.tensor(mr.m, device=d), ct)
    out = net.forward(ct.view(x.shape[0], x.shape[1], ps.n + 1))
    m = torch_cuda.empty(out.shape[0] * out.shape[1], dtype=torch_cuda.int32, device=d)
    ctx.lwe_decrypt(sid, torch_cuda.tensor(kr.s, device=d), out.reshape(-1, ps.n + 1), m)
    ctx.sync()
    got = m.cpu().numpy().reshape(out.shape[0], out.shape[1])
    assert np.array_equal(got, mlp.plain_forward(x, Ws, ps.t))


# ------------------------------------------------------------ multi-table --

def run_gpu_multi(F, torch, ctx, sid, ps, cts, ids2):
    ct_d = F.to_device_words(ps, cts)
    ids_d = torch.tensor(np.ascontiguousarray(ids2, dtype=np.int32), device="cuda")
    out_d = torch.empty((len(cts), ids2.shape[1], ps.n + 1), dtype=ct_d.dtype, device="cuda")
    ctx.bootstrap_multi(sid, ct_d, ids_d, out_d)
    ctx.sync()
    return F.to_host_words(ps, out_d).astype(np.uint64)


def test_multi_table_toy_matches_oracle(F, torch_cuda, ctx, oracle):
    """Several tables per input (one sign rotation shared by k function
    rotations): every (input, table) output equals the oracle's multi-table
    bootstrap bit for bit (set A, 13 inputs x 3 tables)."""
    ps = S.PARAM_SETS["A"]
    K = oracle_keys("A", 0)
    sid = install(ctx, oracle, "A", 0, 4)
    fs, rot = luts("A", 0, 4)
    rng = np.random.default_rng(5)
    ids = rng.integers(0, 4, size=(13, 3)).astype(np.int32)
    mr, cts = fresh_cts("A", 0, 13, K, group=7)
    got = run_gpu_multi(F, torch_cuda, ctx, sid, ps, cts, ids)
    want = oracle.fdfb_batch_multi(ps, K, rot, ids, cts)
    assert np.array_equal(got, want)
    dec = [[oracle.lwe_decrypt(ps.w, ps.t, K.s, o) for o in row] for row in got]
    assert dec == [[int(fs[i][m]) for i in row] for row, m in zip(ids, mr.m)]


def test_multi_table_tfhe_scale(F, torch_cuda, ctx, oracle):
    """Set B, 256 inputs x 4 tables in one call, in the autotuned layout:
    every output equals the single-table bootstrap of its (input, table) on
    the GPU, and sampled inputs equal the oracle's multi-table bootstrap."""
    wl = S.WORKLOADS["tfhe_scale"]
    g = wl.groups[0]
    ps = S.PARAM_SETS[g.set_name]
    K = oracle_keys(g.set_name, wl.seed)
    sid = install(ctx, oracle, g.set_name, wl.seed, g.n_luts)
    fs, rot = luts(g.set_name, wl.seed, g.n_luts)
    ids = np.tile(np.arange(4, dtype=np.int32), (256, 1))
    ids[1::2] = ids[1::2, ::-1]
    mr, cts = fresh_cts(g.set_name, wl.seed, 256, K, group=3)
    ctx.autotune(sid, 1024)
    got = run_gpu_multi(F, torch_cuda, ctx, sid, ps, cts, ids)
    single, _ = run_gpu(F, torch_cuda, ctx, sid, ps, np.repeat(cts, 4, axis=0), ids.reshape(-1),
                        debug=False)
    assert np.array_equal(got.reshape(-1, ps.n + 1), single)
    for c in (0, 1, 255):
        assert np.array_equal(got[c], oracle.fdfb_bootstrap_multi(ps, K, rot[ids[c]], cts[c])), c


def test_multi_table_edge_cases(F, torch_cuda, ctx, oracle):
    """k = 1 is the single-table bootstrap; batch 0 is a no-op; k = 0 and a
    table id out of range are rejected."""
    ps = S.PARAM_SETS["A"]
    K = oracle_keys("A", 0)
    sid = install(ctx, oracle, "A", 0, 4)
    mr, cts = fresh_cts("A", 0, 5, K, group=8)
    ids = np.array([[0], [1], [2], [3], [0]], dtype=np.int32)
    got = run_gpu_multi(F, torch_cuda, ctx, sid, ps, cts, ids)
    single, _ = run_gpu(F, torch_cuda, ctx, sid, ps, cts, ids[:, 0], debug=False)
    assert np.array_equal(got[:, 0], single)
    ct_d = F.to_device_words(ps, cts)
    empty_ids = torch_cuda.empty((0, 2), dtype=torch_cuda.int32, device="cuda")
    empty_out = torch_cuda.empty((0, 2, ps.n + 1), dtype=ct_d.dtype, device="cuda")
    ctx.bootstrap_multi(sid, ct_d[:0], empty_ids, empty_out)
    zero_k = torch_cuda.empty((5, 0), dtype=torch_cuda.int32, device="cuda")
    with pytest.raises(F.FDFBError) as e:
        ctx.bootstrap_multi(sid, ct_d, zero_k, empty_out)
    assert e.value.code == -1
    bad = torch_cuda.tensor([[0, 9]] * 5, dtype=torch_cuda.int32, device="cuda")
    out_d = torch_cuda.empty((5, 2, ps.n + 1), dtype=ct_d.dtype, device="cuda")
    ctx.bootstrap_multi(sid, ct_d, bad, out_d)
    with pytest.raises(F.FDFBError) as e:
        ctx.sync()
    assert e.value.code == -6


# ---------------------------------------------------- layout variants -----

@pytest.mark.parametrize("name,seed,nl,batch", [("A", 0, 2, 50), ("B", 1, 4, 70), ("D", 3, 4, 40),
                                                ("C", 2, 16, 9)])
def test_every_variant_is_bit_exact(F, torch_cuda, ctx, oracle, name, seed, nl, batch):
    """Every register-layout variant of the blind rotation, and the one the
    autotuner picks, produce identical ciphertexts (and variant 0 is checked
    against the oracle on one ciphertext)."""
    ps = S.PARAM_SETS[name]
    K = oracle_keys(name, seed)
    sid = install(ctx, oracle, name, seed, nl)
    fs, rot = luts(name, seed, nl)
    ids = S.lut_assignment(seed, batch, nl, "uniform", group=20)
    mr, cts = fresh_cts(name, seed, batch, K, group=20)
    cur, count, _ = ctx.variant_info(sid)
    outs = []
    for v in range(count):
        ctx.set_variant(sid, v)
        out, _ = run_gpu(F, torch_cuda, ctx, sid, ps, cts, ids, debug=False)
        outs.append(out)
    for v in range(1, count):
        assert np.array_equal(outs[v], outs[0]), f"variant {v}"
    ref = oracle.fdfb_bootstrap(ps, K, rot[ids[0]][0], rot[ids[0]][1], cts[0])
    assert np.array_equal(outs[0][0], ref)
    best, ms = ctx.autotune(sid, 64)
    assert 0 <= best < count and ms > 0
    assert ctx.variant_info(sid)[0] == best
    out, _ = run_gpu(F, torch_cuda, ctx, sid, ps, cts, ids, debug=False)
    assert np.array_equal(out, outs[0])
    ctx.set_variant(sid, cur)


def test_lazy_family_only_where_exact(F, torch_cuda, ctx):
    """Variants on the lazy (28-bit) prime family are offered only for sets
    whose blind-rotation products they lift exactly.  At N = 1024, q = 2^32
    there are eight variants: 0-4 on the 30-bit primes (1 and 3 with 8-bit
    digits) and 5-7 on the lazy family (6 with 8-bit digits).  Set B
    (product bound 2^50.6) gets all eight; a set with B_g = 2^11, l_g = 2
    (bound 2^54.0: above the lazy family's 2^53.7, within the 30-bit primes'
    2^59) keeps only the 16-bit-digit variants 0, 2 and 4."""
    import dataclasses
    ps = S.PARAM_SETS["B"]
    wide = dataclasses.replace(ps, name="Bwide", log2Bg=11, lg=2)
    assert ctx.variant_info(ctx.register(ps))[1] == 8
    assert ctx.variant_info(ctx.register(wide))[1] == 3


def test_degenerate_tables_and_t2(F, torch_cuda, ctx, oracle):
    """Degenerate cases: plaintext modulus t = 2, constant and identity tables,
    and a table equal to its negacyclic extension; bit-exact with the oracle
    and exact output phases (noiseless keys, exact gadgets)."""
    import dataclasses
    ps = dataclasses.replace(S.PARAM_SETS["Z"], name="Z2", t=2)
    kr = S.key_randomness(ps, 9)
    K = oracle.Keys(ps, kr)
    sid = ctx.register(ps)
    ctx.keys_upload(sid, K.bsk, K.pk, K.ksk)
    tables = [[0, 0], [1, 1], [0, 1], [1, 0]]
    for f in tables:
        ctx.lut_setup(sid, f)
    rot = np.stack([np.stack(oracle.setup_polynomial(ps.N, ps.t, f)) for f in tables])
    ms = np.tile([0, 1], 8)
    ids = np.repeat(np.arange(4), 4).astype(np.int32)
    mr = S.message_randomness(ps, 9, len(ms), m=ms)
    cts = oracle.encrypt_messages(ps, K.s, mr)
    out, dbg = run_gpu(F, torch_cuda, ctx, sid, ps, cts, ids)
    check_against_oracle(oracle, ps, K, rot, cts, ids, out, dbg, range(len(ms)))
    for c in range(len(ms)):
        assert oracle.lwe_phase(ps.w, K.s, out[c]) == oracle.delta(ps.w, ps.t) * tables[ids[c]][ms[c]]


def test_bootstrap_captured_in_cuda_graph(F, torch_cuda, ctx, oracle):
    """The mixed bootstrap (forked side streams, joined with events) captures
    into a CUDA graph once scratch exists; replaying it reproduces the
    direct call bit for bit."""
    torch = torch_cuda
    spec = [("A", 3, 3, 20), ("B", 1, 4, 33)]
    groups, refs = [], []
    for gi, (name, seed, nl, batch) in enumerate(spec):
        ps = S.PARAM_SETS[name]
        K = oracle_keys(name, seed)
        sid = install(ctx, oracle, name, seed, nl)
        ids = S.lut_assignment(seed, batch, nl, "uniform", group=30 + gi)
        mr, cts = fresh_cts(name, seed, batch, K, group=30 + gi)
        ref, _ = run_gpu(F, torch, ctx, sid, ps, cts, ids, debug=False)
        groups.append((sid, F.to_device_words(ps, cts), torch.tensor(ids, device="cuda"), None))
        refs.append((ps, ref))
    groups = [(sid, ci, ids, torch.full_like(ci, -1)) for sid, ci, ids, _ in groups]
    ctx.bootstrap_mixed(groups)          # grows scratch and side streams before capture
    ctx.sync()
    for _, _, _, out in groups:
        out.fill_(-1)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            ctx.bootstrap_mixed(groups)
    g.replay()
    torch.cuda.synchronize()
    for (ps, ref), (_, _, _, out) in zip(refs, groups):
        assert np.array_equal(F.to_host_words(ps, out).astype(np.uint64), ref)


def test_chunked_calls_are_bit_exact(F, torch_cuda, ctx, oracle):
    """fdfb_bootstrap and fdfb_bootstrap_multi split a batch into 1-8 slices
    on side streams: every chunk count returns the same ciphertexts (set B, 300
    inputs, and 50 inputs x 3 tables); the union of the blind-rotation launch
    intervals is at most the sum of their durations; a chunked call replays
    from a CUDA graph bit for bit."""
    torch = torch_cuda
    ps = S.PARAM_SETS["B"]
    K = oracle_keys("B", 1)
    sid = install(ctx, oracle, "B", 1, 4)
    fs, rot = luts("B", 1, 4)
    ids = S.lut_assignment(1, 300, 4, "uniform", group=40)
    mr, cts = fresh_cts("B", 1, 300, K, group=40)
    saved = ctx.get_chunks(sid)
    outs = []
    for c in (1, 2, 3, 4, 8):
        ctx.set_chunks(sid, c)
        assert ctx.get_chunks(sid) == c
        out, _ = run_gpu(F, torch, ctx, sid, ps, cts, ids, debug=False)
        outs.append(out)
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    assert np.array_equal(outs[0][7], oracle.fdfb_bootstrap(ps, K, rot[ids[7]][0], rot[ids[7]][1], cts[7]))
    ids2 = np.random.default_rng(9).integers(0, 4, size=(50, 3)).astype(np.int32)
    ctx.set_chunks(sid, 3)
    m3 = run_gpu_multi(F, torch, ctx, sid, ps, cts[:50], ids2)
    ctx.set_chunks(sid, 1)
    m1 = run_gpu_multi(F, torch, ctx, sid, ps, cts[:50], ids2)
    assert np.array_equal(m3, m1)
    # measurement hook: stage 5 is the union of the rotations' intervals
    ctx.set_chunks(sid, 3)
    ctx.profile_enable(True)
    run_gpu(F, torch, ctx, sid, ps, cts, ids, debug=False)
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    total = prof["blind_rotate_sign"][0] + prof["blind_rotate_func"][0]
    assert prof["blind_rotate_sign"][1] == 3 and prof["blind_rotate_func"][1] == 3
    assert prof["blind_rotate_union"][1] == 6
    assert 0 < prof["blind_rotate_union"][0] <= total + 1e-3
    # graph capture of a chunked call (side streams exist from the calls above)
    ctx.set_chunks(sid, 2)
    ct_d = F.to_device_words(ps, cts)
    ids_d = torch.tensor(ids, device="cuda")
    out_d = torch.full_like(ct_d, -1)
    g = torch.cuda.CUDAGraph()
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        with torch.cuda.graph(g, stream=st):
            ctx.bootstrap(sid, ct_d, ids_d, out_d)
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(F.to_host_words(ps, out_d).astype(np.uint64), outs[0])
    with pytest.raises(F.FDFBError):
        ctx.set_chunks(sid, 0)
    with pytest.raises(F.FDFBError):
        ctx.set_chunks(sid, 9)
    ctx.set_chunks(sid, saved)


# ---------------------------------------------------------- TFHE bootstrap --

def test_tfhe_bootstrap_matches_oracle(F, torch_cuda, ctx, oracle):
    """TFHE bootstrap (one blind rotation of a pre-rotation polynomial): set A
    (20 ciphertexts, two polynomials) and set B (sampled from 300, autotuned
    layout) bit for bit against the oracle; set A decrypts to the negacyclic
    function."""
    torch = torch_cuda
    for name, seed, batch, sample in (("A", 0, 20, range(20)), ("B", 1, 300, (0, 1, 299))):
        ps = S.PARAM_SETS[name]
        K = oracle_keys(name, seed)
        sid = install(ctx, oracle, name, seed, 1)
        rng = np.random.default_rng(31)
        f_halves = [rng.integers(0, ps.t, size=ps.t // 2) for _ in range(2)]
        polys = np.stack([oracle.tfhe_test_polynomial(ps, f) for f in f_halves])
        pids = [ctx.tfhe_poly_setup(sid, p) for p in polys]
        ids = rng.integers(0, 2, size=batch).astype(np.int32)
        mr, cts = fresh_cts(name, seed, batch, K, group=50)
        if name == "B":
            ctx.autotune(sid, batch)
        ct_d = F.to_device_words(ps, cts)
        out_d = torch.empty_like(ct_d)
        ctx.tfhe_bootstrap(sid, ct_d, torch.tensor(np.asarray(pids)[ids], dtype=torch.int32, device="cuda"),
                           out_d)
        ctx.sync()
        got = F.to_host_words(ps, out_d).astype(np.uint64)
        for c in sample:
            want = oracle.tfhe_bootstrap(ps, K, polys[ids[c]], cts[c])
            assert np.array_equal(got[c], want), (name, c)
        if name == "A":
            dec = [oracle.lwe_decrypt(ps.w, ps.t, K.s, o) for o in got]
            h = ps.t // 2
            exp = [int(f_halves[i][m]) if m < h else (-int(f_halves[i][m - h])) % ps.t for i, m in zip(ids, mr.m)]
            assert dec == exp


def test_tfhe_bootstrap_errors(F, torch_cuda, ctx, oracle):
    """No polynomial installed -> FDFB_EBADLUT; an id out of range is latched
    and reported by fdfb_sync; batch 0 is a no-op."""
    torch = torch_cuda
    ps = S.PARAM_SETS["A"]
    K = oracle_keys("A", 0)
    sid = ctx.register(ps)
    ctx.keys_upload(sid, K.bsk, K.pk, K.ksk)
    ct = torch.zeros((3, ps.n + 1), dtype=torch.int32, device="cuda")
    out = torch.zeros_like(ct)
    ids = torch.zeros(3, dtype=torch.int32, device="cuda")
    with pytest.raises(F.FDFBError) as e:
        ctx.tfhe_bootstrap(sid, ct, ids, out)
    assert e.value.code == -6
    ctx.tfhe_poly_setup(sid, np.zeros(ps.N, dtype=np.uint32))
    ctx.tfhe_bootstrap(sid, ct[:0], ids[:0], out[:0])
    ctx.tfhe_bootstrap(sid, ct, torch.tensor([0, 5, 0], dtype=torch.int32, device="cuda"), out)
    with pytest.raises(F.FDFBError) as e:
        ctx.sync()
    assert e.value.code == -6
    ctx.sync()


# ---------------------------------------------------------- balanced digits --

def test_signed_digits_match_oracle(F, torch_cuda, ctx, oracle):
    """Balanced blind-rotation digits (signed_digits = 1): sets A and B, every
    layout variant bit for bit equal, and equal to the oracle (A: all 30
    ciphertexts; B: 3 of 40)."""
    import dataclasses
    for name, seed, batch, sample in (("A", 0, 30, range(30)), ("B", 1, 40, (0, 1, 39))):
        ps = dataclasses.replace(S.PARAM_SETS[name], name=name + "s", signed_digits=True)
        K = oracle_keys(name, seed)  # the keys do not depend on the digit form
        sid = ctx.register(ps)
        ctx.keys_upload(sid, K.bsk, K.pk, K.ksk)
        fs, rot = luts(name, seed, 2)
        for f in fs:
            ctx.lut_setup(sid, f)
        ids = S.lut_assignment(seed, batch, 2, "uniform", group=60)
        mr, cts = fresh_cts(name, seed, batch, K, group=60)
        outs = []
        for v in range(ctx.variant_info(sid)[1]):
            ctx.set_variant(sid, v)
            out, _ = run_gpu(F, torch_cuda, ctx, sid, ps, cts, ids, debug=False)
            outs.append(out)
        for v in range(1, len(outs)):
            assert np.array_equal(outs[v], outs[0]), (name, v)
        for c in sample:
            want = oracle.fdfb_bootstrap(ps, K, rot[ids[c]][0], rot[ids[c]][1], cts[c])
            assert np.array_equal(outs[0][c], want), (name, c)


# ------------------------------------------------------ output modulus t' --

@pytest.mark.parametrize("t_out", [2, 16])
def test_other_output_modulus_matches_oracle(F, torch_cuda, ctx, oracle, t_out):
    """f: Z_4 -> Z_t' (noiseless set Z with t_out = t'): the GPU equals the
    oracle bit for bit, and every output decrypts (in Z_t') to f(m)."""
    import dataclasses
    torch = torch_cuda
    ps = dataclasses.replace(S.PARAM_SETS["Z"], name=f"Z{t_out}", t_out=t_out)
    K = oracle_keys("Z", 0)  # keys do not depend on the plaintext moduli
    sid = ctx.register(ps)
    ctx.keys_upload(sid, K.bsk, K.pk, K.ksk)
    rng = np.random.default_rng(40 + t_out)
    fs = rng.integers(0, t_out, size=(6, ps.t))
    rot = np.stack([np.stack(oracle.setup_polynomial(ps.N, ps.t, f)) for f in fs])
    assert [ctx.lut_setup(sid, [int(v) for v in f]) for f in fs] == list(range(6))
    ids = rng.integers(0, 6, size=48).astype(np.int32)
    mr, cts = fresh_cts("Z", 0, 48, K, group=70)
    out, _ = run_gpu(F, torch, ctx, sid, ps, cts, ids, debug=False)
    want = oracle.fdfb_batch(dataclasses.replace(ps), K, rot, ids, cts)
    assert np.array_equal(out, want)
    m_d = torch.empty(48, dtype=torch.int32, device="cuda")
    ctx.lwe_decrypt(sid, torch.tensor(K.s, device="cuda"), F.to_device_words(ps, out), m_d)
    ctx.sync()
    assert m_d.cpu().numpy().tolist() == [int(fs[i][m]) for i, m in zip(ids, mr.m)]
    with pytest.raises(F.FDFBError):
        ctx.lut_setup(sid, [t_out, 0, 0, 0])


# ------------------------------------------------------------ extreme sizes --

@pytest.mark.parametrize("signed", [False, True])
def test_widest_digits_and_largest_t(F, torch_cuda, ctx, oracle, signed):
    """Limits of the parameter space at N = 256: 16-bit digits (B = 2^16, the
    widest the digit buffers hold, l = 2: an exact 32-bit decomposition) in
    every gadget, and t = N (one-coefficient windows).  Every registered
    variant equals the oracle bit for bit; balanced digits reach -2^15."""
    import dataclasses
    base = S.PARAM_SETS["Z"]
    ps = dataclasses.replace(base, name=f"Zmax{int(signed)}", t=256, log2Bg=16, lg=2, log2Bks=16,
                             lks=2, log2Bpk=16, lpk=2, sigma_lwe=2.0 ** 10, sigma_glwe=2.0 ** 6,
                             signed_digits=signed)
    kr = S.key_randomness(ps, 12)
    K = oracle.Keys(ps, kr)
    sid = ctx.register(ps)
    ctx.keys_upload(sid, K.bsk, K.pk, K.ksk)
    fs = S.lut_tables(ps, 12, 2)
    rot = np.stack([np.stack(oracle.setup_polynomial(ps.N, ps.t, f)) for f in fs])
    for f in fs:
        ctx.lut_setup(sid, f)
    ids = S.lut_assignment(12, 21, 2, "uniform")
    mr = S.message_randomness(ps, 12, 21)
    cts = oracle.encrypt_messages(ps, K.s, mr)
    want = oracle.fdfb_batch(ps, K, rot, ids, cts)
    count = ctx.variant_info(sid)[1]
    assert count >= 1
    for v in range(count):
        ctx.set_variant(sid, v)
        out, _ = run_gpu(F, torch_cuda, ctx, sid, ps, cts, ids, debug=False)
        assert np.array_equal(out, want), v

