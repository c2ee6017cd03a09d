"""The key switches on the tensor cores (tcgen05.mma kind::f16 on balanced
key limbs, fp32 partial sums kept below 2^24): bit for bit the oracle's
KeySwitch (figure "Key switching algorithm and its setup") and the CUDA-core
contraction, on random inputs and on inputs that drive every partial sum to
the bound the chunking allows.  Every other GPU test already runs the
bootstrap with the tensor-core key switches."""
import dataclasses

import numpy as np
import pytest

from paper_2109_02731_gb300 import synth as S

from _fdfb_cases import oracle_keys

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("this test needs a CUDA GPU")
    from paper_2109_02731_gb300 import fdfb as F
    ctx = F.Context(0)
    yield torch, F, ctx
    ctx.close()


def _words(r, w, shape):
    if w == 64:
        return r.integers(0, 1 << 63, size=shape, dtype=np.uint64) * np.uint64(2) + \
            r.integers(0, 2, size=shape, dtype=np.uint64)
    return r.integers(0, 1 << 32, size=shape, dtype=np.uint64)


@pytest.mark.parametrize("name,seed,batch", [("A", 0, 130), ("B", 1, 257), ("D", 3, 131), ("C", 2, 5)])
def test_tensor_core_keyswitch_matches_oracle(env, oracle, name, seed, batch):
    torch, F, ctx = env
    ps = S.PARAM_SETS[name]
    K = oracle_keys(name, seed)
    sid = ctx.register(ps)
    ctx.keys_upload(sid, K.bsk, K.pk, K.ksk)
    assert ctx.keyswitch_path(sid) == (1, 1)
    x = _words(np.random.default_rng(seed + 100), ps.w, (batch, ps.N + 1))
    x_d = F.to_device_words(ps, x)
    y_d = torch.empty((batch, ps.n + 1), dtype=F.word_torch(ps), device="cuda")
    ctx.keyswitch(sid, x_d, y_d)
    ctx.sync()
    y = F.to_host_words(ps, y_d).astype(np.uint64)
    for i in sorted({0, batch // 2, batch - 1}):
        assert np.array_equal(y[i], oracle.keyswitch(ps.w, ps.log2Bks, ps.lks, K.ksk, x[i])), i
    # the CUDA-core contraction gives the same words
    ctx.test_hooks(2)
    try:
        assert ctx.keyswitch_path(sid) == (0, 0)
        z_d = torch.empty_like(y_d)
        ctx.keyswitch(sid, x_d, z_d)
        ctx.sync()
    finally:
        ctx.test_hooks(0)
    assert torch.equal(z_d, y_d)


def _limb_pattern(b, negative, w=64):
    """A w-bit word whose balanced base-2^b limbs are all -2^(b-1) (negative)
    or all 2^(b-1) - 1: the largest limb magnitudes there are."""
    v = -(1 << (b - 1)) if negative else (1 << (b - 1)) - 1
    x = 0
    for s in range(-(-w // b)):
        x += v << (b * s)
    return x % (1 << w)


def test_partial_sums_at_their_bound(env, oracle):
    """Digits all B - 1 = 1023 and key words whose limbs all have the largest
    magnitude, for every limb width the library may choose: with N = 2048 and
    10-bit digits each fp32 chunk sum reaches the 2^23 the chunking allows,
    and the result must still be exact."""
    torch, F, ctx = env
    ps = dataclasses.replace(S.PARAM_SETS["D"], name="KSW", n=16, log2Bks=10, lks=4, lpk=1)
    sid = ctx.register(ps)
    N, n, w = ps.N, ps.n, ps.w
    bsk = np.zeros((n, 2 * ps.lg, 2, N), dtype=np.uint64)
    pk = np.zeros((N, ps.lpk, 2, N), dtype=np.uint64)
    # inputs: every rounded mask word has all four digits 1023 (the top 40 bits set)
    batch = 131
    x = np.full((batch, N + 1), ((1 << 40) - 1) << 24, dtype=np.uint64)
    x[:, 0] = np.arange(batch, dtype=np.uint64)
    x_d = F.to_device_words(ps, x)
    for b in range(2, 13):
        for negative in (False, True):
            word = _limb_pattern(b, negative)
            ksk = np.full((N, ps.lks, n + 1), word, dtype=np.uint64)
            ctx.keys_upload(sid, bsk, pk, ksk)
            assert ctx.keyswitch_path(sid)[1] == 1
            y_d = torch.empty((batch, n + 1), dtype=torch.int64, device="cuda")
            ctx.keyswitch(sid, x_d, y_d)
            ctx.sync()
            y = F.to_host_words(ps, y_d).astype(np.uint64)
            ref = oracle.keyswitch(w, ps.log2Bks, ps.lks, ksk, x[0])
            for i in (0, batch - 1):
                want = ref.copy()
                want[0] = (int(ref[0]) + int(x[i, 0]) - int(x[0, 0])) % (1 << w)
                assert np.array_equal(y[i], want), (b, negative, i)


@pytest.mark.parametrize("base,n", [("QZ", 24), ("FDFB-80-6", 16), ("FDFB-100-6", 8)])
def test_prime_set_keyswitch_on_tensor_cores(env, base, n):
    """The prime-modulus form: the tensor cores compute the exact integer sums
    of digit times key residue (limbs covering 65 bits), reduced mod Q after.
    Random residues, and rows whose digits and key words are all Q - 1 (the
    largest sums there are), against the oracle and the CUDA-core path.  The
    packing keys of these sets have 13-bit digits (split into two halves);
    FDFB-100-6's LWE key has 62 binary digits."""
    import oracle.prime_q as OQ
    torch, F, ctx = env
    ps = dataclasses.replace(S.Q_PARAM_SETS[base], name=f"{base}-ks{n}", n=n)
    Q, N = ps.Q, ps.N
    bsk, pk, ksk = S.q_uniform_key_words(ps, 41)
    ksk[:N // 2] = Q - 1
    sid = ctx.register(ps)
    ctx.keys_upload(sid, bsk, pk, ksk)
    assert ctx.keyswitch_path(sid) == (1, 1)
    batch = 70
    x = S.Stream(42, 1).raw(batch * (N + 1)).reshape(batch, N + 1) % np.uint64(Q)
    x[:3] = Q - 1
    x_d = F.to_device_words(ps, x)
    y_d = torch.empty((batch, n + 1), dtype=torch.int64, device="cuda")
    ctx.keyswitch(sid, x_d, y_d)
    ctx.sync()
    y = F.to_host_words(ps, y_d).astype(np.uint64)
    for i in (0, 2, 3, batch - 1):
        assert np.array_equal(y[i], OQ.keyswitch(Q, ps.log2Bks, ps.lks, ksk, x[i])), i
    ctx.test_hooks(2)
    try:
        z_d = torch.empty_like(y_d)
        ctx.keyswitch(sid, x_d, z_d)
        ctx.sync()
    finally:
        ctx.test_hooks(0)
    assert torch.equal(z_d, y_d)
