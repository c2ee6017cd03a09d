"""fdfb_bootstrap_noalloc: the bootstrap for callers that cannot allocate GPU
memory (code under stream capture, real-time or memory-budgeted service
loops).  It must give exactly what fdfb_bootstrap gives, call after call, on
its fixed scratch.  Runs last so a failure here leaves every other test run."""
import numpy as np
import pytest

from paper_2109_02731_gb300 import synth as S

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


def _inputs(torch, F, ctx, sid, ps, kr, seed, count, n_luts):
    dev = "cuda"
    mr = S.message_randomness(ps, seed, count)
    ct = torch.empty((count, ps.n + 1), dtype=F.word_torch(ps), device=dev)
    ctx.lwe_encrypt(sid, torch.tensor(kr.s, device=dev), F.to_device_words(ps, mr.a),
                    torch.tensor(mr.e, device=dev), torch.tensor(mr.m, device=dev), ct)
    ids = torch.tensor(S.lut_assignment(seed, count, n_luts, "uniform"), dtype=torch.int32, device=dev)
    return ct, ids


@pytest.mark.parametrize("name,count", [("A", 40), ("B", 300)])
def test_noalloc_matches_bootstrap_twice(env, name, count):
    torch, F, ctx = env
    ps = S.PARAM_SETS[name]
    sid = ctx.register(ps)
    kr = S.key_randomness(ps, 21)
    ctx.keys_generate(sid, kr)
    for f in S.lut_tables(ps, 21, 3):
        ctx.lut_setup(sid, f)
    assert ctx.noalloc_max_batch(sid) >= count
    for call, seed in enumerate((31, 32)):  # two calls in a row, different inputs
        ct, ids = _inputs(torch, F, ctx, sid, ps, kr, seed, count, 3)
        ref = torch.empty_like(ct)
        got = torch.full_like(ct, -1)
        ctx.bootstrap(sid, ct, ids, ref)
        ctx.bootstrap_noalloc(sid, ct, ids, got)
        ctx.sync()
        assert torch.equal(got, ref), f"call {call}"


def test_noalloc_rejects_batches_beyond_its_scratch(env):
    torch, F, ctx = env
    ps = S.PARAM_SETS["C"]
    sid = ctx.register(ps)
    cap = ctx.noalloc_max_batch(sid)
    assert cap == (32 << 20) // ((6 * ps.N + 2) * 8)
    ct = torch.zeros((cap + 1, ps.n + 1), dtype=torch.int64, device="cuda")
    ids = torch.zeros(cap + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(F.FDFBError) as e:
        ctx.bootstrap_noalloc(sid, ct, ids, torch.empty_like(ct))
    assert e.value.code == -1
