"""fdfb_bootstrap_noalloc: the bootstrap for callers that cannot allocate GPU
memory at call time (host callbacks on a stream, services whose device memory
belongs to a caching allocator or a budget, latency-bound loops).  It must give
exactly what fdfb_bootstrap gives, call after call, on its fixed scratch, for
the power-of-two sets and for the prime-modulus sets (whose pipeline lays the
scratch out differently).  Runs last so a failure here leaves every other test
run."""
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
    prime = isinstance(ps, S.QParamSet)
    mr = (S.q_message_randomness if prime else S.message_randomness)(ps, seed, count)
    ct = torch.empty((count, ps.n + 1), dtype=F.word_torch(ps), device=dev)
    ctx.lwe_encrypt(sid, torch.tensor(kr.s, device=dev), F.to_device_words(ps, mr.a),
                    torch.tensor(mr.e, device=dev), torch.tensor(mr.m, device=dev), ct)
    ids = torch.tensor(S.lut_assignment(seed, count, n_luts, "uniform"), dtype=torch.int32, device=dev)
    return ct, ids


@pytest.mark.parametrize("name,count", [("A", 40), ("B", 300), ("QZ", 40)])
def test_noalloc_matches_bootstrap_twice(env, name, count):
    torch, F, ctx = env
    ps = S.param_set(name)
    prime = isinstance(ps, S.QParamSet)
    sid = ctx.register(ps)
    kr = (S.q_key_randomness if prime else S.key_randomness)(ps, 21)
    ctx.keys_generate(sid, kr)
    for f in (S.q_lut_tables if prime else S.lut_tables)(ps, 21, 3):
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


def test_noalloc_cap_of_a_prime_set(env):
    """The prime-modulus pipeline keeps l_boot sign LWEs, their packing sums
    and packed RLWEs per input: l_boot (7N + 1) + 3N + 1 + 2(n + 1) words,
    44 inputs for FDFB-80-6."""
    torch, F, ctx = env
    ps = S.Q_PARAM_SETS["FDFB-80-6"]
    sid = ctx.register(ps)
    per_input = ps.lboot * (7 * ps.N + 1) + 3 * ps.N + 1 + 2 * (ps.n + 1)
    assert ctx.noalloc_max_batch(sid) == (32 << 20) // (per_input * 8) == 44
