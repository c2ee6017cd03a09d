"""The bounded device-side wait of the staged-key blind rotation (N = 2048,
q = 2^64), made to run out without any fault: fdfb_test_hooks stops the
kernel issuing its bulk key copies, so the wait for them expires with nothing
in flight.  The call must latch FDFB_ETIMEOUT (reported by fdfb_sync), and the
next call on the same context must again be bit-exact."""
import pytest

from paper_2109_02731_gb300 import synth as S

pytestmark = pytest.mark.gpu


def test_staged_key_wait_expires_and_context_recovers():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("this test needs a CUDA GPU")
    from paper_2109_02731_gb300 import fdfb as F
    ps = S.PARAM_SETS["D"]
    ctx = F.Context(0)
    try:
        sid = ctx.register(ps)
        kr = S.key_randomness(ps, 3)
        ctx.keys_generate(sid, kr)
        for f in S.lut_tables(ps, 3, 2):
            ctx.lut_setup(sid, f)
        mr = S.message_randomness(ps, 3, 3, group=40)
        ct = torch.empty((3, ps.n + 1), dtype=torch.int64, device="cuda")
        ctx.lwe_encrypt(sid, torch.tensor(kr.s, device="cuda"), F.to_device_words(ps, mr.a),
                        torch.tensor(mr.e, device="cuda"), torch.tensor(mr.m, device="cuda"), ct)
        ids = torch.tensor([0, 1, 0], dtype=torch.int32, device="cuda")

        def run():
            out = torch.empty_like(ct)
            ctx.bootstrap(sid, ct, ids, out)
            return out

        ctx.set_variant(sid, 0)
        ref = run()
        ctx.sync()
        count = ctx.variant_info(sid)[1]
        expired = []
        for v in range(count):
            ctx.set_variant(sid, v)
            ctx.test_hooks(1)
            run()
            try:
                ctx.sync()
            except F.FDFBError as e:
                assert e.code == -4, f"variant {v}: {e}"  # FDFB_ETIMEOUT
                expired.append(v)
            ctx.test_hooks(0)
            # the context is usable again and exact
            again = run()
            ctx.sync()
            assert torch.equal(again, ref), f"variant {v} after the hook"
        assert len(expired) == 1, f"variants whose staged-key wait expired: {expired}"
        with pytest.raises(F.FDFBError):
            ctx.test_hooks(4)  # unknown bit
    finally:
        ctx.close()
