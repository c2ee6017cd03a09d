"""The benchmark's multi-rank host logic on CPU with gloo, world size 2:
each rank draws its own shard of ciphertext inputs (independent streams, no
data-path collective), the timed region is the slowest rank's, and the
whole-job throughput counts every rank's units.  No GPU involved."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import bench
    from paper_2109_02731_gb300 import synth as S
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ps = S.PARAM_SETS["B"]
    mr = bench.rank_messages(ps, 1, 64, rank)
    # shard fingerprints go through a collective only in the test, to compare them
    fp = torch.tensor([int(mr.a[0, 0]), int(mr.m.sum())], dtype=torch.int64)
    fps = [torch.zeros_like(fp) for _ in range(world)]
    dist.all_gather(fps, fp)
    slow = bench.slowest_rank([10.0 + rank, 3.0 - rank], "cpu")
    out[rank] = (fps[0].tolist(), fps[1].tolist(), slow)
    dist.destroy_process_group()


def test_two_ranks_shard_and_take_the_slowest():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    f0, f1, slow0 = out[0]
    assert out[1][2] == slow0 == [11.0, 3.0]
    assert f0 != f1, "ranks must bootstrap different shards"
    # a rank's shard does not depend on the world size: rank 0 of any run
    # bootstraps the same inputs as a single-GPU run
    import bench
    from paper_2109_02731_gb300 import synth as S
    mr = bench.rank_messages(S.PARAM_SETS["B"], 1, 64, 0)
    assert f0 == [int(mr.a[0, 0]), int(mr.m.sum())]


def _bootstrap_worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import bench
    import oracle as O
    from paper_2109_02731_gb300 import synth as S
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ps = S.PARAM_SETS["A"]
    K = O.Keys(ps, S.key_randomness(ps, 0))           # keys replicated on every rank
    fs = S.lut_tables(ps, 0, 2)
    rot = np.stack([np.stack(O.setup_polynomial(ps.N, ps.t, f)) for f in fs])
    mr = bench.rank_messages(ps, 0, 6, rank)          # this rank's own shard
    ids = (np.arange(6) + rank) % 2
    cts = O.encrypt_messages(ps, K.s, mr)
    outs = O.fdfb_batch(ps, K, rot, ids, cts)        # the data path: no collective
    dec = [O.lwe_decrypt(ps.w, ps.t, K.s, c) for c in outs]
    ok = dec == [int(fs[i][m]) for i, m in zip(ids, mr.m)]
    # only the test gathers anything: per-rank correctness and a fingerprint
    t = torch.tensor([int(ok), int(outs[0][0])], dtype=torch.int64)
    got = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(got, t)
    out[rank] = [g.tolist() for g in got]
    dist.destroy_process_group()


def test_two_ranks_bootstrap_their_own_shards():
    """Weak scaling end to end on CPU: two gloo ranks, keys replicated, each
    bootstraps its own shard of the toy workload through the oracle with no
    collective on the data path; every output of every rank decrypts to
    f(m), and the shards differ."""
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_bootstrap_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    res = out[0]
    assert out[1] == res
    assert res[0][0] == 1 and res[1][0] == 1, "a rank's outputs did not decrypt to f(m)"
    assert res[0][1] != res[1][1], "ranks must bootstrap different shards"
