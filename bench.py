#!/usr/bin/env python3
"""FDFB throughput benchmark: full-domain functional bootstraps per second.

One step = one call of the library's batched bootstrap over the workload's
batch: ModSwitch, sign blind rotation, SampleExtract, packing key switch,
PubMux, function blind rotation, SampleExtract and LWE key switch, for every
ciphertext.  Keys, tables and ciphertexts are made on the GPU from seeded
synthetic randomness before timing (inputs resident in HBM); L2 is flushed
by a 512 MB write before every timed step and the flush is not timed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   # the CPU oracle on a bounded sample

Under torchrun (N > 1) each rank bootstraps its own batch (weak scaling, no
collective on the data path); the timed region is bracketed by barriers and
the slowest rank's time is reported.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2109_02731_gb300 import synth as S  # noqa: E402

METRIC = "FDFB bootstraps/s on 1 GB300 (bit-exact), batched vs plain path; % of roofline"
UNIT = "bootstraps/s"
L2_FLUSH_BYTES = 512 << 20

# Integer multiplier pipe of the GB300: 152 SMs x 64 IMAD lanes per clock x
# 2.07 GHz maximum SM clock; multiply-high issues at half that rate (the
# probe in paper_2109_02731_gb300/probe/int_pipe.cu measures both).
SMS = 152
IMAD_LANES_PER_SM = 64
SM_MAX_GHZ = 2.07


def workload_desc(name: str):
    wl = S.WORKLOADS[name]
    g = wl.groups[0]
    ps = S.PARAM_SETS[g.set_name]
    return wl, g, ps


def br_algorithmic_slots(ps, batch: int) -> float:
    """Integer-multiplier issue slots the blind rotation needs per launch (one
    BR over `batch` ciphertexts), counting only the method's modular products:
    per CMux (2l + 2) P transforms of (N/2) log2 N butterflies, each one Shoup
    product = 1 multiply-high (2 slots: the pipe runs it at half rate) + 2
    multiply-low (1 slot each), and 4 l N P pointwise products, each one
    32x32->64 multiply-add (2 slots); n CMux steps per ciphertext."""
    P = 2 if ps.w == 32 else 3
    bfly = (2 * ps.lg + 2) * P * (ps.N // 2) * ps.logN
    mac = 4 * ps.lg * ps.N * P
    return float(batch) * ps.n * (4.0 * bfly + 2.0 * mac)


def sample_clocks(path: str):
    cmd = ["nvidia-smi",
           "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
           "--format=csv,noheader,nounits", "-lms", "200"]
    try:
        f = open(path, "w")
        return subprocess.Popen(cmd, stdout=f, stderr=subprocess.DEVNULL), f
    except Exception:
        return None, None


def read_clocks(path: str, gpu_index: int):
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    try:
        for ln in open(path):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9 or parts[0] != str(gpu_index):
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
    except OSError:
        pass
    if not sm:
        return None
    return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
            "samples": len(sm)}


def probe_rates(dev_index: int):
    """Measured integer-pipe rates of this GPU (T ops/s): IMAD, IMAD.HI, LOP
    and Harvey butterflies, from paper_2109_02731_gb300/probe/int_pipe.cu."""
    import ctypes
    from paper_2109_02731_gb300 import build as B
    try:
        lib = ctypes.CDLL(B.build_probe())
        rates = (ctypes.c_double * 4)()
        if lib.probe_int_rates(dev_index, rates) != 0:
            return None
        return {"imad": rates[0] / 1e12, "imad_hi": rates[1] / 1e12, "lop": rates[2] / 1e12,
                "butterfly": rates[3] / 1e12, "unit": "T/s"}
    except Exception as e:  # the probe is evidence, not the measurement
        return {"error": str(e)[:200]}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    """The reference arm: the CPU oracle as it stands, on the machine's host cores,
    on a bounded sample of the same workload per step."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import oracle as O
    wl, g, ps = workload_desc(args.workload)
    cores = O.max_threads()
    O.set_threads(cores)
    K = O.Keys(ps, S.key_randomness(ps, wl.seed))
    fs = S.lut_tables(ps, wl.seed, g.n_luts)
    rot = np.stack([np.stack(O.setup_polynomial(ps.N, ps.t, f)) for f in fs])
    ids = S.lut_assignment(wl.seed, g.batch, g.n_luts, g.lut_assign)
    per_step = args.ref_sample
    mr = S.message_randomness(ps, wl.seed, per_step * (args.steps + args.warmup))
    cts = O.encrypt_messages(ps, K.s, mr)

    def step(k):
        sl = slice(k * per_step, (k + 1) * per_step)
        for c in range(sl.start, sl.stop):
            O.fdfb_bootstrap(ps, K, rot[ids[c % g.batch]][0], rot[ids[c % g.batch]][1], cts[c])

    for k in range(args.warmup):
        step(k)
    t0 = time.perf_counter()
    for k in range(args.warmup, args.warmup + args.steps):
        step(k)
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32" if ps.w == 32 else "u64",
        "data": "synthetic (seeded SplitMix64 keys, messages and tables)",
        "config": config_of(args, wl, g, ps),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} ciphertexts per step of the {args.workload} workload, "
                                   f"each bootstrapped by the schoolbook oracle with its ring products "
                                   f"spread over {cores} threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def config_of(args, wl, g, ps):
    return {"workload": f"{wl.name}: FDFB n={ps.n} N={ps.N} q=2^{ps.w} t={ps.t} B_g=2^{ps.log2Bg} "
                        f"l_g={ps.lg} B_ks=2^{ps.log2Bks} l_ks={ps.lks} B_pk=2^{ps.log2Bpk} l_pk={ps.lpk}, "
                        f"{g.batch} ciphertexts per GPU, {g.n_luts} tables ({g.lut_assign})",
            "batch_per_gpu": g.batch, "param_set": ps.name, "seed": wl.seed,
            "l2": "flushed before every timed step (512 MB write, not timed)"}


def cpu_baseline(wl, g, ps, seconds_target=20.0):
    """The oracle timed on a bounded sample (rank 0, one GPU only)."""
    import oracle as O
    cores = O.max_threads()
    O.set_threads(cores)
    K = O.Keys(ps, S.key_randomness(ps, wl.seed))
    fs = S.lut_tables(ps, wl.seed, g.n_luts)
    rot = np.stack([np.stack(O.setup_polynomial(ps.N, ps.t, f)) for f in fs])
    ids = S.lut_assignment(wl.seed, g.batch, g.n_luts, g.lut_assign)
    mr = S.message_randomness(ps, wl.seed, g.batch)
    cts = O.encrypt_messages(ps, K.s, mr)
    t0 = time.perf_counter()
    done = 0
    while done < g.batch:
        c = done
        O.fdfb_bootstrap(ps, K, rot[ids[c]][0], rot[ids[c]][1], cts[c])
        done += 1
        if time.perf_counter() - t0 > seconds_target:
            break
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {done} ciphertexts of the workload, one after another, each bootstrap's "
                      f"ring products spread over {cores} threads ({dt:.1f} s)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tfhe_scale", choices=sorted(S.WORKLOADS))
    ap.add_argument("--ref-sample", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--plain", action="store_true",
                    help="also time the plain path: one ciphertext per bootstrap call")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_2109_02731_gb300 import fdfb as F

    wl, g, ps = workload_desc(args.workload)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    ctx = F.Context(dev.index)
    sid = ctx.register(ps)
    kr = S.key_randomness(ps, wl.seed)
    ctx.keys_generate(sid, kr)
    fs = S.lut_tables(ps, wl.seed, g.n_luts)
    for f in fs:
        ctx.lut_setup(sid, f)
    batch = g.batch
    ids_np = S.lut_assignment(wl.seed, batch, g.n_luts, g.lut_assign)
    mr = S.message_randomness(ps, wl.seed, batch, group=rank)
    s_d = torch.tensor(kr.s, device=dev)
    ct = torch.empty((batch, ps.n + 1), dtype=F.word_torch(ps), device=dev)
    ctx.lwe_encrypt(sid, s_d, F.to_device_words(ps, mr.a, dev), torch.tensor(mr.e, device=dev),
                    torch.tensor(mr.m, device=dev), ct)
    ids = torch.tensor(ids_np, dtype=torch.int32, device=dev)
    out = torch.empty_like(ct)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        ctx.bootstrap(sid, ct, ids, out)
    ctx.sync()
    # correctness of this run: decrypt every output with the secret key
    m_out = torch.empty(batch, dtype=torch.int32, device=dev)
    ctx.lwe_decrypt(sid, s_d, out, m_out)
    ctx.sync()
    want = np.array([fs[i][m] for i, m in zip(ids_np, mr.m)])
    decrypt_ok = float((m_out.cpu().numpy() == want).mean())

    clk_path = os.path.join(tempfile.gettempdir(), f"fdfb_clocks_{os.getpid()}.csv")
    proc, fh = sample_clocks(clk_path)
    time.sleep(0.3)
    ctx.profile_enable(True)
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        ctx.bootstrap(sid, ct, ids, out)
        ev[k][1].record(stream)
    barrier()
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    ms_steps = [a.elapsed_time(b) for a, b in ev]
    ms_total = float(sum(ms_steps))

    # end to end through the public API with host buffers: H2D of the step's
    # ciphertexts and table ids from pinned memory, bootstrap, D2H of outputs.
    ct_h = ct.cpu().pin_memory()
    ids_h = ids.cpu().pin_memory()
    out_h = torch.empty(out.shape, dtype=out.dtype).pin_memory()
    ct_e, ids_e, out_e = torch.empty_like(ct), torch.empty_like(ids), torch.empty_like(out)
    e2e_steps = max(1, args.steps)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_ms = 0.0
    for k in range(e2e_steps):
        flush.zero_()
        e0.record(stream)
        ct_e.copy_(ct_h, non_blocking=True)
        ids_e.copy_(ids_h, non_blocking=True)
        ctx.bootstrap(sid, ct_e, ids_e, out_e)
        out_h.copy_(out_e, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
    barrier()
    if proc is not None:
        proc.terminate()
        proc.wait()
        fh.close()
    clocks = read_clocks(clk_path, dev.index)

    # slowest rank
    if world > 1:
        t = torch.tensor([ms_total, e2e_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_total, e2e_ms = float(t[0]), float(t[1])

    plain = None
    if args.plain and rank == 0:
        reps = 8
        one_ct, one_id, one_out = ct[:1].clone(), ids[:1].clone(), out[:1].clone()
        ctx.bootstrap(sid, one_ct, one_id, one_out)
        barrier()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(reps):
            ctx.bootstrap(sid, one_ct, one_id, one_out)
        p1.record(stream)
        p1.synchronize()
        plain = {"value": reps / (p0.elapsed_time(p1) / 1e3), "unit": UNIT,
                 "what": "one ciphertext per bootstrap call, same kernels"}

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    units = batch * args.steps * world
    value = units / (ms_total / 1e3)
    br_ms, br_n = prof["blind_rotate_sign"]
    br2_ms, br2_n = prof["blind_rotate_func"]
    br_avg_s = (br_ms + br2_ms) / max(1, br_n + br2_n) / 1e3
    slots = br_algorithmic_slots(ps, batch)
    peak = SMS * IMAD_LANES_PER_SM * SM_MAX_GHZ * 1e9 / 1e12  # T slots/s
    achieved = slots / br_avg_s / 1e12
    stage_share = {k: round(v[0] / max(1e-9, sum(x[0] for x in prof.values())), 4) for k, v in prof.items()}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32" if ps.w == 32 else "u64",
        "data": "synthetic (seeded SplitMix64 keys, messages and tables; keys generated on the GPU)",
        "config": config_of(args, wl, g, ps),
        "decrypt_ok": decrypt_ok,
        "roofline": {"bound": "alu", "kernel": "blind_rotate_kernel", "achieved": achieved, "peak": peak,
                     "unit": "T IMAD slots/s", "frac": achieved / peak,
                     "traffic": None, "peak_source": "derived: 152 SMs x 64 IMAD lanes/clock x 2.07 GHz",
                     "launch_ms": br_avg_s * 1e3, "slots_per_launch": slots},
        "stage_share": stage_share,
        "gpu_launches": 5 * args.steps,
        "e2e": {"value": units / (e2e_ms / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": int(ct.numel() * ct.element_size() + ids.numel() * 4),
                "d2h_bytes_per_step": int(out.numel() * out.element_size())},
        "clocks": clocks,
    }
    probe = probe_rates(dev.index)
    if probe:
        line["roofline"]["probe"] = probe
    if plain:
        line["plain_path"] = plain
        line["batched_over_plain"] = value / plain["value"]
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, g, ps)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
