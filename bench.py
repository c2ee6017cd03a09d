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
import dataclasses
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
    ps = S.param_set(g.set_name)
    return wl, g, ps


def is_prime_set(ps) -> bool:
    return isinstance(ps, S.QParamSet)


# The paper's own times per bootstrap for its parameter sets (Table 3: one
# bootstrap, not parallelised, on a 60-core Xeon Cascade Lake VM with a
# 64-bit prime-modulus NTT): context for the prime-modulus workloads.
PAPER_MS_PER_BOOTSTRAP = {"FDFB-80-6": 3655.0, "FDFB-100-6": 4838.0, "FDFB-80-7": 9278.0,
                          "FDFB-100-7": 13781.0, "TFHE-100-7": 7757.0, "TFHE-80-2": 306.0,
                          "TFHE-100-2": 321.0}


# DRAM bytes (read + write) of one blind-rotation launch over the whole batch,
# measured by ncu (dram__bytes_read.sum + dram__bytes_write.sum) on the current
# kernel for (set, variant, batch); reported only for that configuration.
KERNEL_TRAFFIC = {
    ("B", 7, 1024): 86.26e6,    # tfhe_scale workload
    ("D", 6, 1000): 3.19754e9,  # n2048 workload
    # paper_80_6: the sign rotation (6000 items) scaled from a 384-item capture
    # (1.2074 GB): the 413 MB key streams from DRAM once per wave of 152 items
    ("FDFB-80-6", 3, 1000): 1.2074e9 * 6000 / 384,
}
KERNEL_TRAFFIC_SCALED = {("FDFB-80-6", 3, 1000): "sign-rotation launch (batch x l_boot = 6000 items), "
                                                  "scaled by items from an ncu capture of 384 items"}


def br_algorithmic_slots(ps, batch: int) -> float:
    """Integer-multiplier issue slots the blind rotation needs per launch (one
    BR over `batch` ciphertexts), counting only the method's modular products:
    per CMux (2l + 2) P transforms of (N/2) log2 N butterflies, each one Shoup
    product = 1 multiply-high (2 slots: the pipe runs it at half rate) + 2
    multiply-low (1 slot each), and 4 l N P pointwise products, each one
    32x32->64 multiply-add (2 slots); n CMux steps per ciphertext."""
    P = 2 if getattr(ps, "w", 64) == 32 else 3  # prime-modulus sets: three primes
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


def slowest_rank(values, device):
    """Element-wise maximum over all ranks of per-rank timings (the job is as
    fast as its slowest rank)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


def rank_messages(ps, seed: int, batch: int, rank: int, group: int = 0):
    """The message randomness of one rank's shard: every rank bootstraps its
    own batch (weak scaling), drawn from its own sub-stream."""
    if is_prime_set(ps):
        return S.q_message_randomness(ps, seed, batch, group=1000 * rank + group)
    return S.message_randomness(ps, seed, batch, group=1000 * rank + group)


def q_oracle_sample(ps, seconds_target: float = 10.0, tfhe: bool = False):
    """The prime-modulus oracle's time per bootstrap, from a bounded sample:
    one bootstrap of these sets takes the schoolbook oracle hours (about
    (l_boot + 1) n CMux steps of 2 (2 l) N^2 products mod Q), so the sample
    times whole CMux steps of the blind rotation (a ciphertext whose first
    masks are nonzero: the oracle skips steps with a_i = 0), one packing key
    switch, PubMux and the LWE key switch, at full size, and scales each by
    its count per bootstrap.  Key material of the right shapes is drawn
    uniformly mod Q without key generation: the products cost the same for
    any values.  Returns (seconds per bootstrap, description)."""
    import oracle.prime_q as OQ
    rng = np.random.default_rng(0)
    Q, N, n, lg, lb = ps.Q, ps.N, ps.n, ps.lg, ps.lboot
    uni = lambda *shape: rng.integers(0, 2 ** 63, shape, dtype=np.uint64) % np.uint64(Q)
    def cmux_steps(steps):
        pset = dataclasses.replace(ps, n=steps)
        ctN = np.zeros(steps + 1, dtype=np.uint64)
        ctN[1:] = 1 + np.arange(steps)
        bsk, acc = uni(steps, 2 * lg, 2, N), uni(2, N)
        t0 = time.perf_counter()
        OQ.blind_rotate(pset, bsk, acc, ctN)
        return (time.perf_counter() - t0) / steps

    t1 = cmux_steps(1)
    steps = int(min(16, max(1, seconds_target * 0.6 / max(t1, 1e-3))))
    t_step = cmux_steps(steps) if steps > 1 else t1
    lwe = uni(N + 1)
    pk = uni(N, ps.lpk, 2, N)
    t0 = time.perf_counter()
    OQ.keyswitch(Q, ps.log2Bpk, ps.lpk, pk, lwe)
    t_pk = time.perf_counter() - t0
    del pk
    ksk = uni(N, ps.lks, n + 1)
    t0 = time.perf_counter()
    OQ.keyswitch(Q, ps.log2Bks, ps.lks, ksk, lwe)
    t_ks = time.perf_counter() - t0
    cR = uni(lb, 2, N)
    p0 = rng.integers(-ps.t + 1, ps.t, N)
    t0 = time.perf_counter()
    OQ.pubmux(ps, cR, p0, -p0)
    t_pm = time.perf_counter() - t0
    if tfhe:  # the TFHE bootstrap: one rotation and the LWE key switch
        sec = n * t_step + t_ks
        desc = (f"{steps} full-size CMux step(s) ({t_step:.2f} s each, x {n} per TFHE bootstrap) and the "
                f"LWE key switch ({t_ks:.2f} s) of the schoolbook oracle on one core, scaled to one "
                f"bootstrap ({sec / 60:.1f} min)")
        return sec, desc
    sec = (lb + 1) * n * t_step + lb * t_pk + t_pm + t_ks
    desc = (f"{steps} full-size CMux step(s) ({t_step:.2f} s each, x {(lb + 1) * n} per bootstrap), one "
            f"packing key switch ({t_pk:.2f} s, x {lb}), PubMux ({t_pm:.2f} s) and the LWE key switch "
            f"({t_ks:.2f} s) of the schoolbook oracle on one core, scaled to one bootstrap "
            f"({sec / 3600:.2f} h)")
    return sec, desc


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
    if is_prime_set(ps):
        tf = g.mode == "tfhe"
        for _ in range(args.warmup):
            q_oracle_sample(ps, tfhe=tf)
        secs = []
        desc = ""
        for _ in range(args.steps):
            sec, desc = q_oracle_sample(ps, tfhe=tf)
            secs.append(sec)
        value = args.steps / sum(secs)
        line = {
            "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(secs) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic (seeded key-shaped words, no key generation: the oracle's cost does not "
                    "depend on the values)",
            "config": config_of(args, wl, g, ps),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "per step: " + desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line), flush=True)
        return 0
    cores = O.max_threads()
    O.set_threads(cores)
    K = O.Keys(ps, S.key_randomness(ps, wl.seed))
    fs = S.lut_tables(ps, wl.seed, g.n_luts)
    rot = np.stack([np.stack(O.setup_polynomial(ps.N, ps.t, f)) for f in fs])
    ids = S.lut_assignment(wl.seed, g.batch, g.n_luts, g.lut_assign)
    polys = S.tfhe_polynomials(ps, wl.seed, g.n_luts) if g.mode == "tfhe" else None
    per_step = args.ref_sample
    mr = S.message_randomness(ps, wl.seed, per_step * (args.steps + args.warmup))
    cts = O.encrypt_messages(ps, K.s, mr)

    def step(k):
        sl = slice(k * per_step, (k + 1) * per_step)
        for c in range(sl.start, sl.stop):
            if g.mode == "tfhe":
                O.tfhe_bootstrap(ps, K, polys[ids[c % g.batch]], cts[c])
            elif g.tables_per_input > 1:
                O.fdfb_bootstrap_multi(ps, K, rot[ids[c % g.batch]], cts[c])
            else:
                O.fdfb_bootstrap(ps, K, rot[ids[c % g.batch]][0], rot[ids[c % g.batch]][1], cts[c])

    for k in range(args.warmup):
        step(k)
    t0 = time.perf_counter()
    for k in range(args.warmup, args.warmup + args.steps):
        step(k)
    dt = time.perf_counter() - t0
    value = per_step * g.tables_per_input * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32" if ps.w == 32 else "u64",
        "data": "synthetic (seeded SplitMix64 keys, messages and tables)",
        "config": config_of(args, wl, g, ps),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} ciphertexts per step of the {args.workload} workload "
                                   f"({g.tables_per_input} table(s) each), "
                                   f"each bootstrapped by the schoolbook oracle with its ring products "
                                   f"spread over {cores} threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def config_of(args, wl, g, ps):
    if is_prime_set(ps):
        kind = ("TFHE bootstrap (one blind rotation of a pre-rotation polynomial)" if g.mode == "tfhe"
                else "FDFB")
        return {"workload": f"{wl.name}: {kind}, the paper's set {ps.name} (Table 1): n={ps.n} N={ps.N} "
                            f"Q=2^{ps.k}-{(1 << ps.k) - ps.Q} q=2N={ps.q} t={ps.t} B_g=2^{ps.log2Bg} l_g={ps.lg} "
                            f"B_ks=2^{ps.log2Bks} l_ks={ps.lks} B_pk=2^{ps.log2Bpk} l_pk={ps.lpk} "
                            f"L_boot=2^{ps.log2Lboot} l_boot={ps.lboot} (exact decompositions, uniform RLWE "
                            f"key), {g.batch} ciphertexts per GPU, {g.n_luts} tables ({g.lut_assign})",
                "batch_per_gpu": g.batch, "param_set": ps.name, "seed": wl.seed,
                "l2": "flushed before every timed step (512 MB write, not timed)"}
    kind = "TFHE bootstrap (one blind rotation of a test polynomial)" if g.mode == "tfhe" else "FDFB"
    return {"workload": f"{wl.name}: {kind} n={ps.n} N={ps.N} q=2^{ps.w} t={ps.t} B_g=2^{ps.log2Bg} "
                        f"l_g={ps.lg} B_ks=2^{ps.log2Bks} l_ks={ps.lks} B_pk=2^{ps.log2Bpk} l_pk={ps.lpk}, "
                        f"{g.batch} ciphertexts per GPU, {g.n_luts} tables ({g.lut_assign})"
                        + (f", {g.tables_per_input} tables per input sharing one sign rotation"
                           if g.tables_per_input > 1 else ""),
            "batch_per_gpu": g.batch, "param_set": ps.name, "seed": wl.seed,
            "l2": "flushed before every timed step (512 MB write, not timed)"}


def cpu_baseline(wl, g, ps, seconds_target=20.0):
    """The oracle timed on a bounded sample (rank 0, one GPU only)."""
    import oracle as O
    if is_prime_set(ps):
        sec, desc = q_oracle_sample(ps, tfhe=g.mode == "tfhe")
        return {"value": 1.0 / sec, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc}
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
    k = g.tables_per_input
    polys = S.tfhe_polynomials(ps, wl.seed, g.n_luts) if g.mode == "tfhe" else None
    while done < g.batch:
        c = done
        if polys is not None:
            O.tfhe_bootstrap(ps, K, polys[ids[c]], cts[c])
        elif k > 1:
            O.fdfb_bootstrap_multi(ps, K, rot[ids[c]], cts[c])
        else:
            O.fdfb_bootstrap(ps, K, rot[ids[c]][0], rot[ids[c]][1], cts[c])
        done += 1
        if time.perf_counter() - t0 > seconds_target:
            break
    dt = time.perf_counter() - t0
    return {"value": done * k / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {done} ciphertexts of the workload ({k} table(s) each), one after another, "
                      f"each bootstrap's ring products spread over {cores} threads ({dt:.1f} s)"}


class Job:
    """The timed work of one workload on this rank: `step()` queues one step on
    the current stream; `units` bootstraps per step."""

    def __init__(self, torch, F, ctx, dev, args, rank):
        self.torch, self.F, self.ctx, self.dev = torch, F, ctx, dev
        wl = S.WORKLOADS[args.workload]
        self.wl = wl
        self.groups = []
        self.tuned = {}
        if wl.mlp_layers:
            self._prepare_mlp(args, rank)
        else:
            for gi, g in enumerate(wl.groups):
                if args.batch is not None and len(wl.groups) == 1:
                    g = dataclasses.replace(g, batch=args.batch)  # smaller case, e.g. for ncu
                self.groups.append(self._prepare_group(gi, g, args, rank))
            self.units = sum(x["batch"] * x["k"] for x in self.groups)

    def _prepare_group(self, gi, g, args, rank):
        torch, F, ctx, dev, wl = self.torch, self.F, self.ctx, self.dev, self.wl
        ps = S.param_set(g.set_name)
        sid = ctx.register(ps)
        prime = is_prime_set(ps)
        kr = S.q_key_randomness(ps, wl.seed) if prime else S.key_randomness(ps, wl.seed)
        ctx.keys_generate(sid, kr)
        fs = (S.q_lut_tables if prime else S.lut_tables)(ps, wl.seed, g.n_luts, gi)
        for f in fs:
            ctx.lut_setup(sid, f)
        if g.mode == "tfhe":
            polys = (S.q_tfhe_polynomials if prime else S.tfhe_polynomials)(ps, wl.seed, g.n_luts)
            for poly in polys:
                ctx.tfhe_poly_setup(sid, poly)
        ids_np = S.lut_assignment(wl.seed, g.batch, g.n_luts, g.lut_assign, gi)
        mr = rank_messages(ps, wl.seed, g.batch, rank, gi)
        s_d = torch.tensor(kr.s, device=dev)
        ct = torch.empty((g.batch, ps.n + 1), dtype=F.word_torch(ps), device=dev)
        ctx.lwe_encrypt(sid, s_d, F.to_device_words(ps, mr.a, dev), torch.tensor(mr.e, device=dev),
                        torch.tensor(mr.m, device=dev), ct)
        ids = torch.tensor(ids_np, dtype=torch.int32, device=dev)
        if args.variant is not None:
            ctx.set_variant(sid, args.variant)
            cur, cnt, cpt = ctx.variant_info(sid)
            self.tuned[ps.name] = {"variant": cur, "of": cnt, "coeffs_per_thread": cpt, "fixed": True}
        elif not args.no_autotune:
            v, tms, each = ctx.autotune(sid, g.batch, each=True)
            cur, cnt, cpt = ctx.variant_info(sid)
            self.tuned[ps.name] = {"variant": v, "of": cnt, "coeffs_per_thread": cpt,
                                   "trial_blind_rotation_ms": [round(x, 3) for x in each],
                                   "chunks": ctx.get_chunks(sid)}
        k = g.tables_per_input
        if k > 1:
            want = np.array([[fs[i][m] for i in row] for row, m in zip(ids_np, mr.m)]).reshape(-1)
            out = torch.empty((g.batch, k, ps.n + 1), dtype=ct.dtype, device=dev)
        else:
            want = np.array([fs[i][m] for i, m in zip(ids_np, mr.m)])
            out = torch.empty_like(ct)
        return {"sid": sid, "ps": ps, "batch": g.batch, "k": k, "ct": ct, "ids": ids, "out": out,
                "s": s_d, "want": want, "mode": g.mode, "lboot": ps.lboot if prime else 1}

    def _prepare_mlp(self, args, rank):
        from paper_2109_02731_gb300 import mlp
        torch, F, ctx, dev, wl = self.torch, self.F, self.ctx, self.dev, self.wl
        ps = S.PARAM_SETS[wl.groups[0].set_name]
        sid = ctx.register(ps)
        kr = S.key_randomness(ps, wl.seed)
        ctx.keys_generate(sid, kr)
        x, Ws = S.mlp_inputs_and_weights(wl.seed, wl.mlp_layers, wl.mlp_inputs)
        self.net = mlp.EncryptedMLP(ctx, sid, Ws)
        mr = S.message_randomness(ps, wl.seed, x.size, group=rank, m=x.reshape(-1))
        s_d = torch.tensor(kr.s, device=dev)
        ct = torch.empty((x.size, ps.n + 1), dtype=F.word_torch(ps), device=dev)
        ctx.lwe_encrypt(sid, s_d, F.to_device_words(ps, mr.a, dev), torch.tensor(mr.e, device=dev),
                        torch.tensor(mr.m, device=dev), ct)
        if not args.no_autotune:
            v, tms = ctx.autotune(sid, wl.mlp_inputs * wl.mlp_layers[1])
            cur, cnt, cpt = ctx.variant_info(sid)
            self.tuned[ps.name] = {"variant": v, "of": cnt, "coeffs_per_thread": cpt,
                                   "trial_blind_rotation_ms": tms}
        self.mlp_x = ct.view(x.shape[0], x.shape[1], ps.n + 1)
        self.mlp_want = mlp.plain_forward(x, Ws, ps.t)
        self.groups.append({"sid": sid, "ps": ps, "batch": x.size, "k": 1, "ct": ct, "s": s_d})
        self.units = wl.mlp_inputs * sum(wl.mlp_layers[1:])
        self.mlp_batches = [wl.mlp_inputs * k for k in wl.mlp_layers[1:]]

    def step(self, groups=None):
        gs = groups or self.groups
        if self.wl.mlp_layers:
            self.mlp_out = self.net.forward(self.mlp_x)
        elif len(gs) == 1:
            g = gs[0]
            if g.get("mode") == "tfhe":
                self.ctx.tfhe_bootstrap(g["sid"], g["ct"], g["ids"], g["out"])
            elif g["k"] > 1:
                self.ctx.bootstrap_multi(g["sid"], g["ct"], g["ids"], g["out"])
            else:
                self.ctx.bootstrap(g["sid"], g["ct"], g["ids"], g["out"])
        else:
            self.ctx.bootstrap_mixed([(g["sid"], g["ct"], g["ids"], g["out"]) for g in gs])

    def decrypt_ok(self):
        torch, ctx = self.torch, self.ctx
        if self.wl.mlp_layers:
            g = self.groups[0]
            out = self.mlp_out.reshape(-1, g["ps"].n + 1)
            m = torch.empty(out.shape[0], dtype=torch.int32, device=self.dev)
            ctx.lwe_decrypt(g["sid"], g["s"], out, m)
            ctx.sync()
            return float((m.cpu().numpy().reshape(self.mlp_want.shape) == self.mlp_want).mean())
        ok = {}
        if any(g.get("mode") == "tfhe" for g in self.groups):
            return None  # uniform test polynomials: no function to check against
        for g in self.groups:
            m = torch.empty(g["batch"] * g["k"], dtype=torch.int32, device=self.dev)
            ctx.lwe_decrypt(g["sid"], g["s"], g["out"].view(-1, g["ps"].n + 1), m)
            ctx.sync()
            ok[g["ps"].name] = float((m.cpu().numpy() == g["want"]).mean())
        return ok if len(ok) > 1 else next(iter(ok.values()))

    def slots_per_step(self):
        if self.wl.mlp_layers:
            ps = self.groups[0]["ps"]
            return 2 * sum(br_algorithmic_slots(ps, b) for b in self.mlp_batches)
        # one sign rotation per input, one function rotation per (input, table);
        # the TFHE bootstrap has the function rotation only
        # (prime-modulus sets: l_boot sign rotations per input)
        return sum((0 if g.get("mode") == "tfhe" else br_algorithmic_slots(g["ps"], g["batch"] * g.get("lboot", 1)))
                   + br_algorithmic_slots(g["ps"], g["batch"] * g["k"]) for g in self.groups)

    def io_bytes(self):
        if self.wl.mlp_layers:
            g = self.groups[0]
            return (g["ct"].numel() * g["ct"].element_size(),
                    self.mlp_want.size * (g["ps"].n + 1) * g["ct"].element_size())
        h2d = sum(g["ct"].numel() * g["ct"].element_size() + g["ids"].numel() * 4 for g in self.groups)
        d2h = sum(g["out"].numel() * g["out"].element_size() for g in self.groups)
        return h2d, d2h

    def launches_per_step(self):
        """Kernel launches of one step: 5 per pipeline (sign rotation, packing
        key switch, PubMux, function rotation, LWE key switch), one pipeline per
        chunk of a single-set call; plus one affine launch per MLP layer."""
        def pipelines(g, batch):
            c = self.ctx.get_chunks(g["sid"])
            return c if (len(self.groups) == 1 and batch >= 2 * c) else 1
        if self.wl.mlp_layers:
            g = self.groups[0]
            return sum(1 + 5 * pipelines(g, b) for b in self.mlp_batches)
        if any(g.get("mode") == "tfhe" for g in self.groups):
            # accumulator, blind rotation, key switch (+ its finalize kernel mod Q)
            return sum(4 if is_prime_set(g["ps"]) else 3 for g in self.groups)
        # prime-modulus sets: each key switch is a sum kernel and a finalize kernel
        return sum((7 if is_prime_set(g["ps"]) else 5) * pipelines(g, g["batch"]) for g in self.groups)


def config_for(job, args):
    wl = job.wl
    if wl.mlp_layers:
        ps = job.groups[0]["ps"]
        return {"workload": f"{wl.name}: encrypted MLP {'->'.join(map(str, wl.mlp_layers))}, "
                            f"{wl.mlp_inputs} inputs, FDFB set {ps.name} (n={ps.n} N={ps.N} q=2^{ps.w} "
                            f"t={ps.t}); unit = bootstraps ({job.units} per step)",
                "param_set": ps.name, "seed": wl.seed,
                "l2": "flushed before every timed step (512 MB write, not timed)"}
    if len(job.groups) == 1:
        g = wl.groups[0]
        if args.batch is not None:
            g = dataclasses.replace(g, batch=args.batch)
        ps = S.param_set(g.set_name)
        return config_of(args, wl, g, ps)
    return {"workload": f"{wl.name}: " + ", ".join(
                f"set {g['ps'].name} (N={g['ps'].N} q=2^{g['ps'].w} t={g['ps'].t}) x {g['batch']}"
                for g in job.groups) + " in one fdfb_bootstrap_mixed call per step",
            "batch_per_gpu": job.units, "seed": wl.seed,
            "l2": "flushed before every timed step (512 MB write, not timed)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tfhe_scale", choices=sorted(S.WORKLOADS))
    ap.add_argument("--batch", type=int, default=None,
                    help="override the batch of a single-group workload (a smaller case for profiling; "
                         "not the workload's benchmark configuration)")
    ap.add_argument("--ref-sample", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--variant", type=int, default=None,
                    help="use this blind-rotation layout variant instead of autotuning")
    ap.add_argument("--no-plain", dest="plain", action="store_false",
                    help="skip timing the plain path (one ciphertext per bootstrap call, rank 0)")
    ap.add_argument("--plain", dest="plain", action="store_true", help=argparse.SUPPRESS)
    ap.set_defaults(plain=True)
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

    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    ctx = F.Context(dev.index)
    job = Job(torch, F, ctx, dev, args, rank)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        job.step()
    ctx.sync()
    decrypt_ok = job.decrypt_ok()

    clk_path = os.path.join(tempfile.gettempdir(), f"fdfb_clocks_{os.getpid()}.csv")
    proc, fh = sample_clocks(clk_path)
    time.sleep(0.3)
    ctx.profile_enable(True)
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        job.step()
        ev[k][1].record(stream)
    barrier()
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    ms_total = float(sum(a.elapsed_time(b) for a, b in ev))

    # End to end through the public API with host buffers: the step's inputs
    # go host -> device from pinned memory, the outputs come back.
    host_in = [(g["ct"].cpu().pin_memory(), g["ids"].cpu().pin_memory() if "ids" in g else None)
               for g in job.groups]
    dev_in = [(torch.empty_like(g["ct"]), torch.empty_like(g["ids"]) if "ids" in g else None)
              for g in job.groups]
    e2e_groups = []
    for g, (c, i) in zip(job.groups, dev_in):
        e2 = dict(g)
        e2["ct"] = c
        if i is not None:
            e2["ids"] = i
        e2["out"] = torch.empty_like(g["out"]) if "out" in g else None
        e2e_groups.append(e2)
    out_host = [torch.empty((g["out"] if "out" in g else g["ct"]).shape, dtype=g["ct"].dtype).pin_memory()
                for g in job.groups]
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_ms = 0.0
    for k in range(max(1, args.steps)):
        flush.zero_()
        e0.record(stream)
        for (hc, hi), (dc, di) in zip(host_in, dev_in):
            dc.copy_(hc, non_blocking=True)
            if hi is not None:
                di.copy_(hi, non_blocking=True)
        if job.wl.mlp_layers:
            saved = job.mlp_x
            job.mlp_x = dev_in[0][0].view(saved.shape)
            job.step()
            job.mlp_x = saved
            res = job.mlp_out.reshape(-1)
            out_host[0].view(-1)[: res.numel()].copy_(res, non_blocking=True)
        else:
            job.step(e2e_groups)
            for oh, g in zip(out_host, e2e_groups):
                oh.copy_(g["out"], non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
    barrier()
    if proc is not None:
        proc.terminate()
        proc.wait()
        fh.close()
    clocks = read_clocks(clk_path, dev.index)

    if world > 1:
        ms_total, e2e_ms = slowest_rank([ms_total, e2e_ms], dev)

    plain = None
    if (args.plain and rank == 0 and not job.wl.mlp_layers and len(job.groups) == 1
            and job.groups[0]["k"] == 1 and job.groups[0].get("mode") != "tfhe"):
        reps = 8
        g = job.groups[0]
        one_ct, one_id, one_out = g["ct"][:1].clone(), g["ids"][:1].clone(), g["out"][:1].clone()
        ctx.bootstrap(g["sid"], one_ct, one_id, one_out)
        torch.cuda.synchronize()  # rank 0 only: no collective here
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(reps):
            ctx.bootstrap(g["sid"], one_ct, one_id, one_out)
        p1.record(stream)
        p1.synchronize()
        plain = {"value": reps / (p0.elapsed_time(p1) / 1e3), "unit": UNIT,
                 "what": f"one ciphertext per bootstrap call, set {g['ps'].name}, same kernels"}

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    units = job.units * args.steps * world
    value = units / (ms_total / 1e3)
    # wall time with at least one blind-rotation launch in flight (the
    # launches of the chunks of one call overlap on different streams)
    br_ms = prof["blind_rotate_union"][0]
    br_n = prof["blind_rotate_sign"][1] + prof["blind_rotate_func"][1]
    slots = job.slots_per_step() * args.steps
    peak = SMS * IMAD_LANES_PER_SM * SM_MAX_GHZ * 1e9 / 1e12  # T slots/s
    achieved = slots / (br_ms / 1e3) / 1e12
    stages = {k: v for k, v in prof.items() if k != "blind_rotate_union"}
    chunked = any(ctx.get_chunks(g["sid"]) > 1 for g in job.groups) and len(job.groups) == 1
    # launches of different stages overlap when a call is chunked, so their
    # summed durations no longer give shares (a serialised ncu launch list does)
    stage_share = None if chunked else {
        k: round(v[0] / max(1e-9, sum(x[0] for x in stages.values())), 4) for k, v in stages.items()}
    h2d, d2h = job.io_bytes()
    ps0 = job.groups[0]["ps"]
    traffic, traffic_src = None, None
    if len(job.groups) == 1 and not job.wl.mlp_layers and job.groups[0]["k"] == 1:
        g0 = job.groups[0]
        key = (ps0.name, ctx.variant_info(g0["sid"])[0], g0["batch"])
        if key in KERNEL_TRAFFIC:
            traffic = KERNEL_TRAFFIC[key]
            traffic_src = ("dram bytes per unchunked blind-rotation launch over the batch, "
                           f"ncu capture of set {key[0]} variant {key[1]}, {key[2]} ciphertexts")
            if key in KERNEL_TRAFFIC_SCALED:
                traffic_src = "dram bytes per " + KERNEL_TRAFFIC_SCALED[key] + f", set {key[0]} variant {key[1]}"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "u32" if all(getattr(g["ps"], "w", 64) == 32 for g in job.groups) else "u64",
        "data": "synthetic (seeded SplitMix64 keys, messages and tables; keys generated on the GPU)",
        "config": config_for(job, args),
        "decrypt_ok": decrypt_ok,
        "roofline": {"bound": "alu", "kernel": "blind_rotate_kernel", "achieved": achieved, "peak": peak,
                     "unit": "T IMAD slots/s", "frac": achieved / peak,
                     "traffic": traffic, "traffic_source": traffic_src,
                     "peak_source": "derived: 152 SMs x 64 IMAD lanes/clock x 2.07 GHz",
                     "br_ms_per_step": br_ms / args.steps, "launches": br_n,
                     "slots_per_step": job.slots_per_step()},
        "stage_share": stage_share,
        "autotune": job.tuned,
        "gpu_launches": job.launches_per_step() * args.steps,
        "e2e": {"value": units / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "clocks": clocks,
    }
    probe = probe_rates(dev.index)
    if probe:
        line["roofline"]["probe"] = probe
    if plain:
        line["plain_path"] = plain
        line["batched_over_plain"] = value / plain["value"]
    if is_prime_set(ps0) and ps0.name in PAPER_MS_PER_BOOTSTRAP:
        ms = PAPER_MS_PER_BOOTSTRAP[ps0.name]
        line["paper_context"] = {"ms_per_bootstrap": ms, "bootstraps_per_s": 1e3 / ms,
                                 "source": "Table 3 (one bootstrap, not parallelised; 60-core Xeon "
                                           "Cascade Lake VM, 64-bit prime-modulus NTT)"}
    if world == 1 and not args.no_cpu_baseline and len(job.groups) == 1 and not job.wl.mlp_layers:
        g = job.wl.groups[0]
        line["cpu_baseline"] = cpu_baseline(job.wl, g, S.param_set(g.set_name))
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
