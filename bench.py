#!/usr/bin/env python3
"""FDFB throughput benchmark: full-domain functional bootstraps per second.

One step = one call of the library's batched bootstrap over the workload's
batch: ModSwitch, sign blind rotation, SampleExtract, packing key switch,
PubMux, function blind rotation, SampleExtract and LWE key switch, for every
ciphertext.  Keys, tables and ciphertexts are made on the GPU from seeded
synthetic randomness before timing (inputs resident in HBM); L2 is flushed
by a 512 MB write before every timed step and the flush is not timed.

The default workload is large_t: n = 744, N = 4096, q = 2^64, t = 64, 4096
ciphertexts with 16 tables, the largest single-GPU configuration.  Its line
also carries `target_n2048`: the N = 2048, q = 2^64 set on 1000 ciphertexts,
batched and one ciphertext per call (the plain path), with its own roofline.

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
                          "FDFB-100-7": 13781.0, "FDFB-80-8": 33117.0, "FDFB-100-8": 45266.0,
                          "TFHE-100-7": 7757.0, "TFHE-80-2": 306.0,
                          "TFHE-100-2": 321.0}


# DRAM bytes (read + write) of one blind-rotation launch, from ncu
# (dram__bytes_read.sum + dram__bytes_write.sum) on the current kernel, keyed
# by (set, variant): (bytes per wave of resident CTAs, CTAs per wave, what was
# captured).  The transform-domain key streams from DRAM about once per wave,
# so a launch over `items` CTAs moves bytes_per_wave * ceil(items / per_wave).
KERNEL_TRAFFIC = {
    # set C (large_t), variant 4, one CTA per SM: a 152-item capture (one wave)
    ("C", 4): (785.489e6 + 3.880e6, 152, "ncu capture of a 152-item sign rotation (one wave), set C"),
    # set D (target_n2048), variant 9, one CTA per SM: a 152-item capture
    ("D", 9): (294.640e6 + 3.286e6, 152, "ncu capture of a 152-item sign rotation (one wave), set D"),
    # set D, variant 6 (the autotuner's other near-tie): a 1000-item capture
    # (seven waves) read 3.198 GB
    ("D", 6): (3.19754e9 / 7, 152, "ncu capture of a 1000-item sign rotation (7 waves), set D"),
    # FDFB-80-6 sign rotation (variant 3, one CTA per SM): a 384-item capture
    # (three waves) read 1.2074 GB
    ("FDFB-80-6", 3): (1.2074e9 / 3, 152, "ncu capture of a 384-item sign rotation (3 waves), FDFB-80-6"),
    # FDFB-80-8 (N = 2^13, variant 0): a 152-item capture of the small-case
    # driver with n = 64 steps read 302 MB and wrote 5.04 GB; both grow with
    # the steps (key rows and the items' scratch, once per step), so a wave
    # of n = 700 steps moves 700 / 64 of that
    ("FDFB-80-8", 0): ((301.879e6 + 5042.725e6) * 700 / 64, 152,
                       "ncu capture of a 152-item, 64-step sign rotation (probe/n13_rotate.cu), scaled to 700 steps"),
}


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


def br_algorithmic_ops(ps, batch: int):
    """The blind rotation's modular operations per launch over `batch` items
    (n CMux steps each, figure "Blind Rotation and its setup"; extProd of
    Definition "External Product" as exact NTT products over P primes):
    forward butterflies of the 2l digit polynomials, inverse butterflies of
    the 2 output columns, and the 4 l N P pointwise key products.  P = 2
    30-bit primes lift a q = 2^32 product exactly, P = 3 a q = 2^64 or
    prime-Q one."""
    P = 2 if getattr(ps, "w", 64) == 32 else 3
    per_tf = (ps.N // 2) * ps.logN * P
    f = float(batch) * ps.n
    return {"fwd_butterflies": f * 2 * ps.lg * per_tf, "inv_butterflies": f * 2 * per_tf,
            "key_products": f * 4 * ps.lg * ps.N * P}


def opmix_roofline(parts, br_ms: float, probe):
    """Roofline of the blind rotation against the measured rates of its own
    operations (probe): the time the method's butterflies and products need at
    the GPU's rate for each, T_alg = F / R_fwd + I / R_inv + M / R_mac, over
    the measured time.  `parts` lists (parameter set, rotations) -- several
    sets for a mixed call.  Forward butterflies take the faster of the two
    forward forms the kernels use (Harvey's, and for q = 2^32 the lazy
    family's), so the peak is the higher one."""
    F = I = M = t_alg = 0.0
    for ps, batch_items in parts:
        ops = br_algorithmic_ops(ps, 1)
        f, i, m = (ops[k] * batch_items for k in ("fwd_butterflies", "inv_butterflies", "key_products"))
        r_fwd = probe["fwd_butterfly"]
        if getattr(ps, "w", 64) == 32:
            r_fwd = max(r_fwd, probe["lazy_fwd_butterfly"])
        t_alg += f / (r_fwd * 1e12) + i / (probe["inv_butterfly"] * 1e12) + m / (probe["mac64"] * 1e12)
        F, I, M = F + f, I + i, M + m
    total = F + I + M
    peak = total / t_alg / 1e12
    achieved = total / (br_ms / 1e3) / 1e12
    kernel = "blind_rotate_n13_kernel" if any(ps.N == 8192 for ps, _ in parts) else "blind_rotate_kernel"
    return {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak,
            "unit": "T modular ops/s (butterflies + key products)", "frac": achieved / peak,
            "peak_source": "measured in this run: probe of the kernels' own forward and inverse butterflies "
                           "and 32x32->64 key products at full occupancy (probe/int_pipe.cu), combined in the "
                           "method's proportions",
            "ops_per_launch_set": {"fwd_butterflies": F, "inv_butterflies": I, "key_products": M}}


def slot_roofline(slots: float, br_ms: float):
    """The stricter derived roofline: the method's multiplier slots (every
    Shoup product 4 slots, every key product 2) against 152 SMs x 64 integer
    multiply lanes x 2.07 GHz, which leaves out the additions and minimums of
    each butterfly (they issue on the separate ALU pipe)."""
    peak = SMS * IMAD_LANES_PER_SM * SM_MAX_GHZ * 1e9 / 1e12
    achieved = slots / (br_ms / 1e3) / 1e12
    return {"achieved": achieved, "peak": peak, "unit": "T IMAD slots/s", "frac": achieved / peak,
            "peak_source": "derived: 152 SMs x 64 IMAD lanes/clock x 2.07 GHz"}


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


PROBE_KEYS = ("imad", "imad_hi", "lop", "fwd_butterfly", "inv_butterfly", "lazy_fwd_butterfly", "mac64",
              "fp64_flops", "int8_tensor_ops")


def probe_rates(dev_index: int):
    """Measured rates of this GPU's pipes (T ops/s) from
    paper_2109_02731_gb300/probe/int_pipe.cu: single integer instructions,
    the blind rotation's butterflies and key products, FP64 fused
    multiply-adds and 8-bit integer tensor products."""
    import ctypes
    from paper_2109_02731_gb300 import build as B
    try:
        lib = ctypes.CDLL(B.build_probe())
        n = lib.probe_pipe_count()
        rates = (ctypes.c_double * n)()
        rc = lib.probe_pipe_rates(dev_index, rates)
        if rc != 0:
            return {"error": f"probe returned {rc}"}
        out = {k: rates[i] / 1e12 for i, k in enumerate(PROBE_KEYS)}
        out["unit"] = "T/s (fp64_flops: T flop/s; int8_tensor_ops: T op/s, mma.sync m16n8k32)"
        return out
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
    any values.  Returns (seconds per bootstrap, description, seconds the
    sample itself took)."""
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
    measured = t1 + (t_step * steps if steps > 1 else 0.0)
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
    measured += t_pk + t_ks + t_pm
    if tfhe:  # the TFHE bootstrap: one rotation and the LWE key switch
        sec = n * t_step + t_ks
        desc = (f"{steps} full-size CMux step(s) ({t_step:.2f} s each, x {n} per TFHE bootstrap) and the "
                f"LWE key switch ({t_ks:.2f} s) of the schoolbook oracle on one core, scaled to one "
                f"bootstrap ({sec / 60:.1f} min)")
        return sec, desc, measured
    sec = (lb + 1) * n * t_step + lb * t_pk + t_pm + t_ks
    desc = (f"{steps} full-size CMux step(s) ({t_step:.2f} s each, x {(lb + 1) * n} per bootstrap), one "
            f"packing key switch ({t_pk:.2f} s, x {lb}), PubMux ({t_pm:.2f} s) and the LWE key switch "
            f"({t_ks:.2f} s) of the schoolbook oracle on one core, scaled to one bootstrap "
            f"({sec / 3600:.2f} h)")
    return sec, desc, measured


def p2_oracle_sample(ps, seconds_target: float = 10.0):
    """The power-of-two oracle's time per bootstrap from a bounded sample, for
    sets whose single bootstrap takes the schoolbook oracle longer than a
    benchmark step should (2 n CMux steps of 2 (2 l) N^2 word products each):
    whole full-size CMux steps of the blind rotation (the oracle's ring
    products spread over every host core), one packing key switch, PubMux and
    the LWE key switch, each scaled by its count per bootstrap.  Key material
    of the right shapes is drawn uniformly without key generation: the
    products cost the same for any values.  Returns (seconds per bootstrap,
    description, cores, seconds the sample itself took)."""
    import oracle as O
    cores = O.max_threads()
    O.set_threads(cores)
    rng = np.random.default_rng(0)
    N, n, lg, w = ps.N, ps.n, ps.lg, ps.w
    uni = lambda *shape: (rng.integers(0, 2 ** 63, shape, dtype=np.uint64) * np.uint64(2)
                          + rng.integers(0, 2, shape, dtype=np.uint64)) >> np.uint64(64 - w)

    measured = [0.0]

    def cmux_steps(steps):
        pset = dataclasses.replace(ps, n=steps)
        ctN = np.zeros(steps + 1, dtype=np.uint64)
        ctN[1:] = 1 + np.arange(steps)  # nonzero masks: no step is skipped
        bsk, acc = uni(steps, 2 * lg, 2, N), uni(2, N)
        t0 = time.perf_counter()
        O.blind_rotate(pset, bsk, acc, ctN)
        dt = time.perf_counter() - t0
        measured[0] += dt
        return dt / steps

    t1 = cmux_steps(1)
    steps = int(min(16, max(1, seconds_target * 0.6 / max(t1, 1e-3))))
    t_step = cmux_steps(steps) if steps > 1 else t1
    # the key switches' cost is linear in the input dimension: time them on
    # the first N / 8 input words and scale by 8 (keeps the key material small)
    sub = max(1, N // 8)
    lwe = uni(sub + 1)
    pk = uni(sub, ps.lpk, 2, N)
    t0 = time.perf_counter()
    O.keyswitch(w, ps.log2Bpk, ps.lpk, pk, lwe)
    t_pk = time.perf_counter() - t0
    del pk
    ksk = uni(sub, ps.lks, n + 1)
    t0 = time.perf_counter()
    O.keyswitch(w, ps.log2Bks, ps.lks, ksk, lwe)
    t_ks = time.perf_counter() - t0
    cR = uni(2, N)
    p0 = rng.integers(0, ps.t, N)
    t0 = time.perf_counter()
    O.pubmux(w, ps.t, cR, p0, (p0 + 1) % ps.t)
    t_pm = time.perf_counter() - t0
    measured[0] += t_pk + t_ks + t_pm
    t_pk, t_ks = t_pk * N / sub, t_ks * N / sub
    sec = 2 * n * t_step + t_pk + t_pm + t_ks
    desc = (f"{steps} full-size CMux step(s) ({t_step * 1e3:.1f} ms each, x {2 * n} per bootstrap), the "
            f"packing key switch ({t_pk:.2f} s) and the LWE key switch ({t_ks:.2f} s) timed on {sub} of the "
            f"{N} input words and scaled by {N // sub}, and PubMux ({t_pm:.3f} s), of the schoolbook oracle "
            f"with its ring products spread over {cores} threads, scaled to one bootstrap ({sec:.1f} s)")
    return sec, desc, cores, measured[0]


def oracle_bootstrap_macs(ps) -> float:
    """Schoolbook word products of one bootstrap: 2 n CMux steps of 2 (2 l)
    N^2, plus the packing key switch's N l_pk 2N."""
    return 2.0 * ps.n * 2 * (2 * ps.lg) * ps.N ** 2 + ps.N * ps.lpk * 2.0 * ps.N


# Above this many word products a whole bootstrap takes the oracle longer than
# a benchmark step should (set B, 1.6e10, takes about half a second on 16
# cores); larger sets are timed by p2_oracle_sample.
ORACLE_WHOLE_LIMIT = 3e10


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
        units, walls = [], []
        desc = ""
        for _ in range(args.steps):
            sec, desc, wall = q_oracle_sample(ps, tfhe=tf)
            units.append(wall / sec)  # the fraction of one bootstrap the sample did
            walls.append(wall)
        value = sum(units) / sum(walls)
        line = {
            "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(walls) / args.steps,
            "units_per_step": sum(units) / args.steps,
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
    if g.mode == "fdfb" and g.tables_per_input == 1 and oracle_bootstrap_macs(ps) > ORACLE_WHOLE_LIMIT:
        for _ in range(args.warmup):
            p2_oracle_sample(ps, seconds_target=3.0)
        units, walls = [], []
        desc, cores = "", 1
        for _ in range(args.steps):
            sec, desc, cores, wall = p2_oracle_sample(ps, seconds_target=3.0)
            units.append(wall / sec)  # the fraction of one bootstrap the sample did
            walls.append(wall)
        value = sum(units) / sum(walls)
        line = {
            "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(walls) / args.steps,
            "units_per_step": sum(units) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32" if ps.w == 32 else "u64",
            "data": "synthetic (seeded key-shaped words, no key generation: the oracle's cost does not "
                    "depend on the values)",
            "config": config_of(args, wl, g, ps),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
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
        sec, desc, _ = q_oracle_sample(ps, tfhe=g.mode == "tfhe")
        return {"value": 1.0 / sec, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc}
    if g.mode == "fdfb" and g.tables_per_input == 1 and oracle_bootstrap_macs(ps) > ORACLE_WHOLE_LIMIT:
        sec, desc, cores, _ = p2_oracle_sample(ps, seconds_target=seconds_target)
        return {"value": 1.0 / sec, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}
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

    def __init__(self, torch, F, ctx, dev, args, rank, workload=None, batch=None):
        self.torch, self.F, self.ctx, self.dev = torch, F, ctx, dev
        wl = S.WORKLOADS[workload or args.workload]
        self.wl = wl
        self.groups = []
        self.tuned = {}
        if batch is None and workload is None:
            batch = args.batch
        if wl.mlp_layers:
            self._prepare_mlp(args, rank)
        else:
            for gi, g in enumerate(wl.groups):
                if batch is not None and len(wl.groups) == 1:
                    g = dataclasses.replace(g, batch=batch)  # smaller case, e.g. for ncu
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
        if ps.name in self.tuned:
            pk_path, ksk_path = ctx.keyswitch_path(sid)
            self.tuned[ps.name]["keyswitch"] = {
                "packing": "tensor cores (tcgen05)" if pk_path else "CUDA cores",
                "lwe": "tensor cores (tcgen05)" if ksk_path else "CUDA cores"}
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

    def br_items_by_set(self):
        """[(parameter set, blind rotations per step)]: sign and function
        rotations, each n CMux steps."""
        if self.wl.mlp_layers:
            return [(self.groups[0]["ps"], 2 * sum(self.mlp_batches))]
        return [(g["ps"], (0 if g.get("mode") == "tfhe" else g["batch"] * g.get("lboot", 1)) + g["batch"] * g["k"])
                for g in self.groups]

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


def timed_steps(torch, ctx, job, stream, flush, steps, barrier):
    """Times `steps` steps of `job` with CUDA events on the launching stream,
    L2 flushed (not timed) before each; returns (total ms, profile)."""
    ctx.profile_enable(True)
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        job.step()
        ev[k][1].record(stream)
    barrier()
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    return float(sum(a.elapsed_time(b) for a, b in ev)), prof


def time_plain(torch, ctx, job, stream, reps=8):
    """The plain path: one ciphertext per bootstrap call, the same kernels."""
    g = job.groups[0]
    one_ct, one_id, one_out = g["ct"][:1].clone(), g["ids"][:1].clone(), g["out"][:1].clone()
    ctx.bootstrap(g["sid"], one_ct, one_id, one_out)
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(reps):
        ctx.bootstrap(g["sid"], one_ct, one_id, one_out)
    p1.record(stream)
    p1.synchronize()
    return {"value": reps / (p0.elapsed_time(p1) / 1e3), "unit": UNIT,
            "what": f"one ciphertext per bootstrap call, set {g['ps'].name}, same kernels ({reps} calls)"}


def rooflines(job, prof, steps, probe):
    """The op-mix roofline (measured peak) and the slot roofline (derived) of
    the blind rotation launches of `steps` steps of `job`."""
    br_ms = prof["blind_rotate_union"][0]
    out = None
    if probe and "error" not in probe:
        out = opmix_roofline([(ps, n * steps) for ps, n in job.br_items_by_set()], br_ms, probe)
    slots = slot_roofline(job.slots_per_step() * steps, br_ms)
    if out is None:
        out = {"bound": "alu", "kernel": "blind_rotate_kernel", **slots}
        slots = None
    out["br_ms_per_step"] = br_ms / steps
    out["launches"] = prof["blind_rotate_sign"][1] + prof["blind_rotate_func"][1]
    if slots is not None:
        out["slot_model"] = slots
    return out


def kernel_traffic(job, ctx):
    """DRAM bytes of one blind-rotation launch over the workload (sign
    rotation), from the ncu capture of the autotuned variant, or None."""
    if len(job.groups) != 1 or job.wl.mlp_layers or job.groups[0]["k"] != 1:
        return None, None
    g0 = job.groups[0]
    key = (g0["ps"].name, ctx.variant_info(g0["sid"])[0])
    if key not in KERNEL_TRAFFIC:
        return None, None
    per_wave, ctas, src = KERNEL_TRAFFIC[key]
    items = g0["batch"] * g0.get("lboot", 1)
    waves = -(-items // ctas)
    return per_wave * waves, (f"{src}: {per_wave / 1e6:.1f} MB per wave of {ctas} CTAs, x {waves} waves for "
                              f"the {items}-item launch, set {key[0]} variant {key[1]}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large_t", choices=sorted(S.WORKLOADS))
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
    ap.add_argument("--no-target", dest="target", action="store_false",
                    help="skip the N = 2048 target measurement that the large_t line carries")
    ap.set_defaults(plain=True, target=True)
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
    ms_total, prof = timed_steps(torch, ctx, job, stream, flush, args.steps, barrier)

    # End to end through the public API with host buffers: the step's inputs
    # go host -> device from pinned memory, the outputs come back.  Steps
    # longer than half a second are timed five times at most.
    e2e_steps = max(1, min(args.steps, 5 if ms_total / args.steps > 500 else args.steps))
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
    for k in range(e2e_steps):
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

    single = (not job.wl.mlp_layers and len(job.groups) == 1 and job.groups[0]["k"] == 1
              and job.groups[0].get("mode") != "tfhe")
    plain = time_plain(torch, ctx, job, stream) if (args.plain and rank == 0 and single) else None
    launches = job.launches_per_step() * args.steps
    probe = probe_rates(dev.index) if rank == 0 else None

    # The N = 2048 target (rank 0): batched and plain on the same GPU.
    target = None
    if rank == 0 and args.target and args.workload == "large_t" and args.batch is None:
        tjob = Job(torch, F, ctx, dev, args, rank, workload="n2048")
        for _ in range(3):
            tjob.step()
        ctx.sync()
        t_ok = tjob.decrypt_ok()
        t_steps = max(3, min(args.steps, 10))
        t_ms, t_prof = timed_steps(torch, ctx, tjob, stream, flush, t_steps, lambda: torch.cuda.synchronize())
        t_value = tjob.units * t_steps / (t_ms / 1e3)
        t_plain = time_plain(torch, ctx, tjob, stream)
        t_traffic, t_src = kernel_traffic(tjob, ctx)
        t_roof = rooflines(tjob, t_prof, t_steps, probe)
        t_roof["traffic"], t_roof["traffic_source"] = t_traffic, t_src
        target = {"workload": config_for(tjob, args)["workload"], "value": t_value, "unit": UNIT,
                  "steps": t_steps, "ms_per_step": t_ms / t_steps, "decrypt_ok": t_ok,
                  "plain_path": t_plain, "batched_over_plain": t_value / t_plain["value"],
                  "roofline": t_roof, "autotune": tjob.tuned,
                  "goal": "batched >= 10x plain and >= 0.5 of the roofline"}

    # The mixed workload (rank 0): three parameter sets in one call per step.
    mixed = None
    if rank == 0 and args.target and args.workload == "large_t" and args.batch is None:
        mjob = Job(torch, F, ctx, dev, args, rank, workload="mixed")
        for _ in range(2):
            mjob.step()
        ctx.sync()
        m_ok = mjob.decrypt_ok()
        m_steps = 3
        m_ms, m_prof = timed_steps(torch, ctx, mjob, stream, flush, m_steps, lambda: torch.cuda.synchronize())
        mixed = {"workload": config_for(mjob, args)["workload"], "value": mjob.units * m_steps / (m_ms / 1e3),
                 "unit": UNIT, "steps": m_steps, "ms_per_step": m_ms / m_steps, "decrypt_ok": m_ok,
                 "roofline": rooflines(mjob, m_prof, m_steps, probe), "autotune": mjob.tuned}

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    units = job.units * args.steps * world
    value = units / (ms_total / 1e3)
    stages = {k: v for k, v in prof.items() if k != "blind_rotate_union"}
    chunked = any(ctx.get_chunks(g["sid"]) > 1 for g in job.groups) and len(job.groups) == 1
    # launches of different stages overlap when a call is chunked, so their
    # summed durations no longer give shares (a serialised ncu launch list does)
    stage_share = None if chunked else {
        k: round(v[0] / max(1e-9, sum(x[0] for x in stages.values())), 4) for k, v in stages.items()}
    h2d, d2h = job.io_bytes()
    ps0 = job.groups[0]["ps"]
    roof = rooflines(job, prof, args.steps, probe)
    roof["traffic"], roof["traffic_source"] = kernel_traffic(job, ctx)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "u32" if all(getattr(g["ps"], "w", 64) == 32 for g in job.groups) else "u64",
        "data": "synthetic (seeded SplitMix64 keys, messages and tables; keys generated on the GPU)",
        "config": config_for(job, args),
        "decrypt_ok": decrypt_ok,
        "roofline": roof,
        "stage_share": stage_share,
        "autotune": job.tuned,
        "gpu_launches": launches,
        "e2e": {"value": job.units * e2e_steps * world / (e2e_ms / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "steps": e2e_steps},
        "clocks": clocks,
    }
    if probe:
        line["probe"] = probe
    if plain:
        line["plain_path"] = plain
        line["batched_over_plain"] = value / plain["value"]
    if target:
        line["target_n2048"] = target
    if mixed:
        line["mixed"] = mixed
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
