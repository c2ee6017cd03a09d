"""Shared set-up for the GPU parity tests: seeded inputs from the synthetic
generator, oracle keys and expected values, and a CUDA-library context with
the same keys installed."""
from __future__ import annotations

import functools

import numpy as np

from paper_2109_02731_gb300 import synth as S


@functools.lru_cache(maxsize=None)
def oracle_keys(set_name: str, seed: int):
    import oracle as O
    ps = S.PARAM_SETS[set_name]
    return O.Keys(ps, S.key_randomness(ps, seed))


@functools.lru_cache(maxsize=None)
def luts(set_name: str, seed: int, count: int, group: int = 0):
    import oracle as O
    ps = S.PARAM_SETS[set_name]
    fs = S.lut_tables(ps, seed, count, group)
    rot = np.stack([np.stack(O.setup_polynomial(ps.N, ps.t, f)) for f in fs])
    return fs, rot


def fresh_cts(set_name: str, seed: int, count: int, keys, group: int = 0, m=None):
    import oracle as O
    ps = S.PARAM_SETS[set_name]
    mr = S.message_randomness(ps, seed, count, group, m=m)
    return mr, O.encrypt_messages(ps, keys.s, mr)


def mask(ps):
    return np.uint64((1 << ps.w) - 1)
