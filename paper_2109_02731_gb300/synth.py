"""Seeded synthetic inputs for FDFB workloads: parameter sets, workload
definitions and random numbers.  Nothing here computes any part of the
bootstrapping method (no encryption, no products, no decomposition): this
module only draws the random numbers that key generation, encryption and the
workloads consume, so the CUDA library and the CPU oracle can be fed the very
same inputs.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): with a 64-bit state advanced
by the odd constant GAMMA, output i of a stream is MIX(state0 + (i+1)*GAMMA),
where MIX is the published variant-13 finaliser.  Every stream is counter
based, so any slice can be regenerated without the preceding ones, and the
bits are identical on every platform and numpy version.

Gaussian noise is the rounded continuous Gaussian e = floor(sigma*z + 1/2),
z drawn by the Box-Muller transform (Box and Muller, 1958) from two
independent 53-bit uniforms.  The paper leaves the sampler unspecified
(section "Parameters, Performance, and Tests" fixes only the standard
deviation); this is the reading taken.

Parameter sets follow the paper's notation (Table 1): n (LWE dimension),
N (ring degree), q = 2^w (q = Q here), gadget bases B_g = 2^log2Bg with
l_g digits for the bootstrapping key, B_ks/l_ks for the LWE key-switching
key, B_pk/l_pk for the LWE-to-RLWE packing key, plaintext modulus t and the
noise standard deviations.  QParamSet holds the paper's own sets, with a
prime RLWE modulus Q and the LWE side mod q = 2N.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_STREAM_MUL = np.uint64(0xD1B54A32D192ED03)


@dataclasses.dataclass(frozen=True)
class ParamSet:
    """One FDFB parameter set (k = 1, u = {1}, q = Q = 2^w)."""
    name: str
    n: int          # LWE dimension
    N: int          # ring degree, power of two
    w: int          # word bits, q = 2^w (32 or 64)
    t: int          # plaintext modulus, power of two
    log2Bg: int     # bootstrapping-key gadget base
    lg: int
    log2Bks: int    # LWE->LWE key-switching gadget base
    lks: int
    log2Bpk: int    # LWE->RLWE packing-key gadget base
    lpk: int
    sigma_lwe: float   # fresh LWE ciphertexts and the key-switching key
    sigma_glwe: float  # bootstrapping key and packing key
    signed_digits: bool = False  # balanced blind-rotation digits in [-B/2, B/2)
    t_out: int = 0               # output plaintext modulus t' of f: Z_t -> Z_t' (0: t' = t)

    @property
    def logN(self) -> int:
        return int(self.N).bit_length() - 1

    @property
    def word_dtype(self):
        return np.uint32 if self.w == 32 else np.uint64


# Sets A-C are the parameters of the toy, TFHE-scale and large-plaintext
# workloads.  Set D (N = 2048), the packing-key gadgets and the noise levels of
# the 2^64 sets are choices of this library where the workloads leave them
# open.  Z is the noiseless exact-decomposition set used for the exhaustive
# correctness pin.
PARAM_SETS: Dict[str, ParamSet] = {
    "A": ParamSet("A", n=64, N=256, w=32, t=4, log2Bg=8, lg=3, log2Bks=4, lks=5,
                  log2Bpk=8, lpk=3, sigma_lwe=2.0 ** 12, sigma_glwe=2.0 ** 7),
    "B": ParamSet("B", n=630, N=1024, w=32, t=16, log2Bg=7, lg=3, log2Bks=2, lks=8,
                  log2Bpk=7, lpk=3, sigma_lwe=2.0 ** 12, sigma_glwe=2.0 ** 7),
    "C": ParamSet("C", n=744, N=4096, w=64, t=64, log2Bg=10, lg=4, log2Bks=3, lks=10,
                  log2Bpk=10, lpk=4, sigma_lwe=2.0 ** 24, sigma_glwe=2.0 ** 14),
    "D": ParamSet("D", n=744, N=2048, w=64, t=32, log2Bg=10, lg=4, log2Bks=3, lks=10,
                  log2Bpk=10, lpk=4, sigma_lwe=2.0 ** 24, sigma_glwe=2.0 ** 14),
    "Z": ParamSet("Z", n=16, N=256, w=32, t=4, log2Bg=8, lg=4, log2Bks=4, lks=8,
                  log2Bpk=8, lpk=4, sigma_lwe=0.0, sigma_glwe=0.0),
}


@dataclasses.dataclass(frozen=True)
class Group:
    """A batch of ciphertexts under one parameter set."""
    set_name: str
    batch: int
    n_luts: int
    lut_assign: str   # "round_robin", "uniform", or "all" (every input, every table)
    tables_per_input: int = 1
    mode: str = "fdfb"   # "fdfb", or "tfhe" (plain TFHE bootstrap of a test polynomial)


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    seed: int
    groups: List[Group]
    mlp_layers: Optional[List[int]] = None   # config 5 only
    mlp_inputs: int = 0


# Workloads: workload k uses master seed k-1.
WORKLOADS: Dict[str, Workload] = {
    "toy": Workload("toy", 0, [Group("A", 16, 1, "round_robin")]),
    "tfhe_scale": Workload("tfhe_scale", 1, [Group("B", 1024, 4, "round_robin")]),
    "large_t": Workload("large_t", 2, [Group("C", 4096, 16, "uniform")]),
    "mixed": Workload("mixed", 3, [Group("B", 37, 4, "uniform"),
                                   Group("D", 1000, 4, "uniform"),
                                   Group("C", 2900, 4, "uniform")]),
    # the N = 2048 group of the mixed workload on its own
    "n2048": Workload("n2048", 3, [Group("D", 1000, 4, "uniform")]),
    # the TFHE-scale inputs, each evaluated under all four tables with one
    # shared sign rotation (several functions of one input)
    "multi_lut": Workload("multi_lut", 1, [Group("B", 1024, 4, "all", tables_per_input=4)]),
    # the TFHE-scale ciphertexts through the plain TFHE bootstrap (one blind
    # rotation of a test polynomial per ciphertext; negacyclic functions)
    "tfhe_plain": Workload("tfhe_plain", 1, [Group("B", 1024, 4, "round_robin", mode="tfhe")]),
    "mlp": Workload("mlp", 4, [Group("D", 0, 2, "uniform")],
                    mlp_layers=[784, 128, 64, 10], mlp_inputs=64),
    # the paper's own parameter sets (Table 1, prime Q), literal Bootstrap:
    # l_boot = 6 sign rotations and one function rotation per input
    "paper_80_6": Workload("paper_80_6", 5, [Group("FDFB-80-6", 1000, 4, "uniform")]),
    "paper_80_7": Workload("paper_80_7", 6, [Group("FDFB-80-7", 456, 4, "uniform")]),
    # N = 2^13 (split transforms): l_boot = 8 sign rotations per input
    "paper_80_8": Workload("paper_80_8", 8, [Group("FDFB-80-8", 152, 4, "uniform")]),
    "paper_100_8": Workload("paper_100_8", 9, [Group("FDFB-100-8", 152, 4, "uniform")]),
    # Table 1's TFHE:80:2 through the TFHE bootstrap (one rotation)
    "paper_tfhe_80_2": Workload("paper_tfhe_80_2", 7, [Group("TFHE-80-2", 1024, 4, "round_robin",
                                                             mode="tfhe")]),
}

# Sub-stream identifiers (xored into the master seed before mixing).
STREAM_KEYS = 1
STREAM_MESSAGES = 2
STREAM_LUTS = 3
STREAM_LUT_ASSIGN = 4
STREAM_MLP = 5


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Stream:
    """A SplitMix64 stream keyed by (master seed, path of stream ids)."""

    def __init__(self, seed: int, *path: int):
        with np.errstate(over="ignore"):
            s = _mix64(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))
            for p in path:
                s = _mix64(s ^ (np.uint64(p & 0xFFFFFFFFFFFFFFFF) * _STREAM_MUL))
        self.state0 = s[0]

    def sub(self, *path: int) -> "Stream":
        st = Stream.__new__(Stream)
        s = np.array([self.state0], dtype=np.uint64)
        with np.errstate(over="ignore"):
            for p in path:
                s = _mix64(s ^ (np.uint64(p & 0xFFFFFFFFFFFFFFFF) * _STREAM_MUL))
        st.state0 = s[0]
        return st

    def raw(self, count: int, start: int = 0) -> np.ndarray:
        """Outputs start .. start+count-1 of the stream as uint64."""
        out = np.empty(count, dtype=np.uint64)
        chunk = 1 << 22
        with np.errstate(over="ignore"):
            for lo in range(0, count, chunk):
                hi = min(count, lo + chunk)
                idx = np.arange(start + lo + 1, start + hi + 1, dtype=np.uint64)
                out[lo:hi] = _mix64(self.state0 + idx * GAMMA)
        return out

    def words(self, count: int, w: int) -> np.ndarray:
        """Uniform words of Z_{2^w}, dtype uint32 (w=32) or uint64 (w=64)."""
        r = self.raw(count)
        if w == 64:
            return r
        return (r >> np.uint64(64 - w)).astype(np.uint64 if w > 32 else np.uint32)

    def bits(self, count: int) -> np.ndarray:
        return (self.raw(count) >> np.uint64(63)).astype(np.uint8)

    def below(self, count: int, m: int) -> np.ndarray:
        """Integers uniform in [0, m) for m < 2^32 (multiply-high method)."""
        assert 0 < m < (1 << 32)
        r = self.raw(count) >> np.uint64(32)
        return ((r * np.uint64(m)) >> np.uint64(32)).astype(np.int64)

    def uniform01(self, count: int, start: int = 0) -> np.ndarray:
        """Doubles in (0, 1]: ((x >> 11) + 1) * 2^-53."""
        r = self.raw(count, start)
        return ((r >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)

    def gaussian(self, count: int, sigma: float) -> np.ndarray:
        """Rounded Gaussian integers floor(sigma*z + 1/2), int64."""
        if sigma == 0.0 or count == 0:
            return np.zeros(count, dtype=np.int64)
        out = np.empty(count, dtype=np.int64)
        chunk = 1 << 22
        for lo in range(0, count, chunk):
            hi = min(count, lo + chunk)
            u = self.uniform01(2 * (hi - lo), 2 * lo)
            u1, u2 = u[0::2], u[1::2]
            z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)
            out[lo:hi] = np.floor(sigma * z + 0.5).astype(np.int64)
        return out


@dataclasses.dataclass
class KeyRandomness:
    """Everything key generation draws, for one parameter set.

    s      : uint8[n]              binary LWE secret key
    sk     : uint8[N]              binary RLWE secret key (s_F = its coefficients)
    bsk_a  : word[n][2*lg][N]      uniform masks of the GGSW rows
    bsk_e  : int64[n][2*lg][N]     noise of the GGSW rows
    pk_a   : word[N][lpk][N]       uniform masks of the packing key
    pk_e   : int64[N][lpk][N]
    ksk_a  : word[N][lks][n]       uniform masks of the key-switching key
    ksk_e  : int64[N][lks]
    """
    s: np.ndarray
    sk: np.ndarray
    bsk_a: np.ndarray
    bsk_e: np.ndarray
    pk_a: np.ndarray
    pk_e: np.ndarray
    ksk_a: np.ndarray
    ksk_e: np.ndarray


def key_randomness(ps: ParamSet, seed: int) -> KeyRandomness:
    st = Stream(seed, STREAM_KEYS, hash_name(ps.name))
    n, N = ps.n, ps.N
    s = st.sub(1).bits(n)
    sk = st.sub(2).bits(N)
    bsk_a = st.sub(3).words(n * 2 * ps.lg * N, ps.w).reshape(n, 2 * ps.lg, N)
    bsk_e = st.sub(4).gaussian(n * 2 * ps.lg * N, ps.sigma_glwe).reshape(n, 2 * ps.lg, N)
    pk_a = st.sub(5).words(N * ps.lpk * N, ps.w).reshape(N, ps.lpk, N)
    pk_e = st.sub(6).gaussian(N * ps.lpk * N, ps.sigma_glwe).reshape(N, ps.lpk, N)
    ksk_a = st.sub(7).words(N * ps.lks * n, ps.w).reshape(N, ps.lks, n)
    ksk_e = st.sub(8).gaussian(N * ps.lks, ps.sigma_lwe).reshape(N, ps.lks)
    return KeyRandomness(s, sk, bsk_a, bsk_e, pk_a, pk_e, ksk_a, ksk_e)


def hash_name(name: str) -> int:
    h = 0
    for ch in name.encode():
        h = (h * 131 + ch) & 0xFFFFFFFF
    return h


@dataclasses.dataclass
class MessageRandomness:
    """Plaintexts and encryption randomness of a batch of fresh LWE ciphertexts.

    m : int64[count]        messages in Z_t
    a : word[count][n]      uniform masks
    e : int64[count]        noise
    """
    m: np.ndarray
    a: np.ndarray
    e: np.ndarray


def message_randomness(ps: ParamSet, seed: int, count: int, group: int = 0,
                       m: Optional[np.ndarray] = None) -> MessageRandomness:
    st = Stream(seed, STREAM_MESSAGES, hash_name(ps.name), group)
    if m is None:
        m = st.sub(1).below(count, ps.t)
    a = st.sub(2).words(count * ps.n, ps.w).reshape(count, ps.n)
    e = st.sub(3).gaussian(count, ps.sigma_lwe)
    return MessageRandomness(np.asarray(m, dtype=np.int64), a, e)


def lut_tables(ps: ParamSet, seed: int, count: int, group: int = 0) -> np.ndarray:
    """`count` random lookup tables f: Z_t -> Z_t, int64[count][t]."""
    st = Stream(seed, STREAM_LUTS, hash_name(ps.name), group)
    return st.below(count * ps.t, ps.t).reshape(count, ps.t)


def lut_assignment(seed: int, count: int, n_luts: int, how: str, group: int = 0) -> np.ndarray:
    """Table ids: [count], or [count][n_luts] for "all" (input c gets the
    tables in the order c, c+1, ... mod n_luts)."""
    if how == "round_robin":
        return (np.arange(count) % n_luts).astype(np.int32)
    if how == "all":
        return ((np.arange(count)[:, None] + np.arange(n_luts)[None, :]) % n_luts).astype(np.int32)
    st = Stream(seed, STREAM_LUT_ASSIGN, group)
    return st.below(count, n_luts).astype(np.int32)


def tfhe_polynomials(ps: ParamSet, seed: int, count: int) -> np.ndarray:
    """Pre-rotation polynomials for timing the TFHE bootstrap: [count][N]
    words uniform mod q (the bootstrap's cost does not depend on them)."""
    st = Stream(seed, STREAM_LUTS, 100)
    return np.stack([st.sub(i).words(ps.N, ps.w) for i in range(count)])


def mlp_inputs_and_weights(seed: int, layers: List[int], n_inputs: int):
    """Pixels uniform in Z_16 and integer weights uniform in [-8, 7]."""
    st = Stream(seed, STREAM_MLP)
    x = st.sub(0).below(n_inputs * layers[0], 16).reshape(n_inputs, layers[0])
    ws = []
    for i in range(len(layers) - 1):
        w = st.sub(1 + i).below(layers[i + 1] * layers[i], 16).reshape(layers[i + 1], layers[i]) - 8
        ws.append(w.astype(np.int64))
    return x.astype(np.int64), ws


# --------------------------------------------------------------------------
# Prime-modulus parameter sets (the paper's Table 1)
# --------------------------------------------------------------------------

Q1 = (1 << 62) - 65535
Q2 = (1 << 63) - 278527
Q3 = (1 << 48) - 163839
Q4 = (1 << 32) - 139263


@dataclasses.dataclass(frozen=True)
class QParamSet:
    """A parameter set of Table 1: RLWE side modulo a prime Q, LWE side
    modulo q = 2N, exact gadget decompositions, uniform RLWE key in Z_Q^N,
    binary LWE key.  The digit counts lg, lks, lpk (gadget digits) and lboot
    (sign rotations) are stated with each set; the oracle's tests check them
    against the exact decomposition's count and the library re-checks them at
    registration.

    sigma_lwe  : the key-switching key (LWE samples mod Q)
    sigma_glwe : the bootstrapping and packing keys (RLWE samples mod Q)
    sigma_in   : fresh input ciphertexts (LWE samples mod q = 2N)
    """
    name: str
    n: int
    N: int
    Q: int
    t: int
    log2Bg: int
    lg: int
    log2Bks: int
    lks: int
    log2Bpk: int
    lpk: int
    log2Lboot: int
    lboot: int
    sigma_lwe: float
    sigma_glwe: float
    sigma_in: float = 3.2

    @property
    def k(self) -> int:          # Q < 2^k
        return int(self.Q).bit_length()

    @property
    def logN(self) -> int:
        return int(self.N).bit_length() - 1

    @property
    def logq(self) -> int:       # q = 2N
        return self.logN + 1

    @property
    def q(self) -> int:
        return 2 * self.N


# Table 1's columns, and QZ, a small set of the same shape for the
# exhaustive checks.  t is the largest plaintext modulus the paper's
# correctness table gives a negligible error probability for.
Q_PARAM_SETS: Dict[str, QParamSet] = {
    "FDFB-80-6": QParamSet("FDFB-80-6", n=700, N=2048, Q=Q1, t=64, log2Bg=11, lg=6, log2Bks=6, lks=11,
                           log2Bpk=13, lpk=5, log2Lboot=11, lboot=6, sigma_lwe=2.0 ** 38, sigma_glwe=3.2),
    "FDFB-100-6": QParamSet("FDFB-100-6", n=1050, N=2048, Q=Q1, t=64, log2Bg=11, lg=6, log2Bks=1, lks=62,
                            log2Bpk=13, lpk=5, log2Lboot=11, lboot=6, sigma_lwe=2.0 ** 41, sigma_glwe=3.2),
    "FDFB-80-7": QParamSet("FDFB-80-7", n=700, N=4096, Q=Q2, t=128, log2Bg=9, lg=7, log2Bks=4, lks=16,
                           log2Bpk=13, lpk=5, log2Lboot=11, lboot=6, sigma_lwe=2.0 ** 39, sigma_glwe=3.2),
    "FDFB-100-7": QParamSet("FDFB-100-7", n=1100, N=4096, Q=Q2, t=128, log2Bg=9, lg=7, log2Bks=1, lks=63,
                            log2Bpk=13, lpk=5, log2Lboot=11, lboot=6, sigma_lwe=2.0 ** 41, sigma_glwe=3.2),
    "FDFB-80-8": QParamSet("FDFB-80-8", n=700, N=8192, Q=Q2, t=256, log2Bg=9, lg=7, log2Bks=4, lks=16,
                           log2Bpk=13, lpk=5, log2Lboot=8, lboot=8, sigma_lwe=2.0 ** 39, sigma_glwe=3.2),
    "FDFB-100-8": QParamSet("FDFB-100-8", n=1100, N=8192, Q=Q2, t=256, log2Bg=9, lg=7, log2Bks=1, lks=63,
                            log2Bpk=13, lpk=5, log2Lboot=8, lboot=8, sigma_lwe=2.0 ** 41, sigma_glwe=3.2),
    "QZ": QParamSet("QZ", n=24, N=256, Q=Q1, t=8, log2Bg=11, lg=6, log2Bks=6, lks=11, log2Bpk=13, lpk=5,
                    log2Lboot=11, lboot=6,
                    sigma_lwe=2.0 ** 38, sigma_glwe=3.2),
    # Table 1's TFHE columns (the paper's comparison point: one blind
    # rotation of a pre-rotation polynomial, negacyclic functions); they give
    # no packing key or L_boot, so the FDFB-only gadgets take B_RGSW.
    "TFHE-80-2": QParamSet("TFHE-80-2", n=424, N=1024, Q=Q4, t=4, log2Bg=11, lg=3, log2Bks=4, lks=8,
                           log2Bpk=11, lpk=3, log2Lboot=11, lboot=3, sigma_lwe=2.0 ** 16, sigma_glwe=3.2),
    "TFHE-100-2": QParamSet("TFHE-100-2", n=525, N=1024, Q=Q4, t=4, log2Bg=11, lg=3, log2Bks=4, lks=8,
                            log2Bpk=11, lpk=3, log2Lboot=11, lboot=3, sigma_lwe=2.0 ** 16, sigma_glwe=3.2),
    "TFHE-100-7": QParamSet("TFHE-100-7", n=1500, N=4096, Q=Q3, t=128, log2Bg=16, lg=3, log2Bks=1, lks=48,
                            log2Bpk=16, lpk=3, log2Lboot=16, lboot=3, sigma_lwe=2.0 ** 18, sigma_glwe=3.2),
    # small set on Q_4 (k = 32) for the exhaustive checks
    "QT": QParamSet("QT", n=24, N=256, Q=Q4, t=4, log2Bg=11, lg=3, log2Bks=4, lks=8, log2Bpk=11, lpk=3,
                    log2Lboot=11, lboot=3,
                    sigma_lwe=2.0 ** 16, sigma_glwe=3.2),
}


def _below_big(st: Stream, count: int, m: int) -> np.ndarray:
    """Integers in [0, m) for m < 2^64: a raw 64-bit output reduced mod m
    (bias below m / 2^64)."""
    return st.raw(count) % np.uint64(m)


@dataclasses.dataclass
class QKeyRandomness:
    """Everything key generation draws for a prime-Q set.

    s      : uint8[n]            binary LWE key
    sk     : uint64[N]           RLWE key, uniform in Z_Q (s_F = its coefficients)
    bsk_a  : uint64[n][2lg][N]   uniform mod Q;  bsk_e int64 (sigma_glwe)
    pk_a   : uint64[N][lpk][N]   uniform mod Q;  pk_e int64 (sigma_glwe)
    ksk_a  : uint64[N][lks][n]   uniform mod Q;  ksk_e int64[N][lks] (sigma_lwe)
    """
    s: np.ndarray
    sk: np.ndarray
    bsk_a: np.ndarray
    bsk_e: np.ndarray
    pk_a: np.ndarray
    pk_e: np.ndarray
    ksk_a: np.ndarray
    ksk_e: np.ndarray


def q_key_randomness(ps: QParamSet, seed: int) -> QKeyRandomness:
    st = Stream(seed, STREAM_KEYS, hash_name(ps.name))
    n, N, Q = ps.n, ps.N, ps.Q
    s = st.sub(1).bits(n)
    sk = _below_big(st.sub(2), N, Q)
    bsk_a = _below_big(st.sub(3), n * 2 * ps.lg * N, Q).reshape(n, 2 * ps.lg, N)
    bsk_e = st.sub(4).gaussian(n * 2 * ps.lg * N, ps.sigma_glwe).reshape(n, 2 * ps.lg, N)
    pk_a = _below_big(st.sub(5), N * ps.lpk * N, Q).reshape(N, ps.lpk, N)
    pk_e = st.sub(6).gaussian(N * ps.lpk * N, ps.sigma_glwe).reshape(N, ps.lpk, N)
    ksk_a = _below_big(st.sub(7), N * ps.lks * n, Q).reshape(N, ps.lks, n)
    ksk_e = st.sub(8).gaussian(N * ps.lks, ps.sigma_lwe).reshape(N, ps.lks)
    return QKeyRandomness(s, sk, bsk_a, bsk_e, pk_a, pk_e, ksk_a, ksk_e)


def q_uniform_key_words(ps: QParamSet, seed: int):
    """Key-shaped words uniform mod Q in the canonical layouts -- bsk
    [n][2lg][2][N], pK [N][lpk][2][N], ksK [N][lks][n+1] -- that are no
    encryptions at all: the bootstrap's arithmetic is defined for any words,
    so they exercise it at full ring degree and digit counts without the cost
    of key generation (outputs do not decrypt)."""
    st = Stream(seed, STREAM_KEYS, hash_name(ps.name), 99)
    n, N, Q = ps.n, ps.N, ps.Q
    bsk = _below_big(st.sub(1), n * 2 * ps.lg * 2 * N, Q).reshape(n, 2 * ps.lg, 2, N)
    pk = _below_big(st.sub(2), N * ps.lpk * 2 * N, Q).reshape(N, ps.lpk, 2, N)
    ksk = _below_big(st.sub(3), N * ps.lks * (n + 1), Q).reshape(N, ps.lks, n + 1)
    return bsk, pk, ksk


def q_message_randomness(ps: QParamSet, seed: int, count: int, group: int = 0,
                         m: Optional[np.ndarray] = None) -> MessageRandomness:
    """Messages in Z_t, masks uniform mod q = 2N, noise sigma_in."""
    st = Stream(seed, STREAM_MESSAGES, hash_name(ps.name), group)
    if m is None:
        m = st.sub(1).below(count, ps.t)
    a = st.sub(2).below(count * ps.n, ps.q).astype(np.uint64).reshape(count, ps.n)
    e = st.sub(3).gaussian(count, ps.sigma_in)
    return MessageRandomness(np.asarray(m, dtype=np.int64), a, e)


def q_lut_tables(ps: QParamSet, seed: int, count: int, group: int = 0) -> np.ndarray:
    """`count` random lookup tables f: Z_t -> Z_t, int64[count][t]."""
    st = Stream(seed, STREAM_LUTS, hash_name(ps.name), group)
    return st.below(count * ps.t, ps.t).reshape(count, ps.t)


def param_set(name: str):
    """A power-of-two set (PARAM_SETS) or a prime-modulus set (Q_PARAM_SETS)."""
    return PARAM_SETS[name] if name in PARAM_SETS else Q_PARAM_SETS[name]


def crt_sets(base: str, moduli) -> List[QParamSet]:
    """One prime-modulus set per CRT modulus t_i (pairwise coprime), the
    geometry of `base` (Section "Extending the Arithmetic": Z_t with
    t = prod t_i is Z_t1 x ... x Z_tm, one bootstrap per residue)."""
    ps = Q_PARAM_SETS[base]
    return [dataclasses.replace(ps, name=f"{base}-t{t}", t=int(t)) for t in moduli]


def q_tfhe_polynomials(ps: QParamSet, seed: int, count: int) -> np.ndarray:
    """Pre-rotation polynomials for timing the TFHE bootstrap of a prime-modulus
    set: [count][N] residues uniform mod Q (the cost does not depend on them)."""
    st = Stream(seed, STREAM_LUTS, 100)
    return np.stack([_below_big(st.sub(i), ps.N, ps.Q) for i in range(count)])
