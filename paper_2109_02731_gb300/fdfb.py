"""Thin ctypes binding of the FDFB C ABI (include/fdfb.h).

Argument marshalling only: every computation runs in the CUDA library.  Device
buffers are torch CUDA tensors (words stored as int32 for q = 2^32 and int64
for q = 2^64: same bits, torch has no full unsigned support); host buffers are
numpy arrays.  Loading fails loudly when the library cannot be built or no GPU
is present -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional, Sequence

import numpy as np

from . import build as _build
from .synth import KeyRandomness, ParamSet, QKeyRandomness, QParamSet

FDFB_OK = 0
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ETIMEOUT", -5: "ENOKEYS", -6: "EBADLUT"}

SYMBOLS = [
    "fdfb_create", "fdfb_destroy", "fdfb_params_register", "fdfb_key_words", "fdfb_keys_upload",
    "fdfb_keys_generate", "fdfb_keys_download", "fdfb_lut_setup", "fdfb_lut_polys",
    "fdfb_bootstrap", "fdfb_bootstrap_debug", "fdfb_bootstrap_mixed", "fdfb_keyswitch",
    "fdfb_bootstrap_noalloc", "fdfb_noalloc_max_batch", "fdfb_bootstrap_multi",
    "fdfb_tfhe_poly_setup", "fdfb_tfhe_bootstrap",
    "fdfb_lwe_encrypt", "fdfb_lwe_decrypt", "fdfb_lwe_affine", "fdfb_autotune",
    "fdfb_set_variant", "fdfb_variant_info", "fdfb_set_chunks", "fdfb_get_chunks", "fdfb_profile_enable",
    "fdfb_profile_read", "fdfb_test_hooks", "fdfb_keyswitch_path", "fdfb_sync", "fdfb_strerror",
]


class FDFBError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what} failed: {ERRORS.get(code, code)} ({_strerror(code)})")


class fdfb_params(C.Structure):
    _fields_ = [(k, C.c_uint32) for k in ("n", "N", "k", "log2q", "t", "log2Bg", "lg", "log2Bks",
                                          "lks", "log2Bpk", "lpk", "log2Lboot", "lboot", "signed_digits",
                                          "t_out")] + [("Q", C.c_uint64)]


class fdfb_keygen_inputs(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("s", "sk", "bsk_a", "bsk_e", "pk_a", "pk_e", "ksk_a", "ksk_e",
                                          "sk_q")]


class fdfb_debug_bufs(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("ctN", "sgn", "cR", "accF", "cQ", "cKS")]


class fdfb_group(C.Structure):
    _fields_ = [("set_id", C.c_int), ("ct_in", C.c_void_p), ("lut_ids", C.c_void_p),
                ("batch", C.c_int64), ("ct_out", C.c_void_p)]


_lib = None
_lock = threading.Lock()


def lib_path() -> str:
    return _build.LIB


def load(build: bool = True) -> C.CDLL:
    """Builds (if needed) and loads libfdfb.so."""
    global _lib
    with _lock:
        if _lib is None:
            if build:
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError("libfdfb.so is missing; run paper_2109_02731_gb300.build.build()")
            L = C.CDLL(_build.LIB)
            vp, i32, i64 = C.c_void_p, C.c_int, C.c_int64
            sig = {
                "fdfb_create": ([C.POINTER(vp), i32], i32),
                "fdfb_destroy": ([vp], i32),
                "fdfb_params_register": ([vp, C.POINTER(fdfb_params), C.POINTER(i32)], i32),
                "fdfb_key_words": ([C.POINTER(fdfb_params), i32, C.POINTER(C.c_uint64)], i32),
                "fdfb_keys_upload": ([vp, i32, vp, vp, vp, vp], i32),
                "fdfb_keys_generate": ([vp, i32, C.POINTER(fdfb_keygen_inputs), vp], i32),
                "fdfb_keys_download": ([vp, i32, vp, vp, vp, vp], i32),
                "fdfb_lut_setup": ([vp, i32, vp, C.POINTER(i32)], i32),
                "fdfb_lut_polys": ([vp, i32, i32, vp, vp], i32),
                "fdfb_bootstrap": ([vp, i32, vp, vp, i64, vp, vp], i32),
                "fdfb_bootstrap_debug": ([vp, i32, vp, vp, i64, vp, C.POINTER(fdfb_debug_bufs), vp], i32),
                "fdfb_bootstrap_mixed": ([vp, i32, C.POINTER(fdfb_group), vp], i32),
                "fdfb_bootstrap_noalloc": ([vp, i32, vp, vp, i64, vp, vp], i32),
                "fdfb_noalloc_max_batch": ([vp, i32, C.POINTER(i64)], i32),
                "fdfb_bootstrap_multi": ([vp, i32, vp, vp, i64, i32, vp, vp], i32),
                "fdfb_set_chunks": ([vp, i32, i32], i32),
                "fdfb_tfhe_poly_setup": ([vp, i32, vp, C.POINTER(i32)], i32),
                "fdfb_tfhe_bootstrap": ([vp, i32, vp, vp, i64, vp, vp], i32),
                "fdfb_get_chunks": ([vp, i32, C.POINTER(i32)], i32),
                "fdfb_keyswitch": ([vp, i32, vp, i64, vp, vp], i32),
                "fdfb_lwe_encrypt": ([vp, i32, vp, vp, vp, vp, i64, vp, vp], i32),
                "fdfb_lwe_decrypt": ([vp, i32, vp, vp, i64, vp, vp], i32),
                "fdfb_lwe_affine": ([vp, i32, vp, i32, i32, vp, i64, vp, vp], i32),
                "fdfb_autotune": ([vp, i32, i64, vp, C.POINTER(i32), C.POINTER(C.c_double),
                                   C.POINTER(C.c_double), i32], i32),
                "fdfb_set_variant": ([vp, i32, i32], i32),
                "fdfb_variant_info": ([vp, i32, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)], i32),
                "fdfb_profile_enable": ([vp, i32], i32),
                "fdfb_profile_read": ([vp, i32, C.POINTER(C.c_double), C.POINTER(C.c_int64)], i32),
                "fdfb_test_hooks": ([vp, i32], i32),
                "fdfb_keyswitch_path": ([vp, i32, C.POINTER(i32), C.POINTER(i32)], i32),
                "fdfb_sync": ([vp, vp], i32),
                "fdfb_strerror": ([i32], C.c_char_p),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def _strerror(code: int) -> str:
    try:
        return load(build=False).fdfb_strerror(code).decode()
    except Exception:
        return "?"


def _check(rc: int, what: str) -> None:
    if rc != FDFB_OK:
        raise FDFBError(rc, what)


def params_struct(ps) -> fdfb_params:
    if isinstance(ps, QParamSet):
        return fdfb_params(ps.n, ps.N, 1, 64, ps.t, ps.log2Bg, ps.lg, ps.log2Bks, ps.lks, ps.log2Bpk,
                           ps.lpk, ps.log2Lboot, ps.lboot, 0, 0, ps.Q)
    return fdfb_params(ps.n, ps.N, 1, ps.w, ps.t, ps.log2Bg, ps.lg, ps.log2Bks, ps.lks, ps.log2Bpk,
                       ps.lpk, int(ps.t).bit_length() - 1, 1, 1 if ps.signed_digits else 0, ps.t_out, 0)


def key_words(ps: ParamSet, which: int) -> int:
    out = C.c_uint64()
    p = params_struct(ps)
    _check(load().fdfb_key_words(C.byref(p), which, C.byref(out)), "fdfb_key_words")
    return int(out.value)


def _ptr(x) -> Optional[int]:
    """Raw pointer of a torch tensor, numpy array or int (None passes NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    assert x.is_contiguous(), "tensor must be contiguous"
    return x.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def word_np(ps):
    return np.uint32 if getattr(ps, "w", 64) == 32 else np.uint64


def word_torch(ps):
    import torch
    return torch.int32 if getattr(ps, "w", 64) == 32 else torch.int64


def to_host_words(ps: ParamSet, t) -> np.ndarray:
    """Copies a device word tensor to a numpy array of unsigned words."""
    return t.detach().cpu().numpy().view(word_np(ps))


def to_device_words(ps: ParamSet, a: np.ndarray, device="cuda"):
    import torch
    arr = np.ascontiguousarray(np.asarray(a).astype(word_np(ps)))
    sgn = np.int32 if word_np(ps) == np.uint32 else np.int64
    return torch.from_numpy(arr.view(sgn)).to(device)


class Context:
    """One FDFB context (device memory for keys, tables and scratch)."""

    def __init__(self, device: int = 0):
        self.L = load()
        h = C.c_void_p()
        _check(self.L.fdfb_create(C.byref(h), int(device)), "fdfb_create")
        self.h = h
        self.device = device
        self.sets = {}

    def close(self) -> None:
        if self.h:
            self.L.fdfb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def register(self, ps: ParamSet) -> int:
        p = params_struct(ps)
        sid = C.c_int()
        _check(self.L.fdfb_params_register(self.h, C.byref(p), C.byref(sid)), "fdfb_params_register")
        self.sets[sid.value] = ps
        return sid.value

    def keys_upload(self, set_id: int, bsk: np.ndarray, pk: np.ndarray, ksk: np.ndarray, stream=None):
        ps = self.sets[set_id]
        dt = word_np(ps)
        b, p, k = (np.ascontiguousarray(np.asarray(x).astype(dt)) for x in (bsk, pk, ksk))
        _check(self.L.fdfb_keys_upload(self.h, set_id, b.ctypes.data, p.ctypes.data, k.ctypes.data,
                                       _stream(stream)), "fdfb_keys_upload")

    def keys_generate(self, set_id: int, kr, stream=None):
        """kr: KeyRandomness, or QKeyRandomness for a prime-modulus set (its
        RLWE key, uniform mod Q, goes to sk_q)."""
        ps = self.sets[set_id]
        dt = word_np(ps)
        prime = isinstance(kr, QKeyRandomness)
        sk8 = np.zeros(ps.N, np.uint8) if prime else kr.sk.astype(np.uint8)
        keep = [np.ascontiguousarray(kr.s.astype(np.uint8)), np.ascontiguousarray(sk8),
                np.ascontiguousarray(kr.bsk_a.astype(dt)), np.ascontiguousarray(kr.bsk_e.astype(np.int64)),
                np.ascontiguousarray(kr.pk_a.astype(dt)), np.ascontiguousarray(kr.pk_e.astype(np.int64)),
                np.ascontiguousarray(kr.ksk_a.astype(dt)), np.ascontiguousarray(kr.ksk_e.astype(np.int64))]
        keep.append(np.ascontiguousarray(kr.sk.astype(np.uint64)) if prime else None)
        inp = fdfb_keygen_inputs(*[None if a is None else a.ctypes.data for a in keep])
        _check(self.L.fdfb_keys_generate(self.h, set_id, C.byref(inp), _stream(stream)),
               "fdfb_keys_generate")

    def keys_download(self, set_id: int, stream=None):
        ps = self.sets[set_id]
        dt = word_np(ps)
        n, N = ps.n, ps.N
        bsk = np.zeros((n, 2 * ps.lg, 2, N), dtype=dt)
        pk = np.zeros((N, ps.lpk, 2, N), dtype=dt)
        ksk = np.zeros((N, ps.lks, n + 1), dtype=dt)
        _check(self.L.fdfb_keys_download(self.h, set_id, bsk.ctypes.data, pk.ctypes.data,
                                         ksk.ctypes.data, _stream(stream)), "fdfb_keys_download")
        return bsk, pk, ksk

    def lut_setup(self, set_id: int, f: Sequence[int]) -> int:
        arr = np.ascontiguousarray(np.asarray(f, dtype=np.uint32))
        lid = C.c_int()
        _check(self.L.fdfb_lut_setup(self.h, set_id, arr.ctypes.data, C.byref(lid)), "fdfb_lut_setup")
        return lid.value

    def lut_polys(self, set_id: int, lut_id: int):
        N = self.sets[set_id].N
        p0 = np.zeros(N, np.int32)
        p1 = np.zeros(N, np.int32)
        _check(self.L.fdfb_lut_polys(self.h, set_id, lut_id, p0.ctypes.data, p1.ctypes.data),
               "fdfb_lut_polys")
        return p0, p1

    def bootstrap(self, set_id: int, ct_in, lut_ids, ct_out, batch: Optional[int] = None, stream=None):
        b = int(ct_in.shape[0]) if batch is None else batch
        _check(self.L.fdfb_bootstrap(self.h, set_id, _ptr(ct_in), _ptr(lut_ids), b, _ptr(ct_out),
                                     _stream(stream)), "fdfb_bootstrap")

    def bootstrap_multi(self, set_id: int, ct_in, lut_ids, ct_out, stream=None):
        """k tables per input: ct_in [batch][n+1], lut_ids int32 [batch][k] and
        ct_out [batch][k][n+1], all on the device."""
        b, k = int(lut_ids.shape[0]), int(lut_ids.shape[1])
        _check(self.L.fdfb_bootstrap_multi(self.h, set_id, _ptr(ct_in), _ptr(lut_ids), b, k,
                                           _ptr(ct_out), _stream(stream)), "fdfb_bootstrap_multi")

    def tfhe_poly_setup(self, set_id: int, poly) -> int:
        """Installs a TFHE pre-rotation polynomial (N words mod q); returns its id."""
        ps = self.sets[set_id]
        arr = np.ascontiguousarray(np.asarray(poly).astype(word_np(ps)))
        assert arr.shape == (ps.N,)
        out = C.c_int()
        _check(self.L.fdfb_tfhe_poly_setup(self.h, set_id, arr.ctypes.data, C.byref(out)),
               "fdfb_tfhe_poly_setup")
        return out.value

    def tfhe_bootstrap(self, set_id: int, ct_in, poly_ids, ct_out, stream=None):
        _check(self.L.fdfb_tfhe_bootstrap(self.h, set_id, _ptr(ct_in), _ptr(poly_ids), int(ct_in.shape[0]),
                                          _ptr(ct_out), _stream(stream)), "fdfb_tfhe_bootstrap")

    def bootstrap_noalloc(self, set_id: int, ct_in, lut_ids, ct_out, stream=None):
        """fdfb_bootstrap on the library's fixed scratch: allocates nothing."""
        _check(self.L.fdfb_bootstrap_noalloc(self.h, set_id, _ptr(ct_in), _ptr(lut_ids),
                                             int(ct_in.shape[0]), _ptr(ct_out), _stream(stream)),
               "fdfb_bootstrap_noalloc")

    def noalloc_max_batch(self, set_id: int) -> int:
        out = C.c_int64()
        _check(self.L.fdfb_noalloc_max_batch(self.h, set_id, C.byref(out)), "fdfb_noalloc_max_batch")
        return int(out.value)

    def bootstrap_debug(self, set_id: int, ct_in, lut_ids, ct_out, dbg: dict, stream=None):
        d = fdfb_debug_bufs(*[_ptr(dbg.get(k)) for k in ("ctN", "sgn", "cR", "accF", "cQ", "cKS")])
        _check(self.L.fdfb_bootstrap_debug(self.h, set_id, _ptr(ct_in), _ptr(lut_ids),
                                           int(ct_in.shape[0]), _ptr(ct_out), C.byref(d),
                                           _stream(stream)), "fdfb_bootstrap_debug")

    def bootstrap_mixed(self, groups, stream=None):
        """groups: list of (set_id, ct_in, lut_ids, ct_out)."""
        arr = (fdfb_group * max(1, len(groups)))()
        for i, (sid, cin, ids, cout) in enumerate(groups):
            arr[i] = fdfb_group(sid, _ptr(cin), _ptr(ids), int(cin.shape[0]), _ptr(cout))
        _check(self.L.fdfb_bootstrap_mixed(self.h, len(groups), arr, _stream(stream)),
               "fdfb_bootstrap_mixed")

    def keyswitch(self, set_id: int, ct_in, ct_out, stream=None):
        _check(self.L.fdfb_keyswitch(self.h, set_id, _ptr(ct_in), int(ct_in.shape[0]), _ptr(ct_out),
                                     _stream(stream)), "fdfb_keyswitch")

    def lwe_encrypt(self, set_id: int, s, a, e, m, ct_out, stream=None):
        _check(self.L.fdfb_lwe_encrypt(self.h, set_id, _ptr(s), _ptr(a), _ptr(e), _ptr(m),
                                       int(m.shape[0]), _ptr(ct_out), _stream(stream)),
               "fdfb_lwe_encrypt")

    def lwe_decrypt(self, set_id: int, s, ct, m_out, stream=None):
        _check(self.L.fdfb_lwe_decrypt(self.h, set_id, _ptr(s), _ptr(ct), int(ct.shape[0]),
                                       _ptr(m_out), _stream(stream)), "fdfb_lwe_decrypt")

    def lwe_affine(self, set_id: int, W, x, y, stream=None):
        n_out, n_in = int(W.shape[0]), int(W.shape[1])
        _check(self.L.fdfb_lwe_affine(self.h, set_id, _ptr(W), n_in, n_out, _ptr(x), int(x.shape[0]),
                                      _ptr(y), _stream(stream)), "fdfb_lwe_affine")

    def autotune(self, set_id: int, batch: int, stream=None, each: bool = False):
        """Times every blind-rotation variant; keeps and returns (variant, ms)
        (and the list of every variant's ms when `each`)."""
        v, ms = C.c_int(), C.c_double()
        arr = (C.c_double * 16)()
        _check(self.L.fdfb_autotune(self.h, set_id, int(batch), _stream(stream), C.byref(v), C.byref(ms),
                                    arr, 16), "fdfb_autotune")
        if each:
            n = self.variant_info(set_id)[1]
            return v.value, ms.value, [arr[i] for i in range(n)]
        return v.value, ms.value

    def set_variant(self, set_id: int, variant: int) -> None:
        _check(self.L.fdfb_set_variant(self.h, set_id, int(variant)), "fdfb_set_variant")

    def set_chunks(self, set_id: int, chunks: int) -> None:
        _check(self.L.fdfb_set_chunks(self.h, set_id, int(chunks)), "fdfb_set_chunks")

    def get_chunks(self, set_id: int) -> int:
        c = C.c_int()
        _check(self.L.fdfb_get_chunks(self.h, set_id, C.byref(c)), "fdfb_get_chunks")
        return c.value

    def variant_info(self, set_id: int):
        """(current variant, number of variants, coefficients per thread)."""
        cur, cnt, cpt = C.c_int(), C.c_int(), C.c_int()
        _check(self.L.fdfb_variant_info(self.h, set_id, C.byref(cur), C.byref(cnt), C.byref(cpt)),
               "fdfb_variant_info")
        return cur.value, cnt.value, cpt.value

    STAGES = ("blind_rotate_sign", "keyswitch_pk", "pubmux", "blind_rotate_func", "keyswitch_ksk",
              "blind_rotate_union")

    def profile_enable(self, enable: bool = True) -> None:
        _check(self.L.fdfb_profile_enable(self.h, 1 if enable else 0), "fdfb_profile_enable")

    def profile_read(self) -> dict:
        """{stage name: (total ms, launches)} since profile_enable."""
        out = {}
        for i, name in enumerate(self.STAGES):
            ms, n = C.c_double(), C.c_int64()
            _check(self.L.fdfb_profile_read(self.h, i, C.byref(ms), C.byref(n)), "fdfb_profile_read")
            out[name] = (ms.value, n.value)
        return out

    def test_hooks(self, flags: int) -> None:
        """fdfb_test_hooks: bit 0 makes the staged-key blind rotation skip
        its key copies so that its bounded wait expires (error-path tests);
        bit 1 runs the key switches on the CUDA cores instead of the tensor
        cores (comparisons)."""
        _check(self.L.fdfb_test_hooks(self.h, int(flags)), "fdfb_test_hooks")

    def keyswitch_path(self, set_id: int):
        """(packing key, LWE key): 1 = tensor cores, 0 = CUDA cores."""
        a, b = C.c_int(), C.c_int()
        _check(self.L.fdfb_keyswitch_path(self.h, set_id, C.byref(a), C.byref(b)), "fdfb_keyswitch_path")
        return a.value, b.value

    def sync(self, stream=None) -> None:
        _check(self.L.fdfb_sync(self.h, _stream(stream)), "fdfb_sync")
