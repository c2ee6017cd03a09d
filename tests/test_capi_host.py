"""Host-side checks of the CUDA library that need no GPU: the shared library
builds, loads and exports every entry point declared in include/fdfb.h; the
canonical key layouts reproduce the key sizes printed in the paper; and the
library refuses to run without a device."""
import ctypes as C
import math
import os
import re

import pytest

from paper_2109_02731_gb300 import build as B
from paper_2109_02731_gb300 import fdfb as F
from paper_2109_02731_gb300 import synth as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "fdfb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fdfb_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    return F.load()


def test_library_exports_every_declared_entry_point(lib):
    names = declared_entry_points()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(F.SYMBOLS) == names


def test_strerror(lib):
    assert lib.fdfb_strerror(0) == b"ok"
    assert b"lookup" in lib.fdfb_strerror(-6)


def test_create_without_device_fails_loudly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    assert lib.fdfb_create(C.byref(h), 0) == -3


def _ell(B_, Q):
    l = 1
    while B_ ** l < Q:
        l += 1
    return l


def test_key_words_reproduce_table3():
    """Table 3's key sizes = (bsk + pK + ksK words) x 8 bytes, with the
    paper's exact l = ceil(log_B Q): pins the canonical key layouts."""
    Q = {"Q1": 2 ** 62 - 65535, "Q2": 2 ** 63 - 278527}
    rows = [ln.split() for ln in open(os.path.join(ROOT, "tests", "golden", "table3_key_sizes.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 5
    for name, n, N, q, bg, bks, bpk, mb, dec in rows:
        n, N, bg, bks, bpk, dec = int(n), int(N), int(bg), int(bks), int(bpk), int(dec)
        qq = Q[q]
        p = F.fdfb_params(n, N, 1, 64, 64, int(math.log2(bg)), _ell(bg, qq), int(math.log2(bks)),
                          _ell(bks, qq), int(math.log2(bpk)), _ell(bpk, qq), 6, 1)
        words = 0
        for which in range(3):
            out = C.c_uint64()
            assert F.load().fdfb_key_words(C.byref(p), which, C.byref(out)) == 0
            words += out.value
        value = math.floor(words * 8 / 1e6 * 10 ** dec) / 10 ** dec
        assert value == float(mb), (name, value, mb)


def test_key_words_match_canonical_shapes():
    for ps in S.PARAM_SETS.values():
        assert F.key_words(ps, 0) == ps.n * 2 * ps.lg * 2 * ps.N
        assert F.key_words(ps, 1) == ps.N * ps.lpk * 2 * ps.N
        assert F.key_words(ps, 2) == ps.N * ps.lks * (ps.n + 1)
