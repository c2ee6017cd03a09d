"""Host-side facts about the split-precision alternatives, checked with the
toolchain (no GPU): the 8-bit integer form of the fifth-generation tensor-core
MMA (tcgen05.mma kind::i8) does not exist for sm_103a -- ptxas rejects it while
accepting the same instruction with kind::f16 -- so 8-bit integer products on
this GPU can only use the legacy mma.sync path, whose rate the GPU probe
measures.  The probe itself builds for sm_103a."""
import os
import shutil
import subprocess
import tempfile

import pytest

from paper_2109_02731_gb300 import build as B

MMA_SRC = r"""
#include <stdint.h>
__global__ void k(uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t taddr, int acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
               " tcgen05.mma.cta_group::1.kind::KIND [%0], %1, %2, %3, p;\n}"
               :: "r"(taddr), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}
"""


def _compile(kind: str, arch: str = "103a"):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "mma.cu")
        open(src, "w").write(MMA_SRC.replace("KIND", kind))
        return subprocess.run([nvcc, "-gencode", f"arch=compute_{arch},code=sm_{arch}", "-c", src, "-o",
                               os.path.join(d, "mma.o")], capture_output=True, text=True)


def test_tcgen05_int8_mma_is_rejected_for_sm103a():
    r = _compile("i8")
    assert r.returncode != 0
    assert "kind::i8" in (r.stdout + r.stderr) and "sm_103a" in (r.stdout + r.stderr)


def test_tcgen05_f16_mma_compiles_for_sm103a():
    r = _compile("f16")
    assert r.returncode == 0, r.stderr


def test_probe_builds():
    assert os.path.exists(B.build_probe())


def test_n13_rotation_driver_builds_for_sm103a(tmp_path):
    """The small-case driver of the N = 2^13 blind rotation (used for profiler
    captures on a case of a few hundred MB) builds against the library's own
    kernel header."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pkg = os.path.join(root, "paper_2109_02731_gb300")
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O1", "-std", "c++17",
                        "--expt-relaxed-constexpr", "-I", os.path.join(root, "include"), "-I",
                        os.path.join(pkg, "csrc"), "-o", str(tmp_path / "n13_rotate"),
                        os.path.join(pkg, "probe", "n13_rotate.cu")], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
