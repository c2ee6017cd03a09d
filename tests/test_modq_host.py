"""Host check of the CUDA library's modular helpers for the prime-modulus
sets (csrc/fdfb_core.cuh compiled as plain C++ with g++, no GPU): the lift
reduction and its fold counts, and Garner's exact lift, against 128-bit
integer division and the integer the residues came from; and the NTT
constants of both prime families (roots of unity, Shoup and Montgomery
companions, Garner constants) for N = 2^8 .. 2^12."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_modq_helpers_on_the_host(tmp_path):
    exe = str(tmp_path / "host_modq")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2109_02731_gb300", "csrc"),
                           "-o", exe, os.path.join(ROOT, "tests", "host_modq.cpp")])
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr


def test_n13_split_transforms_on_the_host(tmp_path):
    """The N = 2^13 transforms as the kernels run them (split stage, two
    4096-point register transforms on the half tables, joining stage), for
    both register layouts and all three primes, against the schoolbook
    negacyclic product mod p."""
    exe = str(tmp_path / "host_n13")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2109_02731_gb300", "csrc"),
                           "-o", exe, os.path.join(ROOT, "tests", "host_n13.cpp")])
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
