"""Both oracles under AddressSanitizer and UndefinedBehaviorSanitizer: the
driver tests/oracle_sanitize.c runs key generation, encryption and the
full-domain bootstrap of every message on small noiseless sets (power-of-two
modulus with unsigned and balanced digits and an output modulus; prime
modulus Q_1 with l_boot sign rotations) and checks each decrypts to f(m);
any out-of-bounds access, use after free or undefined operation (a shift
past the word, a signed overflow) aborts the run."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_oracles_clean_under_sanitizers(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    exe = str(tmp_path / "oracle_sanitize")
    srcs = [os.path.join(ROOT, "tests", "oracle_sanitize.c"),
            os.path.join(ROOT, "oracle", "fdfb_oracle.c"),
            os.path.join(ROOT, "oracle", "fdfb_oracle_q.c")]
    r = subprocess.run(["gcc", "-std=c11", "-O1", "-g", "-fsanitize=address,undefined",
                        "-fno-sanitize-recover=all", "-fno-omit-frame-pointer", "-o", exe, *srcs],
                       capture_output=True, text=True)
    if r.returncode != 0 and "asan" in (r.stderr or "").lower():
        pytest.skip("sanitizer runtime not available: " + r.stderr.splitlines()[-1])
    assert r.returncode == 0, r.stderr
    run = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert run.returncode == 0 and run.stdout.strip() == "ok", run.stdout + run.stderr
