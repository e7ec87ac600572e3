"""The FP64 oracle under AddressSanitizer and UndefinedBehaviorSanitizer: a C
driver that includes the oracle's source exercises every exported function
(displacement, learned and eight sites, view-dependent colours, fisheye,
candidate lists, neighbour lists, binning) on a small scene; any invalid
access, leak or undefined behaviour fails the run."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_is_clean_under_asan_and_ubsan(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    exe = str(tmp_path / "orc_san")
    cmd = [gcc, "-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
           "-fno-sanitize-recover=undefined", "-fopenmp", "-ffp-contract=off", "-o", exe,
           os.path.join(HERE, "oracle_sanitize_driver.c"), "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "asan" in (r.stderr + r.stdout).lower():
        pytest.skip("this toolchain has no sanitizer runtime")
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, OMP_NUM_THREADS="2", ASAN_OPTIONS="abort_on_error=0:exitcode=23")
    run = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
    assert run.returncode == 0, run.stdout + run.stderr
    assert "sanitized oracle ok" in run.stdout
