"""The C ABI's host code (plans, layouts, validation) under AddressSanitizer:
every translation unit is compiled with a sanitized host side and linked with
a small C driver; any invalid access or leak fails the run.  No GPU call is
made."""
import concurrent.futures as cf
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2604_24994_gb300", "csrc")
from paper_2604_24994_gb300.build import SOURCES  # noqa: E402  (the library's translation units)

UNITS = [u[:-3] for u in SOURCES]


def test_capi_host_code_is_clean_under_asan(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("no nvcc")
    flags = ["-gencode", "arch=compute_103a,code=sm_103a", "-O1", "-std=c++17", "--expt-relaxed-constexpr",
             "-I" + os.path.join(ROOT, "include"), "-Xcompiler", "-fPIC,-fsanitize=address,-fno-omit-frame-pointer"]

    def compile_one(u):
        obj = str(tmp_path / (u + ".o"))
        r = subprocess.run([nvcc, *flags, "-c", os.path.join(CSRC, u + ".cu"), "-o", obj],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS))
    exe = str(tmp_path / "capi_san")
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-I" + os.path.join(ROOT, "include"),
                        "-Xcompiler", "-fsanitize=address", "-o", exe,
                        os.path.join(HERE, "capi_sanitize_driver.c"), *objs, "-lasan"], capture_output=True, text=True)
    if r.returncode != 0 and "asan" in r.stderr.lower():
        pytest.skip("this toolchain has no sanitizer runtime")
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, ASAN_OPTIONS="protect_shadow_gap=0:detect_leaks=1:exitcode=23")
    run = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
    assert run.returncode == 0, run.stdout + run.stderr
    assert "capi ok" in run.stdout
