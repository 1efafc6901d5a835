"""The host side of the C ABI under AddressSanitizer and UndefinedBehaviorSanitizer.

The library is built a second time with its host code instrumented (build --sanitize:
libgpic_asan.so), and the CPU ABI tests run against it in a child process with the gcc
sanitizer runtime preloaded. They cover the argument checks, NULL handles, config
validation and struct layouts, all before any device is touched. Any sanitizer report
fails the test.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _runtime(name):
    gcc = shutil.which("gcc")
    if not gcc:
        return None
    p = subprocess.run([gcc, "-print-file-name=" + name], capture_output=True, text=True).stdout.strip()
    return p if os.path.isabs(p) and os.path.exists(p) else None


@pytest.mark.slow
def test_c_abi_host_code_is_clean_under_asan_and_ubsan():
    if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
        pytest.skip("no nvcc to build the sanitizer variant")
    asan = _runtime("libasan.so")
    if not asan:
        pytest.skip("no gcc AddressSanitizer runtime")
    from paper_2410_18414_gb300 import build
    lib = build.build(sanitize=True)
    env = dict(os.environ, GPIC_LIB=lib, LD_PRELOAD=asan, CUDA_VISIBLE_DEVICES="",
               ASAN_OPTIONS="detect_leaks=0:halt_on_error=1:protect_shadow_gap=0",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    # the child really runs the instrumented library, with the runtime in the process
    probe = ("import ctypes; from paper_2410_18414_gb300 import pic; pic.load_library(); "
             "ctypes.CDLL(None).__asan_init; print(pic.LIB_PATH)")
    r = subprocess.run([sys.executable, "-c", probe], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == lib, r.stdout + r.stderr[-2000:]
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_abi.py", "-q", "-x",
                        "-p", "no:cacheprovider", "-m", "not gpu"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    out = r.stdout[-3000:] + r.stderr[-3000:]
    assert r.returncode == 0, out
    assert "AddressSanitizer" not in r.stderr and "runtime error:" not in r.stderr, out
    assert " passed" in r.stdout, out
