"""Host code under AddressSanitizer and UndefinedBehaviorSanitizer (CPU).

The oracle's C chains and the C ABI's host side (argument validation, work
list planning, the allocation-free entry point's checks) are rebuilt with
-fsanitize=address,undefined -fno-sanitize-recover and their CPU tests rerun
in a child process with the sanitizer runtime preloaded: any out-of-bounds
access, use after free or undefined operation aborts that process.  (Device
code has its own no-trap bounds checks: the SPIN_CHECK build.)"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _asan_runtime():
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    p = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    if not p or not os.path.isabs(p) or not os.path.exists(p):
        pytest.skip("no AddressSanitizer runtime")
    return p


def _run_under_asan(env_extra, tests, timeout=600):
    env = dict(os.environ, LD_PRELOAD=_asan_runtime(),
               ASAN_OPTIONS="detect_leaks=0:protect_shadow_gap=0:abort_on_error=1",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1", **env_extra)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "not gpu",
                        *tests], cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "passed" in r.stdout
    return r.stdout


def test_oracle_pins_under_address_and_undefined_behaviour_sanitizers():
    import oracle
    oracle.build(sanitize=True)
    _run_under_asan({"SPINMC_ORACLE_SANITIZE": "1"},
                    [os.path.join("tests", f) for f in ("test_oracle_ising.py", "test_oracle_potts.py",
                                                        "test_oracle_cpm.py", "test_oracle_philox_accept.py",
                                                        "test_oracle_nnn.py", "test_oracle_triangular.py",
                                                        "test_oracle_dmc.py")])


def test_abi_host_checks_under_address_and_undefined_behaviour_sanitizers():
    from paper_2304_01772_gb300 import build
    lib = build.build(variant="san")
    _run_under_asan({"SPINMC_LIBRARY": lib}, [os.path.join("tests", "test_abi_host.py")])


def test_the_harness_catches_an_out_of_bounds_write(tmp_path):
    """The same flags and runtime turn a one-past-the-end heap write in a
    ctypes-loaded library into an abort with a sanitizer report (UBSan's
    object-size check or ASan's heap-buffer-overflow, whichever fires first)."""
    src = tmp_path / "oob.c"
    src.write_text("#include <stdlib.h>\nint oob(int n) { int *a = malloc(n * sizeof(int)); a[n] = 1;"
                   " int r = a[0]; free(a); return r; }\n")
    so = tmp_path / "liboob.so"
    subprocess.check_call(["gcc", "-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
                           "-fPIC", "-shared", "-o", str(so), str(src)])
    env = dict(os.environ, LD_PRELOAD=_asan_runtime(), ASAN_OPTIONS="detect_leaks=0:abort_on_error=1")
    r = subprocess.run([sys.executable, "-c", f"import ctypes; ctypes.CDLL({str(so)!r}).oob(4)"], env=env,
                       capture_output=True, text=True, timeout=120)
    assert r.returncode != 0
    assert "heap-buffer-overflow" in r.stderr or "runtime error: store to address" in r.stderr
