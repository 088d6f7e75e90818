"""The CPU oracle under AddressSanitizer and UndefinedBehaviorSanitizer: tests/sanitize_oracle.c
drives every oracle entry point on small inputs (orders 0-2, coincident eigenvalues, exact splits,
a diagonal T, padded leading dimensions) with buffers of exactly the documented sizes; any
out-of-bounds access, use after free, leak or undefined arithmetic makes the run fail."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_oracle_is_clean_under_asan_and_ubsan(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    exe = str(tmp_path / "sanitize_oracle")
    cmd = ["gcc", "-std=c99", "-O1", "-g", "-ffp-contract=off", "-fno-fast-math",
           "-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer",
           "-o", exe, os.path.join(HERE, "sanitize_oracle.c"),
           os.path.join(ROOT, "oracle", "tinv_oracle.c"), "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "asan" in (r.stderr or "").lower():
        pytest.skip("sanitizer runtime unavailable: " + r.stderr[-300:])
    assert r.returncode == 0, r.stderr[-2000:]
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    run = subprocess.run([exe], capture_output=True, text=True, timeout=600, env=env)
    assert run.returncode == 0 and run.stdout.strip() == "ok", (run.stdout[-1000:] +
                                                                run.stderr[-4000:])
