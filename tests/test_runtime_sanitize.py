"""The library's host code under AddressSanitizer and UBSan (CPU only): libtinv_asan.so is loaded
in a child process with the ASan runtime preloaded, and everything that runs without a device is
driven through the C ABI -- the tune-cache file parser on malformed and hostile files, the cache
writer, and the argument checks of the entry points.  Any invalid access or undefined operation
aborts the child."""
import json
import os
import shutil
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent(r'''
    import ctypes, json, os, sys
    import numpy as np
    sys.path.insert(0, ROOT)
    from paper_1209_1910_gb300 import binding
    lib = binding.load(LIB)
    tag = "# tinv tune cache v1\n"
    ok_row = "dev\t152\t0\t0\t10\t10\t1\t2\t0\t1.0\n"
    cases = {
        "valid": tag + ok_row,
        "long_line": tag + "x" * 5000 + "\n",
        "long_name": tag + "N" * 1500 + "\t152\t0\t0\t10\t10\t1\t2\t0\t1.0\n",
        "few_fields": tag + "dev\t1\t2\n",
        "non_numeric": tag + "dev\tabc\t0\t0\t10\t10\t1\t2\t0\t1.0\n",
        "trailing_text": tag + "dev\t152\t0\t0\t10\t10\t1\t2\t0\t1.0 junk\n",
        "huge_values": tag + "dev\t99999999999999999999\t0\t0\t99999999999999999999999\t10\t1\t2\t0\t1e999\n",
        "bad_ranges": tag + "dev\t0\t0\t0\t10\t10\t1\t2\t0\t1.0\n",
        "largest_gt_m": tag + "dev\t152\t0\t0\t10\t5\t1\t6\t0\t1.0\n",
        "nan_time": tag + "dev\t152\t0\t0\t10\t10\t1\t2\t0\tnan\n",
        "leading_tab": tag + "\t152\t0\t0\t10\t10\t1\t2\t0\t1.0\n",
        "crlf": tag.replace("\n", "\r\n") + ok_row.replace("\n", "\r\n"),
        "no_final_newline": tag + ok_row.rstrip("\n"),
        "nul_bytes": tag + "\x00\x01\x02\tdev\n" + ok_row,
        "empty": "",
        "tag_only": tag,
        "blank_lines": tag + "\n\n" + ok_row + "\n",
    }
    rcs = {}
    for name, text in cases.items():
        p = os.path.join(TMP, name + ".txt")
        with open(p, "w", newline="") as f:
            f.write(text)
        lib.tinv_tune_clear()
        rcs[name] = lib.tinv_tune_load(p.encode())
    rcs["save"] = lib.tinv_tune_save(os.path.join(TMP, "out.txt").encode())
    rcs["save_bad_dir"] = lib.tinv_tune_save(os.path.join(TMP, "no", "dir.txt").encode())
    # argument checks that return before any device work
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    d, e, w = np.zeros(4), np.ones(3), np.array([3.0, 1.0, 2.0, 4.0])
    Z = np.zeros(16)
    checks = [
        lib.tinv_ex(-1, None, None, 0, None, None, 1, None, None),
        lib.tinv_ex(4, P(d), P(e), 4, P(w), P(Z), 4, None, None),
        lib.tinv_ex(4, P(np.array([0.0, np.nan, 0.0, 0.0])), P(e), 4, P(np.sort(w)), P(Z), 4, None, None),
        lib.tinv_bisect(-1, None, None, None, None),
        lib.tinv_split(-1, None, None, None, None, None),
        lib.tinv_bdsvd(3, P(np.array([1.0, np.inf, 1.0])), P(e), P(d), P(Z), 3, P(Z), 3, None),
        lib.tinv_tune(4, P(d), P(e), 4, P(w), None, 1, None, None, None),
        lib.tinv_tune(0, None, None, 0, None, None, 1, ctypes.byref(ctypes.c_int32()), None, None),
    ]
    for code in range(-110, 4):
        lib.tinv_strerror(code)
    print("RESULT " + json.dumps({"rcs": rcs, "checks": checks}))
''')


def test_host_code_is_clean_under_asan_and_ubsan(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    asan = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True,
                          text=True).stdout.strip()
    if not asan or not os.path.isabs(asan) or not os.path.exists(asan):
        pytest.skip("no ASan runtime")
    from paper_1209_1910_gb300 import build

    lib = build.build(sanitize=True)
    env = dict(os.environ, LD_PRELOAD=asan,
               ASAN_OPTIONS="detect_leaks=0:abort_on_error=0:halt_on_error=1",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    code = "ROOT = %r\nLIB = %r\nTMP = %r\n" % (ROOT, lib, str(tmp_path)) + CHILD
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600,
                       env=env, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-6000:]
    assert "runtime error" not in r.stderr and "AddressSanitizer" not in r.stderr, r.stderr[-6000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    out = json.loads(line[len("RESULT "):])
    rcs = out["rcs"]
    assert rcs["valid"] == 1 and rcs["crlf"] == 1 and rcs["no_final_newline"] == 1
    assert rcs["blank_lines"] == 1 and rcs["tag_only"] == 0 and rcs["nul_bytes"] == 1
    assert rcs["empty"] == -2
    for name in ("long_line", "long_name", "few_fields", "non_numeric", "trailing_text",
                 "huge_values", "bad_ranges", "largest_gt_m", "nan_time", "leading_tab"):
        assert rcs[name] == -3, (name, rcs[name])
    assert rcs["save"] == 0 and rcs["save_bad_dir"] == -2
    assert out["checks"] == [-1, -5, -2, -1, -1, -2, -8, 0]
