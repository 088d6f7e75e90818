"""The library's device-side failure paths on the GPU, none of which faults or hangs it.

* The TINV_DEBUG build (libtinv_debug.so) checks every range of Y, T, Z, the LU factors, the
  team's partial sums and buffers, the team schedule and the distributed solve before it is
  touched.  On small workloads of every entry point that runs the cluster kernel its error word
  stays clear and its results equal the product library's.  With the extent of the factor / Y
  arrays declared one element short (a test hook of the debug build only; the accesses stay
  inside the real allocation and the failed check skips them) the checks fire and the call
  returns TINV_EINTERNAL; the next call in the same process succeeds.
* The bounded team-barrier wait: with tinv_opts.spin_limit = 1 a multi-CTA team's first wait
  gives up at once, the launch ends with TINV_ETIMEDOUT, and the next call succeeds.
The debug library runs in a child process, so the product library stays the one this process
loads."""
import os
import subprocess
import sys

import numpy as np
import pytest

from helpers import clusters_from_heads, orth_ratio, residual_ratio, sin_angle
from paper_1209_1910_gb300 import inputs

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import os, sys
import numpy as np
sys.path.insert(0, %(root)r); sys.path.insert(0, os.path.join(%(root)r, "tests"))
from paper_1209_1910_gb300 import binding, build, inputs
from helpers import residual_ratio, orth_ratio
binding.load(build.build(debug=True))
mode = sys.argv[1]
cases = []
d, e = inputs.uniform(64, seed=3)
cases.append((d, e, inputs.eigenvalues(d, e)[:8], 0))
d, e = inputs.glued_wilkinson(20, 1e-10)
cases.append((d, e, inputs.eigenvalues(d, e), 0))
cases.append((d, e, inputs.eigenvalues(d, e), 1))
if mode == "clear":
    for d, e, w, mt in cases:
        for meth in ("cwy", "mgs"):
            Z, info, *_ = binding.tinv(d, e, w, method=meth, max_team=mt, return_info=True)
            assert info == 0, (len(d), meth, info)
            np.save(os.path.join(sys.argv[2], "%%d_%%s_%%d.npy" %% (len(d), meth, mt)), Z)
    probs = [inputs.uniform(n, seed=n) for n in (7, 30, 64)] + [inputs.glued_wilkinson(3, 1e-10)]
    Zs, rc, info, _ = binding.tinv_batch([p[0] for p in probs], [p[1] for p in probs],
                                          [inputs.eigenvalues(*p) for p in probs], return_info=True)
    assert rc == 0 and np.all(info == 0), (rc, info)
    V = np.random.default_rng(4).standard_normal((300, 40))
    Q = binding.orth(V, "cwy")
    assert np.abs(Q.T @ Q - np.eye(40)).max() < 1e-12
    print("CLEAR_OK")
else:
    d, e, w, _ = cases[1]
    os.environ["TINV_DEBUG_SHRINK_F"] = "1"
    try:
        binding.tinv(d, e, w)
        raise SystemExit("the shortened extent was not detected")
    except binding.TinvError as ex:
        assert ex.code == -109, ex.code  # TINV_EINTERNAL
    del os.environ["TINV_DEBUG_SHRINK_F"]
    Z, info, *_ = binding.tinv(d, e, w, return_info=True)
    assert info == 0 and residual_ratio(d, e, w, Z) <= 10 and orth_ratio(Z) <= 10
    print("FIRED_OK")
'''


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1209_1910_gb300 import binding, build

    build.build()
    build.build(debug=True)
    binding.load()
    return binding


def _child(mode, tmp):
    r = subprocess.run([sys.executable, "-c", CHILD % {"root": ROOT}, mode, str(tmp)],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return r.stdout


def test_debug_build_checks_stay_clear_and_match_the_product(gpu, tmp_path):
    assert "CLEAR_OK" in _child("clear", tmp_path)
    d, e = inputs.uniform(64, seed=3)
    w = inputs.eigenvalues(d, e)[:8]
    for meth in ("cwy", "mgs"):
        assert np.array_equal(np.load(tmp_path / ("64_%s_0.npy" % meth)), gpu.tinv(d, e, w, method=meth))
    d, e = inputs.glued_wilkinson(20, 1e-10)
    w = inputs.eigenvalues(d, e)
    for meth in ("cwy", "mgs"):
        for mt in (0, 1):
            Zd = np.load(tmp_path / ("420_%s_%d.npy" % (meth, mt)))
            Z = gpu.tinv(d, e, w, method=meth, max_team=mt)
            assert np.array_equal(Zd, Z), (meth, mt)


def test_debug_build_check_fires_without_a_fault(gpu, tmp_path):
    assert "FIRED_OK" in _child("fire", tmp_path)


def test_bounded_barrier_wait_gives_up_and_the_next_call_succeeds(gpu):
    d, e = inputs.glued_wilkinson(100, 1e-10)  # n = 2100: CTA teams of several CTAs
    w = inputs.eigenvalues(d, e)
    cnt = np.zeros(4, dtype=np.int64)
    gpu.tinv(d, e, w, counters=cnt.ctypes.data)
    assert cnt[2] > 0  # clusters on CTA teams, so the cluster kernel meets at team barriers
    with pytest.raises(gpu.TinvError) as ex:
        gpu.tinv(d, e, w, spin_limit=1)
    assert ex.value.code == -103  # TINV_ETIMEDOUT
    Z, info, *_ = gpu.tinv(d, e, w, return_info=True)
    assert info == 0 and residual_ratio(d, e, w, Z) <= 10 and orth_ratio(Z) <= 10
    head = gpu.plan(d, e, w)[1]
    Z2 = gpu.tinv(d, e, w)
    for idx in clusters_from_heads(head):
        assert sin_angle(Z[:, idx], Z2[:, idx]) <= 1e-12
