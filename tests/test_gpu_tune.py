"""The team-cap autotuner (tinv_tune through the C ABI): its choice is the automatic rule or a
power-of-two cap, a repeated call on the same shape is served from the tune cache without running
anything, a different spectrum of the same order is a different key, MGS has nothing to tune, and
a call with the chosen cap meets the residual and orthogonality bounds, and choices saved to a
file and loaded again are served from the cache."""
import numpy as np
import pytest

from helpers import orth_ratio, residual_ratio
from paper_1209_1910_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1209_1910_gb300 import binding, build

    build.build()
    binding.load()
    return binding


def test_tune_choice_cache_and_bounds(gpu, orc, tmp_path):
    d, e = inputs.glued_wilkinson(100, 1e-10)  # n = 2100: 7 clusters of 200 and 7 of 100 members
    w = orc.bisect(d, e)
    gpu.tune_clear()
    mt, ms, cached = gpu.tune(d, e, w, reps=1)
    assert not cached and ms > 0.0
    assert mt == 0 or (2 <= mt <= 128 and mt & (mt - 1) == 0)
    mt2, ms2, cached2 = gpu.tune(d, e, w, reps=1)
    assert cached2 and (mt2, ms2) == (mt, ms)
    Z = gpu.tinv(d, e, w, max_team=mt)
    assert residual_ratio(d, e, w, Z) <= 10 and orth_ratio(Z) <= 10
    # the same order with another spectrum (uniform random d, e) is another key: timed anew
    d3, e3 = inputs.uniform(2100, seed=4)
    w3 = orc.bisect(d3, e3)
    _, _, cached3 = gpu.tune(d3, e3, w3, reps=1)
    assert not cached3
    # the cache through a file: the device-name keys written by tinv_tune_save match the keys a
    # later tinv_tune builds, so reloaded choices are served without timing
    path = str(tmp_path / "tune.txt")
    gpu.tune_save(path)
    lines = open(path).read().splitlines()
    assert lines[0] == "# tinv tune cache v2" and len(lines) == 3
    gpu.tune_clear()
    _, _, cached4 = gpu.tune(d, e, w, reps=1)
    assert not cached4
    gpu.tune_clear()
    assert gpu.tune_load(path) == 2
    mt5, ms5, cached5 = gpu.tune(d, e, w, reps=1)
    assert cached5 and mt5 == mt
    gpu.tune_clear()


def test_tune_mgs_keeps_the_automatic_rule(gpu, orc):
    d, e = inputs.glued_wilkinson(10, 1e-10)  # n = 210
    w = orc.bisect(d, e)
    mt, ms, _ = gpu.tune(d, e, w, method="mgs", reps=1)
    assert mt == 0 and ms > 0.0


def test_tune_auto_picks_block_and_cap(gpu, orc):
    # the switch between one member at a time and the blocked compact-WY form, then the cap
    d, e = inputs.glued_wilkinson(100, 1e-10)
    w = orc.bisect(d, e)
    gpu.tune_clear()
    mt, blk, ms, cached = gpu.tune_auto(d, e, w, reps=1)
    assert not cached and ms > 0.0
    assert blk in (0, 4, 8, 16)
    assert mt == 0 or (2 <= mt <= 128 and mt & (mt - 1) == 0)
    assert gpu.tune_auto(d, e, w, reps=1) == (mt, blk, ms, True)
    Z = gpu.tinv(d, e, w, max_team=mt, block=blk)
    assert residual_ratio(d, e, w, Z) <= 10 and orth_ratio(Z) <= 10
    # MGS has neither teams nor blocks
    mt2, blk2, _, _ = gpu.tune_auto(d, e, w, method="mgs", reps=1)
    assert (mt2, blk2) == (0, 0)
    gpu.tune_clear()


def test_tune_batch_is_keyed_by_the_size_profile(gpu, orc):
    probs = [inputs.glued_wilkinson(40, 1e-10), inputs.uniform(300, seed=2), inputs.uniform(97, seed=3)]
    ds, es = [p[0] for p in probs], [p[1] for p in probs]
    ws = [orc.bisect(d, e) for d, e in probs]
    gpu.tune_clear()
    mt, blk, ms, cached = gpu.tune_batch(ds, es, ws, reps=1)
    assert not cached and ms > 0.0 and blk in (0, 4, 8, 16)
    assert gpu.tune_batch(ds, es, ws, reps=1)[3]  # the same profile: served from the cache
    # another size profile is another key
    assert not gpu.tune_batch(ds[:2], es[:2], ws[:2], reps=1)[3]
    Zs = gpu.tinv_batch(ds, es, ws, max_team=mt, block=blk)
    for d, e, w, Z in zip(ds, es, ws, Zs):
        assert residual_ratio(d, e, w, Z) <= 10 and orth_ratio(Z) <= 10
    gpu.tune_clear()
