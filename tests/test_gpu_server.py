"""Serving (tinv_server_*): requests submitted at any time run in waves of the batched path.

Checked here: each result is the same alone and in a mix (bit-identical with one CTA per
cluster, within 1e-10 by subspace angle with CTA teams), requests that arrive while a wave is on
the GPU start in a second wave before the first finishes (two waves in flight), eigenvalues may
be left to the server (GPU bisection, bit-exact with the oracle's), cancellation, back-pressure
and the latency statistics."""
import threading
import time

import numpy as np
import pytest

from helpers import clusters_from_heads, orth_ratio, residual_ratio, sin_angle
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


def _ok(d, e, w, Z):
    """The invariants of a correct eigenvector set: residual <= 10 n eps ||T||_1 and
    orthogonality <= 10 n eps."""
    return residual_ratio(d, e, w, Z) <= 10 and orth_ratio(Z) <= 10


def _mix(count, seed, lo=40, hi=700):
    g = np.random.default_rng(seed)
    out = []
    for q in range(count):
        n = int(np.exp(g.uniform(np.log(lo), np.log(hi))))
        if q % 3 == 2:
            d, e = inputs.glued_wilkinson(max(1, n // 21), 1e-10)
        else:
            d, e = inputs.uniform(n, seed=seed * 100 + q)
        out.append((d, e, inputs.eigenvalues(d, e)))
    return out


def test_server_same_alone_and_in_mix_bit_identical(gpu):
    probs = _mix(12, 1)
    target = probs[5]
    with gpu.Server(max_team=1) as srv:
        t = srv.submit(*target, seed=7)
        Z_alone, info = srv.wait(t)
        assert info == 0
        tickets = [srv.submit(d, e, w, seed=7) for d, e, w in probs]
        results = [srv.wait(t) for t in tickets]
    Z_mix = results[5][0]
    assert np.array_equal(Z_alone, Z_mix)
    Z_single = gpu.tinv(*target, seed=7, max_team=1)
    assert np.array_equal(Z_alone, Z_single)
    for (d, e, w), (Z, info) in zip(probs, results):
        assert info == 0
        assert _ok(d, e, w, Z)


def test_server_same_alone_and_in_mix_with_teams(gpu):
    big = inputs.glued_wilkinson(100, 1e-10)
    big = (big[0], big[1], inputs.eigenvalues(*big))
    others = _mix(10, 2)
    with gpu.Server() as srv:
        Z_alone, info = srv.wait(srv.submit(*big))
        assert info == 0
        ts = [srv.submit(d, e, w) for d, e, w in others[:5]]
        tb = srv.submit(*big)
        ts += [srv.submit(d, e, w) for d, e, w in others[5:]]
        Z_mix, info = srv.wait(tb)
        for t in ts:
            assert srv.wait(t)[1] == 0
    assert info == 0
    d, e, w = big
    assert _ok(d, e, w, Z_mix)
    head = gpu.plan(d, e, w)[1]
    for idx in clusters_from_heads(head):
        assert sin_angle(Z_alone[:, idx], Z_mix[:, idx]) <= 1e-10


def test_server_admits_while_a_wave_runs(gpu):
    big = inputs.glued_wilkinson(120, 1e-10)  # n = 2520: tens of milliseconds on the GPU
    big = (big[0], big[1], inputs.eigenvalues(*big))
    small = _mix(24, 3, lo=32, hi=200)
    with gpu.Server(max_inflight=2) as srv:
        tb = srv.submit(*big)
        time.sleep(0.002)  # the big request's wave is on the GPU now
        ts = [srv.submit(d, e, w) for d, e, w in small]
        done_small = []
        for t in ts:
            srv.wait(t)
            done_small.append((time.perf_counter(), srv.poll(tb) if tb else None))
        Zb, info = srv.wait(tb)
        st = srv.stats()
    assert info == 0
    assert st["completed"] == 25 and st["failed"] == 0
    assert st["waves"] >= 2 and st["max_inflight_seen"] == 2
    # at least some small requests completed while the big one was still running
    assert any(state == "running" for _, state in done_small)
    assert st["p50_ms"] > 0 and st["p99_ms"] >= st["p50_ms"] and st["problems_per_s"] > 0


def test_server_computes_eigenvalues_when_none_given(gpu, orc):
    probs = _mix(6, 4)
    with gpu.Server(max_team=1) as srv:
        ts = [srv.submit(d, e, None, seed=3) for d, e, _ in probs]
        res = [srv.wait(t) for t in ts]
    for (d, e, _), (Z, info) in zip(probs, res):
        assert info == 0
        wo = orc.bisect(d, e)  # the server's bisection is bit-exact with this one
        Z1 = gpu.tinv(d, e, wo, seed=3, max_team=1)
        assert np.array_equal(Z, Z1)


def test_server_cancel_and_backpressure(gpu):
    big = inputs.glued_wilkinson(150, 1e-10)
    big = (big[0], big[1], inputs.eigenvalues(*big))
    small = _mix(6, 5)
    with gpu.Server(max_inflight=1, max_pending=3) as srv:
        tb = srv.submit(*big)
        time.sleep(0.002)
        ts = [srv.submit(*p) for p in small[:3]]
        # three queued: the fourth is refused until the queue drains
        with pytest.raises(gpu.TinvError) as ex:
            srv.submit(*small[3])
        assert ex.value.code == -104  # TINV_EAGAIN
        Zc = srv._bufs[ts[0]]
        Zc[:] = 123.0
        assert srv.cancel(ts[0]) == 0
        with pytest.raises(gpu.TinvError) as ex:
            srv.wait(ts[0])
        assert ex.value.code == -105  # TINV_ECANCELED
        assert np.all(Zc == 123.0)  # a cancelled request's buffer is not written
        for t in ts[1:] + [tb]:
            assert srv.wait(t)[1] == 0
        st = srv.stats()
    assert st["cancelled"] == 1 and st["rejected"] == 1 and st["completed"] == 3


def test_server_concurrent_submitters(gpu):
    probs = _mix(30, 6, lo=20, hi=300)
    out = {}
    with gpu.Server() as srv:
        def worker(lo, hi):
            for q in range(lo, hi):
                d, e, w = probs[q]
                out[q] = srv.submit(d, e, w, seed=q)
        th = [threading.Thread(target=worker, args=(i * 10, i * 10 + 10)) for i in range(3)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        res = {q: srv.wait(t) for q, t in out.items()}
    for q, (Z, info) in res.items():
        d, e, w = probs[q]
        assert info == 0 and _ok(d, e, w, Z)


def test_server_cancel_is_exclusive_with_delivery(gpu):
    # A cancel that races with the copy of a finished wave's result into Z: either it succeeds
    # (returns 0) and Z is never written, or it reports the request as completed (1) and the
    # request delivers a full result.  Cancels are issued at spread-out times around the end of
    # the wave, so some land during the copy into the caller's buffer.
    d, e = inputs.glued_wilkinson(60, 1e-10)  # n = 1260: a 12.7 MB result per request
    w = inputs.eigenvalues(d, e)
    sentinel = 123.0
    outcomes = set()
    with gpu.Server(max_inflight=1) as srv:
        _, info = srv.wait(srv.submit(d, e, w))  # warm-up, and the wave's duration
        assert info == 0
        t0 = time.perf_counter()
        srv.wait(srv.submit(d, e, w))
        dur = time.perf_counter() - t0
        for k in range(24):
            Z = np.full((len(d), len(d)), sentinel, order="F")
            t = srv.submit(d, e, w, out=Z)
            time.sleep(dur * (0.6 + 0.05 * k))
            rc = srv.cancel(t)
            assert rc in (0, 1), rc
            outcomes.add(rc)
            if rc == 0:
                with pytest.raises(gpu.TinvError) as ex:
                    srv.wait(t)
                assert ex.value.code == -105  # TINV_ECANCELED
                time.sleep(0.01)
                assert np.all(Z == sentinel), k  # never written, not even partly
            else:
                Zr, info = srv.wait(t)
                assert info == 0 and not np.any(Zr == sentinel)
                assert _ok(d, e, w, Zr)
    assert outcomes  # at least one cancel was decided
