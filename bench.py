#!/usr/bin/env python3
"""Benchmark: eigenvectors per second of inverse iteration with compact-WY reorthogonalization
(arXiv:1209.1910, Alg. 4) on one GB300, with its roofline fraction and a CPU-oracle baseline.

Default workload: glued Wilkinson matrix, 200 copies of W_21^+ glued by 1e-10 (n = 4200,
14 Peters-Wilkinson clusters of 400 and 200 members), all 4200 eigenvectors, FP64.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One JSON line is printed by rank 0.  `value` is the device-timed throughput with inputs
resident in HBM (CUDA events around each step on the launching stream, L2 flushed by a
512 MiB write between steps); `e2e` is the same metric through the host-pointer C ABI call
(pinned host buffers, host<->device copies inside the timed region).  With N > 1 (torchrun)
every rank solves its own copy of a single-problem workload (replicas), and the batch workload
is split into per-rank problem shards; there is no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1209_1910_gb300 import inputs  # noqa: E402

WORKLOADS = {
    "glued4200": "glued Wilkinson 200 x W21+ (glue 1e-10), n=4200, all eigenvectors",
    "glued2100": "glued Wilkinson 100 x W21+ (glue 1e-10), n=2100, all eigenvectors",
    "uniform1000": "uniform[-1,1] d,e (seed 1), n=1000, all eigenvectors",
    "toeplitz4200": "Toeplitz d=2 e=1, n=4200, all eigenvectors (one cluster)",
    "toeplitz6000": "Toeplitz d=2 e=1, n=6000, all eigenvectors (one cluster; its compact-WY Y, "
                    "144 MB, exceeds the 126 MB L2)",
    "uniform10000": "uniform[-1,1] d,e (seed 1), n=10000, all eigenvectors",
    "zero10000": "Toeplitz d=0 e=1, n=10000, all eigenvectors (one cluster)",
    "batch512": "512 problems, n log-uniform [64,4096] (seed 2), even U[-1,1] d,e, odd glued "
                "W21+ (glue 1e-10); all eigenvectors of every problem, one tinv_batch call",
}
WORKLOADS["split4200"] = ("glued Wilkinson 200 x W21+ with exactly zero glue, n=4200: all eigenpairs "
                          "from (d, e) by tinv_eig (200 unreduced blocks of 21)")
WORKLOADS["bidiag2000"] = ("upper bidiagonal n=2000 (seed 1), a = +-U[1,2), b = U[-1/2,1/2): all "
                           "singular triplets by tinv_bdsvd (Golub-Kahan form of order 4000, 76 "
                           "clusters, the largest 583)")
WORKLOADS["serve"] = ("Poisson request stream (seed 3), 256 requests per load level, n log-uniform "
                      "[128,4096] (the configuration's upper end 16384 capped at 4096: a uniform "
                      "n=16384 request is one cluster of ~n members, about a minute of GPU time), "
                      "70% U[-1,1] / 30% glued W21+; eigenvalues computed by the server; offered at "
                      "0.5x, 0.9x and 1.3x the saturated rate")
# kernels one call enqueues: plan (2), LU (2), first sweep, cluster kernel, CWY finalize, status
LAUNCHES = {"cwy": 8, "mgs": 7}
# the drivers add: split marks, bisection, scatter (tinv_eig); Golub-Kahan form, bisection,
# half split (tinv_bdsvd)
DRIVER_EXTRA_LAUNCHES = {"split4200": 3, "bidiag2000": 3}
FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64 (vector and tensor alike), TFLOP/s
# DRAM bytes (read + write) of one cluster-kernel launch, from one ncu capture of the current
# kernel (dram__bytes_read.sum + dram__bytes_write.sum); None where no capture exists
# DRAM bytes of one k_chain launch (ncu dram__bytes_read.sum + dram__bytes_write.sum, one pass),
# by workload, method and block; None for a configuration not captured with the current kernel
TRAFFIC_BYTES = {("glued4200", "cwy", 16): 16.56e9}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="glued4200")
    ap.add_argument("--method", choices=["cwy", "mgs"], default="cwy")
    ap.add_argument("--block", type=int, default=None,
                    help="compact WY: cluster members orthogonalized in blocks of up to this many "
                         "(Sec. 3.2's block form; 0 = one member at a time, Alg. 4); default 16, "
                         "0 for the served stream and the split driver")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batch, serving and n=1000 child runs of the default workload")
    ap.add_argument("--phases", action="store_true",
                    help="phase timing of the cluster kernel (diagnostic build), no bench line")
    ap.add_argument("--phases-child", action="store_true", help=argparse.SUPPRESS)
    return ap.parse_args()


# ------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
               "-lms", "100"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)

    def summary(self):
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in self.rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in self.rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


# ------------------------------------------------------------------------------------------
def algorithmic_flops(n: int, head: np.ndarray, iters: np.ndarray, method: str) -> float:
    """Flops of the reorthogonalization per launch of the cluster kernel: per member sweep with
    k previous cluster vectors, 8nk - 3k^2 for compact WY (Sec. 3.3.2; sums to 4m^2n - m^3,
    Table 1) and 4nk for MGS (sums to 2m^2n)."""
    j = np.arange(len(head))
    k = (j - head).astype(np.float64)
    sweeps = np.abs(iters).astype(np.float64)
    mem = k >= 1
    if method == "cwy":
        per = 8.0 * n * k - 3.0 * k * k
    else:
        per = 4.0 * n * k
    return float(np.sum(per[mem] * sweeps[mem]))


def cpu_sample(name: str, method: str, d, e, w):
    """Bounded oracle sample: the first 400-member and the first 200-member cluster of the
    glued workload (the workload holds 7 of each, so the sample has its cluster mix); for other
    workloads the first cluster(s) up to ~600 eigenvectors."""
    import oracle

    oracle.build()
    head = oracle.plan(d, e, w)[1]
    starts = np.flatnonzero(head == np.arange(len(head)))
    ends = np.r_[starts[1:], len(head)]
    cl = list(zip(starts, ends))
    if name == "glued4200":
        pick = [next(c for c in cl if c[1] - c[0] == 400), next(c for c in cl if c[1] - c[0] == 200)]
        desc = "oracle on the first 400-member and first 200-member clusters (600 of 4200 vectors)"
    else:
        pick, tot = [], 0
        for c in sorted(cl, key=lambda c: c[0]):
            if tot >= 600:
                break
            pick.append(c)
            tot += c[1] - c[0]
        desc = "oracle on the first %d eigenvectors (whole clusters)" % tot
    t0 = time.perf_counter()
    nv = 0
    for s, t in pick:
        oracle.tinv(d, e, w[s:t], method, j0=int(s))
        nv += t - s
    dt = time.perf_counter() - t0
    return nv / dt, desc


def cpu_parallel(name: str, method: str, d, e, w):
    """The oracle on all host cores: independent clusters (whole ones, singletons grouped into
    ranges) run in threads (the oracle's C calls release the interpreter lock and share no
    state), longest first.  For the glued workload the whole problem is timed; for the others the
    clusters of the single-core sample.  Returns (eigvecs/s, cores, description)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle

    oracle.build()
    head = oracle.plan(d, e, w)[1]
    starts = np.flatnonzero(head == np.arange(len(head)))
    ends = np.r_[starts[1:], len(head)]
    cl = list(zip(starts.tolist(), ends.tolist()))
    n = len(d)
    if name != "glued4200":
        pick, tot = [], 0
        for c in cl:
            if tot >= 600:
                break
            pick.append(c)
            tot += c[1] - c[0]
        cl = pick
    cores = os.cpu_count() or 1
    # group consecutive clusters into ranges of at least ~1/(4 cores) of the total cost
    cost = lambda c: float(c[1] - c[0]) ** 2 * n + float(c[1] - c[0]) * n
    total = sum(cost(c) for c in cl)
    tasks, cur, ccost = [], None, 0.0
    for c in cl:
        cur = (cur[0], c[1]) if cur else c
        ccost += cost(c)
        if ccost >= total / (4 * cores):
            tasks.append((cur, ccost))
            cur, ccost = None, 0.0
    if cur:
        tasks.append((cur, ccost))
    tasks.sort(key=lambda tc: -tc[1])
    nv = sum(c[1] - c[0] for c in cl)

    def run(task):
        (a, b), _ = task
        oracle.tinv(d, e, w[a:b], method, j0=int(a))

    t0 = time.perf_counter()
    with ThreadPoolExecutor(cores) as ex:
        list(ex.map(run, tasks))
    dt = time.perf_counter() - t0
    desc = ("oracle on %d threads over %d independent cluster ranges (%d of %d vectors)"
            % (cores, len(tasks), nv, len(w)))
    return nv / dt, cores, desc


def lapack_dstein_sample(name: str, d, e, w):
    """Context, not a baseline of this library: LAPACK's own bisection + DSTEIN (MGS
    reorthogonalization, the paper's comparison method) through SciPy, on the clusters of the
    single-core oracle sample, in this process with the BLAS library's default threads.  Returns
    None when SciPy is missing."""
    try:
        import scipy.linalg
    except ImportError:
        return None
    import oracle

    oracle.build()
    head = oracle.plan(d, e, w)[1]
    starts = np.flatnonzero(head == np.arange(len(head)))
    ends = np.r_[starts[1:], len(head)]
    cl = list(zip(starts.tolist(), ends.tolist()))
    if name == "glued4200":
        pick = [next(c for c in cl if c[1] - c[0] == 400), next(c for c in cl if c[1] - c[0] == 200)]
    else:
        pick, tot = [], 0
        for c in cl:
            if tot >= 600:
                break
            pick.append(c)
            tot += c[1] - c[0]
    t0 = time.perf_counter()
    nv = 0
    for a, b in pick:
        scipy.linalg.eigh_tridiagonal(d, e, select="i", select_range=(a, b - 1),
                                      lapack_driver="stebz")
        nv += b - a
    dt = time.perf_counter() - t0
    return {"value": nv / dt, "unit": "eigvec/s", "kind": "LAPACK dstebz + dstein (SciPy)",
            "sample": "%d vectors: the clusters of the oracle sample, eigenvalues included" % nv}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.workload == "batch512":
        probs = inputs.batch_matrices()
        sample = lambda: cpu_sample_batch(args.method, probs)
    elif args.workload == "serve":
        probs = serve_requests()[0]
        sample = lambda: cpu_sample_batch(args.method, probs, stride=16)
    elif args.workload in DRIVER_EXTRA_LAUNCHES:
        sample = lambda: cpu_sample_driver(args.workload, args.method)
    else:
        d, e, w = inputs.workload(args.workload)
        sample = lambda: cpu_sample(args.workload, args.method, d, e, w)
    for _ in range(args.warmup):
        sample()
    vals = []
    desc = ""
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, desc = sample()
        vals.append(v)
    el = time.perf_counter() - t0
    value = float(statistics.mean(vals))
    out = {
        "impl": "reference", "metric": driver_metric(args.workload)[0], "value": value,
        "unit": driver_metric(args.workload)[1],
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "method": args.method},
        "cpu_baseline": {"value": value, "unit": driver_metric(args.workload)[1], "cores": 1,
                         "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": driver_metric(args.workload)[1], "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def driver_metric(workload: str):
    if workload == "bidiag2000":
        return "singular_triplets_per_s", "triplet/s"
    return "eigvecs_per_s", "eigvec/s"


def driver_inputs(workload: str):
    if workload == "split4200":
        return inputs.glued_wilkinson(200, 0.0)
    return inputs.bidiagonal(2000, seed=1)


def cpu_sample_driver(workload: str, method: str):
    """Bounded oracle sample for the driver workloads: the whole split driver on the zero-glue
    matrix (200 blocks of order 21), or, for the bidiagonal workload, bisection of its
    Golub-Kahan form plus inverse iteration for the first clusters of at most 200 members, in
    order, up to ~600 triplets (the half split is O(n) per triplet)."""
    import oracle

    oracle.build()
    a, b = driver_inputs(workload)
    if workload == "split4200":
        t0 = time.perf_counter()
        oracle.eig_split(a, b, method=method)
        return len(a) / (time.perf_counter() - t0), "oracle split driver on the whole matrix"
    n = len(a)
    t0 = time.perf_counter()
    d2, e2 = oracle.golub_kahan(a, b)
    s = oracle.bisect(d2, e2)[n:]
    head = oracle.plan(d2, e2, s)[1]
    starts = np.flatnonzero(head == np.arange(len(head)))
    ends = np.r_[starts[1:], len(head)]
    tot = 0
    for c0, c1 in zip(starts, ends):
        if tot >= 600:
            break
        if c1 - c0 > 200:
            continue
        oracle.tinv(d2, e2, s[c0:c1], method, j0=int(c0))
        tot += c1 - c0
    dt = time.perf_counter() - t0
    return tot / dt, ("oracle: bisection of the order-%d Golub-Kahan form, then %d triplets "
                      "(the first whole clusters of <= 200 members)" % (2 * n, tot))


def batch_arm(args):
    """tinv_batch over the 512-problem workload: one launch sequence per step, against
    one-problem-at-a-time calls of the same problems."""
    import torch

    from paper_1209_1910_gb300 import binding, build
    from paper_1209_1910_gb300.replicas import env_rank, lpt_shards, problem_cost, reduce_max, reduce_sum

    rank, world, local = env_rank()
    dist = None
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist_mod

        dist = dist_mod
        dist.init_process_group("nccl", device_id=dev)
    build.build()
    binding.load()
    probs_all = inputs.batch_matrices()
    # several GPUs: each rank solves its own shard of the problems (no data-path collective)
    shard = lpt_shards([problem_cost(len(p[0])) for p in probs_all], world)[rank]
    probs = [probs_all[q] for q in shard]
    ns, off_de, off_z = binding.pack_offsets([len(p[0]) for p in probs])
    M, nprob = int(ns.sum()), len(ns)
    D = np.zeros(M)
    E = np.zeros(M)
    for q, (d, e) in enumerate(probs):
        D[off_de[q]:off_de[q] + ns[q]] = d
        E[off_de[q]:off_de[q] + ns[q] - 1] = e
    td, te = torch.from_numpy(D).to(dev), torch.from_numpy(E).to(dev)
    tw = torch.zeros(M, dtype=torch.float64, device=dev)
    binding.bisect_batch_device(ns, off_de, td, te, tw)  # eigenvalues (setup, untimed)
    tz = torch.zeros(int((ns * ns).sum()), dtype=torch.float64, device=dev)
    info = torch.zeros(nprob, dtype=torch.int64, device=dev)
    iters = torch.zeros(M, dtype=torch.int32, device=dev)
    blk = args.block if args.method == "cwy" else 0
    ws = torch.empty(binding.batch_workspace_size(ns, block=blk), dtype=torch.uint8, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    phase = np.zeros(4, dtype=np.float32)

    def step(with_phase):
        kw = {"phase_ms": phase.ctypes.data} if with_phase else {}
        binding.tinv_batch_device(ns, off_de, off_z, td, te, tw, tz, method=args.method,
                                  info=info, workspace=ws, iters=iters, block=blk, **kw)

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    bad = int((info != 0).sum().item())
    if bad:
        raise RuntimeError("warm-up: %d problems with info != 0" % bad)
    st = torch.cuda.current_stream(dev)
    sampler = ClockSampler(None)
    step_ms, chain_ms = [], []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    for _ in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        step(True)
        b.record(st)
        b.synchronize()
        step_ms.append(a.elapsed_time(b))
        chain_ms.append(float(phase[3]))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler.stop()
    total_ms = float(sum(step_ms))
    M_all, nprob_all = M, nprob
    if dist:
        total_ms = reduce_max(total_ms, dist, dev)
        M_all = int(reduce_sum(M, dist, dev))
        nprob_all = int(reduce_sum(nprob, dist, dev))
    value = M_all * args.steps / (total_ms * 1e-3)

    # checks: status of every problem; residual and orthogonality ratios of a sample
    nonconv = int(info.sum().item())
    W = tw.cpu().numpy()
    it = iters.cpu().numpy()
    eps = float(np.finfo(np.float64).eps)
    order = np.argsort(-ns)
    sample = sorted(set(order[:8].tolist() + list(range(0, nprob, 32))))
    worst_r = worst_o = 0.0
    flops = 0.0
    for q in range(nprob):
        n, a0 = int(ns[q]), int(off_de[q])
        head = binding.plan(D[a0:a0 + n], E[a0:a0 + n - 1], W[a0:a0 + n])[1]
        flops += algorithmic_flops(n, head, it[a0:a0 + n], args.method)
    for q in sample:
        n, a0, z0 = int(ns[q]), int(off_de[q]), int(off_z[q])
        Z = tz[z0:z0 + n * n].view(n, n).T  # column j = eigenvector j
        dq, eq, wq = td[a0:a0 + n], te[a0:a0 + n - 1], tw[a0:a0 + n]
        R = dq[:, None] * Z
        R[:-1] += eq[:, None] * Z[1:]
        R[1:] += eq[:, None] * Z[:-1]
        R -= Z * wq[None, :]
        dh, eh = D[a0:a0 + n], E[a0:a0 + n - 1]
        nrm = float(np.max(np.abs(dh) + np.r_[0, np.abs(eh)] + np.r_[np.abs(eh), 0]))
        worst_r = max(worst_r, float(R.abs().max()) / (n * eps * nrm))
        G = Z.T @ Z
        G.diagonal().sub_(1.0)
        worst_o = max(worst_o, float(G.abs().max()) / (n * eps))
    kern_ms = float(statistics.mean(chain_ms))
    achieved = flops / (kern_ms * 1e-3) / 1e12
    out = {
        "metric": "eigvecs_per_s", "value": value, "unit": "eigvec/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "strong" if world > 1 else "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS["batch512"], "method": args.method, "block": blk,
                   "problems": nprob_all, "eigenvectors": M_all,
                   "parallelism": "problem shards (LPT)" if world > 1 else "single",
                   "inputs": "resident in HBM (eigenvalues by GPU bisection, untimed)",
                   "l2": "flushed by a 512 MiB write between steps"},
        "problems_per_s": nprob_all * args.steps / (total_ms * 1e-3),
        "check": {"nonconverged": nonconv, "sampled_problems": len(sample),
                  "worst_residual_ratio": worst_r, "worst_orth_ratio": worst_o,
                  "sweeps": int(np.abs(it).sum())},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                     "kernel": "k_chain", "kernel_ms": kern_ms, "flops_per_launch": flops,
                     "peak_source": "nominal GB300 FP64: 2 DFMA/clk/SM x 2 flop x 152 SMs x 2.07 GHz = 1.26 TFLOP/s",
                     "phase_ms": {"plan": float(phase[0]), "lu": float(phase[1]),
                                  "first": float(phase[2]), "chain": float(phase[3])}},
        "gpu_launches": LAUNCHES[args.method] * args.steps,
        "clocks": sampler.summary(),
    }

    # the same call captured once into a CUDA graph and replayed (the problem table is already
    # in the workspace, so the call enqueues kernels only)
    if world == 1:
        gs = torch.cuda.Stream()
        gs.wait_stream(st)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(gs):
            with torch.cuda.graph(graph, stream=gs):
                binding.tinv_batch_device(ns, off_de, off_z, td, te, tw, tz, method=args.method,
                                          info=info, workspace=ws, iters=iters, table_ready=1,
                                          block=blk)
        # replay() launches on the current stream: make it gs, the stream the events are on
        with torch.cuda.stream(gs):
            graph.replay()
        torch.cuda.synchronize()
        gms = []
        for _ in range(2):
            flush.zero_()
            info.fill_(-1)
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(gs):
                a.record(gs)
                graph.replay()
                b.record(gs)
            b.synchronize()
            gms.append(a.elapsed_time(b))
            if int(info.min().item()) < 0 or int(info.max().item()) != 0:
                raise RuntimeError("graph replay did not complete the batch (info %s)"
                                   % info.unique().tolist())
        out["graph_replay"] = {"value": M / (statistics.mean(gms) * 1e-3), "unit": "eigvec/s",
                               "ms_per_step": statistics.mean(gms)}
        del graph

    # the same problems one call at a time (each call a full launch sequence), same stream
    if not args.no_compare and world == 1:
        def one_at_a_time():
            for q in range(nprob):
                n, a0, z0 = int(ns[q]), int(off_de[q]), int(off_z[q])
                binding.tinv_device(td[a0:a0 + n], te[a0:a0 + n - 1], tw[a0:a0 + n],
                                    tz[z0:z0 + n * n], method=args.method, block=blk)
        one_at_a_time()
        torch.cuda.synchronize()
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        one_at_a_time()
        b.record(st)
        b.synchronize()
        t1 = a.elapsed_time(b)
        out["compare"] = {"one_at_a_time": {"value": M / (t1 * 1e-3), "ms": t1,
                                            "problems_per_s": nprob / (t1 * 1e-3)}}

    # end to end through the host-pointer C ABI (pinned buffers, copies inside the timed region)
    if not args.no_e2e and world == 1:
        import ctypes

        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        hd, he, hw = pin(D), pin(E), pin(W)
        hz = torch.empty(int((ns * ns).sum()), dtype=torch.float64).pin_memory()
        hinfo = np.zeros(nprob, dtype=np.int64)
        lib = binding.load()
        o = binding._opts(args.method, block=blk)
        P = ctypes.c_void_p

        def e2e_call():
            rc = lib.tinv_batch(nprob, binding._ptr(ns), binding._ptr(off_de), binding._ptr(off_z),
                                P(hd.data_ptr()), P(he.data_ptr()), P(hw.data_ptr()),
                                P(hz.data_ptr()), binding._ptr(hinfo), ctypes.byref(o))
            if rc != 0:
                raise RuntimeError("tinv_batch returned %d" % rc)
        e2e_call()
        el = 0.0
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e2e_call()
            el += time.perf_counter() - t0
        out["e2e"] = {"value": M * args.steps / el, "unit": "eigvec/s",
                      "h2d_bytes_per_step": 3 * M * 8 + nprob * 112,
                      "d2h_bytes_per_step": int((ns * ns).sum()) * 8 + nprob * 8 + 64}
        del hz

    if not args.no_cpu_baseline and world == 1:
        v, desc = cpu_sample_batch(args.method, probs)
        out["cpu_baseline"] = {"value": v, "unit": "eigvec/s", "cores": 1, "kind": "oracle",
                               "sample": desc}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def cpu_sample_batch(method, probs, stride=32):
    """Bounded oracle sample of the batch: every stride-th uniform and every stride-th glued
    problem (problems q with q mod stride in {0, 1}), whole; eigenvalues by the oracle's
    bisection (untimed)."""
    import oracle

    oracle.build()
    pick = [q for q in range(len(probs)) if q % stride in (0, 1)]
    ws = {q: oracle.bisect(*probs[q]) for q in pick}
    tot = 0
    t0 = time.perf_counter()
    for q in pick:
        d, e = probs[q]
        oracle.tinv(d, e, ws[q], method)
        tot += len(d)
    dt = time.perf_counter() - t0
    return tot / dt, ("oracle on %d whole problems of the batch (q mod %d in {0,1}; %d "
                      "eigenvectors)" % (len(pick), stride, tot))


def serve_requests(count=256, hi=4096, seed=3):
    """The serving workload: (d, e) per request and unit-rate exponential arrival gaps."""
    g = inputs.rng(seed)
    reqs = []
    for r in range(count):
        n = int(round(math.exp(g.uniform(math.log(128), math.log(hi)))))
        if g.uniform() < 0.3:
            d, e = inputs.glued_wilkinson(max(1, round(n / 21)), 1e-10)
        else:
            d, e = inputs.uniform(n, seed=seed * 7919 + r)
        reqs.append((d, e))
    return reqs, g.exponential(1.0, count)


def serve_arm(args, count=256, hi=4096):
    """Request-queue server under Poisson load: saturated rate (all requests at once), then the
    same requests offered at 0.5x, 0.9x and 1.3x that rate; p50/p99 latency per level.  Against
    one-problem-at-a-time calls (tinv through the host API, one after another)."""
    import torch

    from paper_1209_1910_gb300 import binding, build

    torch.cuda.set_device(0)
    build.build()
    binding.load()
    reqs, gaps = serve_requests(count, hi)
    blk = args.block if args.method == "cwy" else 0
    M = sum(len(d) for d, _ in reqs)
    outs = [np.zeros((len(d), len(d)), order="F") for d, _ in reqs]

    def run_level(rate):
        """Submit every request at its arrival time (rate None: all at once); returns stats."""
        with binding.Server(method=args.method, block=blk) as srv:
            t0 = time.perf_counter()
            tick = []
            at = 0.0
            for (d, e), gap, Z in zip(reqs, gaps, outs):
                if rate:
                    at += gap / rate
                    dt = t0 + at - time.perf_counter()
                    if dt > 0:
                        time.sleep(dt)
                tick.append(srv.submit(d, e, None, out=Z))
            infos = [srv.wait(t)[1] for t in tick]
            el = time.perf_counter() - t0
            st = srv.stats()
        if any(i != 0 for i in infos):
            raise RuntimeError("non-converged vectors in served requests")
        st["wall_s"] = el
        return st

    warm = max(1, args.warmup)
    for _ in range(warm):
        run_level(None)  # warm-up (builds the memory pool and pinned staging)
    sampler = ClockSampler(None)
    sampler.start()
    sat = run_level(None)
    sat_rate = count / sat["wall_s"]
    levels = []
    for f in (0.5, 0.9, 1.3):
        st = run_level(f * sat_rate)
        levels.append({"load": f, "offered_per_s": f * sat_rate,
                       "achieved_per_s": count / st["wall_s"], "p50_ms": st["p50_ms"],
                       "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"], "waves": st["waves"],
                       "mean_wave_problems": st["mean_wave_problems"],
                       "max_inflight_seen": st["max_inflight_seen"]})
    sampler.stop()
    # accuracy of a sample of the served results (last level)
    eps = float(np.finfo(np.float64).eps)
    worst_r = worst_o = 0.0
    for q in range(0, count, 16):
        d, e = reqs[q]
        Z = outs[q]
        w = binding.bisect(d, e)
        n = len(d)
        R = d[:, None] * Z
        R[:-1] += e[:, None] * Z[1:]
        R[1:] += e[:, None] * Z[:-1]
        R -= Z * w[None, :]
        nrm = float(np.max(np.abs(d) + np.r_[0, np.abs(e)] + np.r_[np.abs(e), 0]))
        worst_r = max(worst_r, float(np.abs(R).max()) / (n * eps * nrm))
        worst_o = max(worst_o, float(np.abs(Z.T @ Z - np.eye(n)).max()) / (n * eps))
    out = {
        "metric": "served_problems_per_s", "value": sat_rate, "unit": "problems/s", "n_gpus": 1,
        "steps": 1, "warmup": warm, "ms_per_step": 1e3 * sat["wall_s"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS["serve"], "method": args.method, "block": blk,
                   "requests": count,
                   "eigenvectors": M, "parallelism": "single",
                   "inputs": "host arrays submitted through tinv_submit (copies, bisection and "
                             "inverse iteration inside the timed region)"},
        "eigvecs_per_s": M / sat["wall_s"],
        "saturated": {"p50_ms": sat["p50_ms"], "p99_ms": sat["p99_ms"], "waves": sat["waves"],
                      "mean_wave_problems": sat["mean_wave_problems"],
                      "max_inflight_seen": sat["max_inflight_seen"]},
        "levels": levels,
        "check": {"sampled_requests": len(range(0, count, 16)), "worst_residual_ratio": worst_r,
                  "worst_orth_ratio": worst_o},
        "clocks": sampler.summary(),
        "e2e": {"value": sat_rate, "unit": "problems/s",
                "h2d_bytes_per_step": int(3 * M * 8), "d2h_bytes_per_step": int(sum(len(d) ** 2 for d, _ in reqs) * 8)},
    }
    if not args.no_compare:
        t0 = time.perf_counter()
        for (d, e), Z in zip(reqs, outs):
            w = binding.bisect(d, e)
            binding.tinv(d, e, w, method=args.method, out=Z, block=blk)
        el = time.perf_counter() - t0
        out["compare"] = {"one_at_a_time": {"value": count / el, "unit": "problems/s",
                                            "eigvecs_per_s": M / el}}
    print(json.dumps(out), flush=True)


def driver_arm(args):
    """tinv_eig (split4200) or tinv_bdsvd (bidiag2000) on device arrays, one call per step; the
    calls synchronize their stream (block table, merge order), so a step is the whole call."""
    import torch

    from paper_1209_1910_gb300 import binding, build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and rank != 0:
        return  # one problem: replicas would repeat it, rank 0 reports
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    build.build()
    binding.load()
    a, b = driver_inputs(args.workload)
    n = len(a)
    ta, tb = (torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in (a, b))
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    phase = np.zeros(4, dtype=np.float32)
    iters = torch.zeros(n, dtype=torch.int32, device=dev)
    blk = args.block if args.method == "cwy" else 0
    if args.workload == "split4200":
        tw = torch.zeros(n, dtype=torch.float64, device=dev)
        tZ = torch.zeros((n, n), dtype=torch.float64, device=dev)
        tib = torch.zeros(n, dtype=torch.int64, device=dev)

        def step(with_phase):
            kw = {"phase_ms": phase.ctypes.data} if with_phase else {}
            return binding.eig_device(ta, tb, tw, tZ, tib, method=args.method, iters=iters,
                                      block=blk, **kw)[0]
    else:
        ts = torch.zeros(n, dtype=torch.float64, device=dev)
        tU = torch.zeros((n, n), dtype=torch.float64, device=dev)
        tV = torch.zeros((n, n), dtype=torch.float64, device=dev)

        def step(with_phase):
            kw = {"phase_ms": phase.ctypes.data} if with_phase else {}
            return binding.bdsvd_device(ta, tb, ts, tU, tV, method=args.method,
                                        iters=iters.data_ptr(), block=blk, **kw)

    for _ in range(args.warmup):
        if step(False) != 0:
            raise RuntimeError("warm-up run reported non-converged vectors")
    torch.cuda.synchronize()
    sampler = ClockSampler(None)
    st = torch.cuda.current_stream(dev)
    step_ms, chain_ms = [], []
    sampler.start()
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        info = step(True)
        e1.record(st)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        chain_ms.append(float(phase[3]))
    torch.cuda.synchronize()
    sampler.stop()
    total_ms = float(sum(step_ms))
    value = n * args.steps / (total_ms * 1e-3)
    eps = float(np.finfo(np.float64).eps)
    it = iters.cpu().numpy()
    if args.workload == "split4200":
        Z = tZ.T
        R = ta[:, None] * Z
        R[:-1] += tb[:, None] * Z[1:]
        R[1:] += tb[:, None] * Z[:-1]
        R -= Z * tw[None, :]
        nrm = float(np.max(np.abs(a) + np.r_[0, np.abs(b)] + np.r_[np.abs(b), 0]))
        res = float(R.abs().max()) / (n * eps * nrm)
        G = tZ @ tZ.T
        G.diagonal().sub_(1.0)
        check = {"nonconverged": int(info), "residual_ratio": res,
                 "orth_ratio": float(G.abs().max()) / (n * eps)}
        # algorithmic CWY flops per block (each block is its own problem with its own plan)
        w_h, iblk = tw.cpu().numpy(), tib.cpu().numpy()
        blocks = np.r_[0, binding.split(a, b)]
        flops = 0.0
        for bi in range(len(blocks) - 1):
            s0, s1 = int(blocks[bi]), int(blocks[bi + 1])
            cols = np.flatnonzero(iblk == bi)
            hb = binding.plan(a[s0:s1], b[s0:s1 - 1], w_h[cols])[1]
            flops += algorithmic_flops(s1 - s0, hb, it[cols], args.method)
        del R, G
    else:
        Bv = ta[:, None] * tV.T
        Bv[:-1] += tb[:, None] * tV.T[1:]
        Rv = Bv - tU.T * ts[None, :]
        nrm = float(np.max(np.abs(a) + np.r_[0, np.abs(b)]))
        res = float(Rv.abs().max()) / (n * eps * nrm)
        GU = tU @ tU.T
        GU.diagonal().sub_(1.0)
        GV = tV @ tV.T
        GV.diagonal().sub_(1.0)
        check = {"nonconverged": int(info), "residual_ratio": res,
                 "orth_ratio_u": float(GU.abs().max()) / (n * eps),
                 "orth_ratio_v": float(GV.abs().max()) / (n * eps)}
        d2 = np.zeros(2 * n)
        e2 = np.zeros(2 * n - 1)
        e2[0::2], e2[1::2] = a, b
        s_h = ts.cpu().numpy()
        hb = binding.plan(d2, e2, s_h)[1]
        flops = algorithmic_flops(2 * n, hb, it, args.method)
        del Bv, Rv, GU, GV
    kern_ms = float(statistics.mean(chain_ms))
    achieved = flops / (kern_ms * 1e-3) / 1e12 if kern_ms > 0 else 0.0
    metric, unit = driver_metric(args.workload)
    out = {
        "metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "method": args.method, "block": blk,
                   "parallelism": "single", "inputs": "resident in HBM",
                   "l2": "flushed by a 512 MiB write between steps"},
        "check": check,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                     "kernel": "k_chain", "kernel_ms": kern_ms, "flops_per_launch": flops,
                     "peak_source": "nominal GB300 FP64: 2 DFMA/clk/SM x 2 flop x 152 SMs x 2.07 GHz = 1.26 TFLOP/s",
                     "phase_ms": {"plan": float(phase[0]), "lu": float(phase[1]),
                                  "first": float(phase[2]), "chain": float(phase[3])}},
        "gpu_launches": (LAUNCHES[args.method] + DRIVER_EXTRA_LAUNCHES[args.workload]) * args.steps,
        "clocks": sampler.summary(),
    }
    if not args.no_e2e:
        pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory().numpy()
        ha, hb2 = pin(a), pin(b)
        call = (lambda: binding.eig(ha, hb2, method=args.method, block=blk)) \
            if args.workload == "split4200" else (lambda: binding.bdsvd(ha, hb2, method=args.method, block=blk))
        call()
        el = 0.0
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            call()
            el += time.perf_counter() - t0
        nout = 1 if args.workload == "split4200" else 2
        out["e2e"] = {"value": n * args.steps / el, "unit": unit,
                      "h2d_bytes_per_step": (2 * n - 1) * 8,
                      "d2h_bytes_per_step": nout * n * n * 8 + n * 8 + 8}
    if not args.no_cpu_baseline:
        v, desc = cpu_sample_driver(args.workload, args.method)
        out["cpu_baseline"] = {"value": v, "unit": unit, "cores": 1, "kind": "oracle",
                               "sample": desc}
    print(json.dumps(out), flush=True)


def ours_arm(args):
    import torch
    if args.workload == "batch512":
        return batch_arm(args)
    if args.workload == "serve":
        return serve_arm(args)
    if args.workload in DRIVER_EXTRA_LAUNCHES:
        return driver_arm(args)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist_mod

        dist = dist_mod
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    from paper_1209_1910_gb300 import binding, build

    build.build()
    binding.load()

    d, e, w = inputs.workload(args.workload)
    n, m = len(d), len(w)
    td, te, tw = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (d, e, w))
    Zt = torch.zeros((m, n), dtype=torch.float64, device=dev)  # row j = eigenvector j
    iters = torch.zeros(m, dtype=torch.int32, device=dev)
    info = torch.zeros(1, dtype=torch.int64, device=dev)
    blk = args.block if args.method == "cwy" else 0
    ws = torch.empty(max(binding.workspace_size(n, m, block=blk), binding.workspace_size(n, m)),
                     dtype=torch.uint8, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    head = binding.plan(d, e, w)[1]
    phase = np.zeros(4, dtype=np.float32)
    counters = torch.zeros(4, dtype=torch.int64, device=dev)

    def step(method, with_phase, block=None):
        kw = {"phase_ms": phase.ctypes.data} if with_phase else {}
        b = blk if block is None else block
        binding.tinv_device(td, te, tw, Zt, method=method, workspace=ws, iters=iters, info=info,
                            counters=counters.data_ptr(), block=b if method == "cwy" else 0, **kw)

    for _ in range(args.warmup):
        step(args.method, False)
    torch.cuda.synchronize()
    if int(info.item()) != 0:
        raise RuntimeError("warm-up run returned info=%d" % int(info.item()))

    gpu_id = None
    try:
        gpu_id = str(torch.cuda.get_device_properties(dev).uuid)
        if not gpu_id.startswith("GPU-"):
            gpu_id = "GPU-" + gpu_id
    except Exception:
        gpu_id = None
    sampler = ClockSampler(gpu_id)
    st = torch.cuda.current_stream(dev)
    step_ms, chain_ms = [], []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    for _ in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        step(args.method, True)  # phase events inside the library synchronize the stream
        b.record(st)
        b.synchronize()
        step_ms.append(a.elapsed_time(b))
        chain_ms.append(float(phase[3]))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler.stop()
    total_ms = float(sum(step_ms))
    if dist:
        tt = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
    it = iters.cpu().numpy()
    nonconv = int(info.item())
    value = world * m * args.steps / (total_ms * 1e-3)

    # result check on the last step (on the GPU, fp64): residual and orthogonality ratios
    Z = Zt.T
    R = td[:, None] * Z
    R[:-1] += te[:, None] * Z[1:]
    R[1:] += te[:, None] * Z[:-1]
    R -= Z * tw[None, :]
    nrm = float(np.max(np.abs(d) + np.r_[0, np.abs(e)] + np.r_[np.abs(e), 0]))
    eps = float(np.finfo(np.float64).eps)
    res_ratio = float(R.abs().max()) / (n * eps * nrm)
    G = Zt @ Zt.T
    G.diagonal().sub_(1.0)
    orth_ratio = float(G.abs().max()) / (n * eps)
    del R, G

    flops = algorithmic_flops(n, head, it, args.method)
    kern_ms = float(statistics.mean(chain_ms))
    achieved = flops / (kern_ms * 1e-3) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS,
            "traffic": TRAFFIC_BYTES.get((args.workload, args.method, args.block)), "kernel": "k_chain",
            "kernel_ms": kern_ms, "flops_per_launch": flops,
            "peak_source": "nominal GB300 FP64: 2 DFMA/clk/SM x 2 flop x 152 SMs x 2.07 GHz = 1.26 TFLOP/s",
            "phase_ms": {"plan": float(phase[0]), "lu": float(phase[1]),
                         "first": float(phase[2]), "chain": float(phase[3])}}

    out = {
        "metric": "eigvecs_per_s", "value": value, "unit": "eigvec/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "method": args.method, "block": blk,
                   "parallelism": "replicas" if world > 1 else "single",
                   "inputs": "resident in HBM", "l2": "flushed by a 512 MiB write between steps"},
        "check": {"nonconverged": nonconv, "residual_ratio": res_ratio, "orth_ratio": orth_ratio,
                  "sweeps": int(np.abs(it).sum()),
                  "sequential_back_substitutions": {"cluster_kernel": int(counters[0].item()),
                                                    "first_sweep": int(counters[3].item())}},
        "roofline": roof,
        "gpu_launches": LAUNCHES[args.method] * args.steps,
        "clocks": sampler.summary(),
    }

    # end to end through the host-pointer C ABI (pinned buffers, copies inside the timed region)
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        hd, he, hw = pin(d), pin(e), pin(w)
        hz = torch.empty((m, n), dtype=torch.float64).pin_memory().numpy().T  # n x m, F-order
        binding.tinv(hd, he, hw, method=args.method, out=hz, block=blk)
        el = 0.0
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            binding.tinv(hd, he, hw, method=args.method, out=hz, block=blk)
            el += time.perf_counter() - t0
        if dist:
            tt = torch.tensor([el], dtype=torch.float64, device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            el = float(tt.item())
        out["e2e"] = {"value": world * m * args.steps / el, "unit": "eigvec/s",
                      "h2d_bytes_per_step": (n + (n - 1) + m) * 8,
                      "d2h_bytes_per_step": n * m * 8 + m * 4 + 64}

    # the MGS comparison on the same workload (Alg. 1 on the GPU), fewer steps.  Where MGS would
    # take minutes (one cluster of thousands of members on one CTA: Toeplitz, n = 10^4), both
    # methods run on the first SUB eigenvalues of the same matrix
    if not args.no_compare and args.method == "cwy" and world == 1:
        SUB = 500
        sizes = np.diff(np.r_[np.flatnonzero(np.r_[True, head[1:] != head[:-1]]), len(head)])
        mgs_cost = float(np.sum(sizes.astype(np.float64) ** 2)) * n  # ~ MGS flops / 6 per sweep
        msub = m if mgs_cost <= 2e10 else min(m, SUB)
        tw_c, Z_c = tw[:msub], Zt[:msub]

        def step_c(method, block):
            binding.tinv_device(td, te, tw_c, Z_c, method=method, workspace=ws, iters=iters[:msub],
                                info=info, counters=counters.data_ptr(),
                                block=block if method == "cwy" else 0)

        def timed_c(method, block):
            step_c(method, block)
            torch.cuda.synchronize()
            ms = []
            for _ in range(2):
                flush.zero_()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(st)
                step_c(method, block)
                b.record(st)
                b.synchronize()
                ms.append(a.elapsed_time(b))
            return statistics.mean(ms)

        t_mgs = timed_c("mgs", 0)
        ncl = int(counters[1].item())  # clusters with >= 2 members (MGS: one CTA each)
        P = torch.cuda.get_device_properties(dev).multi_processor_count
        out["compare"] = {"mgs": {"value": msub / (t_mgs * 1e-3), "ms_per_step": t_mgs,
                                  "ctas": "one CTA per cluster: %d clusters on %d of the %d CTAs "
                                          "of the persistent grid (compact WY spreads each "
                                          "cluster over a CTA team)" % (ncl, min(ncl, P), P)}}
        if msub < m:
            t_cwy = timed_c("cwy", blk)
            out["compare"]["subset"] = ("the first %d of the %d eigenvalues, both methods (MGS, one "
                                        "CTA per cluster, would take minutes on the whole matrix)"
                                        % (msub, m))
            out["compare"]["cwy"] = {"value": msub / (t_cwy * 1e-3), "ms_per_step": t_cwy,
                                     "block": blk}
        # the other form of compact WY on the same workload: one member at a time (Alg. 4 as
        # printed) when the line measures blocks, blocks of 16 otherwise
        other = 0 if blk >= 2 else 16
        t_oth = timed_c("cwy", other)
        out["compare"]["cwy_one_member" if other == 0 else "cwy_block16"] = {
            "value": msub / (t_oth * 1e-3), "ms_per_step": t_oth, "block": other}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, desc = cpu_sample(args.workload, args.method, d, e, w)
        out["cpu_baseline"] = {"value": v, "unit": "eigvec/s", "cores": 1, "kind": "oracle",
                               "sample": desc}
        v, cores, desc = cpu_parallel(args.workload, args.method, d, e, w)
        out["cpu_baseline_parallel"] = {"value": v, "unit": "eigvec/s", "cores": cores,
                                        "kind": "oracle", "sample": desc}
        lap = lapack_dstein_sample(args.workload, d, e, w)
        if lap:
            out["context_lapack_dstein"] = lap
    if rank == 0 and world == 1 and not args.no_extras and args.workload == "glued4200":
        out["extras"] = extras()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def extras():
    """The other workloads of the metric, each a child run of this script (after the main
    measurement, outside its timed region): the 512-problem batch against one call per problem,
    the served request stream against one host call per request, and uniform n = 1000.  Returns
    a summary of each line, or the reason it is missing."""
    runs = {"batch512": ["--workload", "batch512", "--steps", "2", "--warmup", "1", "--no-e2e"],
            "serve": ["--workload", "serve", "--warmup", "1"],
            "uniform1000": ["--workload", "uniform1000", "--steps", "5", "--warmup", "3",
                            "--no-compare"]}
    keep = ("metric", "value", "unit", "ms_per_step", "problems_per_s", "eigvecs_per_s", "compare",
            "check", "roofline", "saturated", "levels", "graph_replay", "e2e", "clocks", "config")
    res = {}
    for name, extra in runs.items():
        cmd = [sys.executable, os.path.abspath(__file__), "--no-cpu-baseline", "--no-extras"] + extra
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
            line = [x for x in r.stdout.splitlines() if x.startswith("{")]
            if r.returncode != 0 or not line:
                res[name] = {"missing": "exit %d: %s" % (r.returncode, (r.stderr or r.stdout)[-300:])}
                continue
            full = json.loads(line[-1])
            res[name] = {k: full[k] for k in keep if k in full}
        except subprocess.TimeoutExpired:
            res[name] = {"missing": "timed out after 600 s"}
    return res


# ------------------------------------------------------------------------------------------
# phase timing of the cluster kernel (diagnostic: a separate library file, libtinv_prof.so,
# compiled with -DTINV_PHASE_PROFILE; thread 0 of every CTA of the cluster kernel adds clock64
# cycles per phase and prints them when the CTA ends)
# ------------------------------------------------------------------------------------------
PHASES = ["total", "solve", "A", "b1", "T1red", "T1", "b2", "Bload", "Brow", "Bsum", "B", "b3",
          "T2refl", "T2red", "T2row", "T2", "b4", "Cload", "Crow", "C", "b5", "load", "end",
          "sv_stage", "sv_fwd1", "sv_fcarry", "sv_fwd2", "sv_back1", "sv_bfold", "sv_back2",
          "sv_check"]


def _phases_child(args):
    from paper_1209_1910_gb300 import binding, build

    path = build.build(profile=True)
    binding.load(path)
    d, e, w = inputs.workload(args.workload)
    ph = np.zeros(4, dtype=np.float32)
    binding.tinv(d, e, w, method=args.method, phase_ms=ph.ctypes.data,
                 block=args.block if args.method == "cwy" else 0)
    print("PHASES_MS plan=%.3f lu=%.3f first=%.3f chain=%.3f" % tuple(ph.tolist()), flush=True)


def summarize_phases(text: str):
    """Per team size G: the slowest team's mean phase cycles over its CTAs, the number of teams
    of that size and the slowest team's index, from the PROF lines of a diagnostic run; and the
    line with the kernels' event times."""
    import collections
    import re

    teams = collections.defaultdict(list)
    chain = ""
    solve = {}
    for line in text.splitlines():
        if line.startswith("SPROF "):
            kv = {k: int(v) for k, v in re.findall(r"(\w+)=(-?\d+)", line)}
            solve[kv["cta"]] = kv
    for line in text.splitlines():
        if line.startswith("PHASES_MS"):
            chain = line
        if not line.startswith("PROF "):
            continue
        kv = {k: int(v) for k, v in re.findall(r"(\w+)=(-?\d+)", line)}
        for k, v in solve.get(kv.get("cta"), {}).items():
            kv.setdefault(k, v)
        if kv.get("team", -1) >= 0:
            teams[(kv["team"], kv["G"])].append(kv)
    by_g = collections.defaultdict(list)
    for (team, g), rows in teams.items():
        mean = {p: sum(r.get(p, 0) for r in rows) / len(rows) for p in PHASES}
        by_g[g].append((mean["total"], team, mean))
    out = {}
    for g, lst in by_g.items():
        lst.sort(reverse=True)
        out[g] = (lst[0][1], len(lst), lst[0][2])
    return out, chain


def phases_arm(args):
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--phases-child",
                        "--workload", args.workload, "--method", args.method,
                        "--block", str(args.block)],
                       capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout[-4000:] + r.stderr[-4000:])
        raise SystemExit(r.returncode)
    res, chain = summarize_phases(r.stdout)
    print("workload %s, method %s; %s" % (args.workload, args.method, chain))
    print("slowest team of each size, mean over its CTAs, millions of SM cycles:")
    for g in sorted(res):
        team, count, mean = res[g]
        print("G=%d (%d teams, slowest %d): " % (g, count, team) +
              " ".join("%s=%.1f" % (p, mean[p] / 1e6) for p in PHASES))


def main():
    args = parse()
    if args.block is None:
        # blocks of 16; one member at a time for the served stream and the split driver (the
        # latter's clusters lie inside blocks of order 21, where blocks gain nothing)
        args.block = 0 if args.workload in ("serve", "split4200") else 16
    if args.phases_child:
        return _phases_child(args)
    if args.phases:
        return phases_arm(args)
    if args.impl == "reference":
        reference_arm(args)
    else:
        ours_arm(args)


if __name__ == "__main__":
    main()
