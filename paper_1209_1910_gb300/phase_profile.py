"""Phase timing of the cluster kernel: where each CTA team's time goes.

    python -m paper_1209_1910_gb300.phase_profile [--workload glued4200] [--method cwy]

Builds the diagnostic variant of the library (libtinv_prof.so, compiled with
-DTINV_PHASE_PROFILE: thread 0 of every CTA of the cluster kernel accumulates clock64 cycles per
phase and prints them when the CTA ends), runs one call on the named workload in a child process,
and prints, per team size, the mean cycles of each phase over the team's CTAs (in millions).
The timed library is a separate file; the product library is not changed.
"""
from __future__ import annotations

import argparse
import collections
import re
import subprocess
import sys

PHASES = ["total", "solve", "A", "b1", "T1red", "T1", "b2", "Bload", "Brow", "Bsum", "B", "b3",
          "T2refl", "T2row", "T2", "b4", "Cload", "Crow", "C", "b5", "load", "end"]


def _child(workload: str, method: str) -> None:
    import numpy as np

    from paper_1209_1910_gb300 import binding, build, inputs

    path = build.build(profile=True)
    binding.load(path)
    d, e, w = inputs.workload(workload)
    ph = np.zeros(4, dtype=np.float32)
    binding.tinv(d, e, w, method=method, phase_ms=ph.ctypes.data)
    print("PHASES_MS plan=%.3f lu=%.3f first=%.3f chain=%.3f" % tuple(ph.tolist()), flush=True)


def summarize(text: str):
    """Per (team, G): the CTAs' phase cycles; returns {G: {phase: mean over the teams' CTAs}}
    for the slowest team of each size, and the chain time line."""
    teams = collections.defaultdict(list)
    chain = ""
    for line in text.splitlines():
        if line.startswith("PHASES_MS"):
            chain = line
        if not line.startswith("PROF "):
            continue
        kv = {k: int(v) for k, v in re.findall(r"(\w+)=(-?\d+)", line)}
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


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="glued4200")
    ap.add_argument("--method", default="cwy")
    ap.add_argument("--child", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.child:
        _child(args.workload, args.method)
        return
    r = subprocess.run([sys.executable, "-m", "paper_1209_1910_gb300.phase_profile", "--child",
                        "--workload", args.workload, "--method", args.method],
                       capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout[-4000:] + r.stderr[-4000:])
        raise SystemExit(r.returncode)
    res, chain = summarize(r.stdout)
    print("workload %s, method %s; %s" % (args.workload, args.method, chain))
    print("slowest team of each size, mean over its CTAs, millions of SM cycles:")
    for g in sorted(res):
        team, count, mean = res[g]
        print("G=%d (%d teams, slowest %d): " % (g, count, team) +
              " ".join("%s=%.1f" % (p, mean[p] / 1e6) for p in PHASES))


if __name__ == "__main__":
    main()
