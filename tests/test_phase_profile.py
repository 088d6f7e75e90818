"""The phase-timing summary of `bench.py --phases` (CPU): per team size, the slowest team's mean
over its CTAs."""
import bench
from bench import PHASES


def _line(cta, team, g, total, solve):
    vals = {p: 0 for p in PHASES}
    vals.update(total=total, solve=solve)
    body = " ".join("%s=%d" % (p, vals[p]) for p in PHASES if p != "total")
    return "PROF cta=%d team=%d G=%d total=%d %s" % (cta, team, g, total, body)


def test_summary_picks_the_slowest_team_of_each_size():
    text = "\n".join([
        "PHASES_MS plan=1.000 lu=2.000 first=3.000 chain=4.000",
        _line(0, 0, 2, 100, 10), _line(1, 0, 2, 110, 30),     # team 0: mean total 105
        _line(2, 1, 2, 120, 40), _line(3, 1, 2, 140, 60),     # team 1: mean total 130
        _line(4, 2, 1, 90, 5),                                 # a team of one CTA
        _line(5, -1, 1, 999, 999),                             # a queue CTA: not a team
        "unrelated output",
    ])
    res, chain = bench.summarize_phases(text)
    assert chain.startswith("PHASES_MS") and "chain=4.000" in chain
    assert sorted(res) == [1, 2]
    team, count, mean = res[2]
    assert team == 1 and count == 2
    assert mean["total"] == 130 and mean["solve"] == 50
    team, count, mean = res[1]
    assert team == 2 and count == 1 and mean["total"] == 90
