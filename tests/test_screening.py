"""The stored screening of the batched tube/ripple draws
(tests/golden/riemann_instances_screened.json, written by
tests/golden/screen_riemann_instances.py with the FP64 oracle) is
consistent and reproduces on a few of the smallest draws."""
import json
import os
import sys

from paper_1004_5442_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _doc():
    with open(os.path.join(GOLD, "riemann_instances_screened.json")) as fh:
        return json.load(fh)


def test_screening_record_is_consistent():
    d = _doc()
    acc, rej = d["accepted"], d["rejected"]
    assert len(acc) == d["count"] == 256 and d["seed"] == 4
    assert sorted(acc + rej) == list(range(len(acc) + len(rej)))
    assert abs(d["acceptance_rate"] - len(acc) / (len(acc) + len(rej))) < 1e-12
    ws = W.riemann_instances(count=256, accepted=acc)
    assert [w.extra["draw"] for w in ws] == acc


def test_screening_verdicts_reproduce(orc):
    sys.path.insert(0, GOLD)
    import screen_riemann_instances as S
    d = _doc()
    last = max(d["accepted"] + d["rejected"])
    draws = {}
    for k, w in W.riemann_candidates(seed=4):
        draws[k] = w
        if k >= last:
            break
    cells = lambda k: draws[k].nx * draws[k].ny
    for k in sorted(d["accepted"], key=cells)[:2]:
        assert S.first_bad_step(draws[k]) is None, k
    for k in sorted(d["rejected"], key=cells)[:2]:
        got = S.first_bad_step(draws[k])
        assert got is not None, k
        if "first_bad_step" in d:
            assert got == d["first_bad_step"][str(k)], (k, got)
