"""HE-DAP selection rules (Alg. 2, Alg. 3): the oracle's plain-Python rules
against hand-applied thresholds on MREs printed in the paper, and the CUDA
library's host implementation of the same rules against the oracle's (host
code only: no GPU is needed)."""
import json
import os
import shutil

import numpy as np
import pytest

from oracle import selector as orule

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "threshold_rule.json")


def test_threshold_rule_on_paper_values():
    for case in json.load(open(GOLDEN))["cases"]:
        assert orule.threshold(case["mre_min"], case["delta"]) == case["threshold"], case["cite"]


def test_getoptiter_picks_first_iteration_within_threshold():
    # MRE curve of a converging Newton run followed by a BTS-induced bump (Sec. 4.3, Fig. 2)
    M = [3e-2, 2e-4, 4.1e-8, 2.97e-8, 2.96e-8, 5e-5, 2.99e-8]
    I, thr = orule.getoptiter_rule(M, 1)
    assert thr == 3e-8 and I == 3
    assert orule.getoptiter_rule([float("inf")] * 3, 1) == (-1, None)
    assert orule.getoptiter_rule([0.0, 1e-9], 1)[0] == 0


def test_level_rule_accuracy_and_speed_choices():
    E = [dict(degree=126, c=0, iters=5, mre=3.06e-8, ms=680.0),
         dict(degree=126, c=1, iters=4, mre=9.25e-7, ms=350.0),
         dict(degree=30, c=0, iters=8, mre=3.9e-8, ms=600.0),
         dict(degree=14, c=0, iters=12, mre=5e-8, ms=600.0)]
    u1, u2, u3 = orule.level_rule(E, 1, 1e-7)
    assert (u1["degree"], u1["c"], u1["iters"]) == (30, 0, 8)    # m <= 4e-8: the degree-14 entry is excluded
    assert (u2["degree"], u2["c"]) == (126, 1)                    # fastest regardless of MRE
    assert (u3["degree"], u3["c"], u3["iters"]) == (14, 0, 12)   # m <= 1e-7; tie at 600 ms goes to smaller d


def _library():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2606_10477_gb300 import build, hedap
    build.build()
    return hedap


def test_library_rules_match_oracle():
    hedap = _library()
    rng = np.random.default_rng(3)
    for _ in range(300):
        M = list(10.0 ** rng.uniform(-12, -2, rng.integers(1, 16)))
        if rng.uniform() < 0.3:
            M[int(rng.integers(len(M)))] = float(f"{rng.integers(1, 10)}e{rng.integers(-12, -3)}")
        delta = float(rng.choice([1, 2, 0.5]))
        oi, othr = orule.getoptiter_rule(M, delta)
        li, lthr = hedap.getoptiter_rule(M, delta)
        assert oi == li and othr == lthr
    for _ in range(200):
        n = int(rng.integers(1, 12))
        E = [dict(level=3, degree=int(2 ** rng.integers(4, 9) - 2), c=int(rng.integers(0, 2)),
                  iters=int(rng.integers(1, 15)), mre=float(10.0 ** rng.uniform(-10, -3)),
                  ms=float(rng.choice([100.0, 200.0, 300.0]))) for _ in range(n)]
        theta = float(rng.choice([1, 2]))
        target = float(rng.choice([0.0, 1e-7, 1e-5]))
        o1, o2, o3 = orule.level_rule(E, theta, target)
        l1, l2, l3 = hedap.select_level_rule(E, theta, target)
        key = ("degree", "c", "iters")
        assert tuple(o1[k] for k in key) == tuple(l1[k] for k in key)
        assert tuple(o2[k] for k in key) == tuple(l2[k] for k in key)
        assert (o3 is None) == (l3 is None)
        if o3:
            assert tuple(o3[k] for k in key) == tuple(l3[k] for k in key)
