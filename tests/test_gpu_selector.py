"""HE-DAP provisioning (Alg. 2 + Alg. 3) on the GPU: the D and R tables the
library returns follow from its own per-iteration trace by the oracle's
plain-Python rules, the profiled levels follow Alg. 3's conditions, and the
MRE curves behave as Sec. 4.3 describes."""
import numpy as np
import pytest

from oracle import selector as orule
from paper_2606_10477_gb300 import hedap, inputs

pytestmark = pytest.mark.gpu


def test_select_tables_follow_from_trace():
    p = inputs.PRESETS["bts12"]
    b = inputs.BTS
    g = hedap.Context(p["log_n"], p["q_bits"], p["p_bits"], p["alpha"], p["log_scale"], p["hw"], 1)
    l_after = g.bts_setup(b["K"], b["r"], b["deg"], b["cts"], b["stc"])
    # paper setting: inputs [0.001, 100], B = 100, theta = delta = 1 (Sec. 4.3)
    D, R, T = g.select(0.001, 100.0, 100.0, 4, 5, 8, theta=1.0, delta=1.0, mre_target=1e-7)
    assert D and R and T
    levels = sorted({e["level"] for e in D})
    assert levels[0] >= 2 and levels[-1] <= l_after
    for e in D:  # Alg. 3 line conditions: c = 0 needs l >= l_BTS + 3, c = 1 needs l < l_afterBTS - 1
        assert (e["c"] == 0 and e["level"] >= 4) or (e["c"] == 1 and e["level"] < l_after - 1)
    # Alg. 2 on the trace reproduces each D entry
    for e in D:
        rows = sorted((t for t in T if (t["level"], t["degree"], t["c"]) == (e["level"], e["degree"], e["c"])),
                      key=lambda t: t["iter"])
        I, _ = orule.getoptiter_rule([t["mre"] for t in rows], 1.0)
        assert I + 1 == e["iters"] and rows[I]["mre"] == e["mre"] and rows[I]["ms"] == e["ms"]
        assert all(rows[k]["ms"] < rows[k + 1]["ms"] for k in range(len(rows) - 1))
    # Alg. 3 on D reproduces R per level
    key = ("degree", "c", "iters")
    for lv in levels:
        Dl = [e for e in D if e["level"] == lv]
        u1, u2, u3 = orule.level_rule(Dl, 1.0, 1e-7)
        Rl = {r["kind"]: r for r in R if r["level"] == lv}
        assert tuple(Rl[1][k] for k in key) == tuple(u1[k] for k in key)
        assert tuple(Rl[2][k] for k in key) == tuple(u2[k] for k in key)
        assert (3 in Rl) == (u3 is not None)
    # with c = 0 at a high level the MRE first falls by orders of magnitude (Newton's quadratic convergence)
    hi = max(lv for lv in levels if any(e["c"] == 0 and e["level"] == lv for e in D))
    rows = sorted((t for t in T if t["level"] == hi and t["c"] == 0 and t["degree"] == 14), key=lambda t: t["iter"])
    assert rows[0]["mre"] > 100 * min(t["mre"] for t in rows)


def test_checkpoint_round_trip_on_a_context(tmp_path):
    """The NTT launch shapes and a table saved from one context are applied to a fresh one with the same key."""
    from paper_2606_10477_gb300 import checkpoint
    p = inputs.PRESETS["toy"]
    a = hedap.Context(p["log_n"], p["q_bits"], p["p_bits"], p["alpha"], p["log_scale"], p["hw"], 1)
    a.ntt_set_variant(2, 5)
    a.ntt_set_role_variant(hedap.NTT_ROLES["finish"], 7)
    path = str(tmp_path / "ckpt.json")
    checkpoint.save(path, a, p, [], device="this GPU", git="rev")
    b = hedap.Context(p["log_n"], p["q_bits"], p["p_bits"], p["alpha"], p["log_scale"], p["hw"], 1)
    b.ntt_set_variant(0, 0)
    assert checkpoint.load(path, b, p, device="this GPU", git="rev")
    assert b.ntt_get_variant() == (2, 5)
    assert b.ntt_get_roles() == {"forward": 2, "inverse": 5, "modup": 2, "finish": 7}
    assert not checkpoint.load(path, b, inputs.PRESETS["n13"], device="this GPU", git="rev")
