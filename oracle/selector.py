"""HE-DAP selection rules (Alg. 2 and Alg. 3) -- TEST INFRASTRUCTURE ONLY.

Plain Python, written from the algorithms' statements:
  Alg. 2: MRE_min = min M; MRE_min = alpha * 10^l (1 <= alpha < 10);
          MRE_delta = (floor(alpha) + delta) * 10^l; I = min{ i : M[i] <= MRE_delta }.
  Alg. 3: per level, m_min over the (d, c, i, m, t) entries, m_theta by the same
          rule with theta; u1 = argmin t over entries with m <= m_theta; u2 = argmin t.
Readings (the paper is silent): l and floor(alpha) come from the shortest
decimal representation of the double (Python's repr), so that an exact power
of ten or a value such as 3e-8 is not misread through log10 rounding; ties go
to smaller t, then smaller d, then c = 0, then smaller i; u3 = argmin t over
entries meeting an absolute MRE target; MRE_min = 0 gives threshold 0.
"""
from __future__ import annotations

import decimal
import math


def decimal_split(v: float):
    """(floor(alpha), l) with v = alpha * 10^l, 1 <= alpha < 10, from repr(v)."""
    d = decimal.Decimal(repr(float(v)))
    return d.as_tuple().digits[0], d.adjusted()


def threshold(mmin: float, delta: float) -> float:
    if mmin == 0:
        return 0.0
    lead, ell = decimal_split(mmin)
    if float(delta).is_integer():
        return float(f"{lead + int(delta)}e{ell}")
    return (lead + delta) * 10.0 ** ell


def getoptiter_rule(M, delta):
    """Index (0-based) of the first iteration within MRE_delta, or -1; and MRE_delta."""
    finite = [m for m in M if math.isfinite(m)]
    if not finite:
        return -1, None
    thr = threshold(min(finite), delta)
    for i, m in enumerate(M):
        if m <= thr:
            return i, thr
    return -1, thr


def _key(e):
    return (e["ms"], e["degree"], e["c"], e["iters"])


def level_rule(entries, theta, mre_target=0.0):
    """(u1, u2, u3 or None) for one level's entries (dicts with degree, c, iters, mre, ms)."""
    mth = threshold(min(e["mre"] for e in entries), theta)
    u1 = min((e for e in entries if e["mre"] <= mth), key=_key)
    u2 = min(entries, key=_key)
    ok = [e for e in entries if mre_target > 0 and e["mre"] <= mre_target]
    return u1, u2, (min(ok, key=_key) if ok else None)
