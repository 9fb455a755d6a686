"""The serving loop (z-score and correlation queries) through the C ABI.

At N = 2^12 every query's result is compared bit for bit with the same
sequence of operations run by the CPU oracle (rotate-and-sum, moments,
CryptoInvSqrt with lazy bootstrapping, the final product), and each result is
checked to be identical alone and grouped with other queries.  At N = 2^16
the decrypted z-scores and correlations are compared with FP64 statistics of
the records.
"""
import numpy as np
import pytest

import oracle
from paper_2606_10477_gb300 import hedap, inputs

pytestmark = pytest.mark.gpu

LAZY = 1 << 63
# (lo, hi, B, degree, Newton steps, Pre-BTS, lazy bootstrapping)
ZCFG = (1e-3, 1.0, 1.0, 31, 4, 0, LAZY)  # var of the records lies in [1e-3, 1]
PCFG = (1e-5, 1e-2, 1e-2, 31, 5, 0, LAZY)  # var_x var_y lies in [1e-5, 1e-2]
ABOVE_BTS = 3  # records arrive 3 levels above a bootstrapped ciphertext's level


def make(name, cls, seed=1):
    p = inputs.PRESETS[name]
    c = cls(p["log_n"], p["q_bits"], p["p_bits"], p["alpha"], p["log_scale"], p["hw"], seed)
    b = inputs.BTS
    lvl = c.bts_setup(b["K"], b["r"], b["deg"], b["cts"], b["stc"])
    return c, lvl + ABOVE_BTS


@pytest.fixture(scope="module")
def pair12():
    g, lvl = make("bts12", hedap.Context)
    o, _ = make("bts12", oracle.Context)
    return g, o, lvl


def encrypt_pair(g, o, vectors, level, seed):
    ocs = [o.encrypt(v, level, seed + k) for k, v in enumerate(vectors)]
    return [g.ct_import(c.limbs(), c.level, c.scale) for c in ocs], ocs


# ------------------------------------------------------------------ the oracle's sequence of the same query
def o_slot_sum(o, a):
    r = 1
    while r < o.N // 2:
        a = o.add(a, o.rotate(a, r))
        r *= 2
    return a


def o_sum(o, cts):
    acc = cts[0]
    for c in cts[1:]:
        acc = o.add(acc, c)
    return acc


def o_central(o, sum_v, mu, mw, n):
    m2 = o.mul(mu, mw)
    ev = o.mul_const(o.drop(sum_v, m2.level + 1), 1.0 / n, m2.scale)
    return o.sub(ev, m2)


def o_invsqrt_final(o, var, cfg):
    lo, hi, B, d, k, pre, mask = cfg
    y = o.invsqrt(var, lo, hi, B, d, k, pre, mask)
    if y.level < 1:  # no level left for the final product: bootstrap y / Y, Y >= 1/sqrt(lo) >= y
        Y = 1
        while Y < 1.0 / np.sqrt(lo):
            Y *= 2
        y = o.bootstrap_scaled(y, Y)
    return y


def o_zscore(o, xs, n, cfg):
    s1 = o_slot_sum(o, o_sum(o, xs))
    s2 = o_slot_sum(o, o_sum(o, [o.mul(x, x) for x in xs]))
    mean = o.mul_const(s1, 1.0 / n, xs[0].scale)
    var = o_central(o, s2, mean, mean, n)
    s = o_invsqrt_final(o, var, cfg)
    return [o.mul(o.sub(x, mean), s) for x in xs]


def o_pcc(o, xs, ys, n, cfg):
    s1 = o_slot_sum(o, o_sum(o, xs))
    s2 = o_slot_sum(o, o_sum(o, [o.mul(x, x) for x in xs]))
    t1 = o_slot_sum(o, o_sum(o, ys))
    t2 = o_slot_sum(o, o_sum(o, [o.mul(y, y) for y in ys]))
    sxy = o_slot_sum(o, o_sum(o, [o.mul(x, y) for x, y in zip(xs, ys)]))
    mx = o.mul_const(s1, 1.0 / n, xs[0].scale)
    my = o.mul_const(t1, 1.0 / n, xs[0].scale)
    var = o.mul(o_central(o, s2, mx, mx, n), o_central(o, t2, my, my, n))
    cov = o_central(o, sxy, mx, my, n)
    return [o.mul(cov, o_invsqrt_final(o, var, cfg))]


def same(gc, oc):
    assert gc.level == oc.level and gc.scale == oc.scale
    assert np.array_equal(gc.limbs(), oc.limbs())


def zscores(x):
    return (x - x.mean()) / x.std()


# ------------------------------------------------------------------ N = 2^12, bit exact
def test_zscore_and_pcc_bit_exact_with_oracle(pair12):
    g, o, lvl = pair12
    slots = o.N // 2
    n = 3000  # two ciphertexts, the second one ragged
    x = inputs.gaussian_records(1, n)
    y = inputs.correlated_records(2, x, 0.6)
    gx, ox = encrypt_pair(g, o, inputs.pack_slots(x, slots), lvl, 10)
    gy, oy = encrypt_pair(g, o, inputs.pack_slots(y, slots), lvl, 20)
    srv = hedap.Server(g, max_batch=4)
    try:
        qz = srv.submit(hedap.QUERY_ZSCORE, gx, n, ZCFG)
        qp = srv.submit(hedap.QUERY_PCC, gx, n, PCFG, ys=gy)
        done, zs, _ = srv.poll(qz)
        assert done and len(zs) == len(gx)
        done, rs, _ = srv.poll(qp)
        assert done and len(rs) == 1
    finally:
        srv.close()
    for gz, oz in zip(zs, o_zscore(o, ox, n, ZCFG)):
        same(gz, oz)
    same(rs[0], o_pcc(o, ox, oy, n, PCFG)[0])
    z = np.concatenate([g.decrypt(c).real for c in zs])[:n]
    assert np.max(np.abs(z - zscores(x))) < 1e-6
    r = g.decrypt(rs[0]).real
    assert np.max(np.abs(r - np.corrcoef(x, y)[0, 1])) < 1e-6


def test_result_identical_alone_and_in_the_mix(pair12):
    g, o, lvl = pair12
    slots = o.N // 2
    data = []
    for k in range(6):
        n = 1500 + 700 * k
        x = inputs.gaussian_records(100 + k, n)
        y = inputs.correlated_records(200 + k, x, 0.3)
        gx, _ = encrypt_pair(g, o, inputs.pack_slots(x, slots), lvl, 1000 + 10 * k)
        gy, _ = encrypt_pair(g, o, inputs.pack_slots(y, slots), lvl, 2000 + 10 * k)
        data.append((n, gx, gy))
    plan = [(hedap.QUERY_ZSCORE, 0), (hedap.QUERY_ZSCORE, 1), (hedap.QUERY_ZSCORE, 2),
            (hedap.QUERY_PCC, 3), (hedap.QUERY_PCC, 1), (hedap.QUERY_PCC, 4), (hedap.QUERY_ZSCORE, 5)]

    def submit(srv, kind, k):
        n, gx, gy = data[k]
        if kind == hedap.QUERY_ZSCORE:
            return srv.submit(kind, gx, n, ZCFG)
        return srv.submit(kind, gx, n, PCFG, ys=gy)

    alone = {}
    srv = hedap.Server(g, max_batch=4)
    try:
        for kind, k in ((hedap.QUERY_ZSCORE, 1), (hedap.QUERY_PCC, 1)):
            done, out, info = srv.poll(submit(srv, kind, k))
            assert info["group_size"] == 1
            alone[kind] = [c.limbs() for c in out]
    finally:
        srv.close()
    srv = hedap.Server(g, max_batch=4, paused=True)
    try:
        ids = [submit(srv, kind, k) for kind, k in plan]
        srv.resume()
        results = [srv.poll(i) for i in ids]
        st = srv.stats()
    finally:
        srv.close()
    sizes = [info["group_size"] for _, _, info in results]
    assert sizes == [4, 4, 4, 3, 3, 3, 4]  # the oldest query with the later ones of its kind
    for (kind, k), (_, out, _) in zip(plan, results):
        if k == 1:
            assert len(out) == len(alone[kind])
            for c, ref in zip(out, alone[kind]):
                assert np.array_equal(c.limbs(), ref)
    assert st["completed"] == len(plan) and 0 < st["p50_ms"] <= st["p99_ms"] and st["qps"] > 0


def test_admission_by_memory_budget(pair12):
    g, o, lvl = pair12
    slots = o.N // 2
    x = inputs.gaussian_records(7, 2000)
    gx, _ = encrypt_pair(g, o, inputs.pack_slots(x, slots), lvl, 70)
    probe = hedap.Server(g, max_batch=4)
    need = probe.estimate(hedap.QUERY_ZSCORE, len(gx), lvl)
    probe.close()
    assert need > 0
    srv = hedap.Server(g, max_batch=4, hbm_budget_bytes=need + need // 2, paused=True)  # room for one at a time
    try:
        ids = [srv.submit(hedap.QUERY_ZSCORE, gx, x.size, ZCFG) for _ in range(3)]
        srv.resume()
        res = [srv.poll(i) for i in ids]
        assert [info["group_size"] for _, _, info in res] == [1, 1, 1]
        ref = [c.limbs() for c in res[0][1]]
        for _, out, _ in res[1:]:
            assert all(np.array_equal(c.limbs(), r) for c, r in zip(out, ref))
    finally:
        srv.close()
    small = hedap.Server(g, max_batch=4, hbm_budget_bytes=need - 1)
    try:
        with pytest.raises(hedap.HedapError) as e:
            small.submit(hedap.QUERY_ZSCORE, gx, x.size, ZCFG)
        assert e.value.code == -4
        with pytest.raises(hedap.HedapError):
            small.submit(hedap.QUERY_ZSCORE, gx, x.size + len(gx) * slots, ZCFG)  # more records than slots
    finally:
        small.close()


# ------------------------------------------------------------------ N = 2^16, accuracy
def test_full_size_zscore_and_pcc_accuracy():
    g, lvl = make("bts16", hedap.Context, seed=3)
    slots = g.N // 2
    srv = hedap.Server(g, max_batch=8)
    try:
        n = 3 * slots - 1000  # three ciphertexts, the last one ragged
        x = inputs.gaussian_records(31, n)
        y = inputs.correlated_records(32, x, -0.45)
        gx = [g.encrypt(v, lvl, 300 + k) for k, v in enumerate(inputs.pack_slots(x, slots))]
        gy = [g.encrypt(v, lvl, 400 + k) for k, v in enumerate(inputs.pack_slots(y, slots))]
        qz = srv.submit(hedap.QUERY_ZSCORE, gx, n, ZCFG)
        qp = srv.submit(hedap.QUERY_PCC, gx, n, PCFG, ys=gy)
        _, zs, _ = srv.poll(qz)
        _, rs, _ = srv.poll(qp)
    finally:
        srv.close()
    z = np.concatenate([g.decrypt(c).real for c in zs])[:n]
    assert np.max(np.abs(z - zscores(x))) < 1e-6
    r = g.decrypt(rs[0]).real
    assert np.max(np.abs(r - np.corrcoef(x, y)[0, 1])) < 1e-6


def test_table_driven_parameters_equal_explicit_ones(pair12):
    """A query that takes (degree, c, iters) from the HE-DAP table (Sec. 4.2) runs
    exactly the query with those parameters written out; the lookup takes the
    variance's level (input - 2 for z-score, - 3 for PCC) or the highest tabled
    level below it."""
    g, o, lvl = pair12
    slots = o.N // 2
    n = 2500
    x = inputs.gaussian_records(31, n)
    y = inputs.correlated_records(32, x, 0.5)
    gx, _ = encrypt_pair(g, o, inputs.pack_slots(x, slots), lvl, 310)
    gy, _ = encrypt_pair(g, o, inputs.pack_slots(y, slots), lvl, 320)

    def entry(level, d, c, i, kind):
        return {"level": level, "degree": d, "c": c, "iters": i, "mre": 0.0, "ms": 0.0, "kind": kind}

    table = [entry(lvl - 3, 31, 0, 4, 2),      # u2: below the z-score variance's level, at the PCC one
             entry(lvl - 4, 15, 0, 6, 2),      # a lower u2 entry, not taken
             entry(lvl - 3, 31, 0, 5, 3),      # u3 for PCC
             entry(lvl + 5, 31, 0, 4, 1)]      # u1 only above every variance level
    other = (ZCFG[0], ZCFG[1], ZCFG[2], 7, 1, 0, 0)  # overridden by the table
    other_p = (PCFG[0], PCFG[1], PCFG[2], 7, 1, 0, 0)
    srv = hedap.Server(g, max_batch=4)
    try:
        srv.set_table(table)
        tz = srv.submit(hedap.QUERY_ZSCORE, gx, n, other, choice=2)
        tp = srv.submit(hedap.QUERY_PCC, gx, n, other_p, ys=gy, choice=3)
        ez = srv.submit(hedap.QUERY_ZSCORE, gx, n, ZCFG)
        ep = srv.submit(hedap.QUERY_PCC, gx, n, PCFG, ys=gy)
        res = {k: srv.poll(k) for k in (tz, tp, ez, ep)}
        with pytest.raises(hedap.HedapError):
            srv.submit(hedap.QUERY_ZSCORE, gx, n, other, choice=1)  # no u1 entry at or below
        with pytest.raises(hedap.HedapError):
            srv.submit(hedap.QUERY_ZSCORE, gx, n, other, choice=4)
        srv.set_table([])
        with pytest.raises(hedap.HedapError):
            srv.submit(hedap.QUERY_ZSCORE, gx, n, other, choice=2)
    finally:
        srv.close()
    for a, b in ((tz, ez), (tp, ep)):
        assert res[a][0] and res[b][0] and len(res[a][1]) == len(res[b][1])
        for c, d in zip(res[a][1], res[b][1]):
            assert np.array_equal(c.limbs(), d.limbs())
    r = g.decrypt(res[tp][1][0]).real
    assert np.max(np.abs(r - np.corrcoef(x, y)[0, 1])) < 1e-6
