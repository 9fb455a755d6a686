"""Serving: continuous batching (groups admitted apart merge at a step boundary)
and host-side failure handling -- a query withdrawn while waiting or in flight,
an allocation failure injected at admission, a bounded host wait, malformed
handles.  Every fault is made on the host; nothing here faults, traps or hangs
the GPU.  Results that survive are compared bit for bit with the same query run
alone.
"""
import ctypes

import numpy as np
import pytest

from paper_2606_10477_gb300 import hedap, inputs

pytestmark = pytest.mark.gpu

LAZY = 1 << 63
ZCFG = (1e-3, 1.0, 1.0, 31, 4, 0, LAZY)
ABOVE_BTS = 3


@pytest.fixture(scope="module")
def ctx12():
    p = inputs.PRESETS["bts12"]
    g = hedap.Context(p["log_n"], p["q_bits"], p["p_bits"], p["alpha"], p["log_scale"], p["hw"], 1)
    b = inputs.BTS
    lvl = g.bts_setup(b["K"], b["r"], b["deg"], b["cts"], b["stc"]) + ABOVE_BTS
    slots = g.N // 2
    data = []
    for k in range(4):
        n = 1200 + 500 * k
        x = inputs.gaussian_records(500 + k, n)
        data.append((n, [g.encrypt(v, lvl, 600 + 10 * k + j) for j, v in enumerate(inputs.pack_slots(x, slots))]))
    return g, data


def alone(g, n, xs):
    srv = hedap.Server(g, max_batch=4)
    try:
        done, out, info = srv.poll(srv.submit(hedap.QUERY_ZSCORE, xs, n, ZCFG))
        assert done and info["group_size"] == 1
        return [c.limbs() for c in out]
    finally:
        srv.close()


def same(out, ref):
    assert len(out) == len(ref)
    for c, r in zip(out, ref):
        assert np.array_equal(c.limbs(), r)


def test_groups_admitted_apart_merge_and_match_alone(ctx12):
    """admit_max = 1: a burst of three queries of one signature is admitted as three groups; the first
    waits at its step boundary for the later ones to catch up, and they run on as one batch of three."""
    g, data = ctx12
    refs = [alone(g, n, xs) for n, xs in data[:3]]
    srv = hedap.Server(g, max_batch=4, paused=True, admit_max=1)
    try:
        ids = [srv.submit(hedap.QUERY_ZSCORE, xs, n, ZCFG) for n, xs in data[:3]]
        srv.resume()
        res = [srv.poll(i) for i in ids]
        assert srv.merges() == 2
    finally:
        srv.close()
    for (done, out, info), ref in zip(res, refs):
        assert done and info["group_size"] == 3
        same(out, ref)


def test_cancel_waiting_and_in_flight(ctx12):
    g, data = ctx12
    ref0 = alone(g, *data[0])
    srv = hedap.Server(g, max_batch=4, paused=True)
    try:
        a = srv.submit(hedap.QUERY_ZSCORE, data[0][1], data[0][0], ZCFG)
        b = srv.submit(hedap.QUERY_ZSCORE, data[1][1], data[1][0], ZCFG)
        c = srv.submit(hedap.QUERY_ZSCORE, data[2][1], data[2][0], ZCFG)
        srv.cancel(b)  # still waiting: withdrawn at once
        with pytest.raises(hedap.HedapError) as e:
            srv.poll(b)
        assert e.value.code == -9
        srv.resume()
        srv.cancel(c)  # admitted with a: withdrawn at a step boundary, a goes on unchanged
        with pytest.raises(hedap.HedapError) as e:
            srv.poll(c)
        assert e.value.code == -9
        done, out, info = srv.poll(a)
        assert done
        same(out, ref0)
        with pytest.raises(hedap.HedapError):
            srv.cancel(a)  # finished and handed over: unknown now
        d = srv.submit(hedap.QUERY_ZSCORE, data[3][1], data[3][0], ZCFG)  # alone in its group: dropped
        srv.cancel(d)
        with pytest.raises(hedap.HedapError) as e:
            srv.poll(d)
        assert e.value.code == -9
        done, out, _ = srv.poll(srv.submit(hedap.QUERY_ZSCORE, data[0][1], data[0][0], ZCFG))  # still serving
        same(out, ref0)
    finally:
        srv.close()


def test_injected_admission_allocation_failure(ctx12):
    g, data = ctx12
    ref0 = alone(g, *data[0])
    srv = hedap.Server(g, max_batch=4)
    try:
        srv.inject(hedap.FAULT_ADMISSION_OOM, 1)
        bad = srv.submit(hedap.QUERY_ZSCORE, data[1][1], data[1][0], ZCFG)
        with pytest.raises(hedap.HedapError) as e:
            srv.poll(bad)
        assert e.value.code == -4
        done, out, _ = srv.poll(srv.submit(hedap.QUERY_ZSCORE, data[0][1], data[0][0], ZCFG))
        assert done
        same(out, ref0)
        with pytest.raises(hedap.HedapError):
            srv.inject(99, 1)  # unknown fault
    finally:
        srv.close()


def test_bounded_wait(ctx12):
    g, data = ctx12
    srv = hedap.Server(g, max_batch=4, paused=True)
    try:
        q = srv.submit(hedap.QUERY_ZSCORE, data[0][1], data[0][0], ZCFG)
        with pytest.raises(hedap.HedapError) as e:
            srv.wait(q, 20.0)  # the server is paused: the query cannot finish
        assert e.value.code == -6
        srv.resume()
        srv.wait(q, 120000.0)
        done, out, _ = srv.poll(q, wait=False)
        assert done and len(out) == len(data[0][1])
    finally:
        srv.close()


def test_malformed_handles_are_refused(ctx12):
    g, data = ctx12
    L = hedap.load()
    out = ctypes.c_void_p()
    junk = (ctypes.c_uint64 * 8)()  # readable memory that is not a handle
    rc = L.hedap_add(g.h, ctypes.cast(junk, ctypes.c_void_p), data[0][1][0].h, ctypes.byref(out))
    assert rc == -1 and "not a live ciphertext handle" in L.hedap_last_error().decode()
    rc = L.hedap_add(ctypes.cast(junk, ctypes.c_void_p), data[0][1][0].h, data[0][1][0].h, ctypes.byref(out))
    assert rc == -1 and "not a live context handle" in L.hedap_last_error().decode()
    p = inputs.PRESETS["toy"]
    other = hedap.Context(p["log_n"], p["q_bits"], p["p_bits"], p["alpha"], p["log_scale"], p["hw"], 2)
    foreign = other.encrypt(inputs.uniform_values(1, other.N // 2, 0, 1), 3, 4)
    rc = L.hedap_rescale(g.h, foreign.h, ctypes.byref(out))
    assert rc == -1 and "another context" in L.hedap_last_error().decode()
    srv = hedap.Server(g, max_batch=2)
    try:
        with pytest.raises(hedap.HedapError) as e:
            srv.submit(hedap.QUERY_ZSCORE, [foreign], 10, ZCFG)
        assert e.value.code == -1
    finally:
        srv.close()
