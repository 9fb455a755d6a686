"""Whole CryptoInvSqrt paths on the GPU (through the C ABI) against the CPU
oracle, bit for bit:

- Pre-BTS (the paper's c = 1, Sec. 4.1) and a forced bootstrap right after the
  Chebyshev step (Alg. 1's BTS placement, bts_mask bit 0) at N = 2^12;
- the benchmarked configuration at N = 2^16 (24 + 2 primes, two per digit,
  degree 15, 4 Newton steps from the top level), one ciphertext through
  hedap_invsqrt and a batch of 8 through a captured CUDA graph, each member
  unpacked and compared with its own oracle run;
- mixed levels grouped by level band (hedap_invsqrt_many): each output against
  the oracle's InvSqrt of its input dropped to the band's lowest level.
"""
import numpy as np
import pytest

import oracle
from paper_2606_10477_gb300 import hedap, inputs

pytestmark = pytest.mark.gpu


def make(name, cls, seed=1, bts=False):
    p = inputs.PRESETS[name]
    c = cls(p["log_n"], p["q_bits"], p["p_bits"], p["alpha"], p["log_scale"], p["hw"], seed)
    lvl = None
    if bts:
        b = inputs.BTS
        lvl = c.bts_setup(b["K"], b["r"], b["deg"], b["cts"], b["stc"])
    return c, lvl


def same(gc, oc, what=""):
    assert gc.level == oc.level, f"{what}: level {gc.level} != {oc.level}"
    assert gc.scale == oc.scale, f"{what}: scale {gc.scale} != {oc.scale}"
    gl, ol = gc.limbs(), oc.limbs()
    bad = np.count_nonzero(gl != ol)
    assert bad == 0, f"{what}: {bad} of {gl.size} residues differ"


def mre(y, a):
    ref = 1 / np.sqrt(a)
    return float(np.mean(np.abs(y - ref) / ref))


# ------------------------------------------------------------------ bootstrapping placements, N = 2^12
@pytest.fixture(scope="module")
def bts12():
    g, lg = make("bts12", hedap.Context, seed=7, bts=True)
    o, lo = make("bts12", oracle.Context, seed=7, bts=True)
    assert lg == lo
    return g, o, lg


def test_pre_bts_bit_exact(bts12):
    """c = 1: a/B is bootstrapped first (scaled to q_0/4096 at level 0, B folded into the constant,
    B = 1 afterwards), from a level too low for c = 0; lazy BTS in the Newton loop; B != 1."""
    g, o, lvl = bts12
    a = inputs.uniform_values(101, o.N // 2, 0.02, 2.0)  # inputs in [0.02, 2], B = 2
    oc = o.encrypt(a, 2, 102)
    gc = g.ct_import(oc.limbs(), oc.level, oc.scale)
    cfg = (0.02, 2.0, 2.0, 7, 2, 1, 1 << 63)
    gy, oy = g.invsqrt(gc, *cfg), o.invsqrt(oc, *cfg)
    same(gy, oy, "pre-BTS")
    y = g.decrypt(gy).real
    assert mre(y, a) < 1e-2  # degree 7 and two Newton steps on a 100x interval, through a bootstrap


def test_forced_bootstrap_after_chebyshev_bit_exact(bts12):
    """bts_mask bit 0: BTS of y right after the Chebyshev step (Alg. 1), then Newton steps."""
    g, o, lvl = bts12
    a = inputs.uniform_values(103, o.N // 2, 0.05, 1.0)
    oc = o.encrypt(a, lvl, 104)
    gc = g.ct_import(oc.limbs(), oc.level, oc.scale)
    cfg = (0.05, 1.0, 1.0, 7, 2, 0, 1)
    gy, oy = g.invsqrt(gc, *cfg), o.invsqrt(oc, *cfg)
    same(gy, oy, "bts_mask bit 0")
    # y bootstrapped to l_afterBTS; ct_x = 0.5 a sits one level below the input, and each Newton step
    # takes two levels below min(level(x), level(y))
    assert gy.level == lvl - 1 - 4
    y = g.decrypt(gy).real
    assert mre(y, a) < 1e-4


# ------------------------------------------------------------------ the benchmarked configuration, N = 2^16
BENCH_CFG = (1e-3, 1.0, 1.0, 15, 4)
N16_BATCH = 8


@pytest.fixture(scope="module")
def n16_runs():
    """8 oracle-encrypted inputs at the top level and the oracle's CryptoInvSqrt of each."""
    g, _ = make("n16", hedap.Context, seed=11)
    o, _ = make("n16", oracle.Context, seed=11)
    L = o.n_q - 1
    vals = [inputs.uniform_values(900 + k, o.N // 2, 1e-3, 1.0) for k in range(N16_BATCH)]
    ocs = [o.encrypt(v, L, 950 + k) for k, v in enumerate(vals)]
    oys = [o.invsqrt(c, *BENCH_CFG) for c in ocs]
    gcs = [g.ct_import(c.limbs(), c.level, c.scale) for c in ocs]
    return g, vals, gcs, oys


def test_invsqrt_bench_config_full_size_bit_exact(n16_runs):
    g, vals, gcs, oys = n16_runs
    gy = g.invsqrt(gcs[0], *BENCH_CFG)
    same(gy, oys[0], "single ciphertext")
    assert mre(g.decrypt(gy).real, vals[0]) <= 1e-7


def test_batched_graph_replay_full_size_bit_exact_per_member(n16_runs):
    """The bench's timed step: a batch of 8 packed ciphertexts through a captured CUDA graph."""
    g, vals, gcs, oys = n16_runs
    batch = g.pack(gcs)
    graph = g.invsqrt_graph(batch, *BENCH_CFG)
    try:
        out = graph.run(batch)
        assert out.batch == N16_BATCH
        for k in range(N16_BATCH):
            same(g.unpack(out, k), oys[k], f"member {k}")
    finally:
        graph.close()


# ------------------------------------------------------------------ mixed levels by level band
def test_invsqrt_many_level_bands_against_oracle():
    g, _ = make("toy", hedap.Context, seed=3)
    o, _ = make("toy", oracle.Context, seed=3)
    L = o.n_q - 1
    levels = [L, L - 1, L - 2, L, L - 3, L - 1, L - 4]
    vals = [inputs.uniform_values(700 + i, o.N // 2, 0.01, 1.0) for i in range(len(levels))]
    ocs = [o.encrypt(v, l, 800 + i) for i, (v, l) in enumerate(zip(vals, levels))]
    gcs = [g.ct_import(c.limbs(), c.level, c.scale) for c in ocs]
    cfg = (0.01, 1.0, 1.0, 7, 1, 0, 0)
    band = 2
    outs = g.invsqrt_many(gcs, [cfg] * len(gcs), band)
    for i, (oc, out) in enumerate(zip(ocs, outs)):
        floor = min(l for l in levels if l // band == levels[i] // band)
        same(out, o.invsqrt(o.drop(oc, floor), *cfg), f"input {i} (level {levels[i]}, band floor {floor})")


# ------------------------------------------------------------------ mixed levels, none dropped
def test_invsqrt_mixed_levels_against_oracle(bts12):
    """Single ciphertexts at their own levels with their own configurations (Pre-BTS for the low ones,
    sparse packing for one): each output equals the oracle's CryptoInvSqrt of that input alone, through
    hedap_invsqrt_mixed and through its captured CUDA graph."""
    g, o, lvl = bts12
    lazy = 1 << 63
    pre = (0.05, 1.0, 1.0, 7, 2, 1, lazy, 0)
    top = (0.05, 1.0, 1.0, 7, 2, 0, lazy, 0)
    sparse = (0.05, 1.0, 1.0, 7, 2, 1, lazy, 7)
    plan = [(3, pre), (5, pre), (lvl, top), (lvl, top), (lvl - 2, top), (4, sparse)]
    ocs, cfgs = [], []
    for i, (level, cfg) in enumerate(plan):
        n = 1 << cfg[7] if cfg[7] else o.N // 2
        a = np.tile(inputs.uniform_values(130 + i, n, 0.05, 1.0), o.N // 2 // n)
        ocs.append(o.encrypt(a, level, 140 + i))
        cfgs.append(cfg)
    gcs = [g.ct_import(c.limbs(), c.level, c.scale) for c in ocs]
    outs = g.invsqrt_mixed(gcs, cfgs)
    for i, (oc, cfg, out) in enumerate(zip(ocs, cfgs, outs)):
        same(out, o.invsqrt(oc, *cfg), f"input {i} (level {oc.level})")
    graph = g.invsqrt_mixed_graph(gcs, cfgs)
    try:
        again = graph.run_many(gcs)
        for i, (a, b) in enumerate(zip(outs, again)):
            assert np.array_equal(a.limbs(), b.limbs()), f"graph replay, input {i}"
    finally:
        graph.close()
