"""Batched ciphertexts: every operation on a packed batch equals the same
operation on each ciphertext alone, bit for bit (CUDA library through its C ABI)."""
import numpy as np
import pytest

from paper_2606_10477_gb300 import hedap, inputs

pytestmark = pytest.mark.gpu


def ctx(name, seed=1):
    p = inputs.PRESETS[name]
    return hedap.Context(p["log_n"], p["q_bits"], p["p_bits"], p["alpha"], p["log_scale"], p["hw"], seed)


def imported(g, seed, level, n):
    pr = g.primes()
    return [g.ct_import(inputs.random_ciphertext_limbs(seed + i, pr, level, g.N), level, g.scale) for i in range(n)]


def check(g, batch_out, singles):
    assert batch_out.batch == len(singles)
    for k, s in enumerate(singles):
        u = g.unpack(batch_out, k)
        assert u.level == s.level and u.scale == s.scale
        assert np.array_equal(u.limbs(), s.limbs()), f"ciphertext {k}"


@pytest.mark.parametrize("name,n", [("n13", 3), ("toy", 16)])
def test_batched_ring_ops_equal_single_ops(name, n):
    g = ctx(name)
    L = g.n_q - 1
    a, b = imported(g, 100, L, n), imported(g, 200, L, n)
    A, B = g.pack(a), g.pack(b)
    assert A.batch == n
    check(g, g.add(A, B), [g.add(x, y) for x, y in zip(a, b)])
    check(g, g.sub(A, B), [g.sub(x, y) for x, y in zip(a, b)])
    check(g, g.mul(A, B), [g.mul(x, y) for x, y in zip(a, b)])
    check(g, g.rescale(A), [g.rescale(x) for x in a])
    check(g, g.rotate(A, 3), [g.rotate(x, 3) for x in a])
    check(g, g.conjugate(A), [g.conjugate(x) for x in a])
    check(g, g.mul_const(A, 0.75, g.scale), [g.mul_const(x, 0.75, g.scale) for x in a])
    check(g, g.add_const(A, -0.25), [g.add_const(x, -0.25) for x in a])
    check(g, g.mul_int(A, 3), [g.mul_int(x, 3) for x in a])


def test_invsqrt_batch_groups_and_matches_single():
    g = ctx("toy")
    L = g.n_q - 1
    vals = [inputs.uniform_values(300 + i, g.N // 2, 0.01, 1.0) for i in range(5)]
    cts = [g.encrypt(v, L if i != 2 else L - 1, 400 + i) for i, v in enumerate(vals)]
    cfgs = [(0.01, 1.0, 1.0, 15, 2, 0, 0)] * 5
    cfgs[4] = (0.01, 1.0, 1.0, 7, 2, 0, 0)  # a different configuration forms its own group
    outs = g.invsqrt_batch(cts, cfgs)
    for ct, cfg, o in zip(cts, cfgs, outs):
        s = g.invsqrt(ct, *cfg)
        assert o.level == s.level and np.array_equal(o.limbs(), s.limbs())


def test_bootstrap_batch_equals_single():
    p = inputs.PRESETS["bts12"]
    g = ctx("bts12")
    b = inputs.BTS
    g.bts_setup(b["K"], b["r"], b["deg"], b["cts"], b["stc"])
    cts = [g.encrypt(inputs.uniform_values(500 + i, g.N // 2, -1, 1), 1, 600 + i) for i in range(3)]
    check(g, g.bootstrap_scaled(g.pack(cts), 1), [g.bootstrap_scaled(c, 1) for c in cts])


def test_invsqrt_many_level_bands():
    """Mixed levels: a band groups the inputs it holds and drops them to its lowest level; each
    result equals the single-ciphertext InvSqrt of the input dropped to that level."""
    g = ctx("toy")
    L = g.n_q - 1
    levels = [L, L - 1, L - 2, L, L - 3, L - 1]
    vals = [inputs.uniform_values(700 + i, g.N // 2, 0.01, 1.0) for i in range(len(levels))]
    cts = [g.encrypt(v, l, 800 + i) for i, (v, l) in enumerate(zip(vals, levels))]
    cfg = (0.01, 1.0, 1.0, 7, 1, 0, 0)  # the lowest band ends at level 1 (decryptable)
    band = 2
    outs = g.invsqrt_many(cts, [cfg] * len(cts), band)
    for i, (ct, o) in enumerate(zip(cts, outs)):
        floor = min(l for l in levels if l // band == levels[i] // band)
        s = g.invsqrt(g.drop(ct, floor), *cfg)
        assert o.level == s.level and np.array_equal(o.limbs(), s.limbs())
        y = g.decrypt(o).real
        assert np.mean(np.abs(y * np.sqrt(vals[i]) - 1)) < 1e-2  # degree 7, one Newton step
    same = g.invsqrt_many(cts, [cfg] * len(cts), 0)  # band 0: exact levels, as invsqrt_batch
    for ct, o in zip(cts, same):
        assert np.array_equal(o.limbs(), g.invsqrt(ct, *cfg).limbs())


def test_batch_import_export_in_one_copy():
    """hedap_batch_import / hedap_batch_export move a whole batch [n][2][level+1][N] in one copy each way: the
    imported batch equals the single imports packed, the export equals the members' exports (also for a batch whose
    parts are more limbs apart than its level needs, after a rescale), and bad input is refused."""
    g = ctx("n13")
    L = g.n_q - 1
    pr = g.primes()
    host = np.stack([inputs.random_ciphertext_limbs(300 + i, pr, L, g.N) for i in range(5)])
    b = g.batch_import(host, 5, L, g.scale)
    check(g, b, [g.ct_import(host[i], L, g.scale) for i in range(5)])
    out = np.zeros_like(host)
    g.batch_export(b, out)
    assert np.array_equal(out, host)
    r = g.rescale(g.mul(b, b))  # a derived batch two levels down
    want = np.stack([g.unpack(r, k).limbs() for k in range(5)])
    got = np.zeros((5, 2, r.level + 1, g.N), dtype=np.uint64)
    g.batch_export(r, got)
    assert np.array_equal(got, want)
    with pytest.raises(hedap.HedapError):
        g.batch_export(r, np.zeros((4, 2, r.level + 1, g.N), dtype=np.uint64))  # capacity below 5 ciphertexts
    bad = host.copy()
    bad[3, 1, 2, 7] = pr[2]  # not below its prime
    with pytest.raises(hedap.HedapError) as e:
        g.batch_import(bad, 5, L, g.scale)
    assert e.value.code == -7
    with pytest.raises(hedap.HedapError):
        g.batch_import(host, 17, L, g.scale)
