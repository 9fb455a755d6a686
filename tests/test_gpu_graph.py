"""CryptoInvSqrt replayed from a CUDA graph equals the ordinary launch sequence bit for bit."""
import numpy as np
import pytest

from paper_2606_10477_gb300 import hedap, inputs

pytestmark = pytest.mark.gpu


def make(name, seed=1):
    p = inputs.PRESETS[name]
    return hedap.Context(p["log_n"], p["q_bits"], p["p_bits"], p["alpha"], p["log_scale"], p["hw"], seed)


@pytest.mark.parametrize("name,batch,degree,iters", [("toy", 1, 15, 2), ("n13", 3, 7, 1)])
def test_graph_replay_bit_exact(name, batch, degree, iters):
    g = make(name)
    L = g.n_q - 1
    cts = [g.encrypt(inputs.uniform_values(60 + k, g.N // 2, 0.01, 1.0), L, 70 + k) for k in range(2 * batch)]
    first = g.pack(cts[:batch]) if batch > 1 else cts[0]
    second = g.pack(cts[batch:]) if batch > 1 else cts[1]
    graph = g.invsqrt_graph(first, 0.01, 1.0, 1.0, degree, iters)
    try:
        assert graph.kernels > 0
        for ct in (first, second, first):  # replays on new inputs, then on the first again
            ref = g.invsqrt(ct, 0.01, 1.0, 1.0, degree, iters)
            got = graph.run(ct)
            assert got.level == ref.level and got.scale == ref.scale
            assert np.array_equal(got.limbs(), ref.limbs())
        assert graph.run(want_output=False) is None  # replay on the previous input
    finally:
        graph.close()


def test_graph_with_bootstrapping_bit_exact():
    g = make("bts12")
    b = inputs.BTS
    lvl = g.bts_setup(b["K"], b["r"], b["deg"], b["cts"], b["stc"])
    ct = g.encrypt(inputs.log_uniform_values(80, g.N // 2, 1e-3, 1.0), lvl, 81)
    cfg = (1e-3, 1.0, 1.0, 31, 3, 0, 1 << 63)
    graph = g.invsqrt_graph(ct, *cfg)
    try:
        ref = g.invsqrt(ct, *cfg)
        got = graph.run(ct)
        assert np.array_equal(got.limbs(), ref.limbs())
    finally:
        graph.close()


def test_graph_rejects_mismatched_input():
    g = make("toy")
    L = g.n_q - 1
    a = g.encrypt(inputs.uniform_values(90, g.N // 2, 0.01, 1.0), L, 91)
    graph = g.invsqrt_graph(a, 0.01, 1.0, 1.0, 7, 1)
    try:
        with pytest.raises(hedap.HedapError):
            graph.run(g.encrypt(inputs.uniform_values(92, g.N // 2, 0.01, 1.0), L - 1, 93))
    finally:
        graph.close()
