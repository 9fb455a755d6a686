"""Bit-exact parity of the individual hybrid key-switching steps and of rescale
(CUDA library through its C ABI vs the CPU oracle, same seeded inputs)."""
import numpy as np
import pytest

import oracle
from paper_2606_10477_gb300 import hedap, inputs

pytestmark = pytest.mark.gpu


def make_pair(name, seed=1):
    p = inputs.PRESETS[name]
    args = (p["log_n"], p["q_bits"], p["p_bits"], p["alpha"], p["log_scale"], p["hw"], seed)
    return hedap.Context(*args), oracle.Context(*args)


@pytest.fixture(scope="module", params=["n10", "toy"])
def pair(request):
    return make_pair(request.param)


def ext_primes(o, level):
    pr = o.primes()
    return np.concatenate([pr[:level + 1], pr[o.n_q:]])


def test_modup_bit_exact(pair):
    g, o = pair
    for level in (o.n_q - 1, 2, 0):
        x = inputs.random_limbs(60 + level, o.primes()[:level + 1], o.N)
        gy = g.modup_coeff(x, level)
        for j in range(gy.shape[0]):
            assert np.array_equal(gy[j], o.modup_coeff(x, level, j)), f"level {level}, digit {j}"


def test_moddown_bit_exact(pair):
    g, o = pair
    for level in (o.n_q - 1, 1):
        pr = ext_primes(o, level)
        x = np.stack([inputs.random_limbs(70 + level + p, pr, o.N) for p in range(2)])
        gd = g.moddown_coeff(x, level)
        for p in range(2):
            assert np.array_equal(gd[p], o.moddown_coeff(x[p], level)), f"level {level}, part {p}"


def test_key_switch_bit_exact(pair):
    g, o = pair
    for level in (o.n_q - 1, 3):
        d = inputs.random_limbs(80 + level, o.primes()[:level + 1], o.N)
        for gal in (0, o.galois_of_rotation(1)):
            assert np.array_equal(g.key_switch(d, level, gal), o.key_switch(d, level, gal)), f"level {level}, g {gal}"


def test_rescale_bit_exact(pair):
    g, o = pair
    for level in (o.n_q - 1, 1):
        limbs = inputs.random_ciphertext_limbs(90 + level, o.primes(), level, o.N)
        gc, oc = g.ct_import(limbs, level, o.scale), o.ct_import(limbs, level, o.scale)
        gr, orr = g.rescale(gc), o.rescale(oc)
        assert gr.scale == orr.scale and np.array_equal(gr.limbs(), orr.limbs())
