"""Bootstrapping on the GPU (through the C ABI) against the CPU oracle.

ModRaise, the monomial products, EvalMod, the grouped CoeffToSlot /
SlotToCoeff transforms and the whole bootstrap are compared bit for bit at
N = 2^12 (the plaintext diagonals come from two independently written FP64
encoders that perform the same operations in the same order); at N = 2^16 by
the decrypted error and CryptoInvSqrt's MRE.
"""
import numpy as np
import pytest

import oracle
from paper_2606_10477_gb300 import hedap, inputs

# levels a bootstrap consumes: CoeffToSlot, the EvalMod interpolant (ceil(log2(deg+1)) levels), the double
# angles, SlotToCoeff
BTS_LEVELS = (inputs.BTS["cts"] + inputs.BTS["deg"].bit_length() + inputs.BTS["r"]
              + inputs.BTS["stc"])

pytestmark = pytest.mark.gpu


def make(name, cls, seed=1):
    p = inputs.PRESETS[name]
    c = cls(p["log_n"], p["q_bits"], p["p_bits"], p["alpha"], p["log_scale"], p["hw"], seed)
    b = inputs.BTS
    lvl = c.bts_setup(b["K"], b["r"], b["deg"], b["cts"], b["stc"])
    return c, lvl


@pytest.fixture(scope="module")
def pair12():
    g, lg = make("bts12", hedap.Context)
    o, lo = make("bts12", oracle.Context)
    return g, o


def same(gc, oc):
    assert gc.level == oc.level and gc.scale == oc.scale
    assert np.array_equal(gc.limbs(), oc.limbs())


def level0_pair(g, o, seed, values):
    """Oracle-encrypted ciphertext at level 0 with scale q_0 / 2^12, imported into the library."""
    q0 = float(o.primes()[0])
    oc = o.mul_const(o.encrypt(values, 1, seed), 1.0, q0 / 4096)
    return g.ct_import(oc.limbs(), 0, oc.scale), oc


def test_mod_raise_and_monomials_bit_exact(pair12):
    g, o = pair12
    gc, oc = level0_pair(g, o, 3, inputs.uniform_values(3, o.N // 2, -1, 1))
    same(g.mod_raise(gc), o.mod_raise(oc))
    L = o.n_q - 1
    limbs = inputs.random_ciphertext_limbs(4, o.primes(), L, o.N)
    ga, oa = g.ct_import(limbs, L, o.scale), o.ct_import(limbs, L, o.scale)
    for e in (o.N // 2, 3 * o.N // 2):
        same(g.mul_monomial(ga, e), o.mul_monomial(oa, e))


def test_eval_mod_bit_exact(pair12):
    g, o = pair12
    lvl = o.n_q - 1 - 3
    u = inputs.uniform_values(5, o.N // 2, -1, 1)
    scale = float(o.primes()[lvl])
    oc = o.mul_const(o.encrypt(u, lvl + 1, 6), 1.0, scale)
    gc = g.ct_import(oc.limbs(), oc.level, oc.scale)
    gm, om = g.eval_mod(gc), o.eval_mod(oc)
    same(gm, om)
    K = inputs.BTS["K"]
    assert np.max(np.abs(o.decrypt(om).real - np.sin(2 * np.pi * K * u))) < 1e-6


@pytest.mark.parametrize("inverse", [True, False])
def test_linear_transform_groups_match_oracle(pair12, inverse):
    g, o = pair12
    L = o.n_q - 1
    z = inputs.uniform_values(7, o.N // 2, -1, 1) + 1j * inputs.uniform_values(8, o.N // 2, -1, 1)
    oc = o.encrypt(z, L, 9)
    gc = g.ct_import(oc.limbs(), L, oc.scale)
    for grp in range(inputs.BTS["cts" if inverse else "stc"]):
        target = oc.scale / 16  # plaintext scale q_l / 16 keeps the encoded diagonals below 2^63
        oc = o.linear_transform_group(oc, 3, inverse, grp, target)
        gc = g.linear_transform_group(gc, 3, inverse, grp, target)
        same(gc, oc)


def test_bootstrap_matches_oracle_and_input(pair12):
    g, o = pair12
    z = inputs.uniform_values(10, o.N // 2, -1, 1) + 1j * inputs.uniform_values(11, o.N // 2, -1, 1)
    gc, oc = level0_pair(g, o, 12, z)
    gb, ob = g.bootstrap(gc), o.bootstrap(oc)
    assert gb.level == o.n_q - 1 - BTS_LEVELS
    same(gb, ob)
    assert np.max(np.abs(g.decrypt(gb) - z)) < 1e-4


def test_bootstrap_full_size():
    """N = 2^16, 32768 complex slots, log2(QP) = 1555, h = 192."""
    g, lvl = make("bts16", hedap.Context)
    assert lvl == g.n_q - 1 - BTS_LEVELS
    z = inputs.uniform_values(13, g.N // 2, -1, 1) + 1j * inputs.uniform_values(14, g.N // 2, -1, 1)
    ct = g.encrypt(z, 1, 15)
    b = g.bootstrap_scaled(ct, 1)
    assert b.level == lvl
    err = np.abs(g.decrypt(b) - z)
    assert np.max(err) < 1e-3 and np.mean(err) < 1e-4


def test_invsqrt_with_bootstrapping_full_size():
    """N = 2^16, inputs log-uniform in [1e-4, 1] at l_max, Chebyshev degree 63, 4 Newton steps,
    lazy bootstrapping: decrypted MRE <= 1e-7."""
    g, lvl = make("bts16", hedap.Context, seed=2)
    a = inputs.log_uniform_values(16, g.N // 2, 1e-4, 1.0)
    ct = g.encrypt(a, lvl, 17)
    y = g.decrypt(g.invsqrt(ct, 1e-4, 1.0, 1.0, 63, 4, 0, 1 << 63)).real
    ref = 1 / np.sqrt(a)
    mre = float(np.mean(np.abs(y - ref) / ref))
    assert mre <= 1e-7, mre


def test_encoder_and_diagonals_match_oracle(pair12):
    g, o = pair12
    z = inputs.uniform_values(20, o.N // 2, -1, 1) + 1j * inputs.uniform_values(21, o.N // 2, -1, 1)
    for sc in (2.0 ** 40, 2.0 ** 56):
        assert np.array_equal(g.encode_coeffs(z.real, z.imag, sc), o.encode_coeffs(z.real, z.imag, sc).astype(np.int64))
    for inverse in (True, False):
        for grp in range(3):
            for off, d in o.fft_group(3, inverse, grp).items():
                assert np.array_equal(g.bts_diagonal(inverse, grp, off), d)


def test_ct_x_rebootstrapping_variant_bit_exact(pair12):
    g, o = pair12
    a = inputs.uniform_values(5, o.N // 2, 0.1, 1.0)
    oc = o.encrypt(a, 5, 6)
    gc = g.ct_import(oc.limbs(), oc.level, oc.scale)
    mask = (1 << 63) | (1 << 62)
    same(g.invsqrt(gc, 0.1, 1.0, 1.0, 3, 5, 0, mask), o.invsqrt(oc, 0.1, 1.0, 1.0, 3, 5, 0, mask))


# ------------------------------------------------------------------ dense secret, sparse-secret encapsulation
@pytest.fixture(scope="module")
def dense12():
    g, _ = make("bts12d", hedap.Context)
    o, _ = make("bts12d", oracle.Context)
    g.bts_encapsulate(inputs.ENC_HW)
    o.bts_encapsulate(inputs.ENC_HW)
    return g, o


def test_encapsulation_switches_bit_exact(dense12):
    g, o = dense12
    z = inputs.uniform_values(20, o.N // 2, -1, 1)
    gc, oc = level0_pair(g, o, 21, z)
    gs, os_ = g.encapsulation_switch(gc, True), o.encapsulation_switch(oc, True)
    same(gs, os_)
    L = o.n_q - 1
    limbs = inputs.random_ciphertext_limbs(22, o.primes(), L, o.N)
    ga, oa = g.ct_import(limbs, L, o.scale), o.ct_import(limbs, L, o.scale)
    same(g.encapsulation_switch(ga, False), o.encapsulation_switch(oa, False))


def test_dense_secret_bootstrap_matches_oracle(dense12):
    g, o = dense12
    z = inputs.uniform_values(23, o.N // 2, -1, 1) + 1j * inputs.uniform_values(24, o.N // 2, -1, 1)
    gc, oc = level0_pair(g, o, 25, z)
    gb, ob = g.bootstrap(gc), o.bootstrap(oc)
    same(gb, ob)
    assert np.max(np.abs(g.decrypt(gb) - z)) < 1e-4


def test_dense_secret_bootstrap_full_size():
    """N = 2^16 under a dense ternary secret, bootstrapped through an encapsulated weight-192 secret."""
    g, lvl = make("bts16d", hedap.Context, seed=3)
    g.bts_encapsulate(inputs.ENC_HW)
    z = inputs.uniform_values(26, g.N // 2, -1, 1) + 1j * inputs.uniform_values(27, g.N // 2, -1, 1)
    b = g.bootstrap_scaled(g.encrypt(z, 1, 28), 1)
    assert b.level == lvl
    err = np.abs(g.decrypt(b) - z)
    assert np.max(err) < 1e-3 and np.mean(err) < 1e-4


# ------------------------------------------------------------------ sparse packing
@pytest.mark.parametrize("ls", [7, 10])
def test_sub_sum_bit_exact(pair12, ls):
    g, o = pair12
    L = o.n_q - 1
    limbs = inputs.random_ciphertext_limbs(30 + ls, o.primes(), L, o.N)
    ga, oa = g.ct_import(limbs, L, o.scale), o.ct_import(limbs, L, o.scale)
    same(g.sub_sum(ga, ls), o.sub_sum(oa, ls))


@pytest.mark.parametrize("ls", [7, 10])
def test_sparse_slot_bootstrap_bit_exact(pair12, ls):
    g, o = pair12
    n = 1 << ls
    v = inputs.uniform_values(40 + ls, n, -1, 1) + 1j * inputs.uniform_values(50 + ls, n, -1, 1)
    zt = np.tile(v, o.N // 2 // n)
    gc, oc = level0_pair(g, o, 60 + ls, zt)
    gb, ob = g.bootstrap_slots(gc, ls), o.bootstrap_slots(oc, ls)
    same(gb, ob)
    assert np.max(np.abs(g.decrypt(gb) - zt)) < 1e-4


def test_sparse_slot_invsqrt_bit_exact(pair12):
    g, o = pair12
    n = 1 << 8
    a = np.tile(inputs.log_uniform_values(70, n, 1e-4, 1.0), o.N // 2 // n)
    lvl = o.n_q - 1 - BTS_LEVELS
    oc = o.encrypt(a, lvl, 71)
    gc = g.ct_import(oc.limbs(), oc.level, oc.scale)
    cfg = (1e-4, 1.0, 1.0, 15, 5, 0, 1 << 63, 8)
    same(g.invsqrt(gc, *cfg), o.invsqrt(oc, *cfg))


def test_sparse_slot_bootstrap_full_size():
    """N = 2^16 with 2^10 values repeated over the 32768 slots: five rotations of SubSum, then
    CoeffToSlot / SlotToCoeff on 1024 slots."""
    g, lvl = make("bts16", hedap.Context, seed=4)
    n = 1 << 10
    v = inputs.uniform_values(72, n, -1, 1) + 1j * inputs.uniform_values(73, n, -1, 1)
    zt = np.tile(v, g.N // 2 // n)
    b = g.bootstrap_scaled_slots(g.encrypt(zt, 1, 74), 1, 10)
    assert b.level == lvl
    err = np.abs(g.decrypt(b) - zt)
    assert np.max(err) < 1e-3 and np.mean(err) < 1e-4


def test_bootstrap_full_size_bit_exact():
    """N = 2^16, 32768 complex slots, log2(QP) = 1555, h = 192: one scaled bootstrap through the library
    and through the CPU oracle from the same ciphertext, compared bit for bit (the oracle takes about a
    minute here), and decrypting to its input."""
    g, lvl = make("bts16", hedap.Context, seed=6)
    o, lo = make("bts16", oracle.Context, seed=6)
    assert lvl == lo
    z = inputs.uniform_values(81, o.N // 2, -1, 1) + 1j * inputs.uniform_values(82, o.N // 2, -1, 1)
    oc = o.encrypt(z, 1, 83)
    gc = g.ct_import(oc.limbs(), oc.level, oc.scale)
    gb, ob = g.bootstrap_scaled(gc, 1), o.bootstrap_scaled(oc, 1)
    same(gb, ob)
    assert np.max(np.abs(g.decrypt(gb) - z)) < 1e-3
