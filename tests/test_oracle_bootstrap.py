"""Pins of the oracle's bootstrapping against facts outside the oracle.

The grouped FFT factors multiply to the decoding matrix V (and its inverse,
up to the bit-reversal permutation), checked against numpy's dense matrix
algebra; X^(N/2) acts as i on every slot; ModRaise adds a multiple of q_0
below K; EvalMod approximates sin(2 pi K u); the whole bootstrap returns its
input within a stated error, and CryptoInvSqrt with bootstrapping inside the
Newton loop reproduces its FP64 model.
"""
import numpy as np
import pytest

import oracle
from paper_2606_10477_gb300 import inputs

# levels a bootstrap consumes: CoeffToSlot, the EvalMod interpolant (ceil(log2(deg+1)) levels), the double
# angles, SlotToCoeff
BTS_LEVELS = (inputs.BTS["cts"] + inputs.BTS["deg"].bit_length() + inputs.BTS["r"]
              + inputs.BTS["stc"])


@pytest.fixture(scope="module")
def ctx():
    p = inputs.PRESETS["bts12"]
    b = inputs.BTS
    o = oracle.Context(p["log_n"], p["q_bits"], p["p_bits"], p["alpha"], p["log_scale"], p["hw"], 1)
    o.bts_setup(b["K"], b["r"], b["deg"], b["cts"], b["stc"])
    return o


def decoding_matrix(N):
    n = N // 2
    g5 = np.array([pow(5, j, 2 * N) for j in range(n)])
    return np.exp(1j * np.pi * (np.outer(g5, np.arange(n)) % (2 * N)) / N)


def bitrev_perm(n):
    bits = int(np.log2(n))
    return np.array([int(format(i, f"0{bits}b")[::-1], 2) for i in range(n)])


def apply(D, x):
    return sum(d * np.roll(x, -off) for off, d in D.items())


def test_grouped_factors_are_the_decoding_matrix(ctx):
    n = ctx.N // 2
    V = decoding_matrix(ctx.N)
    perm = bitrev_perm(n)
    rng = np.random.default_rng(1)
    v = rng.normal(size=n) + 1j * rng.normal(size=n)
    w = np.linalg.solve(V, v)
    x = v.copy()
    for g in range(3):
        x = apply(ctx.fft_group(3, True, g), x)
    assert np.max(np.abs(x - w[perm])) < 1e-12  # CoeffToSlot = bit-reversed V^-1
    y = w[perm].copy()
    for g in range(3):
        y = apply(ctx.fft_group(3, False, g), y)
    assert np.max(np.abs(y - v)) < 1e-11       # SlotToCoeff = V on bit-reversed input
    # a group of r stages has at most 2^(r+1) - 1 diagonals
    assert all(len(ctx.fft_group(3, inv, g)) <= 31 for inv in (True, False) for g in range(3))


@pytest.mark.parametrize("inverse", [True, False])
def test_linear_transform_decrypts_to_the_diagonal_product(ctx, inverse):
    """Each CoeffToSlot / SlotToCoeff group applied homomorphically (baby steps hoisted and kept over Q_l u P, one
    ModDown per giant step, one rescale) decrypts to the group's diagonals applied to the decrypted input in numpy,
    within CKKS noise: a dropped baby or giant step, a wrong rotation offset or a misplaced ModDown fails it."""
    n = ctx.N // 2
    z = inputs.uniform_values(21, n, -1, 1) + 1j * inputs.uniform_values(22, n, -1, 1)
    c = ctx.encrypt(z, ctx.n_q - 1, 23)
    x = ctx.decrypt(c)
    for g in range(3):
        target = c.scale / 16  # plaintext scale q_l / 16 keeps the encoded diagonals below 2^63
        c = ctx.linear_transform_group(c, 3, inverse, g, target)
        want = apply(ctx.fft_group(3, inverse, g), x)
        got = ctx.decrypt(c)
        assert np.max(np.abs(got - want)) < 1e-6, f"group {g}"
        x = got


def test_monomial_half_n_is_i_in_every_slot(ctx):
    z = inputs.uniform_values(2, ctx.N // 2, -1, 1) + 1j * inputs.uniform_values(3, ctx.N // 2, -1, 1)
    ct = ctx.encrypt(z, 3, 4)
    assert np.max(np.abs(ctx.decrypt(ctx.mul_monomial(ct, ctx.N // 2)) - 1j * z)) < 1e-8
    assert np.max(np.abs(ctx.decrypt(ctx.mul_monomial(ct, 3 * ctx.N // 2)) + 1j * z)) < 1e-8


def test_mod_raise_adds_small_multiple_of_q0(ctx):
    q0 = int(ctx.primes()[0])
    z = inputs.uniform_values(5, ctx.N // 2, -1, 1)
    ct0 = ctx.mul_const(ctx.encrypt(z, 1, 6), 1.0, q0 / 4096)
    m = ctx.decrypt_coeffs(ct0)
    t = ctx.decrypt_coeffs(ctx.mod_raise(ct0))
    I = np.round((t - m) / q0)
    assert np.max(np.abs(t - m - q0 * I)) <= 4096  # FP64 resolution of values ~ K q_0 ~ 2^65
    assert 0 < np.max(np.abs(I)) < inputs.BTS["K"]


def test_eval_mod_approximates_scaled_sine(ctx):
    K = inputs.BTS["K"]
    lvl = ctx.n_q - 1 - 3
    u = inputs.uniform_values(7, ctx.N // 2, -1, 1)
    ct = ctx.mul_const(ctx.encrypt(u, lvl + 1, 8), 1.0, float(ctx.primes()[lvl]))
    out = ctx.decrypt(ctx.eval_mod(ct)).real
    assert np.max(np.abs(out - np.sin(2 * np.pi * K * u))) < 1e-8


def test_bootstrap_returns_its_input(ctx):
    q0 = float(ctx.primes()[0])
    z = inputs.uniform_values(9, ctx.N // 2, -1, 1) + 1j * inputs.uniform_values(10, ctx.N // 2, -1, 1)
    ct0 = ctx.mul_const(ctx.encrypt(z, 1, 11), 1.0, q0 / 4096)
    b = ctx.bootstrap(ct0)
    assert b.level == ctx.n_q - 1 - BTS_LEVELS
    assert np.max(np.abs(ctx.decrypt(b) - z)) < 1e-4


def test_invsqrt_with_lazy_bootstrapping_reproduces_fp64_model(ctx):
    a = inputs.log_uniform_values(16, ctx.N // 2, 1e-4, 1.0)
    L_after = ctx.n_q - 1 - BTS_LEVELS
    y = ctx.decrypt(ctx.invsqrt(ctx.encrypt(a, L_after, 17), 1e-4, 1.0, 1.0, 15, 5, 0, 1 << 63)).real
    plain = oracle.plain_invsqrt(a, 1e-4, 1.0, 1.0, 15, 5)
    assert np.max(np.abs(y - plain) / plain) < 1e-4


def test_ct_x_rebootstrapping_variant(ctx):
    """Bit 62: ct_x is bootstrapped with y when it has fewer than 5 levels.  From level 5 (x at 4)
    every Alg. 1 Newton step needs a bootstrap of y; with the variant the refreshed x lets steps run
    from the bootstrapped level, so the result sits higher, and its error is that of one bootstrap of
    x (Newton does not correct x), far above Alg. 1's."""
    a = inputs.uniform_values(5, ctx.N // 2, 0.1, 1.0)
    ct = ctx.encrypt(a, 5, 6)
    lazy = 1 << 63
    alg1 = ctx.invsqrt(ct, 0.1, 1.0, 1.0, 3, 5, 0, lazy)
    var = ctx.invsqrt(ct, 0.1, 1.0, 1.0, 3, 5, 0, lazy | (1 << 62))
    assert var.level > alg1.level
    err_alg1 = np.mean(np.abs(ctx.decrypt(alg1).real * np.sqrt(a) - 1))
    err_var = np.mean(np.abs(ctx.decrypt(var).real * np.sqrt(a) - 1))
    assert err_alg1 < 1e-8 and err_var < 1e-4


# ------------------------------------------------------------------ dense secret, sparse-secret encapsulation
@pytest.fixture(scope="module")
def dense():
    p = inputs.PRESETS["bts12d"]
    b = inputs.BTS
    o = oracle.Context(p["log_n"], p["q_bits"], p["p_bits"], p["alpha"], p["log_scale"], p["hw"], 1)
    o.bts_setup(b["K"], b["r"], b["deg"], b["cts"], b["stc"])
    o.bts_encapsulate(inputs.ENC_HW)
    return o


def level0(o, seed):
    q0 = int(o.primes()[0])
    z = inputs.uniform_values(seed, o.N // 2, -1, 1) + 1j * inputs.uniform_values(seed + 1, o.N // 2, -1, 1)
    return z, o.mul_const(o.encrypt(z, 1, seed + 2), 1.0, q0 / 4096)


def test_switch_to_sparse_secret_keeps_the_message(dense):
    """After the key switch s -> s~ the level-0 ciphertext decrypts to its message under s~ and
    to noise under s; switching back to s restores decryption under s."""
    z, ct0 = level0(dense, 40)
    sw = dense.encapsulation_switch(ct0, True)
    assert sw.level == 0
    assert np.max(np.abs(dense.decrypt_sparse(sw) - z)) < 1e-6
    assert np.max(np.abs(dense.decrypt(sw) - z)) > 1.0
    back = dense.encapsulation_switch(sw, False)
    assert np.max(np.abs(dense.decrypt(back) - z)) < 1e-6


def test_encapsulation_bounds_the_mod_raise_overflow(dense):
    """Under the dense secret ModRaise's overflow I (t = m + q_0 I) exceeds the K of a weight-192
    secret (its spread is about sqrt(2N/3 / 12) ~ 15); raised under s~ and switched back, it stays
    below K (spread about sqrt(192 / 12) = 4)."""
    q0 = int(dense.primes()[0])
    K = inputs.BTS["K"]
    _, ct0 = level0(dense, 50)
    m = dense.decrypt_coeffs(ct0)

    def overflow(t):
        d = dense.decrypt_coeffs(t) - m
        I = np.round(d / q0)
        assert np.max(np.abs(d - q0 * I)) <= 1e6  # key-switch noise and FP64 resolution, far below q_0
        return np.max(np.abs(I))

    assert overflow(dense.mod_raise(ct0)) > K
    t = dense.encapsulation_switch(dense.mod_raise(dense.encapsulation_switch(ct0, True)), False)
    assert t.level == dense.n_q - 1
    assert 0 < overflow(t) < K


def test_dense_secret_bootstrap_returns_its_input(dense):
    z, ct0 = level0(dense, 60)
    b = dense.bootstrap(ct0)
    assert b.level == dense.n_q - 1 - BTS_LEVELS
    assert np.max(np.abs(dense.decrypt(b) - z)) < 1e-4


# ------------------------------------------------------------------ sparse packing (2^log_slots slots repeated)
def test_sub_sum_projects_onto_the_subring(ctx):
    """Rotating by n, 2n, ..., N/4 and adding maps a plaintext m to (N/2n) times its part in
    Z[X^(N/2n)]: coefficients at multiples of N/2n multiplied by N/2n, all others zero (within
    the noise of the rotations' key switches)."""
    half = ctx.N // 2
    z = inputs.uniform_values(70, half, -1, 1) + 1j * inputs.uniform_values(71, half, -1, 1)
    ct = ctx.encrypt(z, 5, 72)
    m = ctx.decrypt_coeffs(ct)
    for ls in (7, 10):
        g = half >> ls
        d = ctx.decrypt_coeffs(ctx.sub_sum(ct, ls))
        expect = np.where(np.arange(ctx.N) % g == 0, g * m, 0.0)
        assert np.max(np.abs(d - expect)) < 4096  # against coefficients up to ~1.5e12


@pytest.mark.parametrize("ls", [7, 10])
def test_sparse_slot_bootstrap_returns_its_input(ctx, ls):
    """2^ls values repeated over the N/2 slots: the bootstrap returns them within 1e-4, still
    repeated with period 2^ls, at the level of a full-slot bootstrap."""
    half = ctx.N // 2
    n = 1 << ls
    q0 = float(ctx.primes()[0])
    v = inputs.uniform_values(80 + ls, n, -1, 1) + 1j * inputs.uniform_values(90 + ls, n, -1, 1)
    zt = np.tile(v, half // n)
    b = ctx.bootstrap_slots(ctx.mul_const(ctx.encrypt(zt, 1, 100 + ls), 1.0, q0 / 4096), ls)
    assert b.level == ctx.n_q - 1 - BTS_LEVELS
    out = ctx.decrypt(b)
    assert np.max(np.abs(out - zt)) < 1e-4
    assert np.max(np.abs(out - np.tile(out[:n], half // n))) < 1e-4


def test_sparse_slot_invsqrt_with_lazy_bootstrapping(ctx):
    n = 1 << 8
    a = inputs.log_uniform_values(110, n, 1e-4, 1.0)
    at = np.tile(a, ctx.N // 2 // n)
    L_after = ctx.n_q - 1 - BTS_LEVELS
    y = ctx.decrypt(ctx.invsqrt(ctx.encrypt(at, L_after, 111), 1e-4, 1.0, 1.0, 15, 5, 0, 1 << 63, 8)).real
    plain = oracle.plain_invsqrt(at, 1e-4, 1.0, 1.0, 15, 5)
    assert np.max(np.abs(y - plain) / plain) < 1e-4


def apply_period(D, x):
    """sum over offsets o of d_o * (x rotated left by o), x of the diagonals' length"""
    return sum(d * np.roll(x, -off) for off, d in D.items())


def test_sparse_groups_are_the_small_decoding_matrix(ctx):
    """For n = 2^7 slots the grouped factors are those of the ring of dimension 2n: CoeffToSlot is the
    bit-reversed inverse of V_n (z_j = m(zeta_4n^(5^j))), SlotToCoeff is V_n on bit-reversed input."""
    ls = 7
    n = 1 << ls
    V = decoding_matrix(2 * n)
    perm = bitrev_perm(n)
    rng = np.random.default_rng(3)
    v = rng.normal(size=n) + 1j * rng.normal(size=n)
    w = np.linalg.solve(V, v)
    x = v.copy()
    for g in range(3):
        x = apply_period(ctx.fft_group_ex(3, True, g, ls), x)
    assert np.max(np.abs(x - w[perm])) < 1e-12
    y = w[perm].copy()
    for g in range(3):
        y = apply_period(ctx.fft_group_ex(3, False, g, ls), y)
    assert np.max(np.abs(y - v)) < 1e-11


def test_packed_groups_split_real_and_imaginary_parts(ctx):
    """Packed sparse slots: the last CoeffToSlot group of period 2n gives (1 | -i) times the plain group's
    output, so that s + conj(s) is 2 Re | 2 Im; the first SlotToCoeff group of period 2n applied to y equals
    the plain group applied to z_m = y_m + i y_(m+n), on both halves."""
    ls = 7
    n = 1 << ls
    rng = np.random.default_rng(4)
    v = rng.normal(size=n) + 1j * rng.normal(size=n)
    plain = apply_period(ctx.fft_group_ex(3, True, 2, ls), v)
    packed = apply_period(ctx.fft_group_ex(3, True, 2, ls, packed=True), np.tile(v, 2))
    mask = np.concatenate([np.ones(n), -1j * np.ones(n)])
    assert np.max(np.abs(packed - mask * np.tile(plain, 2))) < 1e-12
    s = packed + np.conj(packed)
    assert np.max(np.abs(s[:n] - 2 * plain.real)) < 1e-12 and np.max(np.abs(s[n:] - 2 * plain.imag)) < 1e-12
    y = rng.normal(size=2 * n)
    z = y[:n] + 1j * y[n:]
    ref = apply_period(ctx.fft_group_ex(3, False, 0, ls), z)
    got = apply_period(ctx.fft_group_ex(3, False, 0, ls, packed=True), y.astype(complex))
    assert np.max(np.abs(got - np.tile(ref, 2))) < 1e-12
