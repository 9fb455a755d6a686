"""Parity of the CUDA library (through its C ABI) with the CPU oracle.

Ring-level results are compared bit for bit on the same seeded inputs; the
decrypted CryptoInvSqrt output is compared with FP64 1/sqrt(a) (MRE <= 1e-7)
and with the oracle's FP64 model of the same algorithm.
"""
import numpy as np
import pytest

import oracle
from paper_2606_10477_gb300 import hedap, inputs

pytestmark = pytest.mark.gpu

MRE_TARGET = 1e-7


def make_pair(name, seed=1):
    p = inputs.PRESETS[name]
    args = (p["log_n"], p["q_bits"], p["p_bits"], p["alpha"], p["log_scale"], p["hw"], seed)
    return hedap.Context(*args), oracle.Context(*args)


@pytest.fixture(scope="module")
def toy():
    return make_pair("toy")


@pytest.fixture(scope="module")
def n13():
    return make_pair("n13")


@pytest.fixture(scope="module")
def n10():
    return make_pair("n10")


def mre(y, a):
    ref = 1 / np.sqrt(a)
    return float(np.mean(np.abs(y - ref) / ref))


def same_ct(g_ct, o_ct):
    assert g_ct.level == o_ct.level
    assert g_ct.scale == o_ct.scale
    gl, ol = g_ct.limbs(), o_ct.limbs()
    assert gl.shape == ol.shape
    bad = np.count_nonzero(gl != ol)
    assert bad == 0, f"{bad} of {gl.size} residues differ"


def imported_pair(g, o, seed, level, scale=None):
    limbs = inputs.random_ciphertext_limbs(seed, o.primes(), level, o.N)
    scale = scale or o.scale
    return g.ct_import(limbs, level, scale), o.ct_import(limbs, level, scale)


# ---------------------------------------------------------------- parameters and keys
@pytest.mark.parametrize("name", ["toy", "n13", "n10"])
def test_prime_chain_matches(name, request):
    g, o = request.getfixturevalue(name)
    assert np.array_equal(g.primes(), o.primes())


def test_relinearisation_key_bit_exact(toy, n10):
    for g, o in (toy, n10):
        dn = -(-o.n_q // o.alpha)
        for j in range(dn):
            gb, ga = g.key_digit(0, j)
            ob, oa = o.key_digit(0, j)
            assert np.array_equal(ga, oa) and np.array_equal(gb, ob)


def test_galois_elements_from_the_library(n10):
    """The library's Galois elements (hedap_galois_element) against the oracle's, including negative
    steps, zero and steps beyond N/2 (rotation is periodic in N/2), and conjugation 2N - 1."""
    g, o = n10
    for r in (1, -5, 0, 7, o.N // 2, o.N // 2 + 3, -(o.N // 2) - 1):
        assert g.galois_of_rotation(r) == o.galois_of_rotation(r), r
    assert g.galois_of_conjugation() == 2 * o.N - 1


def test_rotation_key_bit_exact(n10):
    g, o = n10
    for r in (1, -5):
        gal = g.galois_of_rotation(r)
        assert gal == o.galois_of_rotation(r)
        for j in (0, 2):
            gb, ga = g.key_digit(gal, j)
            ob, oa = o.key_digit(gal, j)
            assert np.array_equal(ga, oa) and np.array_equal(gb, ob)


# ---------------------------------------------------------------- NTT
@pytest.mark.parametrize("name", ["n10", "toy", "n13"])
def test_ntt_bit_exact_every_prime(name, request):
    g, o = request.getfixturevalue(name)
    primes = o.primes()
    x = inputs.random_limbs(7, primes, o.N)
    fwd = g.ntt(x, 0)
    inv = g.ntt(x, 0, inverse=True)
    for i in range(len(primes)):
        assert np.array_equal(fwd[i], o.ntt(x[i], i)), f"forward, prime {i}"
        assert np.array_equal(inv[i], o.ntt(x[i], i, inverse=True)), f"inverse, prime {i}"
    assert np.array_equal(g.ntt(fwd, 0, inverse=True), x)


@pytest.mark.parametrize("name", ["n10", "n13"])
def test_every_ntt_launch_shape_is_bit_exact(name, request):
    g, o = request.getfixturevalue(name)
    primes = o.primes()
    x = inputs.random_limbs(17, primes, o.N)
    ref_f = np.stack([o.ntt(x[i], i) for i in range(len(primes))])
    ref_i = np.stack([o.ntt(x[i], i, inverse=True) for i in range(len(primes))])
    try:
        for v in range(8):
            g.ntt_set_variant(v, v)
            assert np.array_equal(g.ntt(x, 0), ref_f), f"forward variant {v}"
            assert np.array_equal(g.ntt(x, 0, inverse=True), ref_i), f"inverse variant {v}"
    finally:
        g.ntt_tune(4 * g.n_q, 1)


@pytest.mark.parametrize("name", ["n10", "n13"])
def test_fused_roles_every_launch_shape_bit_exact(name, request):
    """The key switch's ModUp column phase and the fused ModDown / rescale run in the shape of their own
    role: every shape of each role gives the oracle's HMult, rescale and rotation bit for bit."""
    g, o = request.getfixturevalue(name)
    L = o.n_q - 1
    ga, oa = imported_pair(g, o, 41, L)
    gb, ob = imported_pair(g, o, 42, L)
    want = (o.mul(oa, ob), o.rotate(oa, 3))
    saved = g.ntt_get_roles()
    try:
        for role in ("modup", "finish"):
            for v in range(8):
                g.ntt_set_role_variant(hedap.NTT_ROLES[role], v)
                same_ct(g.mul(ga, gb), want[0])
                same_ct(g.rotate(ga, 3), want[1])
            g.ntt_set_roles(saved)
    finally:
        g.ntt_set_roles(saved)
    with pytest.raises(hedap.HedapError):
        g.ntt_set_role_variant(4, 0)
    with pytest.raises(hedap.HedapError):
        g.ntt_set_role_variant(hedap.NTT_ROLES["modup"], 8)


def test_ntt_ragged_batch_offset_primes(n13):
    g, o = n13
    primes = o.primes()
    first = 3
    x = inputs.random_limbs(8, primes[first:first + 7], o.N)  # 7 limbs: not a power of two
    fwd = g.ntt(x, first)
    for i in range(7):
        assert np.array_equal(fwd[i], o.ntt(x[i], first + i))
    assert g.ntt(np.zeros((0, o.N), dtype=np.uint64), 0).size == 0  # empty batch is a no-op
    with pytest.raises(hedap.HedapError):
        g.ntt(x, len(primes) - 2)  # runs past the last prime


def test_ntt_full_size_device_batch():
    torch = pytest.importorskip("torch")
    p = inputs.PRESETS["n16"]
    g = hedap.Context(p["log_n"], p["q_bits"], p["p_bits"], p["alpha"], p["log_scale"], 0, 1)
    o = oracle.Context(p["log_n"], p["q_bits"][:2], p["p_bits"][:1], 1, p["log_scale"], 0, 1)  # same first primes
    primes = g.primes()
    assert np.array_equal(primes[:2], o.primes()[:2])
    x = inputs.random_limbs(9, primes, g.N)  # 26 limbs at N = 2^16
    t = torch.from_numpy(x.view(np.int64)).cuda()
    g.ntt(t, 0)
    g.sync()
    out = t.cpu().numpy().view(np.uint64)
    for i in (0, 1):  # sampled limbs, recomputed by the oracle
        assert np.array_equal(out[i], o.ntt(x[i], i))
    g.ntt(t, 0, inverse=True)
    g.sync()
    assert np.array_equal(t.cpu().numpy().view(np.uint64), x)


# ---------------------------------------------------------------- ring operations, bit exact
@pytest.mark.parametrize("name", ["n10", "toy", "n13"])
def test_add_sub_mul_rescale_bit_exact(name, request):
    g, o = request.getfixturevalue(name)
    L = o.n_q - 1
    ga, oa = imported_pair(g, o, 11, L)
    gb, ob = imported_pair(g, o, 12, L - 1)  # different levels: the higher one is dropped
    same_ct(g.add(ga, gb), o.add(oa, ob))
    same_ct(g.sub(ga, gb), o.sub(oa, ob))
    same_ct(g.mul_relin(ga, gb), o.mul_relin(oa, ob))
    same_ct(g.mul(ga, gb), o.mul(oa, ob))
    same_ct(g.rescale(ga), o.rescale(oa))
    same_ct(g.drop(ga, 1), o.drop(oa, 1))


def test_mul_with_rescale_at_every_level_bit_exact(n10):
    """HMult with its ModDown and rescale in one transform, at every level down to 1 (the last digit partial at
    every other level), against the oracle's relinearised product followed by its rescale."""
    g, o = n10
    for level in range(o.n_q - 1, 0, -1):
        ga, oa = imported_pair(g, o, 300 + level, level)
        gb, ob = imported_pair(g, o, 400 + level, level)
        same_ct(g.mul(ga, gb), o.mul(oa, ob))


def test_mul_with_rescale_bootstrapping_chain_bit_exact():
    """The bts12 chain: three special primes (four staged tiles in the fused column phase) and primes of 45, 55 and 60
    bits, so that some ModUp factors cannot be folded into the key (their bound check fails)."""
    g, o = make_pair("bts12")
    for level in (o.n_q - 1, o.n_q - 5, 12, 3, 1):
        ga, oa = imported_pair(g, o, 500 + level, level)
        gb, ob = imported_pair(g, o, 600 + level, level)
        same_ct(g.mul(ga, gb), o.mul(oa, ob))


@pytest.mark.parametrize("name", ["n10", "toy"])
def test_constants_bit_exact(name, request):
    g, o = request.getfixturevalue(name)
    L = o.n_q - 1
    ga, oa = imported_pair(g, o, 13, L)
    for c in (0.5, -1.25, 3.0e-3):
        same_ct(g.mul_const(ga, c, o.scale * 1.5), o.mul_const(oa, c, o.scale * 1.5))
        same_ct(g.add_const(ga, c), o.add_const(oa, c))
    for m in (2, -3, 0):
        same_ct(g.mul_int(ga, m), o.mul_int(oa, m))


@pytest.mark.parametrize("name", ["n10", "toy"])
def test_rotation_conjugation_bit_exact(name, request):
    g, o = request.getfixturevalue(name)
    L = o.n_q - 1
    for level in (L, 1):
        ga, oa = imported_pair(g, o, 14 + level, level)
        for r in (1, -3, 7):
            same_ct(g.rotate(ga, r), o.rotate(oa, r))
        same_ct(g.conjugate(ga), o.conjugate(oa))


@pytest.mark.parametrize("name", ["n10", "toy"])
def test_hoisted_rotations_bit_exact(name, request):
    g, o = request.getfixturevalue(name)
    L = o.n_q - 1
    for level in (L, 1):
        ga, oa = imported_pair(g, o, 31 + level, level)
        steps = [1, -3, 7, 0]
        for gc, oc in zip(g.rotate_hoisted(ga, steps), o.rotate_hoisted(oa, steps)):
            same_ct(gc, oc)


@pytest.mark.parametrize("name", ["n12a4", "n12a8"])
def test_wide_digits_bit_exact(name):
    """Digits of 4 and 8 primes (5 and 7 special primes): lazy and canonical terms in the fused conversions."""
    g, o = make_pair(name)
    L = o.n_q - 1
    for level in (L, 4):
        ga, oa = imported_pair(g, o, 41 + level, level)
        gb, ob = imported_pair(g, o, 42 + level, level)
        same_ct(g.mul(ga, gb), o.mul(oa, ob))
        same_ct(g.rotate(ga, 3), o.rotate(oa, 3))
        for gc, oc in zip(g.rotate_hoisted(ga, [1, -2]), o.rotate_hoisted(oa, [1, -2])):
            same_ct(gc, oc)


def test_invsqrt_n16_three_digits():
    """N = 2^16, 24 x 50-bit primes, dnum = 3 (7 special primes): MRE <= 1e-7."""
    p = inputs.PRESETS["n16d3"]
    g = hedap.Context(p["log_n"], p["q_bits"], p["p_bits"], p["alpha"], p["log_scale"], 0, 5)
    a = inputs.uniform_values(43, g.N // 2, 1e-3, 1.0)
    y = g.decrypt(g.invsqrt(g.encrypt(a, g.n_q - 1, 44), 1e-3, 1.0, 1.0, 31, 3)).real
    assert mre(y, a) <= MRE_TARGET


def test_ring_ops_bit_exact_at_full_size():
    """N = 2^16, 24 + 2 primes, two primes per digit: one HMult, one rotation, one rescale."""
    p = inputs.PRESETS["n16"]
    g, o = make_pair("n16")
    L = p["q_bits"].__len__() - 1
    ga, oa = imported_pair(g, o, 21, L)
    gb, ob = imported_pair(g, o, 22, L)
    same_ct(g.mul(ga, gb), o.mul(oa, ob))
    same_ct(g.rotate(ga, 5), o.rotate(oa, 5))


# ---------------------------------------------------------------- encryption / decryption
def test_encrypt_decrypt_against_oracle(toy):
    g, o = toy
    a = inputs.uniform_values(31, o.N // 2, -1, 1)
    L = o.n_q - 1
    gc, oc = g.encrypt(a, L, 5), o.encrypt(a, L, 5)
    gl, ol = gc.limbs(), oc.limbs()
    assert np.array_equal(gl[1], ol[1])  # the uniform part a is the same draw
    # the FP64 encodings may differ by one unit in rare coefficients
    diff = o.decrypt_coeffs(o.ct_import(gl, L, gc.scale)) - o.decrypt_coeffs(oc)
    assert np.max(np.abs(diff)) <= 1
    assert np.max(np.abs(g.decrypt(gc).real - a)) < 1e-9
    # the library decrypts the oracle's ciphertext to the oracle's values
    assert np.max(np.abs(g.decrypt(g.ct_import(ol, L, oc.scale)) - o.decrypt(oc))) < 1e-12


# ---------------------------------------------------------------- CryptoInvSqrt
def test_invsqrt_toy_bit_exact_and_accurate(toy):
    """Toy preset: N = 2^12, degree 15, 2 Newton steps on U[0.01, 1]."""
    g, o = toy
    a = inputs.uniform_values(41, o.N // 2, 0.01, 1.0)
    L = o.n_q - 1
    oc = o.encrypt(a, L, 9)
    gc = g.ct_import(oc.limbs(), L, oc.scale)
    gy = g.invsqrt(gc, 0.01, 1.0, 1.0, 15, 2)
    oy = o.invsqrt(oc, 0.01, 1.0, 1.0, 15, 2)
    same_ct(gy, oy)
    y = g.decrypt(gy).real
    assert mre(y, a) <= MRE_TARGET
    plain = oracle.plain_invsqrt(a, 0.01, 1.0, 1.0, 15, 2)
    assert np.max(np.abs(y - plain) / plain) < 1e-6


@pytest.mark.parametrize("d,k", [(31, 3), (63, 2), (15, 4)])
def test_invsqrt_n16_meets_mre_target(d, k):
    """N = 2^16, 32768 slots, U[1e-3, 1]: decrypted MRE <= 1e-7 and close to the FP64 model."""
    p = inputs.PRESETS["n16"]
    g = hedap.Context(p["log_n"], p["q_bits"], p["p_bits"], p["alpha"], p["log_scale"], 0, 3)
    a = inputs.uniform_values(42, g.N // 2, 1e-3, 1.0)
    ct = g.encrypt(a, g.n_q - 1, 17)
    y = g.decrypt(g.invsqrt(ct, 1e-3, 1.0, 1.0, d, k)).real
    plain = oracle.plain_invsqrt(a, 1e-3, 1.0, 1.0, d, k)
    assert mre(y, a) <= MRE_TARGET
    assert np.max(np.abs(y - plain) / plain) < 1e-6


# ---------------------------------------------------------------- errors
def test_error_codes(toy):
    g, o = toy
    ga, _ = imported_pair(g, o, 51, 0)
    with pytest.raises(hedap.HedapError) as e:
        g.rescale(ga)
    assert e.value.code == -2
    gb, _ = imported_pair(g, o, 52, 0, scale=o.scale * 2)
    with pytest.raises(hedap.HedapError) as e:
        g.add(ga, gb)
    assert e.value.code == -3
    bad = inputs.random_ciphertext_limbs(53, o.primes(), 0, o.N)
    bad[0, 0, 0] = o.primes()[0]
    with pytest.raises(hedap.HedapError) as e:
        g.ct_import(bad, 0, o.scale)
    assert e.value.code == -7
    bad = inputs.random_ciphertext_limbs(54, o.primes(), 3, o.N)  # the last word of part 1's last limb
    bad[1, 3, o.N - 1] = int(o.primes()[3]) + 5
    with pytest.raises(hedap.HedapError) as e:
        g.ct_import(bad, 3, o.scale)
    assert e.value.code == -7
    with pytest.raises(hedap.HedapError) as e:
        g.invsqrt(ga, 0.01, 1.0, 1.0, 15, 2)  # level 0 input
    assert e.value.code == -2
    for lvl in (1, 2, 3):  # too few levels for the Chebyshev products: a level error, which the selector skips
        gl, _ = imported_pair(g, o, 60 + lvl, lvl)
        with pytest.raises(hedap.HedapError) as e:
            g.invsqrt(gl, 0.01, 1.0, 1.0, 15, 2)
        assert e.value.code == -2
