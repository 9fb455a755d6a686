"""Seeded synthetic inputs and CKKS parameter presets.

This module holds no arithmetic of the method: it draws input values and
random residues with numpy and names the parameter sets.  Both the CUDA path
and the CPU oracle take their inputs from here.
"""
from __future__ import annotations

import numpy as np

# CKKS parameter presets (bit sizes of the Q primes q_0.., of the special primes,
# primes per key-switching digit, log2 of the scale, secret Hamming weight (0 = dense)).
PRESETS = {
    # toy, correctness only: N = 2^12, 12 primes of ~40 bits + one 60-bit special prime
    "toy": dict(log_n=12, q_bits=[40] * 12, p_bits=[60], alpha=1, log_scale=40, hw=0),
    # N = 2^16, 24 primes of ~50 bits + 2 special primes of ~60 bits, 2 primes per digit
    "n16": dict(log_n=16, q_bits=[50] * 24, p_bits=[60, 60], alpha=2, log_scale=50, hw=0),
    # the same ring with three key-switching digits (8 primes each, dnum = 3 as the workload names it);
    # 7 special primes of 60 bits keep P (420 bits) above a digit (400 bits)
    "n16d3": dict(log_n=16, q_bits=[50] * 24, p_bits=[60] * 7, alpha=8, log_scale=50, hw=0),
    # small rings with the same prime shapes, for fast parity checks
    "n12a8": dict(log_n=12, q_bits=[40] * 10, p_bits=[60] * 7, alpha=8, log_scale=40, hw=0),
    "n12a4": dict(log_n=12, q_bits=[40] * 10, p_bits=[60] * 5, alpha=4, log_scale=40, hw=0),
    "n13": dict(log_n=13, q_bits=[50] * 8, p_bits=[60, 60], alpha=2, log_scale=50, hw=0),
    "n10": dict(log_n=10, q_bits=[45, 36, 36, 36, 36, 36], p_bits=[50, 50], alpha=2, log_scale=36, hw=0),
    # N = 2^16 with bootstrapping: q_0 (60 bits), 10 compute primes (45), 3 x 45, 10 x 55, 3 x 60, P = 3 x 60;
    # log2(QP) = 1555; sparse ternary secret h = 192.  A bootstrap consumes 15 levels (CoeffToSlot the three
    # 60-bit primes, EvalMod nine 55-bit ones, SlotToCoeff the last 55-bit and two 45-bit ones), so a
    # bootstrapped ciphertext sits at level 11
    "bts16": dict(log_n=16, q_bits=[60] + [45] * 10 + [45] * 3 + [55] * 10 + [60] * 3, p_bits=[60] * 3, alpha=3,
                  log_scale=45, hw=192),
    # N = 2^16 shaped like the paper's HEaaN "FGb" parameters (Delta = 2^42, l_max = 12 after bootstrapping,
    # Sec. 3): q_0 (60 bits), 12 compute primes (42), SlotToCoeff 3 x 42, EvalMod 9 x 55, CoeffToSlot 3 x 60,
    # P = 3 x 60; log2(QP) = 1545; sparse ternary secret h = 192
    "bts16f": dict(log_n=16, q_bits=[60] + [42] * 12 + [42] * 3 + [55] * 9 + [60] * 3, p_bits=[60] * 3, alpha=3,
                   log_scale=42, hw=192),
    # the same chain shape at N = 2^12, for parity with the CPU oracle
    "bts12": dict(log_n=12, q_bits=[60] + [45] * 8 + [45] * 3 + [55] * 10 + [60] * 3, p_bits=[60] * 3, alpha=3,
                  log_scale=45, hw=192),
    # the same chains under a dense ternary secret; bootstrapping then runs with sparse-secret
    # encapsulation (an ephemeral secret of weight ENC_HW), which keeps the sparse chain's K.  The
    # rounding noise of rescaling grows with the secret's norm (sqrt(2N/3) against sqrt(h)), so EvalMod
    # runs on 60-bit primes here (log2(QP) = 1605, within the 128-bit bound for a dense ternary secret
    # at N = 2^16); with 55-bit ones the mean error was 4.4 times the sparse chain's at N = 2^14 (1.6
    # times at N = 2^12) and the maximum passed 1e-3 at N = 2^16
    "bts16d": dict(log_n=16, q_bits=[60] + [45] * 10 + [45] * 3 + [60] * 10 + [60] * 3, p_bits=[60] * 3, alpha=3,
                   log_scale=45, hw=0),
    "bts12d": dict(log_n=12, q_bits=[60] + [45] * 8 + [45] * 3 + [60] * 10 + [60] * 3, p_bits=[60] * 3, alpha=3,
                   log_scale=45, hw=0),
}

# bootstrapping parameters: ModRaise overflow bound K, double angles r, EvalMod
# Chebyshev degree, CoeffToSlot and SlotToCoeff levels
BTS = dict(K=28, r=4, deg=31, cts=3, stc=3)
ENC_HW = 192  # weight of the ephemeral sparse secret of the encapsulation


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def uniform_values(seed: int, n: int, lo: float, hi: float) -> np.ndarray:
    """n values uniform in [lo, hi]."""
    return rng(seed).uniform(lo, hi, n)


def log_uniform_values(seed: int, n: int, lo: float, hi: float) -> np.ndarray:
    """n values with log10 uniform in [log10 lo, log10 hi]."""
    return 10.0 ** rng(seed).uniform(np.log10(lo), np.log10(hi), n)


def linspace_values(n: int, lo: float, hi: float) -> np.ndarray:
    """The paper's provisioning input: n evenly spaced points in [lo, hi]."""
    return np.linspace(lo, hi, n)


def random_limbs(seed: int, primes, n_coeffs: int) -> np.ndarray:
    """Uniform residues: one row of n_coeffs words per prime, row i below primes[i]."""
    g = rng(seed)
    return np.stack([g.integers(0, int(q), n_coeffs, dtype=np.uint64) for q in primes])


def random_ciphertext_limbs(seed: int, primes, level: int, n_coeffs: int) -> np.ndarray:
    """[2][level+1][N] uniform residues (a valid-shaped NTT-domain ciphertext)."""
    g = rng(seed)
    return np.stack([np.stack([g.integers(0, int(primes[i]), n_coeffs, dtype=np.uint64) for i in range(level + 1)])
                     for _ in range(2)])


def gaussian_records(seed: int, n: int, mean: float = 50.0, sd: float = 10.0, unit: float = 0.01) -> np.ndarray:
    """n records drawn from N(mean, sd^2), expressed in `unit`s of 100 (0.5 +- 0.1 by default)."""
    return rng(seed).normal(mean, sd, n) * unit


def correlated_records(seed: int, x: np.ndarray, rho: float, mean: float = 50.0, sd: float = 10.0,
                       unit: float = 0.01) -> np.ndarray:
    """Records paired with x (same distribution) with correlation about rho."""
    z = (x / unit - mean) / sd
    e = rng(seed).normal(0.0, 1.0, x.size)
    return (mean + sd * (rho * z + np.sqrt(1.0 - rho * rho) * e)) * unit


def pack_slots(values: np.ndarray, slots: int) -> list:
    """Split records into ceil(n / slots) slot vectors, the last one zero-padded."""
    n_ct = max(1, -(-values.size // slots))
    buf = np.zeros(n_ct * slots)
    buf[:values.size] = values
    return [buf[k * slots:(k + 1) * slots].copy() for k in range(n_ct)]
