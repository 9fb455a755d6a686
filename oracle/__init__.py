"""CPU oracle for the RNS-CKKS / CryptoInvSqrt hot path -- TEST INFRASTRUCTURE ONLY.

The arithmetic lives in ``ckks_oracle.cpp`` (plain C++, ``unsigned __int128``
modular arithmetic, FP64).  This module compiles it with the host ``g++`` and
exposes it through ``ctypes``.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it; the GPU library never does.

Functions whose results no independent check pins are listed in the C++ file's
header; every function exported here is pinned by ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ckks_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "libckks_oracle.so")
_lock = threading.Lock()
_lib = None

u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libckks_oracle.so`` (g++, -O2)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    base = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-fvisibility=hidden", _SRC]
    r = subprocess.run(base + ["-fopenmp", "-o", tmp], capture_output=True)
    if r.returncode != 0:  # no OpenMP runtime: the same code, one thread
        subprocess.run(base + ["-o", tmp], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


def _declare(L):
    vp = C.c_void_p
    sig = {
        "orc_last_error": (C.c_char_p, []),
        "orc_ctx_create": (vp, [C.c_uint32, C.c_uint32, u32p, C.c_uint32, u32p, C.c_uint32, C.c_double,
                                C.c_uint32, C.c_uint64]),
        "orc_ctx_destroy": (None, [vp]),
        "orc_ctx_primes": (C.c_int, [vp, u64p]),
        "orc_ctx_psi": (C.c_int, [vp, u64p]),
        "orc_export_secret": (C.c_int, [vp, i64p]),
        "orc_export_sparse_secret": (C.c_int, [vp, i64p]),
        "orc_gen_galois_key": (C.c_int, [vp, C.c_uint64]),
        "orc_galois_of_rotation": (C.c_uint64, [vp, C.c_int64]),
        "orc_export_key": (C.c_int, [vp, C.c_uint64, C.c_uint32, u64p, u64p]),
        "orc_ntt": (C.c_int, [vp, u64p, C.c_uint32, C.c_int]),
        "orc_modup_coeff": (C.c_int, [vp, u64p, C.c_int, C.c_int, u64p]),
        "orc_moddown_coeff": (C.c_int, [vp, u64p, C.c_int, u64p]),
        "orc_rescale_ntt": (C.c_int, [vp, u64p, C.c_int, u64p]),
        "orc_encode_coeffs": (C.c_int, [vp, f64p, f64p, C.c_double, f64p]),
        "orc_decode_coeffs": (C.c_int, [vp, f64p, C.c_double, f64p, f64p]),
        "orc_ct_import": (vp, [vp, u64p, C.c_int, C.c_double]),
        "orc_ct_info": (C.c_int, [vp, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
        "orc_ct_export": (C.c_int, [vp, vp, u64p]),
        "orc_ct_free": (None, [vp]),
        "orc_encrypt": (vp, [vp, f64p, f64p, C.c_uint64, C.c_int, C.c_uint64]),
        "orc_decrypt": (C.c_int, [vp, vp, f64p, f64p]),
        "orc_decrypt_coeffs": (C.c_int, [vp, vp, f64p]),
        "orc_add": (vp, [vp, vp, vp]),
        "orc_sub": (vp, [vp, vp, vp]),
        "orc_mul_relin": (vp, [vp, vp, vp]),
        "orc_mul": (vp, [vp, vp, vp]),
        "orc_rescale": (vp, [vp, vp]),
        "orc_rotate": (vp, [vp, vp, C.c_int64]),
        "orc_rotate_hoisted": (C.c_int, [vp, vp, C.POINTER(C.c_int64), C.c_int, C.POINTER(vp)]),
        "orc_conjugate": (vp, [vp, vp]),
        "orc_mul_const": (vp, [vp, vp, C.c_double, C.c_double]),
        "orc_add_const": (vp, [vp, vp, C.c_double]),
        "orc_mul_int": (vp, [vp, vp, C.c_int64]),
        "orc_drop": (vp, [vp, vp, C.c_int]),
        "orc_invsqrt": (vp, [vp, vp, C.c_double, C.c_double, C.c_double, C.c_uint32, C.c_uint32, C.c_uint32,
                             C.c_uint64, C.c_uint32]),
        "orc_bootstrap_slots": (vp, [vp, vp, C.c_int]),
        "orc_bootstrap_scaled_slots": (vp, [vp, vp, C.c_int64, C.c_int]),
        "orc_sub_sum": (vp, [vp, vp, C.c_int]),
        "orc_cheb_coeffs": (C.c_int, [C.c_double, C.c_double, C.c_uint32, f64p]),
        "orc_cheb_eval": (vp, [vp, vp, f64p, C.c_uint32, C.c_int]),
        "orc_clenshaw": (C.c_double, [f64p, C.c_uint32, C.c_double]),
        "orc_plain_invsqrt": (C.c_int, [f64p, C.c_uint64, C.c_double, C.c_double, C.c_double, C.c_uint32,
                                        C.c_uint32, f64p]),
        "orc_key_switch": (C.c_int, [vp, u64p, C.c_int, C.c_uint64, u64p]),
        "orc_threads": (C.c_int, []),
        "orc_bts_setup": (C.c_int, [vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]),
        "orc_bootstrap": (vp, [vp, vp]),
        "orc_bts_encapsulate": (C.c_int, [vp, C.c_int]),
        "orc_encapsulation_switch": (vp, [vp, vp, C.c_int]),
        "orc_decrypt_sparse": (C.c_int, [vp, vp, f64p, f64p]),
        "orc_bootstrap_scaled": (vp, [vp, vp, C.c_int64]),
        "orc_mod_raise": (vp, [vp, vp]),
        "orc_linear_transform_group": (vp, [vp, vp, C.c_int, C.c_int, C.c_int, C.c_double]),
        "orc_eval_mod": (vp, [vp, vp]),
        "orc_set_scale": (vp, [vp, vp, C.c_double]),
        "orc_mul_monomial": (vp, [vp, vp, C.c_uint64]),
        "orc_fft_group_offsets": (C.c_int, [vp, C.c_int, C.c_int, C.c_int, i64p, C.c_int]),
        "orc_fft_group_diag": (C.c_int, [vp, C.c_int, C.c_int, C.c_int, C.c_int64, f64p, f64p]),
        "orc_fft_group_ex_offsets": (C.c_int, [vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, i64p, C.c_int]),
        "orc_fft_group_ex_diag": (C.c_int, [vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int64, f64p, f64p,
                                            C.c_int]),
        "orc_splitmix_stream": (C.c_uint64, [C.c_uint64, C.c_uint64, C.c_uint64, u64p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


class OracleError(RuntimeError):
    pass


def _check(rc):
    if rc is None or (isinstance(rc, int) and rc < 0):
        raise OracleError(lib().orc_last_error().decode())
    return rc


class Ciphertext:
    """Oracle ciphertext handle: (c0, c1) in the NTT domain at ``level`` with ``scale``."""

    def __init__(self, ctx: "Context", handle):
        if not handle:
            raise OracleError(lib().orc_last_error().decode())
        self.ctx = ctx
        self.h = handle

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_ct_free(self.h)
            self.h = None

    @property
    def level(self) -> int:
        lv, sc = C.c_int(), C.c_double()
        lib().orc_ct_info(self.h, C.byref(lv), C.byref(sc))
        return lv.value

    @property
    def scale(self) -> float:
        lv, sc = C.c_int(), C.c_double()
        lib().orc_ct_info(self.h, C.byref(lv), C.byref(sc))
        return sc.value

    def limbs(self) -> np.ndarray:
        out = np.empty((2, self.level + 1, self.ctx.N), dtype=np.uint64)
        lib().orc_ct_export(self.ctx.h, self.h, out)
        return out


class Context:
    """Oracle CKKS context: prime chain, secret key and switching keys from ``seed``."""

    def __init__(self, log_n, q_bits, p_bits, alpha, log_scale, hw=0, seed=1):
        qb = np.ascontiguousarray(q_bits, dtype=np.uint32)
        pb = np.ascontiguousarray(p_bits, dtype=np.uint32)
        h = lib().orc_ctx_create(log_n, len(qb), qb, len(pb), pb, alpha, float(log_scale), hw, seed)
        if not h:
            raise OracleError(lib().orc_last_error().decode())
        self.h = h
        self.log_n, self.N = log_n, 1 << log_n
        self.n_q, self.n_p, self.alpha = len(qb), len(pb), alpha
        self.scale = 2.0 ** log_scale
        self.seed = seed

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_ctx_destroy(self.h)
            self.h = None

    # ---- parameters and keys
    def primes(self) -> np.ndarray:
        out = np.empty(self.n_q + self.n_p, dtype=np.uint64)
        lib().orc_ctx_primes(self.h, out)
        return out

    def psi(self) -> np.ndarray:
        out = np.empty(self.n_q + self.n_p, dtype=np.uint64)
        lib().orc_ctx_psi(self.h, out)
        return out

    def secret(self) -> np.ndarray:
        out = np.empty(self.N, dtype=np.int64)
        lib().orc_export_secret(self.h, out)
        return out

    def sparse_secret(self) -> np.ndarray:
        """The ephemeral secret of the bootstrapping encapsulation (coefficients)."""
        out = np.empty(self.N, dtype=np.int64)
        _check(lib().orc_export_sparse_secret(self.h, out))
        return out

    def galois_of_rotation(self, r: int) -> int:
        return int(lib().orc_galois_of_rotation(self.h, r))

    def key_digit(self, g: int, j: int):
        tot = self.n_q + self.n_p
        b = np.empty((tot, self.N), dtype=np.uint64)
        a = np.empty((tot, self.N), dtype=np.uint64)
        _check(lib().orc_export_key(self.h, g, j, b, a))
        return b, a

    # ---- ring helpers
    def ntt(self, limb: np.ndarray, prime_idx: int, inverse=False) -> np.ndarray:
        a = np.ascontiguousarray(limb, dtype=np.uint64).copy()
        lib().orc_ntt(self.h, a, prime_idx, int(inverse))
        return a

    def modup_coeff(self, digit_limbs: np.ndarray, level: int, digit: int) -> np.ndarray:
        x = np.ascontiguousarray(digit_limbs, dtype=np.uint64)
        out = np.empty((level + 1 + self.n_p, self.N), dtype=np.uint64)
        _check(lib().orc_modup_coeff(self.h, x, level, digit, out))
        return out

    def moddown_coeff(self, ext_limbs: np.ndarray, level: int) -> np.ndarray:
        x = np.ascontiguousarray(ext_limbs, dtype=np.uint64)
        out = np.empty((level + 1, self.N), dtype=np.uint64)
        _check(lib().orc_moddown_coeff(self.h, x, level, out))
        return out

    def rescale_ntt(self, limbs: np.ndarray, level: int) -> np.ndarray:
        x = np.ascontiguousarray(limbs, dtype=np.uint64)
        out = np.empty((level, self.N), dtype=np.uint64)
        _check(lib().orc_rescale_ntt(self.h, x, level, out))
        return out

    def key_switch(self, d: np.ndarray, level: int, galois: int) -> np.ndarray:
        x = np.ascontiguousarray(d, dtype=np.uint64)
        out = np.empty((2, level + 1, self.N), dtype=np.uint64)
        _check(lib().orc_key_switch(self.h, x, level, galois, out))
        return out

    def encode_coeffs(self, re, im=None, scale=None) -> np.ndarray:
        re = np.ascontiguousarray(re, dtype=np.float64)
        im = np.zeros_like(re) if im is None else np.ascontiguousarray(im, dtype=np.float64)
        out = np.empty(self.N, dtype=np.float64)
        _check(lib().orc_encode_coeffs(self.h, re, im, float(scale or self.scale), out))
        return out

    def decode_coeffs(self, m, scale=None):
        m = np.ascontiguousarray(m, dtype=np.float64)
        re = np.empty(self.N // 2)
        im = np.empty(self.N // 2)
        _check(lib().orc_decode_coeffs(self.h, m, float(scale or self.scale), re, im))
        return re + 1j * im

    # ---- ciphertexts
    def encrypt(self, values, level: int, seed: int) -> Ciphertext:
        v = np.asarray(values)
        re = np.ascontiguousarray(v.real, dtype=np.float64)
        im = np.ascontiguousarray(v.imag if np.iscomplexobj(v) else np.zeros_like(re), dtype=np.float64)
        return Ciphertext(self, lib().orc_encrypt(self.h, re, im, len(re), level, seed))

    def decrypt(self, ct: Ciphertext) -> np.ndarray:
        re = np.empty(self.N // 2)
        im = np.empty(self.N // 2)
        _check(lib().orc_decrypt(self.h, ct.h, re, im))
        return re + 1j * im

    def decrypt_coeffs(self, ct: Ciphertext) -> np.ndarray:
        out = np.empty(self.N)
        _check(lib().orc_decrypt_coeffs(self.h, ct.h, out))
        return out

    def ct_import(self, limbs: np.ndarray, level: int, scale: float) -> Ciphertext:
        x = np.ascontiguousarray(limbs, dtype=np.uint64)
        return Ciphertext(self, lib().orc_ct_import(self.h, x, level, float(scale)))

    def add(self, a, b):
        return Ciphertext(self, lib().orc_add(self.h, a.h, b.h))

    def sub(self, a, b):
        return Ciphertext(self, lib().orc_sub(self.h, a.h, b.h))

    def mul_relin(self, a, b):
        return Ciphertext(self, lib().orc_mul_relin(self.h, a.h, b.h))

    def mul(self, a, b):
        return Ciphertext(self, lib().orc_mul(self.h, a.h, b.h))

    def rescale(self, a):
        return Ciphertext(self, lib().orc_rescale(self.h, a.h))

    def rotate(self, a, steps: int):
        return Ciphertext(self, lib().orc_rotate(self.h, a.h, steps))

    def rotate_hoisted(self, a, steps):
        """Rotations of one ciphertext sharing one ModUp (hoisting), one per entry of steps."""
        st = (C.c_int64 * len(steps))(*steps)
        out = (C.c_void_p * len(steps))()
        if lib().orc_rotate_hoisted(self.h, a.h, st, len(steps), out) != 0:
            raise OracleError(lib().orc_last_error().decode())
        return [Ciphertext(self, out[i]) for i in range(len(steps))]

    def conjugate(self, a):
        return Ciphertext(self, lib().orc_conjugate(self.h, a.h))

    def mul_const(self, a, c: float, target_scale: float):
        return Ciphertext(self, lib().orc_mul_const(self.h, a.h, c, target_scale))

    def add_const(self, a, c: float):
        return Ciphertext(self, lib().orc_add_const(self.h, a.h, c))

    def mul_int(self, a, m: int):
        return Ciphertext(self, lib().orc_mul_int(self.h, a.h, m))

    def drop(self, a, level: int):
        return Ciphertext(self, lib().orc_drop(self.h, a.h, level))

    def bts_setup(self, K=28, r=4, deg=31, cts=3, stc=3) -> int:
        """Enable bootstrapping; returns the level of a bootstrapped ciphertext."""
        return _check(lib().orc_bts_setup(self.h, K, r, deg, cts, stc))

    def bootstrap(self, a):
        return Ciphertext(self, lib().orc_bootstrap(self.h, a.h))

    def bootstrap_slots(self, a, log_slots: int):
        """Sparse-slot bootstrapping of a level-0 ciphertext holding 2^log_slots values repeated."""
        return Ciphertext(self, lib().orc_bootstrap_slots(self.h, a.h, log_slots))

    def bootstrap_scaled_slots(self, a, Y: int, log_slots: int):
        return Ciphertext(self, lib().orc_bootstrap_scaled_slots(self.h, a.h, Y, log_slots))

    def sub_sum(self, a, log_slots: int):
        """Sum of the rotations by 2^log_slots, 2^(log_slots+1), ..., N/4 (projection onto the subring)."""
        return Ciphertext(self, lib().orc_sub_sum(self.h, a.h, log_slots))

    def bts_encapsulate(self, h: int) -> None:
        """Sparse-secret encapsulation of bootstrapping: an ephemeral secret of weight h and its two keys."""
        _check(lib().orc_bts_encapsulate(self.h, h))

    def encapsulation_switch(self, a, to_sparse: bool):
        return Ciphertext(self, lib().orc_encapsulation_switch(self.h, a.h, 1 if to_sparse else 0))

    def decrypt_sparse(self, ct: Ciphertext) -> np.ndarray:
        """Decryption under the ephemeral sparse secret of the encapsulation."""
        re = np.empty(self.N // 2)
        im = np.empty(self.N // 2)
        _check(lib().orc_decrypt_sparse(self.h, ct.h, re, im))
        return re + 1j * im

    def bootstrap_scaled(self, a, Y: int):
        return Ciphertext(self, lib().orc_bootstrap_scaled(self.h, a.h, Y))

    def linear_transform_group(self, a, groups: int, inverse: bool, g: int, target: float):
        return Ciphertext(self, lib().orc_linear_transform_group(self.h, a.h, groups, int(inverse), g, target))

    def eval_mod(self, a):
        return Ciphertext(self, lib().orc_eval_mod(self.h, a.h))

    def with_scale(self, a, scale: float):
        return Ciphertext(self, lib().orc_set_scale(self.h, a.h, scale))

    def mod_raise(self, a):
        return Ciphertext(self, lib().orc_mod_raise(self.h, a.h))

    def mul_monomial(self, a, e: int):
        return Ciphertext(self, lib().orc_mul_monomial(self.h, a.h, e))

    def fft_group(self, groups: int, inverse: bool, g: int) -> dict:
        """{offset: complex diagonal} of group g of the grouped special-FFT factors."""
        offs = np.empty(4096, dtype=np.int64)
        k = _check(lib().orc_fft_group_offsets(self.h, groups, int(inverse), g, offs, len(offs)))
        out = {}
        for o in offs[:k]:
            re, im = np.empty(self.N // 2), np.empty(self.N // 2)
            _check(lib().orc_fft_group_diag(self.h, groups, int(inverse), g, int(o), re, im))
            out[int(o)] = re + 1j * im
        return out

    def fft_group_ex(self, groups: int, inverse: bool, g: int, log_slots: int, packed: bool = False) -> dict:
        """{offset: diagonal} of group g for 2^log_slots slots; packed: the 2n-periodic form used when the
        real and imaginary parts share one ciphertext (last CoeffToSlot / first SlotToCoeff group)."""
        offs = np.empty(1 << 16, dtype=np.int64)
        k = _check(lib().orc_fft_group_ex_offsets(self.h, groups, int(inverse), g, log_slots, int(packed), offs,
                                                  len(offs)))
        out = {}
        cap = self.N  # a diagonal has at most 2n <= N entries
        for o in offs[:k]:
            re, im = np.empty(cap), np.empty(cap)
            m = _check(lib().orc_fft_group_ex_diag(self.h, groups, int(inverse), g, log_slots, int(packed), int(o),
                                                   re, im, cap))
            out[int(o)] = re[:m] + 1j * im[:m]
        return out

    def cheb_eval(self, t, coeffs, need: int = -1):
        """sum_j c_j T_j(t) (t in [-1, 1]); need < 0: the fewest-levels plan, else the fewest-products plan
        when it ends at level >= need."""
        c = np.ascontiguousarray(coeffs, dtype=np.float64)
        return Ciphertext(self, lib().orc_cheb_eval(self.h, t.h, c, len(c) - 1, need))

    def invsqrt(self, a, lo, hi, B, degree, iters, pre_bts=0, bts_mask=0, log_slots=0):
        return Ciphertext(self, lib().orc_invsqrt(self.h, a.h, lo, hi, B, degree, iters, pre_bts, bts_mask,
                                                  log_slots))


def cheb_coeffs(lo: float, hi: float, d: int) -> np.ndarray:
    out = np.empty(d + 1)
    lib().orc_cheb_coeffs(lo, hi, d, out)
    return out


def clenshaw(c: np.ndarray, t: float) -> float:
    c = np.ascontiguousarray(c, dtype=np.float64)
    return float(lib().orc_clenshaw(c, len(c) - 1, t))


def plain_invsqrt(a, lo, hi, B, degree, iters) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    out = np.empty_like(a)
    lib().orc_plain_invsqrt(a, len(a), lo, hi, B, degree, iters, out)
    return out


def splitmix_stream(seed: int, tag: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.uint64)
    lib().orc_splitmix_stream(seed, tag, n, out)
    return out


def threads() -> int:
    """Host threads the oracle's per-limb loops use."""
    return int(lib().orc_threads())
