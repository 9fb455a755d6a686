"""ctypes binding of the GB300 RNS-CKKS library (``include/hedap.h``).

Argument marshalling only: every operation runs in the CUDA library.  Importing
this module does not load the library; the first ``Context`` does, and fails
loudly when ``_build/libhedap.so`` is missing (run ``build()`` first) or no
CUDA device is present.  There is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhedap.so")
_lock = threading.Lock()
_lib = None

STATUS = {0: "ok", -1: "invalid argument", -2: "not enough levels", -3: "scale mismatch", -4: "out of device memory",
          -5: "CUDA error", -6: "wait timed out", -7: "input out of range", -8: "missing switching key",
          -9: "cancelled"}
FAULT_ADMISSION_OOM = 1
# NTT launch-shape roles (HEDAP_NTT_ROLE_*)
NTT_ROLES = {"forward": 0, "inverse": 1, "modup": 2, "finish": 3}

EXPORTED = [
    "hedap_status_str", "hedap_last_error", "hedap_ctx_create", "hedap_ctx_destroy", "hedap_ctx_primes", "hedap_sync",
    "hedap_gen_galois_key", "hedap_galois_element", "hedap_export_key", "hedap_encrypt", "hedap_decrypt", "hedap_ct_import",
    "hedap_ct_export", "hedap_batch_import", "hedap_batch_export", "hedap_ct_info", "hedap_ct_free", "hedap_add", "hedap_sub", "hedap_mul_relin", "hedap_mul",
    "hedap_rescale", "hedap_rotate", "hedap_rotate_hoisted", "hedap_conjugate", "hedap_mul_const", "hedap_add_const", "hedap_mul_int",
    "hedap_drop_level", "hedap_invsqrt", "hedap_ntt", "hedap_profile_enable", "hedap_profile_read", "hedap_profile_read_slots",
    "hedap_launch_count", "hedap_modup", "hedap_moddown", "hedap_key_switch", "hedap_rescale_noalloc",
    "hedap_bootstrap_setup", "hedap_bootstrap", "hedap_bootstrap_scaled", "hedap_bootstrap_encapsulate",
    "hedap_encapsulation_switch", "hedap_bootstrap_slots", "hedap_bootstrap_scaled_slots", "hedap_sub_sum", "hedap_mod_raise", "hedap_mul_monomial",
    "hedap_bts_linear_transform", "hedap_eval_mod", "hedap_set_scale", "hedap_encode", "hedap_bts_diagonal",
    "hedap_batch_pack", "hedap_batch_unpack", "hedap_ct_batch_size", "hedap_invsqrt_batch", "hedap_invsqrt_many", "hedap_invsqrt_mixed", "hedap_ntt_batch",
    "hedap_ntt_tune", "hedap_ntt_set_variant", "hedap_ntt_get_variant", "hedap_ntt_set_role_variant",
    "hedap_ntt_get_role_variant", "hedap_butterfly_rate", "hedap_select", "hedap_getoptiter_rule", "hedap_select_level_rule",
    "hedap_server_create", "hedap_server_submit", "hedap_server_poll", "hedap_server_stats", "hedap_server_destroy",
    "hedap_server_resume", "hedap_server_estimate", "hedap_server_wait", "hedap_server_cancel", "hedap_server_inject",
    "hedap_server_merges", "hedap_server_set_table", "hedap_invsqrt_graph_create", "hedap_graph_run",
    "hedap_graph_kernels", "hedap_graph_destroy", "hedap_invsqrt_mixed_graph_create", "hedap_graph_run_many",
]


class SelectCfg(C.Structure):
    _fields_ = [("A", C.c_double), ("B_max", C.c_double), ("B", C.c_double), ("d_e_min", C.c_uint32),
                ("d_e_max", C.c_uint32), ("i_max", C.c_uint32), ("theta", C.c_double), ("delta", C.c_double),
                ("mre_target", C.c_double), ("level_min", C.c_int32), ("level_max", C.c_int32),
                ("seed", C.c_uint64)]


class SelectEntry(C.Structure):
    _fields_ = [("level", C.c_int32), ("degree", C.c_uint32), ("c", C.c_uint32), ("iters", C.c_uint32),
                ("mre", C.c_double), ("ms", C.c_double), ("kind", C.c_uint32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SelectTrace(C.Structure):
    _fields_ = [("level", C.c_int32), ("degree", C.c_uint32), ("c", C.c_uint32), ("iter", C.c_uint32),
                ("mre", C.c_double), ("ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class BtsParams(C.Structure):
    _fields_ = [("K", C.c_uint32), ("double_angles", C.c_uint32), ("mod_degree", C.c_uint32),
                ("cts_levels", C.c_uint32), ("stc_levels", C.c_uint32)]


class HedapError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [("log_n", C.c_uint32), ("n_q", C.c_uint32), ("q_bits", C.POINTER(C.c_uint32)),
                ("n_p", C.c_uint32), ("p_bits", C.POINTER(C.c_uint32)), ("alpha", C.c_uint32),
                ("log_scale", C.c_double), ("secret_hw", C.c_uint32)]


class InvSqrtCfg(C.Structure):
    _fields_ = [("lo", C.c_double), ("hi", C.c_double), ("B", C.c_double), ("degree", C.c_uint32),
                ("newton_iters", C.c_uint32), ("pre_bts", C.c_uint32), ("bts_mask", C.c_uint64),
                ("log_slots", C.c_uint32)]


class ServerCfg(C.Structure):
    _fields_ = [("max_batch", C.c_uint32), ("start_paused", C.c_uint32), ("hbm_budget_bytes", C.c_uint64),
                ("admit_max", C.c_uint32)]


class Query(C.Structure):
    _fields_ = [("kind", C.c_uint32), ("x", C.POINTER(C.c_void_p)), ("y", C.POINTER(C.c_void_p)),
                ("n_ct", C.c_uint32), ("n_records", C.c_uint64), ("invsqrt", InvSqrtCfg), ("choice", C.c_uint32)]


QUERY_ZSCORE, QUERY_PCC = 1, 2


def load(path: str = LIB_PATH):
    """Load the shared library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
            L = C.CDLL(path)
            _declare(L)
            _lib = L
    return _lib


def _declare(L):
    vp, pp = C.c_void_p, C.POINTER(C.c_void_p)
    u64p = C.POINTER(C.c_uint64)
    dp = C.POINTER(C.c_double)
    st = C.c_int
    sig = {
        "hedap_status_str": (C.c_char_p, [C.c_int]),
        "hedap_last_error": (C.c_char_p, []),
        "hedap_ctx_create": (st, [C.POINTER(Params), C.c_uint64, vp, pp]),
        "hedap_ctx_destroy": (None, [vp]),
        "hedap_ctx_primes": (st, [vp, u64p, C.c_size_t]),
        "hedap_sync": (st, [vp]),
        "hedap_gen_galois_key": (st, [vp, C.c_uint64]),
        "hedap_galois_element": (st, [vp, C.c_int64, C.c_int, u64p]),
        "hedap_export_key": (st, [vp, C.c_uint64, C.c_uint32, u64p, u64p]),
        "hedap_encrypt": (st, [vp, dp, dp, C.c_size_t, C.c_int, C.c_uint64, pp]),
        "hedap_decrypt": (st, [vp, vp, dp, dp, C.c_size_t]),
        "hedap_ct_import": (st, [vp, u64p, C.c_int, C.c_double, C.c_int, pp]),
        "hedap_ct_export": (st, [vp, vp, u64p, C.c_size_t, C.c_int]),
        "hedap_batch_import": (st, [vp, u64p, C.c_size_t, C.c_int, C.c_double, C.c_int, pp]),
        "hedap_batch_export": (st, [vp, vp, u64p, C.c_size_t, C.c_int]),
        "hedap_ct_info": (st, [vp, C.POINTER(C.c_int), dp]),
        "hedap_ct_free": (None, [vp]),
        "hedap_add": (st, [vp, vp, vp, pp]),
        "hedap_sub": (st, [vp, vp, vp, pp]),
        "hedap_mul_relin": (st, [vp, vp, vp, pp]),
        "hedap_mul": (st, [vp, vp, vp, pp]),
        "hedap_rescale": (st, [vp, vp, pp]),
        "hedap_rotate": (st, [vp, vp, C.c_int64, pp]),
        "hedap_rotate_hoisted": (st, [vp, vp, C.POINTER(C.c_int64), C.c_size_t, pp]),
        "hedap_conjugate": (st, [vp, vp, pp]),
        "hedap_mul_const": (st, [vp, vp, C.c_double, C.c_double, pp]),
        "hedap_add_const": (st, [vp, vp, C.c_double, pp]),
        "hedap_mul_int": (st, [vp, vp, C.c_int64, pp]),
        "hedap_drop_level": (st, [vp, vp, C.c_int, pp]),
        "hedap_invsqrt": (st, [vp, vp, C.POINTER(InvSqrtCfg), pp]),
        "hedap_ntt": (st, [vp, u64p, C.c_size_t, C.c_uint32, C.c_int, C.c_int]),
        "hedap_profile_enable": (st, [C.c_int]),
        "hedap_profile_read": (st, [C.c_char_p, u64p, dp, dp]),
        "hedap_profile_read_slots": (st, [C.c_char_p, dp]),
        "hedap_launch_count": (st, [u64p]),
        "hedap_modup": (st, [vp, u64p, C.c_int, u64p]),
        "hedap_moddown": (st, [vp, u64p, C.c_int, u64p]),
        "hedap_key_switch": (st, [vp, u64p, C.c_int, C.c_uint64, u64p]),
        "hedap_rescale_noalloc": (st, [vp, u64p, C.c_int, u64p]),
        "hedap_bootstrap_setup": (st, [vp, C.POINTER(BtsParams), C.POINTER(C.c_int)]),
        "hedap_bootstrap": (st, [vp, vp, pp]),
        "hedap_bootstrap_scaled": (st, [vp, vp, C.c_int64, pp]),
        "hedap_bootstrap_encapsulate": (st, [vp, C.c_uint32]),
        "hedap_bootstrap_slots": (st, [vp, vp, C.c_uint32, pp]),
        "hedap_bootstrap_scaled_slots": (st, [vp, vp, C.c_int64, C.c_uint32, pp]),
        "hedap_sub_sum": (st, [vp, vp, C.c_uint32, pp]),
        "hedap_encapsulation_switch": (st, [vp, vp, C.c_int, pp]),
        "hedap_mod_raise": (st, [vp, vp, pp]),
        "hedap_mul_monomial": (st, [vp, vp, C.c_uint64, pp]),
        "hedap_bts_linear_transform": (st, [vp, vp, C.c_int, C.c_int, C.c_double, pp]),
        "hedap_eval_mod": (st, [vp, vp, pp]),
        "hedap_set_scale": (st, [vp, vp, C.c_double]),
        "hedap_encode": (st, [vp, dp, dp, C.c_size_t, C.c_double, C.POINTER(C.c_int64)]),
        "hedap_bts_diagonal": (st, [vp, C.c_int, C.c_int, C.c_int64, dp, dp]),
        "hedap_batch_pack": (st, [vp, pp, C.c_size_t, pp]),
        "hedap_batch_unpack": (st, [vp, vp, C.c_size_t, pp]),
        "hedap_ct_batch_size": (st, [vp, C.POINTER(C.c_int)]),
        "hedap_invsqrt_batch": (st, [vp, pp, C.POINTER(InvSqrtCfg), C.c_size_t, pp]),
        "hedap_invsqrt_many": (st, [vp, pp, C.POINTER(InvSqrtCfg), C.c_size_t, C.c_int, pp]),
        "hedap_invsqrt_mixed": (st, [vp, pp, C.POINTER(InvSqrtCfg), C.c_size_t, pp]),
        "hedap_ntt_batch": (st, [vp, u64p, C.c_size_t, C.c_size_t, C.c_uint32, C.c_int, C.c_int]),
        "hedap_ntt_tune": (st, [vp, C.c_int, C.c_int, C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_int,
                                C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "hedap_ntt_set_variant": (st, [vp, C.c_int, C.c_int]),
        "hedap_ntt_get_variant": (st, [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "hedap_ntt_set_role_variant": (st, [vp, C.c_int, C.c_int]),
        "hedap_ntt_get_role_variant": (st, [vp, C.c_int, C.POINTER(C.c_int)]),
        "hedap_butterfly_rate": (st, [vp, dp]),
        "hedap_select": (st, [vp, C.POINTER(SelectCfg), C.POINTER(SelectEntry), C.c_size_t, C.POINTER(C.c_size_t),
                              C.POINTER(SelectEntry), C.c_size_t, C.POINTER(C.c_size_t), C.POINTER(SelectTrace),
                              C.c_size_t, C.POINTER(C.c_size_t)]),
        "hedap_getoptiter_rule": (st, [dp, C.c_size_t, C.c_double, C.POINTER(C.c_int), dp]),
        "hedap_select_level_rule": (st, [C.POINTER(SelectEntry), C.c_size_t, C.c_double, C.c_double,
                                         C.POINTER(SelectEntry), C.POINTER(SelectEntry), C.POINTER(SelectEntry),
                                         C.POINTER(C.c_int)]),
        "hedap_server_create": (st, [vp, C.POINTER(ServerCfg), pp]),
        "hedap_server_submit": (st, [vp, C.POINTER(Query), u64p]),
        "hedap_server_poll": (st, [vp, C.c_uint64, C.c_int, C.POINTER(C.c_int), pp, C.c_size_t,
                                   C.POINTER(C.c_size_t), dp, C.POINTER(C.c_uint32)]),
        "hedap_server_resume": (st, [vp]),
        "hedap_server_wait": (st, [vp, C.c_uint64, C.c_double]),
        "hedap_server_cancel": (st, [vp, C.c_uint64]),
        "hedap_server_inject": (st, [vp, C.c_uint32, C.c_uint32]),
        "hedap_server_merges": (st, [vp, u64p]),
        "hedap_server_set_table": (st, [vp, C.POINTER(SelectEntry), C.c_size_t]),
        "hedap_invsqrt_graph_create": (st, [vp, vp, C.POINTER(InvSqrtCfg), pp]),
        "hedap_graph_run": (st, [vp, vp, pp]),
        "hedap_invsqrt_mixed_graph_create": (st, [vp, pp, C.POINTER(InvSqrtCfg), C.c_size_t, pp]),
        "hedap_graph_run_many": (st, [vp, pp, C.c_size_t, pp]),
        "hedap_graph_kernels": (st, [vp, u64p]),
        "hedap_graph_destroy": (None, [vp]),
        "hedap_server_estimate": (st, [vp, C.c_uint32, C.c_uint32, C.c_int, u64p]),
        "hedap_server_stats": (st, [vp, dp, dp, dp, u64p]),
        "hedap_server_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _check(rc):
    if rc != 0:
        raise HedapError(rc, load().hedap_last_error().decode())


def _u64ptr(arr):
    """Pointer and on_device flag for a numpy array or a CUDA torch tensor of uint64/int64."""
    if isinstance(arr, np.ndarray):
        assert arr.dtype == np.uint64 and arr.flags.c_contiguous
        return arr.ctypes.data_as(C.POINTER(C.c_uint64)), 0
    if hasattr(arr, "data_ptr"):  # torch tensor
        assert arr.is_contiguous() and arr.element_size() == 8
        return C.cast(C.c_void_p(arr.data_ptr()), C.POINTER(C.c_uint64)), 1 if arr.is_cuda else 0
    raise TypeError("expected a numpy uint64 array or a torch tensor")


class Ciphertext:
    def __init__(self, ctx: "Context", handle: C.c_void_p):
        self.ctx = ctx
        self.h = handle

    def __del__(self):
        h = getattr(self, "h", None)
        if h and _lib is not None:
            _lib.hedap_ct_free(h)
            self.h = None

    def _info(self):
        lv, sc = C.c_int(), C.c_double()
        _check(load().hedap_ct_info(self.h, C.byref(lv), C.byref(sc)))
        return lv.value, sc.value

    @property
    def level(self) -> int:
        return self._info()[0]

    @property
    def scale(self) -> float:
        return self._info()[1]

    @property
    def batch(self) -> int:
        n = C.c_int()
        _check(load().hedap_ct_batch_size(self.h, C.byref(n)))
        return n.value

    def limbs(self) -> np.ndarray:
        out = np.empty((2, self.level + 1, self.ctx.N), dtype=np.uint64)
        p, _ = _u64ptr(out)
        _check(load().hedap_ct_export(self.ctx.h, self.h, p, out.size, 0))
        return out

    def export_to(self, dst) -> None:
        """Copy [2][level+1][N] words into dst (numpy array, host or CUDA torch tensor)."""
        p, dev = _u64ptr(dst)
        cap = dst.size if isinstance(dst, np.ndarray) else dst.numel()
        _check(load().hedap_ct_export(self.ctx.h, self.h, p, cap, dev))


class Context:
    """A CKKS context on the current CUDA device (keys generated from ``seed``)."""

    def __init__(self, log_n, q_bits, p_bits, alpha, log_scale, hw=0, seed=1, stream=None):
        L = load()
        self._qb = (C.c_uint32 * len(q_bits))(*q_bits)
        self._pb = (C.c_uint32 * len(p_bits))(*p_bits)
        prm = Params(log_n, len(q_bits), self._qb, len(p_bits), self._pb, alpha, float(log_scale), hw)
        h = C.c_void_p()
        _check(L.hedap_ctx_create(C.byref(prm), seed, C.c_void_p(stream or 0), C.byref(h)))
        self.h = h
        self.log_n, self.N = log_n, 1 << log_n
        self.n_q, self.n_p, self.alpha = len(q_bits), len(p_bits), alpha
        self.scale = 2.0 ** log_scale
        self.seed = seed

    def close(self):
        if getattr(self, "h", None):
            load().hedap_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        if _lib is not None:
            self.close()

    def _ct(self, fn, *args) -> Ciphertext:
        out = C.c_void_p()
        _check(fn(self.h, *args, C.byref(out)))
        return Ciphertext(self, out)

    # ---- parameters and keys
    def primes(self) -> np.ndarray:
        out = np.empty(self.n_q + self.n_p, dtype=np.uint64)
        _check(load().hedap_ctx_primes(self.h, out.ctypes.data_as(C.POINTER(C.c_uint64)), out.size))
        return out

    def gen_galois_key(self, g: int):
        _check(load().hedap_gen_galois_key(self.h, g))

    def galois_of_rotation(self, r: int) -> int:
        out = C.c_uint64()
        _check(load().hedap_galois_element(self.h, r, 0, C.byref(out)))
        return out.value

    def galois_of_conjugation(self) -> int:
        out = C.c_uint64()
        _check(load().hedap_galois_element(self.h, 0, 1, C.byref(out)))
        return out.value

    def key_digit(self, g: int, j: int):
        tot = self.n_q + self.n_p
        b = np.empty((tot, self.N), dtype=np.uint64)
        a = np.empty((tot, self.N), dtype=np.uint64)
        _check(load().hedap_export_key(self.h, g, j, _u64ptr(b)[0], _u64ptr(a)[0]))
        return b, a

    def sync(self):
        _check(load().hedap_sync(self.h))

    # ---- ring helpers
    def ntt(self, limbs, first_prime: int, inverse=False):
        """In-place NTT of consecutive limbs (numpy: returns a transformed copy)."""
        if isinstance(limbs, np.ndarray):
            x = np.ascontiguousarray(limbs, dtype=np.uint64).copy()
            n = x.size // self.N
            _check(load().hedap_ntt(self.h, _u64ptr(x)[0], n, first_prime, int(inverse), 0))
            return x
        p, dev = _u64ptr(limbs)
        _check(load().hedap_ntt(self.h, p, limbs.numel() // self.N, first_prime, int(inverse), dev))
        return limbs

    def ntt_tune(self, limbs=384, reps=3):
        """Autotune the NTT launch shape; returns (fwd ms per variant, inv ms per variant, chosen fwd, chosen inv)."""
        f, i = (C.c_float * 16)(), (C.c_float * 16)()
        fv, iv = C.c_int(), C.c_int()
        _check(load().hedap_ntt_tune(self.h, limbs, reps, f, i, 16, C.byref(fv), C.byref(iv)))
        n = 8
        return list(f[:n]), list(i[:n]), fv.value, iv.value

    def butterfly_rate(self) -> float:
        """Butterflies per second of a register-only loop of the NTT butterfly."""
        r = C.c_double()
        _check(load().hedap_butterfly_rate(self.h, C.byref(r)))
        return r.value

    def ntt_set_variant(self, fwd: int, inv: int):
        _check(load().hedap_ntt_set_variant(self.h, fwd, inv))

    def ntt_get_variant(self):
        """(forward, inverse) NTT launch shapes in use."""
        f, i = C.c_int(), C.c_int()
        _check(load().hedap_ntt_get_variant(self.h, C.byref(f), C.byref(i)))
        return f.value, i.value

    def ntt_set_role_variant(self, role: int, variant: int):
        _check(load().hedap_ntt_set_role_variant(self.h, role, variant))

    def ntt_get_roles(self) -> dict:
        """Launch shape of every NTT role, by role name."""
        out = {}
        for name, role in NTT_ROLES.items():
            v = C.c_int()
            _check(load().hedap_ntt_get_role_variant(self.h, role, C.byref(v)))
            out[name] = v.value
        return out

    def ntt_set_roles(self, roles: dict):
        for name, v in roles.items():
            self.ntt_set_role_variant(NTT_ROLES[name], int(v))

    def ntt_batch(self, limbs, n_limbs: int, first_prime: int, inverse=False):
        """In-place NTT of a CUDA tensor holding polynomials of n_limbs limbs each."""
        p, dev = _u64ptr(limbs)
        _check(load().hedap_ntt_batch(self.h, p, n_limbs, limbs.numel() // (n_limbs * self.N), first_prime,
                                      int(inverse), dev))
        return limbs

    # ---- key-switching steps
    def modup_coeff(self, limbs: np.ndarray, level: int) -> np.ndarray:
        x = np.ascontiguousarray(limbs, dtype=np.uint64)
        dn = -(-(level + 1) // self.alpha)
        out = np.empty((dn, level + 1 + self.n_p, self.N), dtype=np.uint64)
        _check(load().hedap_modup(self.h, _u64ptr(x)[0], level, _u64ptr(out)[0]))
        return out

    def moddown_coeff(self, limbs: np.ndarray, level: int) -> np.ndarray:
        x = np.ascontiguousarray(limbs, dtype=np.uint64)
        out = np.empty((2, level + 1, self.N), dtype=np.uint64)
        _check(load().hedap_moddown(self.h, _u64ptr(x)[0], level, _u64ptr(out)[0]))
        return out

    def key_switch(self, d: np.ndarray, level: int, galois: int) -> np.ndarray:
        x = np.ascontiguousarray(d, dtype=np.uint64)
        out = np.empty((2, level + 1, self.N), dtype=np.uint64)
        _check(load().hedap_key_switch(self.h, _u64ptr(x)[0], level, galois, _u64ptr(out)[0]))
        return out

    # ---- ciphertexts
    def encrypt(self, values, level: int, seed: int) -> Ciphertext:
        v = np.asarray(values)
        re = np.ascontiguousarray(v.real, dtype=np.float64)
        im = np.ascontiguousarray(v.imag if np.iscomplexobj(v) else np.zeros_like(re), dtype=np.float64)
        dp = C.POINTER(C.c_double)
        return self._ct(load().hedap_encrypt, re.ctypes.data_as(dp), im.ctypes.data_as(dp), len(re), level, seed)

    def decrypt(self, ct: Ciphertext) -> np.ndarray:
        n = self.N // 2
        re, im = np.empty(n), np.empty(n)
        dp = C.POINTER(C.c_double)
        _check(load().hedap_decrypt(self.h, ct.h, re.ctypes.data_as(dp), im.ctypes.data_as(dp), n))
        return re + 1j * im

    def ct_import(self, limbs, level: int, scale: float) -> Ciphertext:
        if isinstance(limbs, np.ndarray):
            limbs = np.ascontiguousarray(limbs, dtype=np.uint64)
        p, dev = _u64ptr(limbs)
        return self._ct(load().hedap_ct_import, p, level, float(scale), dev)

    def add(self, a, b):
        return self._ct(load().hedap_add, a.h, b.h)

    def sub(self, a, b):
        return self._ct(load().hedap_sub, a.h, b.h)

    def mul_relin(self, a, b):
        return self._ct(load().hedap_mul_relin, a.h, b.h)

    def mul(self, a, b):
        return self._ct(load().hedap_mul, a.h, b.h)

    def rescale(self, a):
        return self._ct(load().hedap_rescale, a.h)

    def rotate(self, a, steps: int):
        return self._ct(load().hedap_rotate, a.h, steps)

    def rotate_hoisted(self, a: Ciphertext, steps) -> list:
        st = (C.c_int64 * len(steps))(*steps)
        out = (C.c_void_p * len(steps))()
        _check(load().hedap_rotate_hoisted(self.h, a.h, st, len(steps), out))
        return [Ciphertext(self, C.c_void_p(out[i])) for i in range(len(steps))]

    def conjugate(self, a):
        return self._ct(load().hedap_conjugate, a.h)

    def mul_const(self, a, c: float, target_scale: float):
        return self._ct(load().hedap_mul_const, a.h, c, target_scale)

    def add_const(self, a, c: float):
        return self._ct(load().hedap_add_const, a.h, c)

    def mul_int(self, a, m: int):
        return self._ct(load().hedap_mul_int, a.h, m)

    def drop(self, a, level: int):
        return self._ct(load().hedap_drop_level, a.h, level)

    # ---- bootstrapping
    def bts_setup(self, K=28, r=4, deg=31, cts=3, stc=3) -> int:
        """Enable bootstrapping; returns the level of a bootstrapped ciphertext."""
        lv = C.c_int()
        _check(load().hedap_bootstrap_setup(self.h, C.byref(BtsParams(K, r, deg, cts, stc)), C.byref(lv)))
        return lv.value

    def bootstrap(self, a):
        return self._ct(load().hedap_bootstrap, a.h)

    def bootstrap_slots(self, a, log_slots: int):
        """Sparse-slot bootstrapping (2^log_slots values repeated over the N/2 slots)."""
        return self._ct(load().hedap_bootstrap_slots, a.h, log_slots)

    def bootstrap_scaled_slots(self, a, Y: int, log_slots: int):
        return self._ct(load().hedap_bootstrap_scaled_slots, a.h, Y, log_slots)

    def sub_sum(self, a, log_slots: int):
        return self._ct(load().hedap_sub_sum, a.h, log_slots)

    def bts_encapsulate(self, h: int) -> None:
        """Sparse-secret encapsulation of bootstrapping (ephemeral secret of weight h)."""
        _check(load().hedap_bootstrap_encapsulate(self.h, h))

    def encapsulation_switch(self, a, to_sparse: bool):
        return self._ct(load().hedap_encapsulation_switch, a.h, 1 if to_sparse else 0)

    def bootstrap_scaled(self, a, Y: int):
        return self._ct(load().hedap_bootstrap_scaled, a.h, Y)

    def mod_raise(self, a):
        return self._ct(load().hedap_mod_raise, a.h)

    def mul_monomial(self, a, e: int):
        return self._ct(load().hedap_mul_monomial, a.h, e)

    def linear_transform_group(self, a, groups_unused: int, inverse: bool, g: int, target: float):
        return self._ct(load().hedap_bts_linear_transform, a.h, int(inverse), g, target)

    def eval_mod(self, a):
        return self._ct(load().hedap_eval_mod, a.h)

    def encode_coeffs(self, re, im=None, scale=None) -> np.ndarray:
        re = np.ascontiguousarray(re, dtype=np.float64)
        im = np.zeros_like(re) if im is None else np.ascontiguousarray(im, dtype=np.float64)
        out = np.empty(self.N, dtype=np.int64)
        dp = C.POINTER(C.c_double)
        _check(load().hedap_encode(self.h, re.ctypes.data_as(dp), im.ctypes.data_as(dp), len(re),
                                   float(scale or self.scale), out.ctypes.data_as(C.POINTER(C.c_int64))))
        return out

    def bts_diagonal(self, inverse: bool, g: int, offset: int):
        n = self.N // 2
        re, im = np.empty(n), np.empty(n)
        dp = C.POINTER(C.c_double)
        _check(load().hedap_bts_diagonal(self.h, int(inverse), g, offset, re.ctypes.data_as(dp),
                                         im.ctypes.data_as(dp)))
        return re + 1j * im

    def with_scale(self, a, scale: float):
        b = self.drop(a, a.level)
        _check(load().hedap_set_scale(self.h, b.h, scale))
        return b

    def invsqrt(self, a, lo, hi, B, degree, iters, pre_bts=0, bts_mask=0, log_slots=0):
        cfg = InvSqrtCfg(lo, hi, B, degree, iters, pre_bts, bts_mask, log_slots)
        return self._ct(load().hedap_invsqrt, a.h, C.byref(cfg))

    def invsqrt_graph(self, example, lo, hi, B, degree, iters, pre_bts=0, bts_mask=0) -> "Graph":
        """CryptoInvSqrt captured as a CUDA graph for the example's level, batch and scale."""
        cfg = InvSqrtCfg(lo, hi, B, degree, iters, pre_bts, bts_mask)
        h = C.c_void_p()
        _check(load().hedap_invsqrt_graph_create(self.h, example.h, C.byref(cfg), C.byref(h)))
        return Graph(self, h)

    # ---- batches
    def batch_import(self, limbs, n: int, level: int, scale: float) -> Ciphertext:
        """n ciphertexts [n][2][level+1][N] (numpy array or torch tensor, host or CUDA) as one batch, one copy."""
        if isinstance(limbs, np.ndarray):
            limbs = np.ascontiguousarray(limbs, dtype=np.uint64)
        p, dev = _u64ptr(limbs)
        return self._ct(load().hedap_batch_import, p, n, level, float(scale), dev)

    def batch_export(self, b: Ciphertext, dst) -> None:
        """Copy a batch's [n][2][level+1][N] words into dst (numpy array or torch tensor, host or CUDA)."""
        p, dev = _u64ptr(dst)
        cap = dst.size if isinstance(dst, np.ndarray) else dst.numel()
        _check(load().hedap_batch_export(self.h, b.h, p, cap, dev))

    def pack(self, cts) -> Ciphertext:
        arr = (C.c_void_p * len(cts))(*[c.h for c in cts])
        return self._ct(load().hedap_batch_pack, arr, len(cts))

    def unpack(self, b: Ciphertext, k: int) -> Ciphertext:
        return self._ct(load().hedap_batch_unpack, b.h, k)

    def select(self, A, B_max, B, d_e_min, d_e_max, i_max, theta=1.0, delta=1.0, mre_target=0.0,
               level_min=0, level_max=0, seed=7):
        """Run HE-DAP provisioning (Alg. 2 + Alg. 3); returns (D, R, trace) as lists of dicts."""
        cfg = SelectCfg(A, B_max, B, d_e_min, d_e_max, i_max, theta, delta, mre_target, level_min, level_max, seed)
        cap_d = 64 * (d_e_max - d_e_min + 1) * 2
        D, R, T = (SelectEntry * cap_d)(), (SelectEntry * (64 * 3))(), (SelectTrace * (cap_d * i_max))()
        nd, nr, nt = C.c_size_t(), C.c_size_t(), C.c_size_t()
        _check(load().hedap_select(self.h, C.byref(cfg), D, len(D), C.byref(nd), R, len(R), C.byref(nr), T, len(T),
                                   C.byref(nt)))
        return ([D[i].as_dict() for i in range(nd.value)], [R[i].as_dict() for i in range(nr.value)],
                [T[i].as_dict() for i in range(nt.value)])

    def invsqrt_batch(self, cts, cfgs):
        """cfgs: list of (lo, hi, B, degree, iters, pre_bts, bts_mask), one per ciphertext."""
        n = len(cts)
        arr = (C.c_void_p * n)(*[c.h for c in cts])
        cf = (InvSqrtCfg * n)(*[InvSqrtCfg(*c) for c in cfgs])
        outs = (C.c_void_p * n)()
        _check(load().hedap_invsqrt_batch(self.h, arr, cf, n, outs))
        return [Ciphertext(self, C.c_void_p(o)) for o in outs]

    def invsqrt_many(self, cts, cfgs, level_band: int):
        """Mixed levels: groups by level band (dropping to the band's lowest level), see hedap.h."""
        n = len(cts)
        arr = (C.c_void_p * n)(*[c.h for c in cts])
        cf = (InvSqrtCfg * n)(*[InvSqrtCfg(*c) for c in cfgs])
        outs = (C.c_void_p * n)()
        _check(load().hedap_invsqrt_many(self.h, arr, cf, n, level_band, outs))
        return [Ciphertext(self, C.c_void_p(o)) for o in outs]


    def invsqrt_mixed(self, cts, cfgs):
        """Single ciphertexts at their own levels (none dropped), batched where their states meet (see
        hedap.h, hedap_invsqrt_mixed); cfgs as for invsqrt_batch (an 8th entry is log_slots)."""
        n = len(cts)
        arr = (C.c_void_p * n)(*[c.h for c in cts])
        cf = (InvSqrtCfg * n)(*[InvSqrtCfg(*c) for c in cfgs])
        outs = (C.c_void_p * n)()
        _check(load().hedap_invsqrt_mixed(self.h, arr, cf, n, outs))
        return [Ciphertext(self, C.c_void_p(o)) for o in outs]

    def invsqrt_mixed_graph(self, cts, cfgs) -> "Graph":
        """invsqrt_mixed captured as one CUDA graph for these inputs' levels and scales."""
        n = len(cts)
        arr = (C.c_void_p * n)(*[c.h for c in cts])
        cf = (InvSqrtCfg * n)(*[InvSqrtCfg(*c) for c in cfgs])
        h = C.c_void_p()
        _check(load().hedap_invsqrt_mixed_graph_create(self.h, arr, cf, n, C.byref(h)))
        g = Graph(self, h)
        g.n = n
        return g


PROFILE_CLASSES = ("ntt", "modup", "ksk_inner", "moddown", "tensor", "rescale", "automorph", "elementwise")


class Graph:
    """A captured CryptoInvSqrt (see Context.invsqrt_graph)."""

    def __init__(self, ctx: Context, handle):
        self.ctx = ctx
        self.h = handle

    def run(self, a=None, want_output=True):
        """Replay on `a` (or on the previous input); returns the result ciphertext or None."""
        out = C.c_void_p()
        _check(load().hedap_graph_run(self.h, a.h if a is not None else None,
                                      C.byref(out) if want_output else None))
        return Ciphertext(self.ctx, out) if want_output else None

    def run_many(self, cts=None, want_output=True):
        """Replay a graph of many ciphertexts (Context.invsqrt_mixed_graph) on `cts` (or the previous inputs)."""
        n = self.n
        arr = (C.c_void_p * n)(*[c.h for c in cts]) if cts is not None else None
        outs = (C.c_void_p * n)()
        _check(load().hedap_graph_run_many(self.h, arr, n, outs if want_output else None))
        return [Ciphertext(self.ctx, C.c_void_p(o)) for o in outs] if want_output else None

    @property
    def kernels(self) -> int:
        n = C.c_uint64()
        _check(load().hedap_graph_kernels(self.h, C.byref(n)))
        return n.value

    def close(self) -> None:
        if getattr(self, "h", None):
            load().hedap_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        if _lib is not None:
            self.close()


class Server:
    """Continuous-batching server for z-score / correlation queries on one context.

    Inputs are borrowed by the library until a query is done; this wrapper
    keeps references to them until then."""

    def __init__(self, ctx: Context, max_batch: int = 8, hbm_budget_bytes: int = 64 << 30, paused: bool = False,
                 admit_max: int = 0):
        self.ctx = ctx
        self._held = {}
        h = C.c_void_p()
        cfg = ServerCfg(max_batch, 1 if paused else 0, hbm_budget_bytes, admit_max)
        _check(load().hedap_server_create(ctx.h, C.byref(cfg), C.byref(h)))
        self.h = h

    def submit(self, kind: int, xs, n_records: int, cfg, ys=None, choice: int = 0) -> int:
        """Submit a query; cfg = (lo, hi, B, degree, iters, pre_bts, bts_mask); choice 1/2/3 takes
        (degree, c, iters) from the HE-DAP table (u1/u2/u3). Returns its id."""
        xa = (C.c_void_p * len(xs))(*[c.h for c in xs])
        ya = (C.c_void_p * len(ys))(*[c.h for c in ys]) if ys is not None else None
        q = Query(kind, C.cast(xa, C.POINTER(C.c_void_p)),
                  C.cast(ya, C.POINTER(C.c_void_p)) if ya is not None else None,
                  len(xs), n_records, InvSqrtCfg(*cfg), choice)
        qid = C.c_uint64()
        _check(load().hedap_server_submit(self.h, C.byref(q), C.byref(qid)))
        self._held[qid.value] = (list(xs), list(ys or []))
        return qid.value

    def poll(self, qid: int, wait: bool = True):
        """(done, results, info); results are handed over once done; info = {latency_ms, group_size}."""
        done, n, lat, gs = C.c_int(), C.c_size_t(), C.c_double(), C.c_uint32()
        try:
            _check(load().hedap_server_poll(self.h, qid, 1 if wait else 0, C.byref(done), None, 0, C.byref(n),
                                            C.byref(lat), C.byref(gs)))
        except HedapError:
            self._held.pop(qid, None)
            raise
        if not done.value:
            return False, None, None
        out = (C.c_void_p * n.value)()
        _check(load().hedap_server_poll(self.h, qid, 0, C.byref(done), out, n.value, None, None, None))
        self._held.pop(qid, None)
        return True, [Ciphertext(self.ctx, C.c_void_p(v)) for v in out], {"latency_ms": lat.value,
                                                                          "group_size": gs.value}

    def resume(self) -> None:
        _check(load().hedap_server_resume(self.h))

    def wait(self, qid: int, timeout_ms: float) -> None:
        """Block until the query is done (HedapError code -6 when timeout_ms passes first)."""
        _check(load().hedap_server_wait(self.h, qid, float(timeout_ms)))

    def cancel(self, qid: int) -> None:
        _check(load().hedap_server_cancel(self.h, qid))

    def inject(self, fault: int, count: int) -> None:
        """Host-side fault injection (FAULT_ADMISSION_OOM: the next `count` admissions fail)."""
        _check(load().hedap_server_inject(self.h, fault, count))

    def merges(self) -> int:
        n = C.c_uint64()
        _check(load().hedap_server_merges(self.h, C.byref(n)))
        return n.value

    def set_table(self, R) -> None:
        """Install HE-DAP's per-level table (list of dicts as returned by Context.select)."""
        arr = (SelectEntry * max(1, len(R)))(*[SelectEntry(e["level"], e["degree"], e["c"], e["iters"], e["mre"],
                                                           e["ms"], e["kind"]) for e in R])
        _check(load().hedap_server_set_table(self.h, arr, len(R)))

    def estimate(self, kind: int, n_ct: int, level: int) -> int:
        b = C.c_uint64()
        _check(load().hedap_server_estimate(self.h, kind, n_ct, level, C.byref(b)))
        return b.value

    def stats(self) -> dict:
        p50, p99, qps, n = C.c_double(), C.c_double(), C.c_double(), C.c_uint64()
        _check(load().hedap_server_stats(self.h, C.byref(p50), C.byref(p99), C.byref(qps), C.byref(n)))
        return {"p50_ms": p50.value, "p99_ms": p99.value, "qps": qps.value, "completed": n.value}

    def close(self) -> None:
        if getattr(self, "h", None):
            load().hedap_server_destroy(self.h)
            self.h = None
            self._held.clear()

    def __del__(self):
        if _lib is not None:
            self.close()


def profile_enable(on: bool) -> None:
    _check(load().hedap_profile_enable(int(on)))


def profile_read() -> dict:
    """{class: (timed launch groups, total ms, algorithmic bytes)} since profile_enable(True)."""
    out = {}
    for c in PROFILE_CLASSES:
        n, ms, by = C.c_uint64(), C.c_double(), C.c_double()
        _check(load().hedap_profile_read(c.encode(), C.byref(n), C.byref(ms), C.byref(by)))
        out[c] = (n.value, ms.value, by.value)
    return out


def profile_read_slots(kernel_class: str) -> float:
    """Algorithmic multiply work (32-bit multiply-pipe slots) of a class since profile_enable(True)."""
    v = C.c_double()
    _check(load().hedap_profile_read_slots(kernel_class.encode(), C.byref(v)))
    return v.value


def launch_count() -> int:
    n = C.c_uint64()
    _check(load().hedap_launch_count(C.byref(n)))
    return n.value


def getoptiter_rule(M, delta: float):
    """Alg. 2's threshold rule (host code of the library): (I 0-based or -1, MRE_delta)."""
    m = np.ascontiguousarray(M, dtype=np.float64)
    I, thr = C.c_int(), C.c_double()
    _check(load().hedap_getoptiter_rule(m.ctypes.data_as(C.POINTER(C.c_double)), len(m), delta, C.byref(I),
                                        C.byref(thr)))
    return I.value, thr.value


def select_level_rule(entries, theta: float, mre_target: float = 0.0):
    """Alg. 3's per-level rule: entries are dicts (level, degree, c, iters, mre, ms); returns (u1, u2, u3 or None)."""
    arr = (SelectEntry * len(entries))(*[SelectEntry(e["level"], e["degree"], e["c"], e["iters"], e["mre"], e["ms"], 0)
                                         for e in entries])
    u1, u2, u3, h = SelectEntry(), SelectEntry(), SelectEntry(), C.c_int()
    _check(load().hedap_select_level_rule(arr, len(entries), theta, mre_target, C.byref(u1), C.byref(u2),
                                          C.byref(u3), C.byref(h)))
    return u1.as_dict(), u2.as_dict(), (u3.as_dict() if h.value else None)
