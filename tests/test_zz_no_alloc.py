"""hedap_rescale_noalloc: the rescale variant for callers that cannot allocate
device memory during an operation (a serving loop admitted against a fixed HBM
budget, a host framework whose allocator owns device memory, code that must not
let a cudaMalloc/cudaFree synchronise the device).  Its scratch is a
library-held device array.

It must give exactly what hedap_rescale and the oracle's rescale give, on
consecutive calls that reuse the shared scratch; it must not move the device
memory pool (nor, once its kernels are loaded, the device's free memory); it
must refuse sizes beyond the scratch maximum and overlapping buffers.  This
file is collected last so that a stop-at-first-failure run has already run the
rest.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2606_10477_gb300 import hedap, inputs

pytestmark = pytest.mark.gpu


def _u64p(t):
    return ctypes.cast(ctypes.c_void_p(t.data_ptr()), ctypes.POINTER(ctypes.c_uint64))


def _noalloc(ctx, din, level, dout):
    return hedap.load().hedap_rescale_noalloc(ctx.h, _u64p(din), level, _u64p(dout))


def _device_memory():
    """(reserved, used) bytes of the current device's default memory pool (where the library's
    stream-ordered allocations come from) and the device's free bytes, read through the driver."""
    cu = ctypes.CDLL("libcuda.so.1")
    dev = ctypes.c_int()
    assert cu.cuCtxGetDevice(ctypes.byref(dev)) == 0
    pool = ctypes.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    vals = []
    for attr in (5, 7):  # CU_MEMPOOL_ATTR_RESERVED_MEM_CURRENT, CU_MEMPOOL_ATTR_USED_MEM_CURRENT
        v = ctypes.c_uint64()
        assert cu.cuMemPoolGetAttribute(pool, attr, ctypes.byref(v)) == 0
        vals.append(v.value)
    free, total = ctypes.c_size_t(), ctypes.c_size_t()
    assert cu.cuMemGetInfo_v2(ctypes.byref(free), ctypes.byref(total)) == 0
    return vals[0], vals[1], free.value


@pytest.mark.parametrize("name", ["n13", "n16"])
def test_rescale_noalloc_matches_rescale_and_oracle_without_allocating(name):
    torch = pytest.importorskip("torch")
    p = inputs.PRESETS[name]
    args = (p["log_n"], p["q_bits"], p["p_bits"], p["alpha"], p["log_scale"], p["hw"], 5)
    ctx, orc = hedap.Context(*args), oracle.Context(*args)
    primes = ctx.primes()
    for call, level in enumerate((ctx.n_q - 1, ctx.n_q - 3)):
        limbs = inputs.random_ciphertext_limbs(200 + call, primes, level, ctx.N)
        expect = ctx.rescale(ctx.ct_import(limbs, level, ctx.scale)).limbs()
        ref = orc.rescale(orc.ct_import(limbs, level, orc.scale)).limbs()
        assert np.array_equal(expect, ref), "hedap_rescale differs from the oracle"
        din = torch.from_numpy(limbs.view(np.int64)).cuda()
        dout = torch.empty((2, level, ctx.N), dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        ctx.sync()
        before = _device_memory()
        assert _noalloc(ctx, din, level, dout) == 0, hedap.load().hedap_last_error().decode()
        ctx.sync()
        after = _device_memory()
        assert before[:2] == after[:2], f"call {call}: the memory pool moved {before[:2]} -> {after[:2]}"
        if call > 0:  # the first call may load its kernels' code; later ones take nothing
            assert before[2] == after[2], f"call {call}: free device memory {before[2]} -> {after[2]}"
        got = dout.cpu().numpy().view(np.uint64)
        assert np.array_equal(got, expect), f"call {call}: {np.count_nonzero(got != expect)} residues differ"


def test_rescale_noalloc_rejects_sizes_beyond_its_scratch_and_overlap():
    torch = pytest.importorskip("torch")
    # N = 2^16 and level 33: (2 + 2*33) * 2^16 words > 4 Mi words of scratch
    ctx = hedap.Context(16, [33] * 34, [60], 8, 30, 0, 1)
    din = torch.zeros((2, 34, ctx.N), dtype=torch.int64, device="cuda")
    dout = torch.zeros((2, 33, ctx.N), dtype=torch.int64, device="cuda")
    assert _noalloc(ctx, din, 33, dout) == -1
    assert "exceeds the scratch maximum" in hedap.load().hedap_last_error().decode()
    # an output that overlaps the input is refused before any work is queued
    assert _noalloc(ctx, din, 4, din[0, 2]) == -1
    assert "overlaps" in hedap.load().hedap_last_error().decode()
