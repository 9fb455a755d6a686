"""hedap_rescale_noalloc: the rescale variant for callers that cannot allocate
device memory during an operation (its scratch is a library-held device array).

It must give exactly what hedap_rescale gives, on consecutive calls that reuse
the shared scratch, and refuse sizes beyond the scratch maximum.  This file is
collected last so that a stop-at-first-failure run has already run the rest.
"""
import ctypes

import numpy as np
import pytest

from paper_2606_10477_gb300 import hedap, inputs

pytestmark = pytest.mark.gpu


def _noalloc(ctx, din, level, dout):
    rc = hedap.load().hedap_rescale_noalloc(ctx.h, ctypes.cast(ctypes.c_void_p(din.data_ptr()),
                                                               ctypes.POINTER(ctypes.c_uint64)),
                                            level, ctypes.cast(ctypes.c_void_p(dout.data_ptr()),
                                                               ctypes.POINTER(ctypes.c_uint64)))
    return rc


@pytest.mark.parametrize("name", ["n13", "n16"])
def test_rescale_noalloc_matches_rescale_on_consecutive_calls(name):
    torch = pytest.importorskip("torch")
    p = inputs.PRESETS[name]
    ctx = hedap.Context(p["log_n"], p["q_bits"], p["p_bits"], p["alpha"], p["log_scale"], p["hw"], 5)
    primes = ctx.primes()
    for call, level in enumerate((ctx.n_q - 1, ctx.n_q - 3)):
        limbs = inputs.random_ciphertext_limbs(200 + call, primes, level, ctx.N)
        expect = ctx.rescale(ctx.ct_import(limbs, level, ctx.scale)).limbs()
        din = torch.from_numpy(limbs.view(np.int64)).cuda()
        dout = torch.empty((2, level, ctx.N), dtype=torch.int64, device="cuda")
        assert _noalloc(ctx, din, level, dout) == 0, hedap.load().hedap_last_error().decode()
        torch.cuda.synchronize()
        got = dout.cpu().numpy().view(np.uint64)
        assert np.array_equal(got, expect), f"call {call}: {np.count_nonzero(got != expect)} residues differ"


def test_rescale_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    # N = 2^16 and level 33: (2 + 2*33) * 2^16 words > 4 Mi words of scratch
    ctx = hedap.Context(16, [33] * 34, [60], 8, 30, 0, 1)
    din = torch.zeros((2, 34, ctx.N), dtype=torch.int64, device="cuda")
    dout = torch.zeros((2, 33, ctx.N), dtype=torch.int64, device="cuda")
    rc = _noalloc(ctx, din, 33, dout)
    assert rc == -1
    assert "exceeds the scratch maximum" in hedap.load().hedap_last_error().decode()
