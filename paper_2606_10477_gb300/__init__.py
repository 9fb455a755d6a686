"""GB300 (sm_103a) RNS-CKKS arithmetic behind the encrypted inverse square root
of HE-DAP: batched negacyclic NTT, hybrid key switching, rescale, rotation and
CryptoInvSqrt, behind the C ABI of ``include/hedap.h``.

``hedap`` is the ctypes binding; ``inputs`` holds the seeded synthetic inputs
and parameter presets.  Nothing here computes on the CPU.
"""
from . import inputs  # noqa: F401
