"""GB300-native haemoglobin estimation via Haar decomposition (Jones et al., Section 2).

The estimator itself lives in ``libhb.so`` (CUDA, sm_103a) behind the C ABI of
``include/hb.h``; ``binding`` is its ctypes wrapper and ``synth`` the seeded
synthetic workload generator.  Build the library with ``build.build()``.
"""
from .binding import Context, HbError, Server, load, strerror  # noqa: F401
