"""GB300 library for MLMC with stabilised leapfrog local time-stepping.

Hot path (CUDA, sm_103a, ``csrc/``): per-sample random coefficient, coarse
apply, inner LTS substeps on the refined region, outer update, QoI and MLMC
level sums, behind the C ABI declared in ``include/lflts.h``.
``lflts`` is the ctypes binding, ``mlmc`` the host-side Alg. 1 driver.
"""
from . import lflts  # noqa: F401  (binding; loads the .so lazily)

__all__ = ["lflts"]
