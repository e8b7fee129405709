"""GB300-native damped acoustic wave modelling, adjoint and FWI gradient.

Implements the hot path of Kukreja et al., "Devito: automated fast finite
difference computation" (arXiv 1608.08658): the leapfrog stencil of Listing 1,
its adjoint (Listing 2) and the adjoint-state gradient (Eq. 3), as hand-written
CUDA for sm_103a behind a C ABI (``include/wave.h``).  This package holds the
ctypes binding (``wave``), the torch-facing helpers and the seeded synthetic
input generators (``inputs``).  The CUDA library is loaded lazily on first use;
there is no CPU fallback.
"""

__all__ = ["wave", "inputs"]
