"""GB300-native analytic-pulse gather + relativistic Boris push.

Method: Weichman et al., "Analytic pulse technique for computational
electromagnetics" (arXiv:2307.04843).  Each macroparticle evaluates the
closed-form laser field E1/B1 at its own position and time, adds the field
gathered from a static grid (E = E1 + E2, Sec. 2), and takes a relativistic
Boris step; hand-written sm_103a CUDA kernels behind the C ABI in
include/ap.h, reached from Python through the ctypes binding in ``_lib``.

Submodules are imported lazily so that the seeded input generators in
``workloads`` can be used without the compiled library.
"""
__all__ = ["workloads"]
