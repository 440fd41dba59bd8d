"""GB300-native periodic kernel-independent FMM (Yan & Shelley, Algorithm 2).

The compute path is the CUDA library ``_build/libpkifmm.so`` (C ABI in
``include/pkifmm.h``); this package only marshals arguments to it.  Importing
the package does not load the library; the first call does, and fails loudly
if it is missing.
"""

LAPLACE, STOKES = 0, 1
LAPLACE_FIELD, STOKES_PRESSURE = 2, 3  # targets get (potential, gradient) / (velocity, pressure)
FP64, MIXED = 0, 1
FAR_L2L, FAR_DIRECT = 0, 1


def __getattr__(name):
    if name.startswith("pkifmm_") or name in ("PeriodicKIFMM", "load_library", "PKIFMMError"):
        from . import _binding
        return getattr(_binding, name)
    raise AttributeError(name)
