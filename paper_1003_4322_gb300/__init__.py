"""GB300-native hot path of the pseudospectral incompressible Navier-Stokes
solver of Mininni, Rosenberg, Reddy and Pouquet (Sec. 2, Eqs. 1-2): 3D
r2c/c2r FFTs of the (2 pi)^3 periodic box, the dealiased nonlinear term
u x w, and the integrating-factor RK2 update with 2/3-rule truncation,
Leray projection and exact viscous factor; with the extensions of Sec. 5
(rotation, MHD, boxes of other aspect ratios on N_x x N_y x N_z grids),
helicity and the spherical and phase-shift dealiasing variants.

The compute path is libns.so (hand-written CUDA for sm_103a behind the C ABI
of include/ns.h); ``_native`` is its ctypes binding and ``solver`` a small
convenience layer over it.  Importing this package does not load the library;
``load()`` does, and raises when it is missing.
"""
from . import inputs  # noqa: F401  (seeded synthetic inputs; no method arithmetic)


def load():
    """Load libns.so; raises ImportError if it has not been built."""
    from . import _native
    return _native.load()


def __getattr__(name):
    if name.startswith("ns_") or name.startswith("NS_") or name in ("NsError", "SYMBOLS"):
        from . import _native
        return getattr(_native, name)
    if name in ("Solver",):
        from . import solver
        return getattr(solver, name)
    raise AttributeError(name)
