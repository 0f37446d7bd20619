"""A small object layer over the C ABI: one context, its runs and their
states as numpy/torch arrays.  Argument marshalling only; every step of the
method runs in libns."""
from __future__ import annotations

import numpy as np

from . import _native as nat


class Solver:
    """Integrating-factor RK2 pseudospectral solver for one or more runs.

    runs: list of dicts with keys n, nu, dt and optionally force_amp,
    force_k, dealias, rot, and eta with mhd = 1 for MHD runs.
    prec: "fp64" (plain form) or "fp32" (fused form; plain form when a run
    is MHD).
    """

    def __init__(self, runs, prec: str = "fp32", stream=None):
        self.runs = [dict(r) for r in runs]
        self.prec = nat.NS_FP64 if prec == "fp64" else nat.NS_FP32
        self.ctx = nat.ns_init(self.runs, self.prec, stream)

    def close(self) -> None:
        if self.ctx is not None:
            nat.ns_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def n(self, run: int = 0) -> int:
        return int(self.runs[run]["n"])

    def set_state(self, uhat, run: int = 0) -> None:
        """uhat: complex128 half layout [3][N][N][N/2+1] (numpy or torch)."""
        if isinstance(uhat, np.ndarray):
            uhat = np.ascontiguousarray(uhat, dtype=np.complex128)
        nat.ns_set_state(self.ctx, run, uhat)

    def get_state(self, run: int = 0, out=None):
        n = self.n(run)
        if out is None:
            out = np.empty((3, n, n, n // 2 + 1), dtype=np.complex128)
        nat.ns_get_state(self.ctx, run, out)
        return out

    def set_field(self, field: int, uhat, run: int = 0) -> None:
        """field 0: velocity, 1: magnetic field of an MHD run."""
        if isinstance(uhat, np.ndarray):
            uhat = np.ascontiguousarray(uhat, dtype=np.complex128)
        nat.ns_set_field(self.ctx, run, field, uhat)

    def get_field(self, field: int, run: int = 0, out=None):
        n = self.n(run)
        if out is None:
            out = np.empty((3, n, n, n // 2 + 1), dtype=np.complex128)
        nat.ns_get_field(self.ctx, run, field, out)
        return out

    def field_spectrum(self, field: int, run: int = 0):
        return nat.ns_field_spectrum(self.ctx, run, field, self.n(run))

    def step(self, nsteps: int = 1) -> None:
        nat.ns_step(self.ctx, nsteps)

    def energy_spectrum(self, run: int = 0):
        return nat.ns_energy_spectrum(self.ctx, run, self.n(run))

    def helicity(self, run: int = 0):
        return nat.ns_helicity(self.ctx, run, self.n(run))

    def series(self, run: int = 0, count: int = 4096):
        return nat.ns_series(self.ctx, run, count)

    def sync(self) -> None:
        nat.ns_sync(self.ctx)

    def fft_r2c(self, u, out) -> None:
        n = u.shape[-1]
        nat.ns_fft_r2c(self.ctx, n, u.numel() // n ** 3, u, out)

    def fft_c2r(self, uh, out) -> None:
        n = uh.shape[-2]
        nat.ns_fft_c2r(self.ctx, n, out.numel() // n ** 3, uh, out)
