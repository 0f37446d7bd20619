"""A small object layer over the C ABI: one context, its runs and their
states as numpy/torch arrays.  Argument marshalling only; every step of the
method runs in libns."""
from __future__ import annotations

import numpy as np

from . import _native as nat


class Solver:
    """Integrating-factor RK2 pseudospectral solver for one or more runs.

    runs: list of dicts with keys n, nu, dt and optionally force_amp,
    force_k, dealias, rot, eta with mhd = 1 for MHD runs, and ny, nz, lx,
    ly, lz for a grid of n x ny x nz points on the box of sides
    2 pi (lx, ly, lz).
    prec: "fp64" (plain form) or "fp32" (fused form; plain FP32 form when a
    run is MHD at a size without a fused kernel, uses phase shifts, or is not
    the (2 pi)^3 cube).
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

    def dims(self, run: int = 0) -> tuple:
        """Grid points (N_x, N_y, N_z) of a run."""
        r = self.runs[run]
        n = int(r["n"])
        return (n, int(r.get("ny", 0)) or n, int(r.get("nz", 0)) or n)

    def half_shape(self, run: int = 0, ncomp: int = 3) -> tuple:
        nx, ny, nz = self.dims(run)
        return (ncomp, nx, ny, nz // 2 + 1)

    def _checked(self, a, run: int, out: bool = False):
        """The buffer must hold exactly the run's half layout in complex128
        (an output buffer as it is: it is written in place)."""
        if isinstance(a, np.ndarray):
            if out and (a.dtype != np.complex128 or not a.flags["C_CONTIGUOUS"]):
                raise TypeError("output buffers are C-contiguous complex128")
            a = np.ascontiguousarray(a, dtype=np.complex128)
        elif str(getattr(a, "dtype", "")) != "torch.complex128":
            raise TypeError("state buffers are complex128")
        if tuple(a.shape) != self.half_shape(run):
            raise ValueError(f"state has shape {tuple(a.shape)}, run {run} wants {self.half_shape(run)}")
        return a

    def set_state(self, uhat, run: int = 0) -> None:
        """uhat: complex128 half layout [3][N_x][N_y][N_z/2+1] (numpy or torch)."""
        nat.ns_set_state(self.ctx, run, self._checked(uhat, run))

    def get_state(self, run: int = 0, out=None):
        if out is None:
            out = np.empty(self.half_shape(run), dtype=np.complex128)
        out = self._checked(out, run, out=True)
        nat.ns_get_state(self.ctx, run, out)
        return out

    def set_states(self, uhats, first: int = 0) -> None:
        """The velocity states of runs first, first + 1, ... in one call (one
        synchronisation for page-locked host or device buffers)."""
        nat.ns_set_states(self.ctx, first, [self._checked(u, first + i) for i, u in enumerate(uhats)])

    def energy_spectra(self, first: int = 0, count: int | None = None):
        """(E, Omega, spectra) of runs first .. first + count - 1 in one round
        trip; spectra rows are zero-padded to the widest run's shells."""
        count = len(self.runs) - first if count is None else count
        nb = max(nat.ns_run_nbins(self.runs[first + i]) for i in range(count))
        return nat.ns_energy_spectra(self.ctx, first, count, nb)

    def set_field(self, field: int, uhat, run: int = 0) -> None:
        """field 0: velocity, 1: magnetic field of an MHD run."""
        nat.ns_set_field(self.ctx, run, field, self._checked(uhat, run))

    def get_field(self, field: int, run: int = 0, out=None):
        if out is None:
            out = np.empty(self.half_shape(run), dtype=np.complex128)
        out = self._checked(out, run, out=True)
        nat.ns_get_field(self.ctx, run, field, out)
        return out

    def field_spectrum(self, field: int, run: int = 0):
        return nat.ns_field_spectrum(self.ctx, run, field, self.runs[run])

    def step(self, nsteps: int = 1) -> None:
        nat.ns_step(self.ctx, nsteps)

    def energy_spectrum(self, run: int = 0):
        return nat.ns_energy_spectrum(self.ctx, run, self.runs[run])

    def helicity(self, run: int = 0):
        return nat.ns_helicity(self.ctx, run, self.runs[run])

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

    def fft_r2c_grid(self, u, out) -> None:
        """r2c of device fields [ncomp][N_x][N_y][N_z] into [ncomp][N_x][N_y][N_z/2+1]."""
        nx, ny, nz = u.shape[-3:]
        nc = u.numel() // (nx * ny * nz)
        if tuple(out.shape[-3:]) != (nx, ny, nz // 2 + 1) or out.numel() != nc * nx * ny * (nz // 2 + 1):
            raise ValueError("output shape does not match the input grid")
        nat.ns_fft_r2c_grid(self.ctx, nx, ny, nz, nc, u, out)

    def fft_c2r_grid(self, uh, out) -> None:
        """c2r of device fields [ncomp][N_x][N_y][N_z/2+1] into [ncomp][N_x][N_y][N_z]."""
        nx, ny, nz = out.shape[-3:]
        nc = out.numel() // (nx * ny * nz)
        if tuple(uh.shape[-3:]) != (nx, ny, nz // 2 + 1) or uh.numel() != nc * nx * ny * (nz // 2 + 1):
            raise ValueError("input shape does not match the output grid")
        nat.ns_fft_c2r_grid(self.ctx, nx, ny, nz, nc, uh, out)
