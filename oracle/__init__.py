"""FP64 CPU oracle of the pseudospectral Navier-Stokes hot path (Sec. 2,
Eqs. 1-2), loaded through ctypes from ``ns_oracle.c``.

TEST INFRASTRUCTURE, NOT PRODUCT CODE: only the test suite, the smoke check
of the package entry file and the benchmark's CPU-baseline / reference leg may
import this module.  The CUDA path never imports, links or executes it, and it
never imports the CUDA path.  It shares nothing with the CUDA path; inputs
reach both sides from ``paper_1003_4322_gb300.inputs`` as plain arrays.

Arrays use the half layout ``[3][N][N][N//2+1]`` complex128 for spectral
vector fields (normalised coefficients, u(x) = sum_k a(k) e^{ik.x}) and
``[ncomp][N][N][N]`` float64 for fields on the grid; on a grid of
N_x x N_y x N_z points (``Params.ny``, ``Params.nz``) and a box of sides
2 pi l_i (``Params.lx``, ``ly``, ``lz``; the boxes of aspect ratio other than
one of Sec. 5) they are ``[3][N_x][N_y][N_z//2+1]`` and
``[ncomp][N_x][N_y][N_z]``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ns_oracle.c")
_SO = os.path.join(_HERE, "libns_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP loops over lines/modes)."""
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class _Params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("nu", ctypes.c_double),
                ("dt", ctypes.c_double), ("force_amp", ctypes.c_double),
                ("force_k", ctypes.c_int), ("dealias", ctypes.c_int),
                ("rot", ctypes.c_double), ("eta", ctypes.c_double),
                ("mhd", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double),
                ("lz", ctypes.c_double)]


@dataclass
class Params:
    n: int
    nu: float = 0.0
    dt: float = 0.0
    force_amp: float = 0.0
    force_k: int = 0
    dealias: int = 0
    rot: float = 0.0
    eta: float = 0.0
    mhd: int = 0
    ny: int = 0        # grid points along y (0: n)
    nz: int = 0        # grid points along z (0: n)
    lx: float = 0.0    # box side along x in units of 2 pi (0: 1)
    ly: float = 0.0
    lz: float = 0.0

    def c(self) -> _Params:
        return _Params(self.n, self.nu, self.dt, self.force_amp,
                       self.force_k, self.dealias, self.rot, self.eta, self.mhd,
                       self.ny, self.nz, self.lx, self.ly, self.lz)

    def ncomp(self) -> int:
        return 6 if self.mhd else 3

    def dims(self) -> tuple:
        """Grid points (N_x, N_y, N_z)."""
        return (self.n, self.ny or self.n, self.nz or self.n)

    def half_shape(self, ncomp: int = 3) -> tuple:
        nx, ny, nz = self.dims()
        return (ncomp, nx, ny, nz // 2 + 1)


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.c_void_p
        L.or_set_threads.argtypes = [ctypes.c_int]
        I = ctypes.c_int
        PP = ctypes.POINTER(_Params)
        L.or_fft3_r2c.argtypes = [I, I, P, P]
        L.or_fft3_c2r.argtypes = [I, I, P, P]
        L.or_fft3_r2c_grid.argtypes = [I, I, I, I, P, P]
        L.or_fft3_c2r_grid.argtypes = [I, I, I, I, P, P]
        L.or_project.argtypes = [I, I, P]
        L.or_project_p.argtypes = [PP, P]
        L.or_curl.argtypes = [I, P, P]
        L.or_curl_p.argtypes = [PP, P, P]
        L.or_nbins_p.argtypes = [PP]
        L.or_diagnostics_p.argtypes = [PP, P, P, P, P, I]
        L.or_helicity_p.argtypes = [PP, P, P, P, I]
        L.or_forcing.argtypes = [ctypes.POINTER(_Params), P]
        L.or_nonlinear.argtypes = [ctypes.POINTER(_Params), P, P]
        L.or_step.argtypes = [ctypes.POINTER(_Params), P, ctypes.c_int]
        L.or_step_with.argtypes = [ctypes.POINTER(_Params), ctypes.c_int, P, ctypes.c_int]
        L.or_nbins.argtypes = [ctypes.c_int]
        L.or_diagnostics.argtypes = [ctypes.c_int, P, P, P, P, ctypes.c_int]
        L.or_helicity.argtypes = [ctypes.c_int, P, P, P, ctypes.c_int]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def set_threads(nthreads: int) -> int:
    """Set the OpenMP thread count; returns the count in effect."""
    return lib().or_set_threads(int(nthreads))


def fft3_r2c(u: np.ndarray) -> np.ndarray:
    """Unnormalised forward r2c of real fields [ncomp][N_x][N_y][N_z] (or
    [N_x][N_y][N_z]) into the half layout [ncomp][N_x][N_y][N_z/2+1]."""
    squeeze = u.ndim == 3
    u = np.ascontiguousarray(u.reshape((1,) + u.shape) if squeeze else u,
                             dtype=np.float64)
    nc, nx, ny, nz = u.shape
    out = np.empty((nc, nx, ny, nz // 2 + 1), dtype=np.complex128)
    _check(lib().or_fft3_r2c_grid(nx, ny, nz, nc, _ptr(u), _ptr(out)), "r2c")
    return out[0] if squeeze else out


def fft3_c2r(a: np.ndarray) -> np.ndarray:
    """Unnormalised inverse c2r of half-layout arrays [ncomp][N_x][N_y][N_z/2+1]
    (N_z even, so N_z = 2 (last extent - 1))."""
    squeeze = a.ndim == 3
    a = np.ascontiguousarray(a.reshape((1,) + a.shape) if squeeze else a,
                             dtype=np.complex128)
    nc, nx, ny, nzh = a.shape
    nz = 2 * (nzh - 1)
    out = np.empty((nc, nx, ny, nz), dtype=np.float64)
    _check(lib().or_fft3_c2r_grid(nx, ny, nz, nc, _ptr(a), _ptr(out)), "c2r")
    return out[0] if squeeze else out


def project(a: np.ndarray, dealias: int = 0, p: Params | None = None) -> np.ndarray:
    """Pi then P(k) v = v - k (k.v)/|k|^2 of a half-layout vector field (on
    the grid and box of p, with p's dealiasing rule, when p is given)."""
    v = np.array(a, dtype=np.complex128, order="C", copy=True)
    if p is None:
        _check(lib().or_project(v.shape[1], dealias, _ptr(v)), "project")
    else:
        cp = p.c()
        _check(lib().or_project_p(ctypes.byref(cp), _ptr(v)), "project")
    return v


def curl(a: np.ndarray, p: Params | None = None) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.complex128)
    w = np.empty_like(a)
    if p is None:
        _check(lib().or_curl(a.shape[1], _ptr(a), _ptr(w)), "curl")
    else:
        cp = p.c()
        _check(lib().or_curl_p(ctypes.byref(cp), _ptr(a), _ptr(w)), "curl")
    return w


def forcing(p: Params) -> np.ndarray:
    fh = np.empty(p.half_shape(), dtype=np.complex128)
    cp = p.c()
    _check(lib().or_forcing(ctypes.byref(cp), _ptr(fh)), "forcing")
    return fh


def _check_shape(a: np.ndarray, p: Params) -> None:
    want = p.half_shape(p.ncomp())
    if a.shape != want:
        raise ValueError(f"state has shape {a.shape}, parameters want {want}")


def nonlinear(a: np.ndarray, p: Params) -> np.ndarray:
    """N(a) = P Pi [FFT(u x w)/N^3 + 2 rot (a_y, -a_x, 0)] + f_hat; with
    p.mhd the six-component [N_u; N_b] of the state [u; b]."""
    a = np.ascontiguousarray(a, dtype=np.complex128)
    _check_shape(a, p)
    out = np.empty_like(a)
    cp = p.c()
    _check(lib().or_nonlinear(ctypes.byref(cp), _ptr(a), _ptr(out)), "nonlinear")
    return out


INTEGRATORS = {"if-heun": 0, "if-midpoint": 1, "rk2": 2}


def step(a: np.ndarray, p: Params, nsteps: int, integrator: str = "if-heun") -> np.ndarray:
    """nsteps RK2 steps; returns the new state (a copy).  integrator:
    "if-heun" (integrating-factor Heun, the reading of the unnamed integrator
    that the solver uses), or for comparison only "if-midpoint"
    (integrating factor with the midpoint rule) and "rk2" (Heun with the
    viscous term explicit)."""
    v = np.array(a, dtype=np.complex128, order="C", copy=True)
    _check_shape(v, p)
    cp = p.c()
    if integrator == "if-heun":
        _check(lib().or_step(ctypes.byref(cp), _ptr(v), int(nsteps)), "step")
    else:
        _check(lib().or_step_with(ctypes.byref(cp), INTEGRATORS[integrator], _ptr(v), int(nsteps)),
               "step")
    return v


def nbins(n) -> int:
    """Number of shells of the cube N^3 (n an int) or of the grid and box of
    n (a Params)."""
    if isinstance(n, Params):
        cp = n.c()
        return lib().or_nbins_p(ctypes.byref(cp))
    return lib().or_nbins(n)


def diagnostics(a: np.ndarray, p: Params | None = None):
    """(E, Omega, E(K)) with K = round-half-up(|k| / k_min), K = 0..nbins-1
    (k_min = 1 on the (2 pi)^3 box)."""
    a = np.ascontiguousarray(a, dtype=np.complex128)
    e = ctypes.c_double()
    om = ctypes.c_double()
    if p is None:
        n = a.shape[1]
        nb = nbins(n)
        spec = np.empty(nb, dtype=np.float64)
        _check(lib().or_diagnostics(n, _ptr(a), ctypes.byref(e), ctypes.byref(om),
                                    _ptr(spec), nb), "diagnostics")
    else:
        nb = nbins(p)
        spec = np.empty(nb, dtype=np.float64)
        cp = p.c()
        _check(lib().or_diagnostics_p(ctypes.byref(cp), _ptr(a), ctypes.byref(e),
                                      ctypes.byref(om), _ptr(spec), nb), "diagnostics")
    return e.value, om.value, spec


def helicity(a: np.ndarray, p: Params | None = None):
    """(H, H(K)): helicity 1/2 <u . w> and its shell spectrum."""
    a = np.ascontiguousarray(a, dtype=np.complex128)
    h = ctypes.c_double()
    if p is None:
        n = a.shape[1]
        nb = nbins(n)
        spec = np.empty(nb, dtype=np.float64)
        _check(lib().or_helicity(n, _ptr(a), ctypes.byref(h), _ptr(spec), nb), "helicity")
    else:
        nb = nbins(p)
        spec = np.empty(nb, dtype=np.float64)
        cp = p.c()
        _check(lib().or_helicity_p(ctypes.byref(cp), _ptr(a), ctypes.byref(h), _ptr(spec), nb),
               "helicity")
    return h.value, spec


def rel_l2(test: np.ndarray, ref: np.ndarray) -> float:
    """Relative L2 distance of two half-layout spectral arrays, each mode
    weighted by its multiplicity in the full spectrum (2 for 0 < kz < N_z/2;
    N_z is even, so the last kz plane is the Nyquist plane)."""
    w = np.full(ref.shape[-1], 2.0)
    w[0] = 1.0
    w[-1] = 1.0
    num = np.sum(w * np.abs(test - ref) ** 2)
    den = np.sum(w * np.abs(ref) ** 2)
    return math.sqrt(num / den) if den > 0 else math.sqrt(num)
