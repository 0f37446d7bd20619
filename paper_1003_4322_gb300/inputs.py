"""Seeded synthetic inputs for the pseudospectral Navier-Stokes hot path.

This module builds initial conditions and test fields only.  It holds none of
the method's arithmetic (no transform, nonlinear term, projection, dealiasing
step, time stepping or diagnostic): every field is written down from its
closed-form Fourier coefficients or drawn from a counter-based generator, so
that the FP64 CPU oracle and the CUDA path can be fed the very same array.

Conventions (shared by both sides through the data only):

* grid x_j = 2*pi*j/N on the (2*pi)^3 periodic box (Sec. 2, Eqs. 1-2);
* a field is stored as its normalised Fourier coefficients a(k), so that
  u(x) = sum_k a(k) exp(i k.x), in the r2c half layout
  ``[3][N][N][N//2+1]`` complex128, index ``[c][kx mod N][ky mod N][kz]``
  with kz in [0, N/2] (the half storage of Sec. 2, Fig. 1);
* the kz = 0 and kz = N/2 planes hold both k and -k, with a(-k) = conj(a(k));
* on a grid of N_x x N_y x N_z points and a box of sides 2*pi*l_i (the boxes
  of aspect ratio other than one of Sec. 5) the layout is
  ``[3][N_x][N_y][N_z//2+1]`` and index m along axis i stands for the
  wavenumber m / l_i.

Counter-based generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a pure function of
(seed, counter).  The counter of draw ``d`` of wavevector ``k`` is
``1 + 3*mode_id(k) + d`` with an N-independent ``mode_id``, so one seed gives
the same low-wavenumber field at every grid size.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

_MASK64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


def splitmix64(seed: int, counter: int) -> int:
    """SplitMix64 output number ``counter`` of the stream started at ``seed``."""
    z = (seed + _GOLDEN * counter) & _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def uniform(seed: int, ident: int, draw: int) -> float:
    """Uniform in [0, 1): the top 53 bits of SplitMix64 times 2**-53."""
    return (splitmix64(seed, 1 + 3 * ident + draw) >> 11) * (1.0 / (1 << 53))


def mode_id(kx: int, ky: int, kz: int) -> int:
    """Grid-size independent identifier of a wavevector with |k_i| < 512."""
    return ((kx + 512) * 1024 + (ky + 512)) * 1024 + (kz + 512)


def half_shape(n: int, ncomp: int = 3) -> tuple:
    return (ncomp, n, n, n // 2 + 1)


class _Spectrum:
    """Accumulates the full-space coefficient list of a real vector field
    (n: N of the cube, or the grid (N_x, N_y, N_z))."""

    def __init__(self, n):
        self.dims = (n, n, n) if isinstance(n, int) else tuple(n)
        self.terms: dict = {}

    def add_real_term(self, c: int, k: tuple, a: complex) -> None:
        """Add a*exp(i k.x) + conj(a)*exp(-i k.x) to component c."""
        kx, ky, kz = k
        for kk, v in (((kx, ky, kz), a), ((-kx, -ky, -kz), np.conj(a))):
            key = (c,) + kk
            self.terms[key] = self.terms.get(key, 0.0) + v

    def sum_sq(self) -> float:
        return float(sum(abs(v) ** 2 for v in self.terms.values()))

    def to_half(self, scale: float = 1.0) -> np.ndarray:
        nx, ny, nz = self.dims
        out = np.zeros((3, nx, ny, nz // 2 + 1), dtype=np.complex128)
        for (c, kx, ky, kz), v in self.terms.items():
            if kz < 0:
                continue  # its partner -k (kz > 0) carries the same information
            out[c, kx % nx, ky % ny, kz] += scale * v
        return out


def abc_state(n: int, A: float = 1.0, B: float = 1.0, C: float = 1.0,
              k: int = 1) -> np.ndarray:
    """Arnold-Beltrami-Childress flow
    u = (A sin kz + C cos ky, B sin kx + A cos kz, C sin ky + B cos kx),
    whose vorticity is k*u (a Beltrami field, u x w = 0)."""
    s = _Spectrum(n)
    sin, cos = -0.5j, 0.5  # sin t = (-i/2) e^{it} + c.c.; cos t = (1/2) e^{it} + c.c.
    s.add_real_term(0, (0, 0, k), A * sin)
    s.add_real_term(0, (0, k, 0), C * cos)
    s.add_real_term(1, (k, 0, 0), B * sin)
    s.add_real_term(1, (0, 0, k), A * cos)
    s.add_real_term(2, (0, k, 0), C * sin)
    s.add_real_term(2, (k, 0, 0), B * cos)
    return s.to_half()


def taylor_green_state(n: int) -> np.ndarray:
    """Taylor-Green vortex u = (sin x cos y cos z, -cos x sin y cos z, 0)."""
    s = _Spectrum(n)
    # sin x cos y cos z = sum over sx,sy,sz = +-1 of (sx/(8i)) e^{i(sx x+sy y+sz z)};
    # each real term below adds one (k, -k) pair, so sz = +1 covers all eight.
    for sx in (-1, 1):
        for sy in (-1, 1):
            s.add_real_term(0, (sx, sy, 1), sx / 8j)
            s.add_real_term(1, (sx, sy, 1), -sy / 8j)
    return s.to_half()


def _in_box(k: tuple, n: int, dealias: int) -> bool:
    """Modes the generator may populate: strictly inside the 2/3-rule cube
    (and sphere, for dealias=1), or the sphere 9|k|^2 < 2 n^2 without the
    Nyquist index (dealias=2), so that the field is representable."""
    kx, ky, kz = k
    if dealias == 2:
        return 2 * max(abs(kx), abs(ky), abs(kz)) < n and 9 * (kx * kx + ky * ky + kz * kz) < 2 * n * n
    if 3 * max(abs(kx), abs(ky), abs(kz)) >= n:
        return False
    if dealias == 1 and 9 * (kx * kx + ky * ky + kz * kz) >= n * n:
        return False
    return True


def random_solenoidal_spectrum(n: int, lo: float, hi: float, rms: float,
                               seed: int, dealias: int = 0) -> _Spectrum:
    """Random divergence-free field with per-mode amplitude |k|^-2 on the
    shells lo <= |k| <= hi (shell spectrum E(K) ~ K^-2), random phases and a
    random split between the two transverse directions, scaled so that the
    per-component rms velocity sqrt(2E/3) equals ``rms``."""
    s = _Spectrum(n)
    kmax = int(math.floor(hi))
    for kx in range(-kmax, kmax + 1):
        for ky in range(-kmax, kmax + 1):
            for kz in range(0, kmax + 1):
                # half space: kz > 0, or kz == 0 with (ky > 0 or (ky == 0 and kx > 0))
                if kz == 0 and not (ky > 0 or (ky == 0 and kx > 0)):
                    continue
                kk = kx * kx + ky * ky + kz * kz
                kmag = math.sqrt(kk)
                if kmag < lo or kmag > hi or not _in_box((kx, ky, kz), n, dealias):
                    continue
                kv = np.array([kx, ky, kz], dtype=np.float64)
                zhat = np.array([0.0, 0.0, 1.0])
                e1 = np.cross(kv, zhat)
                if np.linalg.norm(e1) == 0.0:
                    e1 = np.cross(kv, np.array([1.0, 0.0, 0.0]))
                e1 /= np.linalg.norm(e1)
                e2 = np.cross(kv / kmag, e1)
                mid = mode_id(kx, ky, kz)
                r1, r2, r3 = (uniform(seed, mid, d) for d in range(3))
                amp = kmag ** -2
                vec = amp * (e1 * np.exp(2j * math.pi * r1) * math.cos(2 * math.pi * r3)
                             + e2 * np.exp(2j * math.pi * r2) * math.sin(2 * math.pi * r3))
                for c in range(3):
                    s.add_real_term(c, (kx, ky, kz), vec[c])
    e_now = 0.5 * s.sum_sq()
    e_target = 1.5 * rms * rms
    s.scale = math.sqrt(e_target / e_now) if e_now > 0 else 0.0
    return s


def _in_grid(m: tuple, dims: tuple, dealias: int) -> bool:
    """Index vectors the grid generator may populate: inside the 2/3 rule of
    every axis, 3 |m_i| < N_i (and the ellipsoid sum_i (3 m_i / N_i)^2 < 1,
    for dealias=1), or the ellipsoid sum_i (3 m_i / N_i)^2 < 2 without the
    Nyquist index (dealias=2); the ellipsoid in exact rationals."""
    s = sum(Fraction(3 * abs(mi), ni) ** 2 for mi, ni in zip(m, dims))
    if dealias == 2:
        return all(2 * abs(mi) < ni for mi, ni in zip(m, dims)) and s < 2
    if not all(3 * abs(mi) < ni for mi, ni in zip(m, dims)):
        return False
    return not (dealias == 1 and s >= 1)


def random_solenoidal_grid(dims: tuple, box: tuple, lo: float, hi: float, rms: float,
                           seed: int, dealias: int = 0) -> np.ndarray:
    """The random solenoidal field of ``random_solenoidal_spectrum`` on an
    N_x x N_y x N_z grid of the box of sides 2*pi*l_i: index vector m stands
    for k = m / l, per-mode amplitude |k|^-2 on lo <= |k| <= hi, the same
    draws per index vector (mode_id of m), per-component rms ``rms``.
    Returns the half layout [3][N_x][N_y][N_z//2+1]."""
    dims = tuple(int(d) for d in dims)
    box = tuple(float(b) for b in box)
    s = _Spectrum(dims)
    lim = [int(math.floor(hi * b)) for b in box]
    for mx in range(-lim[0], lim[0] + 1):
        for my in range(-lim[1], lim[1] + 1):
            for mz in range(0, lim[2] + 1):
                if mz == 0 and not (my > 0 or (my == 0 and mx > 0)):
                    continue
                if not _in_grid((mx, my, mz), dims, dealias):
                    continue
                kv = np.array([mx / box[0], my / box[1], mz / box[2]])
                kmag = float(np.linalg.norm(kv))
                if kmag < lo or kmag > hi:
                    continue
                e1 = np.cross(kv, np.array([0.0, 0.0, 1.0]))
                if np.linalg.norm(e1) == 0.0:
                    e1 = np.cross(kv, np.array([1.0, 0.0, 0.0]))
                e1 /= np.linalg.norm(e1)
                e2 = np.cross(kv / kmag, e1)
                mid = mode_id(mx, my, mz)
                r1, r2, r3 = (uniform(seed, mid, d) for d in range(3))
                vec = kmag ** -2 * (e1 * np.exp(2j * math.pi * r1) * math.cos(2 * math.pi * r3)
                                    + e2 * np.exp(2j * math.pi * r2) * math.sin(2 * math.pi * r3))
                for c in range(3):
                    s.add_real_term(c, (mx, my, mz), vec[c])
    e_now = 0.5 * s.sum_sq()
    scale = math.sqrt(1.5 * rms * rms / e_now) if e_now > 0 else 0.0
    return s.to_half(scale)


def random_real_grid(dims: tuple, ncomp: int, seed: int) -> np.ndarray:
    """Gaussian real fields, shape [ncomp][N_x][N_y][N_z] (z fastest)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((ncomp,) + tuple(dims))


def random_hermitian_half_grid(dims: tuple, ncomp: int, seed: int) -> np.ndarray:
    """Random half-layout array [ncomp][N_x][N_y][N_z/2+1] whose kz = 0 and
    kz = N_z/2 planes satisfy a(-k) = conj(a(k))."""
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    nh = nz // 2 + 1
    a = rng.standard_normal((ncomp, nx, ny, nh)) + 1j * rng.standard_normal((ncomp, nx, ny, nh))
    negx, negy = (-np.arange(nx)) % nx, (-np.arange(ny)) % ny
    for p in (0, nz // 2):
        plane = a[:, :, :, p]
        partner = np.conj(plane[:, negx][:, :, negy])
        a[:, :, :, p] = 0.5 * (plane + partner)
    return a


def random_solenoidal_state(n: int, lo: float, hi: float, rms: float,
                            seed: int, dealias: int = 0) -> np.ndarray:
    s = random_solenoidal_spectrum(n, lo, hi, rms, seed, dealias)
    return s.to_half(s.scale)


def config1_state(n: int = 32, seed: int = 1) -> np.ndarray:
    """ABC (A=B=C=1, k=1) plus a random solenoidal perturbation on
    2 <= |k| <= 4 with per-component rms 0.1."""
    return abc_state(n) + random_solenoidal_state(n, 2.0, 4.0, 0.1, seed)


def turbulence_state(n: int, seed: int, rms: float = 1.0,
                     dealias: int = 0) -> np.ndarray:
    """Seeded solenoidal start with spectrum K^-2 on 1 <= |k| <= 4."""
    return random_solenoidal_state(n, 1.0, 4.0, rms, seed, dealias)


def ensemble_nu(r: int, seed: int = 4999) -> float:
    """Viscosity of ensemble member r: 5e-3 + 1.5e-2 * U(seed, r)."""
    return 5e-3 + 1.5e-2 * uniform(seed, r, 0)


def random_real(n: int, ncomp: int, seed: int) -> np.ndarray:
    """Gaussian real fields, shape [ncomp][n][n][n] (z fastest)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((ncomp, n, n, n))


def random_hermitian_half(n: int, ncomp: int, seed: int) -> np.ndarray:
    """Random half-layout array whose kz = 0 and kz = N/2 planes satisfy
    a(-k) = conj(a(k)), i.e. the r2c image of some real field."""
    rng = np.random.default_rng(seed)
    nh = n // 2 + 1
    a = rng.standard_normal((ncomp, n, n, nh)) + 1j * rng.standard_normal((ncomp, n, n, nh))
    neg = (-np.arange(n)) % n
    for p in (0, n // 2):
        plane = a[:, :, :, p]
        partner = np.conj(plane[:, neg][:, :, neg])
        a[:, :, :, p] = 0.5 * (plane + partner)
    return a


def subsample_stride(n: int, m: int) -> int:
    """Stride of the m^3 sub-lattice of an n^3 grid (every n/m-th point)."""
    if n % m:
        raise ValueError("sub-lattice size must divide the grid size")
    return n // m
