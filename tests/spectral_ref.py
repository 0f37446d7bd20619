"""Independent references used to pin the oracle: brute-force sums written
from the definitions (O(N^6) DFT, the triad convolution of the nonlinear
term), half-layout <-> full-spectrum bookkeeping and the error metric.

Grids may have N_x x N_y x N_z points and the box sides 2 pi l_i (the boxes
of aspect ratio other than one of Sec. 5): index m along axis i stands for
the wavenumber m / l_i; the dealiasing rules hold in grid indices per axis."""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np


def wavenumbers(n: int) -> np.ndarray:
    """Signed wavenumber of each full index (index n/2 -> -n/2)."""
    i = np.arange(n)
    return np.where(2 * i < n, i, i - n)


def brute_dft3(u: np.ndarray, sign: int = -1) -> np.ndarray:
    """X(k) = sum_x u(x) exp(sign i k.x) for every k of the N_x x N_y x N_z
    grid, by one dense phase matrix (the definition, O(N^6))."""
    nx, ny, nz = u.shape
    X, Y, Z = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1).astype(np.float64)
    scaled = pos / np.array([nx, ny, nz], dtype=np.float64)
    phase = np.exp(sign * 2j * math.pi * (pos @ scaled.T))  # k and x share index sets
    return (phase @ u.ravel().astype(np.complex128)).reshape(nx, ny, nz)


def half_to_full(a: np.ndarray) -> np.ndarray:
    """Complete a half-layout array [..][N_x][N_y][N_z/2+1] (N_z even) to the
    full spectrum with a(-k) = conj(a(k))."""
    nx, ny, nzh = a.shape[-3:]
    nz = 2 * (nzh - 1)
    full = np.zeros(a.shape[:-1] + (nz,), dtype=np.complex128)
    full[..., :nzh] = a
    negx, negy = (-np.arange(nx)) % nx, (-np.arange(ny)) % ny
    for z in range(nzh, nz):
        b = a[..., nz - z]
        full[..., z] = np.conj(b[..., negx, :][..., :, negy])
    return full


def keep(k: np.ndarray, n, dealias: int = 0) -> np.ndarray:
    """2/3-rule mask of signed grid indices k (rows): cube 3 |k_i| < N_i,
    the ellipsoid sum_i (3 k_i / N_i)^2 < 1 in addition (dealias=1); dealias=2:
    the ellipsoid sum_i (3 k_i / N_i)^2 < 2 without the Nyquist index.  n is
    N (cube) or (N_x, N_y, N_z); the ellipsoid is tested in exact rationals."""
    dims = (n, n, n) if np.isscalar(n) else tuple(n)
    k = np.asarray(k)
    m = np.abs(k)
    out = np.empty(k.shape[0], dtype=bool)
    for r in range(k.shape[0]):
        s = sum(Fraction(3 * int(m[r, i]), dims[i]) ** 2 for i in range(3))
        if dealias == 2:
            out[r] = all(2 * m[r, i] < dims[i] for i in range(3)) and s < 2
            continue
        ok = all(3 * m[r, i] < dims[i] for i in range(3))
        if dealias == 1:
            ok = ok and s < 1
        out[r] = ok
    return out


def kept_modes(n, dealias: int = 0):
    """All kept signed index vectors of the full spectrum, as an (M, 3) int
    array (n: N or (N_x, N_y, N_z))."""
    dims = (n, n, n) if np.isscalar(n) else tuple(n)
    KX, KY, KZ = np.meshgrid(*(wavenumbers(d) for d in dims), indexing="ij")
    K = np.stack([KX.ravel(), KY.ravel(), KZ.ravel()], axis=1)
    if dealias == 0:   # the plain cube rule, vectorised
        return K[np.all(3 * np.abs(K) < np.array(dims), axis=1)]
    return K[keep(K, dims, dealias)]


def _dims(a_half: np.ndarray) -> tuple:
    nx, ny, nzh = a_half.shape[-3:]
    return (nx, ny, 2 * (nzh - 1))


def full_coeffs(a_half: np.ndarray, K: np.ndarray) -> np.ndarray:
    """Coefficients (M, 3) of a half-layout vector field at index vectors K."""
    nx, ny, nz = _dims(a_half)
    full = half_to_full(a_half)
    return full[:, K[:, 0] % nx, K[:, 1] % ny, K[:, 2] % nz].T


def triad_nonlinear(a_half: np.ndarray, dealias: int = 0, l=(1.0, 1.0, 1.0)) -> np.ndarray:
    """N(k) = P(k) sum_{p+q=k; p,q,k kept} a(p) x (i q x a(q)) for every kept
    k, written into a half-layout array (no forcing).  Exact convolution:
    no transform, hence no aliasing.  On a box of sides 2 pi l_i the
    wavevector of index m is m / l (the convolution runs over indices)."""
    dims = _dims(a_half)
    K = kept_modes(dims, dealias)
    Kf = K.astype(np.float64) / np.array(l, dtype=np.float64)
    A = full_coeffs(a_half, K)                       # (M, 3)
    W = 1j * np.cross(Kf, A)                         # vorticity coefficients i q x a(q)
    M = len(K)
    off = max(dims)
    span = 3 * off
    lut = -np.ones((span, span, span), dtype=np.int64)
    lut[K[:, 0] + off, K[:, 1] + off, K[:, 2] + off] = np.arange(M)
    out = np.zeros((M, 3), dtype=np.complex128)
    for i in range(M):                               # p = K[i]
        s = K[i] + K                                 # p + q for all q
        tgt = lut[s[:, 0] + off, s[:, 1] + off, s[:, 2] + off]
        ok = tgt >= 0
        contrib = np.cross(np.broadcast_to(A[i], (M, 3))[ok], W[ok])
        np.add.at(out, tgt[ok], contrib)
    k2 = np.sum(Kf * Kf, axis=1)
    kv = np.sum(Kf * out, axis=1)
    nz = k2 > 0
    out[nz] -= Kf[nz] * (kv[nz] / k2[nz])[:, None]
    out[~nz] = 0
    return _to_half(out, K, a_half)


def half_weights(n: int) -> np.ndarray:
    """Multiplicity weights of the kz planes 0..N_z/2 (n = N_z)."""
    w = np.full(n // 2 + 1, 2.0)
    w[0] = 1.0
    w[n // 2] = 1.0
    return w


def energy_half(a: np.ndarray) -> float:
    return float(0.5 * np.sum(half_weights(_dims(a)[2]) * np.abs(a) ** 2))


def rel_l2(test: np.ndarray, ref: np.ndarray) -> float:
    w = half_weights(_dims(ref)[2])
    num = np.sum(w * np.abs(test - ref) ** 2)
    den = np.sum(w * np.abs(ref) ** 2)
    return math.sqrt(num / den)


def helical_mode(n, k, s, amp=0.3):
    """Half-layout state with one helical mode at wavevector k (kz > 0): the
    eigenvector of the curl symbol i k x with eigenvalue s |k|, found by
    numpy's eig, so that w = s |k| u and u x w vanishes."""
    kv = np.array(k, dtype=float)
    cross = np.array([[0.0, -kv[2], kv[1]], [kv[2], 0.0, -kv[0]], [-kv[1], kv[0], 0.0]])
    w, V = np.linalg.eig(1j * cross)
    h = V[:, np.argmin(abs(w - s * np.linalg.norm(kv)))]
    h = h / np.linalg.norm(h)
    a = np.zeros((3, n, n, n // 2 + 1), dtype=np.complex128)
    a[:, k[0] % n, k[1] % n, k[2]] = amp * h
    return a


def _triad_cross(A, B, K, n):
    """sum_{p+q=k; p,q,k kept} A(p) x B(q) for every kept k (rows of K)."""
    M = len(K)
    off = n
    lut = -np.ones((3 * n, 3 * n, 3 * n), dtype=np.int64)
    lut[K[:, 0] + off, K[:, 1] + off, K[:, 2] + off] = np.arange(M)
    out = np.zeros((M, 3), dtype=np.complex128)
    for i in range(M):
        s = K[i] + K
        tgt = lut[s[:, 0] + off, s[:, 1] + off, s[:, 2] + off]
        ok = tgt >= 0
        np.add.at(out, tgt[ok], np.cross(np.broadcast_to(A[i], (M, 3))[ok], B[ok]))
    return out


def _to_half(out, K, like):
    nx, ny, _ = _dims(like)
    res = np.zeros_like(like)
    sel = K[:, 2] >= 0
    for c in range(3):
        res[c, K[sel, 0] % nx, K[sel, 1] % ny, K[sel, 2]] = out[sel, c]
    return res


def triad_mhd(a_half: np.ndarray, dealias: int = 0):
    """Exact convolutions of the MHD nonlinear terms of a six-component
    half-layout state [u; b] (Alfven units, j = i k x b):
    N_u(k) = P(k) sum_{p+q=k} [u(p) x (i q x u(q)) + (i p x b(p)) x b(q)],
    N_b(k) = i k x sum_{p+q=k} u(p) x b(q);  no transform, no aliasing."""
    n = a_half.shape[1]
    K = kept_modes(n, dealias)
    Kf = K.astype(np.float64)
    U = full_coeffs(a_half[:3], K)
    B = full_coeffs(a_half[3:], K)
    W = 1j * np.cross(Kf, U)
    J = 1j * np.cross(Kf, B)
    nu = _triad_cross(U, W, K, n) + _triad_cross(J, B, K, n)
    k2 = np.sum(Kf * Kf, axis=1)
    kv = np.sum(Kf * nu, axis=1)
    nz = k2 > 0
    nu[nz] -= Kf[nz] * (kv[nz] / k2[nz])[:, None]
    nu[~nz] = 0
    nb = 1j * np.cross(Kf, _triad_cross(U, B, K, n))
    return np.concatenate([_to_half(nu, K, a_half[:3]), _to_half(nb, K, a_half[3:])])


def _shell_of_half(nx: int, ny: int, nz: int):
    """Shell index round-half-up(|k|) and the cube-rule kept mask of every
    half-layout mode, (N_x, N_y, N_z/2+1) arrays."""
    kx = wavenumbers(nx)[:, None, None].astype(np.float64)
    ky = wavenumbers(ny)[None, :, None].astype(np.float64)
    kz = np.arange(nz // 2 + 1, dtype=np.float64)[None, None, :]
    shell = np.floor(np.sqrt(kx * kx + ky * ky + kz * kz) + 0.5).astype(np.int64)
    keep = (3 * np.abs(kx) < nx) & (3 * np.abs(ky) < ny) & (3 * kz < nz)
    return shell, keep


def shell_error_ratios(test: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """Per-shell error bound of an FP32 state against its FP64 reference:
    for every shell K (round-half-up |k|) with kept modes,
        err_K / sqrt(E_K + (n_K / n) E),
    where err_K^2 and E_K are the weighted sums of |test - ref|^2 and |ref|^2
    over the shell, E the sum over all modes, and n_K / n the shell's share of
    the kept modes (multiplicity-weighted).  A bound tol on every ratio admits
    the two errors FP32 arithmetic makes -- rounding proportional to each
    mode's own amplitude, and transform noise spread evenly over the modes --
    but not an error confined to a few shells, which the global relative L2
    distance misses when those shells hold little energy."""
    nx, ny, nz = _dims(ref)
    shell, keep = _shell_of_half(nx, ny, nz)
    w = np.broadcast_to(half_weights(nz)[None, None, :], shell.shape)
    d2 = (w * np.sum(np.abs(test - ref) ** 2, axis=0))[keep]
    r2 = (w * np.sum(np.abs(ref) ** 2, axis=0))[keep]
    s = shell[keep]
    nb = int(s.max()) + 1
    err = np.bincount(s, weights=d2, minlength=nb)
    ek = np.bincount(s, weights=r2, minlength=nb)
    nk = np.bincount(s, weights=w[keep], minlength=nb)
    has = nk > 0
    return np.sqrt(err[has] / (ek[has] + nk[has] / nk.sum() * ek.sum()))


def shell_error_ratios_device(got, ref, planes: int = 32):
    """shell_error_ratios of two device half-layout states (torch complex
    tensors [3][N_x][N_y][N_z/2+1]), accumulated in FP64 over slabs of x
    planes, so that 1024^3 states need no host copy."""
    import torch
    nx, ny, nzh = ref.shape[-3:]
    nz = 2 * (nzh - 1)
    dev = ref.device
    ky = torch.as_tensor(wavenumbers(ny), dtype=torch.float64, device=dev)[None, :, None]
    kz = torch.arange(nzh, dtype=torch.float64, device=dev)[None, None, :]
    wz = torch.as_tensor(half_weights(nz), dtype=torch.float64, device=dev)[None, None, :]
    kxs = torch.as_tensor(wavenumbers(nx), dtype=torch.float64, device=dev)
    nb = int(math.floor(math.sqrt(3) * (nx // 2) + 0.5)) + 2
    err = torch.zeros(nb, dtype=torch.float64, device=dev)
    ek = torch.zeros_like(err)
    nk = torch.zeros_like(err)
    for x0 in range(0, nx, planes):
        kx = kxs[x0:x0 + planes][:, None, None]
        k2 = kx * kx + ky * ky + kz * kz
        shell = torch.floor(torch.sqrt(k2) + 0.5).long()
        keep = (3 * kx.abs() < nx) & (3 * ky.abs() < ny) & (3 * kz < nz)
        w = wz.expand(shell.shape)
        d2 = torch.zeros(shell.shape, dtype=torch.float64, device=dev)
        r2 = torch.zeros_like(d2)
        for c in range(ref.shape[0]):
            d2 += (got[c, x0:x0 + planes].to(torch.complex128)
                   - ref[c, x0:x0 + planes].to(torch.complex128)).abs().square()
            r2 += ref[c, x0:x0 + planes].to(torch.complex128).abs().square()
        s = shell[keep]
        err += torch.bincount(s, weights=(w * d2)[keep], minlength=nb)[:nb]
        ek += torch.bincount(s, weights=(w * r2)[keep], minlength=nb)[:nb]
        nk += torch.bincount(s, weights=w[keep], minlength=nb)[:nb]
    has = nk > 0
    r = torch.sqrt(err[has] / (ek[has] + nk[has] / nk.sum() * ek.sum()))
    return r.cpu().numpy()
