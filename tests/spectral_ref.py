"""Independent references used to pin the oracle: brute-force sums written
from the definitions (O(N^6) DFT, the triad convolution of the nonlinear
term), half-layout <-> full-spectrum bookkeeping and the error metric."""
from __future__ import annotations

import math

import numpy as np


def wavenumbers(n: int) -> np.ndarray:
    """Signed wavenumber of each full index (index n/2 -> -n/2)."""
    i = np.arange(n)
    return np.where(2 * i < n, i, i - n)


def brute_dft3(u: np.ndarray, sign: int = -1) -> np.ndarray:
    """X(k) = sum_x u(x) exp(sign i k.x) for every k of the n^3 grid, by one
    dense phase matrix (the definition, O(N^6))."""
    n = u.shape[0]
    g = np.arange(n)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1).astype(np.float64)
    phase = np.exp(sign * 2j * math.pi * (pos @ pos.T) / n)  # k and x share index sets
    return (phase @ u.ravel().astype(np.complex128)).reshape(n, n, n)


def half_to_full(a: np.ndarray) -> np.ndarray:
    """Complete a half-layout array [..][n][n][n/2+1] to the full n^3
    spectrum with a(-k) = conj(a(k))."""
    n = a.shape[-3]
    nh = n // 2 + 1
    full = np.zeros(a.shape[:-1] + (n,), dtype=np.complex128)
    full[..., :nh] = a
    neg = (-np.arange(n)) % n
    for z in range(nh, n):
        b = a[..., n - z]
        full[..., z] = np.conj(b[..., neg, :][..., :, neg])
    return full


def keep(k: np.ndarray, n: int, dealias: int = 0) -> np.ndarray:
    """2/3-rule mask: cube 3 max|k_i| < n, sphere 9|k|^2 < n^2 in addition;
    dealias=2: the sphere 9|k|^2 < 2 n^2 without the Nyquist index."""
    m = np.max(np.abs(k), axis=-1)
    if dealias == 2:
        return (2 * m < n) & (9 * np.sum(k * k, axis=-1) < 2 * n * n)
    ok = 3 * m < n
    if dealias == 1:
        ok &= 9 * np.sum(k * k, axis=-1) < n * n
    return ok


def kept_modes(n: int, dealias: int = 0):
    """All kept wavevectors of the full spectrum, as an (M, 3) int array."""
    kk = wavenumbers(n)
    KX, KY, KZ = np.meshgrid(kk, kk, kk, indexing="ij")
    K = np.stack([KX.ravel(), KY.ravel(), KZ.ravel()], axis=1)
    return K[keep(K, n, dealias)]


def full_coeffs(a_half: np.ndarray, K: np.ndarray) -> np.ndarray:
    """Coefficients (M, 3) of a half-layout vector field at wavevectors K."""
    n = a_half.shape[1]
    full = half_to_full(a_half)
    return full[:, K[:, 0] % n, K[:, 1] % n, K[:, 2] % n].T


def triad_nonlinear(a_half: np.ndarray, dealias: int = 0) -> np.ndarray:
    """N(k) = P(k) sum_{p+q=k; p,q,k kept} a(p) x (i q x a(q)) for every kept
    k, written into a half-layout array (no forcing).  Exact convolution:
    no transform, hence no aliasing."""
    n = a_half.shape[1]
    K = kept_modes(n, dealias)
    A = full_coeffs(a_half, K)                       # (M, 3)
    W = 1j * np.cross(K.astype(np.float64), A)       # vorticity coefficients i q x a(q)
    M = len(K)
    off = n
    lut = -np.ones((3 * n, 3 * n, 3 * n), dtype=np.int64)
    lut[K[:, 0] + off, K[:, 1] + off, K[:, 2] + off] = np.arange(M)
    out = np.zeros((M, 3), dtype=np.complex128)
    for i in range(M):                               # p = K[i]
        s = K[i] + K                                 # p + q for all q
        tgt = lut[s[:, 0] + off, s[:, 1] + off, s[:, 2] + off]
        ok = tgt >= 0
        contrib = np.cross(np.broadcast_to(A[i], (M, 3))[ok], W[ok])
        np.add.at(out, tgt[ok], contrib)
    Kf = K.astype(np.float64)
    k2 = np.sum(Kf * Kf, axis=1)
    kv = np.sum(Kf * out, axis=1)
    nz = k2 > 0
    out[nz] -= Kf[nz] * (kv[nz] / k2[nz])[:, None]
    out[~nz] = 0
    res = np.zeros_like(a_half)
    sel = K[:, 2] >= 0
    for c in range(3):
        res[c, K[sel, 0] % n, K[sel, 1] % n, K[sel, 2]] = out[sel, c]
    return res


def half_weights(n: int) -> np.ndarray:
    w = np.full(n // 2 + 1, 2.0)
    w[0] = 1.0
    w[n // 2] = 1.0
    return w


def energy_half(a: np.ndarray) -> float:
    return float(0.5 * np.sum(half_weights(a.shape[1]) * np.abs(a) ** 2))


def rel_l2(test: np.ndarray, ref: np.ndarray) -> float:
    w = half_weights(ref.shape[1])
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
    n = like.shape[1]
    res = np.zeros_like(like)
    sel = K[:, 2] >= 0
    for c in range(3):
        res[c, K[sel, 0] % n, K[sel, 1] % n, K[sel, 2]] = out[sel, c]
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
