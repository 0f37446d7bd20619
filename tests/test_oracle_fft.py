"""Pins of the oracle's 3D transforms (Sec. 2: r2c into the (N/2+1) x N x N
half array, c2r back).  Each test checks the oracle against something other
than itself: the O(N^6) definition, closed forms, Parseval, numpy's FFT."""
import math

import numpy as np
import pytest

import oracle
from paper_1003_4322_gb300 import inputs
from tests.spectral_ref import brute_dft3


@pytest.mark.parametrize("n", [6, 8, 12])
def test_r2c_matches_brute_force_dft(n):
    u = inputs.random_real(n, 1, 10 + n)[0]
    ref = brute_dft3(u, -1)[:, :, : n // 2 + 1]
    got = oracle.fft3_r2c(u)
    assert np.abs(got - ref).max() < 1e-11 * n ** 3


@pytest.mark.parametrize("n", [6, 8])
def test_c2r_matches_brute_force_inverse(n):
    a = inputs.random_hermitian_half(n, 1, 3)[0]
    from tests.spectral_ref import half_to_full
    full = half_to_full(a)
    ref = brute_dft3(full, +1)
    assert np.abs(ref.imag).max() < 1e-10       # Hermitian input, real output
    got = oracle.fft3_c2r(a)
    assert np.abs(got - ref.real).max() < 1e-11 * n ** 3


@pytest.mark.parametrize("n", [16, 24, 32, 18])
def test_r2c_matches_numpy(n):
    u = inputs.random_real(n, 2, n)
    ref = np.fft.rfftn(u, axes=(1, 2, 3))
    got = oracle.fft3_r2c(u)
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-13


@pytest.mark.parametrize("n", [8, 12, 32])
def test_round_trip_and_parseval(n):
    u = inputs.random_real(n, 1, 7)[0]
    X = oracle.fft3_r2c(u)
    back = oracle.fft3_c2r(X)
    assert np.abs(back - n ** 3 * u).max() < 1e-12 * n ** 3
    w = np.full(n // 2 + 1, 2.0)
    w[0] = w[n // 2] = 1.0
    lhs = np.sum(u * u)
    rhs = np.sum(w * np.abs(X) ** 2) / n ** 3
    assert abs(lhs - rhs) < 1e-12 * lhs


def test_single_mode_closed_form():
    n = 16
    g = 2 * math.pi * np.arange(n) / n
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    # cos(2x + 3y - z) = (e^{ik.x} + e^{-ik.x})/2 with k = (2, 3, -1): the half
    # layout holds -k = (-2, -3, 1) at kz = 1 with value N^3/2.
    u = np.cos(2 * X + 3 * Y - Z) + 0.25 * np.sin(5 * Z)
    A = oracle.fft3_r2c(u)
    expect = np.zeros_like(A)
    expect[(-2) % n, (-3) % n, 1] = n ** 3 / 2
    expect[0, 0, 5] = 0.25 * n ** 3 / 2j
    assert np.abs(A - expect).max() < 1e-10
    # inverse of a single stored coefficient: a e^{ik.x} + conj(a) e^{-ik.x}
    B = np.zeros_like(A)
    B[1, 2, 3] = 0.5 - 0.25j
    v = oracle.fft3_c2r(B)
    ref = 2 * (0.5 * np.cos(X + 2 * Y + 3 * Z) + 0.25 * np.sin(X + 2 * Y + 3 * Z))
    assert np.abs(v - ref).max() < 1e-13


def test_nyquist_plane_taken_as_given():
    n = 8
    a = np.zeros((n, n, n // 2 + 1), dtype=np.complex128)
    a[0, 0, n // 2] = 1.0          # cos(4z) sampled: (-1)^z, self-conjugate
    v = oracle.fft3_c2r(a)
    z = np.arange(n)
    assert np.abs(v - (-1.0) ** z[None, None, :]).max() < 1e-14
