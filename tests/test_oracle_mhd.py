"""Pins of the oracle's MHD nonlinear terms and step (the magnetohydrodynamic
equations of the same code, Sec. 5; Alfven units, state [u; b]).  CPU only."""
import math

import numpy as np
import pytest

import oracle
from paper_1003_4322_gb300 import inputs
from tests.spectral_ref import half_weights, helical_mode, triad_mhd


def _mhd_state(n, seed, rms_u=0.6, rms_b=0.5):
    u = inputs.random_solenoidal_state(n, 1.0, n / 3.0, rms_u, seed=seed)
    b = inputs.random_solenoidal_state(n, 1.0, n / 3.0, rms_b, seed=seed + 100)
    return np.concatenate([u, b])


def _dot(x, y):
    """sum over the full spectrum of Re(conj(x) . y) for half-layout fields."""
    w = half_weights(x.shape[1])
    return float(np.sum(w * np.real(np.conj(x) * y)))


@pytest.mark.parametrize("dealias", [0, 1])
def test_mhd_nonlinear_equals_exact_triad_sum(dealias):
    a = _mhd_state(8, 3)
    got = oracle.nonlinear(a, oracle.Params(n=8, mhd=1, dealias=dealias))
    want = triad_mhd(a, dealias)
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()


def test_mhd_ideal_invariants_are_conserved_semidiscretely():
    """With nu = eta = 0, no forcing and no rotation, the Galerkin-truncated
    system conserves the total energy, the cross helicity u.b and the
    magnetic helicity A.b (A = i k x b / k^2): N is orthogonal to each."""
    n = 12
    a = _mhd_state(n, 5)
    N = oracle.nonlinear(a, oracle.Params(n=n, mhd=1))
    u, b, Nu, Nb = a[:3], a[3:], N[:3], N[3:]
    scale = math.sqrt(_dot(a, a) * _dot(N, N))
    assert abs(_dot(u, Nu) + _dot(b, Nb)) < 1e-13 * scale      # energy
    assert abs(_dot(u, Nb) + _dot(b, Nu)) < 1e-13 * scale      # cross helicity
    k = np.fft.fftfreq(n, 1.0 / n)
    KX, KY, KZ = np.meshgrid(k, k, np.arange(n // 2 + 1), indexing="ij")
    K = np.stack([KX, KY, KZ])
    k2 = np.where(KX ** 2 + KY ** 2 + KZ ** 2 > 0, KX ** 2 + KY ** 2 + KZ ** 2, 1.0)
    A = 1j * np.cross(K, b, axis=0) / k2
    assert abs(_dot(A, Nb)) < 1e-13 * scale                   # magnetic helicity
    # and they are not trivially zero: the transfers themselves are not
    assert abs(_dot(u, Nu)) > 1e-3 * scale and abs(_dot(b, Nu)) > 1e-3 * scale


def test_force_free_field_decays_exactly():
    """u = 0 and b = ABC (k = 1): j = b, so j x b = 0 and u x b = 0; b decays
    as exp(-eta t) at any dt and u stays zero."""
    n, eta, dt, steps = 16, 0.02, 0.05, 6
    a = np.concatenate([np.zeros_like(inputs.abc_state(n)), inputs.abc_state(n)])
    b = oracle.step(a, oracle.Params(n=n, nu=0.01, eta=eta, dt=dt, mhd=1), steps)
    assert np.abs(b[:3]).max() < 1e-15
    assert np.abs(b[3:] - a[3:] * math.exp(-eta * dt * steps)).max() < 1e-14


@pytest.mark.parametrize("k", [(0, 0, 2), (1, 2, 3), (-2, 1, 1)])
@pytest.mark.parametrize("s", [1, -1])
def test_alfven_wave_is_exact(k, s):
    """Mean field B0 z and one helical mode in both u and b: u x w, u x b'
    and j' x b' vanish, and what is left is the linear Alfven coupling
    d u/dt = i kz B0 b, d b/dt = i kz B0 u, i.e. the Elsasser fields
    z+- = u +- b turn at +-kz B0.  With nu = eta, IF-Heun multiplies z+- by
    exp(-nu k^2 dt)(1 + z + z^2/2), z = +-i kz B0 dt, per step exactly."""
    n, nu, dt, B0, steps = 16, 0.01, 0.01, 1.7, 15
    h = helical_mode(n, k, s, amp=1.0)
    al, be = 0.3, -0.1 + 0.2j
    a = np.concatenate([al * h, be * h])
    a[5, 0, 0, 0] = B0
    out = oracle.step(a, oracle.Params(n=n, nu=nu, eta=nu, dt=dt, mhd=1), steps)
    kk = np.linalg.norm(k)
    E = math.exp(-nu * kk ** 2 * dt)
    g = [E * (1 + z + z * z / 2) for z in (1j * k[2] * B0 * dt, -1j * k[2] * B0 * dt)]
    zp, zm = (al + be) * g[0] ** steps, (al - be) * g[1] ** steps
    assert np.abs(out[:3] - 0.5 * (zp + zm) * h).max() < 1e-14
    want_b = 0.5 * (zp - zm) * h
    want_b[2, 0, 0, 0] = B0
    assert np.abs(out[3:] - want_b).max() < 1e-14


def test_mhd_step_is_second_order():
    a0 = _mhd_state(8, 9, 1.0, 0.8)
    res = [oracle.step(a0, oracle.Params(n=8, nu=0.05, eta=0.03, dt=0.2 / m, mhd=1), m)
           for m in (10, 20, 40)]
    d1 = math.sqrt(_dot(res[0] - res[1], res[0] - res[1]))
    d2 = math.sqrt(_dot(res[1] - res[2], res[1] - res[2]))
    assert 3.6 < d1 / d2 < 4.4
