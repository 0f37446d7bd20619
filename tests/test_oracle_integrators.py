"""The oracle's comparison integrators (the paper names no time integrator,
Sec. 3; integrating-factor Heun is the reading the solver uses): the same
IF-Heun through both entry points, exact linear behaviour on a single
solenoidal mode (whose nonlinear term vanishes), second-order convergence to
the Galerkin ODE solution, and the order of the inviscid energy drift that
tells the two integrating-factor rules apart."""
import ctypes
import math

import numpy as np
import pytest

import oracle
from paper_1003_4322_gb300 import inputs
from tests.spectral_ref import rel_l2
from tests.test_oracle_solver import _galerkin_rhs_factory


def _single_mode(n):
    a = np.zeros((3, n, n, n // 2 + 1), dtype=np.complex128)
    # k = (1, 2, 2) with amplitude along (2, -1, 0)/sqrt5, normal to k
    a[0, 1, 2, 2] = 0.4 * 2 / math.sqrt(5)
    a[1, 1, 2, 2] = -0.4 / math.sqrt(5)
    return a


def test_if_heun_is_the_same_through_both_entry_points():
    n = 12
    p = oracle.Params(n=n, nu=0.02, dt=2e-3, force_amp=0.5, force_k=2)
    a0 = inputs.turbulence_state(n, 5)
    want = oracle.step(a0, p, 3)
    v = a0.copy()
    cp = p.c()
    assert oracle.lib().or_step_with(ctypes.byref(cp), 0, v.ctypes.data_as(ctypes.c_void_p), 3) == 0
    assert np.array_equal(v, want)


def test_unknown_integrator_is_refused():
    n = 8
    p = oracle.Params(n=n, nu=0.02, dt=1e-3)
    v = np.zeros((3, n, n, n // 2 + 1), dtype=np.complex128)
    cp = p.c()
    for bad in (-1, 3):
        assert oracle.lib().or_step_with(ctypes.byref(cp), bad, v.ctypes.data_as(ctypes.c_void_p), 1) != 0
    with pytest.raises(KeyError):
        oracle.step(v, p, 1, integrator="euler")


def test_single_mode_linear_behaviour():
    n, nu, dt, steps = 16, 0.03, 0.02, 7
    a = _single_mode(n)
    z = nu * 9 * dt                       # nu |k|^2 dt, |k|^2 = 9
    mid = oracle.step(a, oracle.Params(n=n, nu=nu, dt=dt), steps, integrator="if-midpoint")
    assert np.abs(mid - a * math.exp(-z * steps)).max() < 1e-16
    rk2 = oracle.step(a, oracle.Params(n=n, nu=nu, dt=dt), steps, integrator="rk2")
    assert np.abs(rk2 - a * (1 - z + z * z / 2) ** steps).max() < 4e-16   # a few ulps of 0.36
    # and rk2 is not exact: its amplification differs from exp(-z) at O(z^3)
    assert np.abs(rk2 - a * math.exp(-z * steps)).max() > 1e-8


@pytest.mark.parametrize("integrator", ["if-midpoint", "rk2"])
def test_second_order_convergence_to_the_galerkin_ode(integrator):
    scipy_integrate = pytest.importorskip("scipy.integrate")
    n, nu, T = 8, 0.05, 0.2
    a0 = inputs.random_solenoidal_state(n, 1.0, 3.5, 1.5, seed=21)
    sol = scipy_integrate.solve_ivp(_galerkin_rhs_factory(n, nu), (0.0, T),
                                    a0.ravel().view(np.float64), method="DOP853",
                                    rtol=1e-12, atol=1e-14)
    exact = sol.y[:, -1].view(np.complex128).reshape(a0.shape)
    errs = []
    for steps in (10, 20, 40):
        b = oracle.step(a0, oracle.Params(n=n, nu=nu, dt=T / steps), steps, integrator=integrator)
        errs.append(rel_l2(b, exact))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.6 < r2 < 4.4, errs


def _weights(n):
    w = np.full(n // 2 + 1, 2.0)
    w[0] = w[n // 2] = 1.0
    return w


def test_inviscid_energy_change_of_each_rule_is_its_exact_identity():
    # With nu = 0 and no forcing, Re<b, N(b)> = 0 for every b, so one step
    # changes sum |a|^2 (full spectrum) by exactly
    #   IF-Heun:     (dt^2/4) |N(a) - N(a1)|^2          >= 0,  a1 = a + dt N(a)
    #   IF-midpoint: dt^2 Re<N(a_h) - N(a), N(a_h)>,          a_h = a + dt/2 N(a)
    # (exact algebra, no truncation error): a dropped stage, a wrong weight
    # or a full-step factor at the midpoint breaks them.
    n, dt = 16, 0.01
    p = oracle.Params(n=n, nu=0.0, dt=dt)
    a = inputs.turbulence_state(n, 31, rms=1.0)
    w = _weights(n)

    def dot(x, y):
        return float(np.sum(w * (x * np.conj(y)).real))

    Na = oracle.nonlinear(a, p)
    heun = oracle.step(a, p, 1)
    a1 = a + dt * Na
    want = dt * dt / 4 * dot(Na - oracle.nonlinear(a1, p), Na - oracle.nonlinear(a1, p))
    got = dot(heun, heun) - dot(a, a)
    assert want > 0 and abs(got - want) < 1e-9 * want + 1e-15 * dot(a, a)
    mid = oracle.step(a, p, 1, integrator="if-midpoint")
    ah = a + dt / 2 * Na
    Nh = oracle.nonlinear(ah, p)
    want = dt * dt * dot(Nh - Na, Nh)
    got = dot(mid, mid) - dot(a, a)
    assert abs(got - want) < 1e-9 * abs(want) + 1e-15 * dot(a, a), (got, want)
