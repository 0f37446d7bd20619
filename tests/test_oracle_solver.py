"""Pins of the oracle's nonlinear term, projection, forcing, time step and
diagnostics (Sec. 2, Eqs. 1-2; reductions for global quantities and spectra,
Sec. 3).  None of these re-types the oracle: they use the exact triad
convolution, exact solutions, conservation laws, convergence orders and a
high-order ODE integrator on the Galerkin system."""
import math

import numpy as np
import pytest

import oracle
from paper_1003_4322_gb300 import inputs
from tests.spectral_ref import (energy_half, half_to_full, helical_mode, kept_modes, rel_l2,
                                triad_nonlinear, wavenumbers)


def _kvec(n):
    k = wavenumbers(n).astype(np.float64)
    kz = np.arange(n // 2 + 1, dtype=np.float64)
    return np.meshgrid(k, k, kz, indexing="ij")


# ---------------------------------------------------------------- nonlinear term

@pytest.mark.parametrize("n,dealias", [(8, 0), (12, 0), (12, 1)])
def test_nonlinear_equals_triad_sum(n, dealias):
    a = inputs.random_solenoidal_state(n, 1.0, 4.0, 0.7, seed=n + dealias, dealias=dealias)
    p = oracle.Params(n=n, dealias=dealias)
    got = oracle.nonlinear(a, p)
    ref = triad_nonlinear(a, dealias)
    assert np.abs(got - ref).max() < 1e-14 * max(1.0, np.abs(ref).max()) * n
    assert np.abs(ref).max() > 1e-3          # a non-trivial case


def test_nonlinear_masks_input_modes():
    # a field with energy outside the kept set: only its kept part acts
    n = 12
    a = inputs.random_hermitian_half(n, 3, 5)
    got = oracle.nonlinear(a, oracle.Params(n=n))
    ref = triad_nonlinear(a, 0)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_abc_is_a_fixed_point_of_the_nonlinear_term():
    a = inputs.abc_state(16)
    assert np.abs(oracle.nonlinear(a, oracle.Params(n=16))).max() < 1e-15


def test_projection_is_idempotent_and_solenoidal():
    n = 12
    v = inputs.random_hermitian_half(n, 3, 11)
    pv = oracle.project(v)
    ppv = oracle.project(pv)
    assert np.abs(ppv - pv).max() < 1e-15
    KX, KY, KZ = _kvec(n)
    div = KX * pv[0] + KY * pv[1] + KZ * pv[2]
    assert np.abs(div).max() < 1e-13
    # a solenoidal kept field is unchanged
    s = inputs.random_solenoidal_state(n, 1, 3, 1.0, 4)
    assert np.abs(oracle.project(s) - s).max() < 1e-15


def test_nonlinear_output_is_divergence_free_and_dealiased():
    n = 24
    a = inputs.turbulence_state(n, 2)
    N = oracle.nonlinear(a, oracle.Params(n=n, force_amp=0.5, force_k=3))
    KX, KY, KZ = _kvec(n)
    assert np.abs(KX * N[0] + KY * N[1] + KZ * N[2]).max() < 1e-13
    outside = 3 * np.maximum(np.maximum(abs(KX), abs(KY)), KZ) >= n
    assert np.abs(N[:, outside]).max() == 0.0


def test_forcing_closed_form():
    # f = F (sin kf z + cos kf y, sin kf x + cos kf z, sin kf y + cos kf x)
    n, kf, F = 16, 3, 0.5
    fh = oracle.forcing(oracle.Params(n=n, force_amp=F, force_k=kf))
    ex = np.zeros_like(fh)
    ex[0, 0, 0, kf] = F / 2j
    ex[0, 0, kf, 0] = ex[0, 0, n - kf, 0] = F / 2
    ex[1, kf, 0, 0] = F / 2j
    ex[1, n - kf, 0, 0] = -F / 2j
    ex[1, 0, 0, kf] = F / 2
    ex[2, 0, kf, 0] = F / 2j
    ex[2, 0, n - kf, 0] = -F / 2j
    ex[2, kf, 0, 0] = ex[2, n - kf, 0, 0] = F / 2
    assert np.abs(fh - ex).max() < 1e-15
    # and it enters the nonlinear term additively (f is solenoidal)
    a = inputs.turbulence_state(n, 9)
    d = oracle.nonlinear(a, oracle.Params(n=n, force_amp=F, force_k=kf)) - \
        oracle.nonlinear(a, oracle.Params(n=n))
    assert np.abs(d - ex).max() < 1e-15


# ---------------------------------------------------------------- time stepping

@pytest.mark.parametrize("dt", [1e-3, 0.05])
def test_abc_decays_exactly(dt):
    n, nu, steps = 16, 0.01, 20
    a = inputs.abc_state(n)
    b = oracle.step(a, oracle.Params(n=n, nu=nu, dt=dt), steps)
    E, Om, _ = oracle.diagnostics(b)
    t = steps * dt
    assert abs(E - 1.5 * math.exp(-2 * nu * t)) < 1e-14
    assert abs(Om - 1.5 * math.exp(-2 * nu * t)) < 1e-14
    assert np.abs(b - a * math.exp(-nu * t)).max() < 1e-15


def test_single_solenoidal_mode_decays_exactly():
    n, nu, dt = 16, 0.03, 0.02
    a = np.zeros((3, n, n, n // 2 + 1), dtype=np.complex128)
    # k = (1, 2, 2): amplitude along e = (2, -1, 0)/sqrt5, which is normal to k
    a[0, 1, 2, 2] = 0.4 * 2 / math.sqrt(5)
    a[1, 1, 2, 2] = -0.4 / math.sqrt(5)
    b = oracle.step(a, oracle.Params(n=n, nu=nu, dt=dt), 7)
    assert np.abs(b - a * math.exp(-nu * 9 * dt * 7)).max() < 1e-16


def _galerkin_rhs_factory(n, nu):
    """Right-hand side of the dealiased Galerkin ODE system
    da/dt = -nu k^2 a + N(a) on the half layout, N by the triad sum."""
    KX, KY, KZ = _kvec(n)
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    shape = (3, n, n, n // 2 + 1)

    def rhs(t, y):
        a = y.view(np.complex128).reshape(shape)
        d = -nu * k2 * a + triad_nonlinear(a)
        return d.ravel().view(np.float64)
    return rhs


def test_time_step_converges_at_second_order_to_galerkin_ode():
    scipy_integrate = pytest.importorskip("scipy.integrate")
    n, nu, T = 8, 0.05, 0.2
    a0 = inputs.random_solenoidal_state(n, 1.0, 3.5, 1.5, seed=21)
    sol = scipy_integrate.solve_ivp(_galerkin_rhs_factory(n, nu), (0.0, T),
                                    a0.ravel().view(np.float64), method="DOP853",
                                    rtol=1e-12, atol=1e-14)
    exact = sol.y[:, -1].view(np.complex128).reshape(a0.shape)
    errs = []
    for steps in (10, 20, 40):
        b = oracle.step(a0, oracle.Params(n=n, nu=nu, dt=T / steps), steps)
        errs.append(rel_l2(b, exact))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.6 < r2 < 4.4, errs
    assert errs[2] < 1e-4


def test_inviscid_energy_drift_is_third_order_and_positive():
    # With nu = 0 and no forcing, <a, N(a)> = 0.  One Heun step then changes
    # |a|^2 by exactly (dt^2/4)|N(a) - N(a1)|^2 = O(dt^4) >= 0, so the drift
    # over a fixed time is O(dt^3) and never negative.  Another RK2 (explicit
    # midpoint) or a dropped stage would change the order or the sign.
    n, T = 16, 0.4
    a0 = inputs.turbulence_state(n, 31, rms=1.0)
    E0 = oracle.diagnostics(a0)[0]
    drift = []
    for steps in (20, 40, 80):
        b = oracle.step(a0, oracle.Params(n=n, nu=0.0, dt=T / steps), steps)
        drift.append(oracle.diagnostics(b)[0] - E0)
    assert all(d > 0 for d in drift)
    assert drift[2] < 1e-5 * E0
    assert 7.5 < drift[0] / drift[1] < 8.5 and 7.5 < drift[1] / drift[2] < 8.5, drift


def test_energy_budget():
    # dE/dt = -2 nu Omega + <u.f>, checked with a centred difference
    n, nu, dt, F, kf = 16, 0.02, 1e-3, 0.5, 3
    p = oracle.Params(n=n, nu=nu, dt=dt, force_amp=F, force_k=kf)
    a0 = inputs.turbulence_state(n, 8)
    a1 = oracle.step(a0, p, 1)
    fh = oracle.forcing(p)

    def budget(a):
        _, Om, _ = oracle.diagnostics(a)
        w = np.full(n // 2 + 1, 2.0)
        w[0] = w[n // 2] = 1.0
        uf = float(np.sum(w * np.real(a * np.conj(fh))))
        return -2 * nu * Om + uf
    lhs = (oracle.diagnostics(a1)[0] - oracle.diagnostics(a0)[0]) / dt
    rhs = 0.5 * (budget(a0) + budget(a1))
    assert abs(lhs - rhs) < 1e-5 * max(1.0, abs(rhs))


def test_taylor_green_invariants():
    n, nu, dt = 32, 1 / 1600, 2e-3
    a0 = inputs.taylor_green_state(n)
    E0, Om0, spec = oracle.diagnostics(a0)
    assert abs(E0 - 0.125) < 1e-15 and abs(Om0 - 0.375) < 1e-15
    assert abs(spec[2] - 0.125) < 1e-15        # all energy at |k| = sqrt3 -> shell 2
    a1 = oracle.step(a0, oracle.Params(n=n, nu=nu, dt=dt), 1)
    dEdt = (oracle.diagnostics(a1)[0] - E0) / dt
    assert abs(dEdt - (-2 * nu * Om0)) < 1e-6
    # mirror symmetries of TG survive: u_x odd in x, even in y and z (grid space)
    a5 = oracle.step(a0, oracle.Params(n=n, nu=nu, dt=dt), 5)
    u = oracle.fft3_c2r(a5)
    ux = u[0]
    neg = (-np.arange(n)) % n
    assert np.abs(ux[neg] + ux).max() < 1e-14
    assert np.abs(ux[:, neg] - ux).max() < 1e-14
    assert np.abs(ux[:, :, neg] - ux).max() < 1e-14


# ---------------------------------------------------------------- diagnostics

def test_diagnostics_parseval_and_spectrum():
    n = 16
    a = inputs.turbulence_state(n, 4, rms=0.8)
    E, Om, spec = oracle.diagnostics(a)
    assert abs(E - 1.5 * 0.8 ** 2) < 1e-14
    u = np.fft.irfftn(a, s=(n, n, n), axes=(1, 2, 3)) * n ** 3
    assert abs(0.5 * np.mean(np.sum(u * u, axis=0)) - E) < 1e-13
    assert abs(spec.sum() - E) < 1e-14
    assert len(spec) == math.ceil(math.sqrt(3) * n / 2) + 1
    # single mode k = (3, 4, 0): |k| = 5
    b = np.zeros_like(a)
    b[2, 3, 4, 0] = 0.5
    b[2, n - 3, n - 4, 0] = 0.5
    E, Om, spec = oracle.diagnostics(b)
    assert abs(E - 0.25) < 1e-16 and abs(Om - 25 * 0.25) < 1e-13
    assert abs(spec[5] - 0.25) < 1e-16 and abs(spec.sum() - 0.25) < 1e-16
    # round half up: |k| = 2.5 goes to shell 3 (k = (0, 1.5?)): use (1, 2, 2)/|k|=3
    c = np.zeros_like(a)
    c[0, 1, 2, 2] = 1.0
    _, _, spec = oracle.diagnostics(c)
    assert spec[3] == 1.0


def test_energy_half_helper_agrees_with_oracle():
    a = inputs.config1_state(32)
    assert abs(energy_half(a) - oracle.diagnostics(a)[0]) < 1e-14
    assert len(kept_modes(32)) == 21 ** 3
    assert np.allclose(half_to_full(a)[:, :, :, :17], a)


# ---------------------------------------------------------------- helicity

def test_helicity_of_beltrami_and_taylor_green():
    # ABC with k = 1 is a Beltrami field, w = u: H = 1/2 <u . u> = E = 1.5,
    # all in shell 1; Taylor-Green carries no helicity.
    H, spec = oracle.helicity(inputs.abc_state(16))
    assert abs(H - 1.5) < 1e-14 and abs(spec[1] - 1.5) < 1e-14
    H, _ = oracle.helicity(inputs.taylor_green_state(16))
    assert abs(H) < 1e-15
    # ABC at k = 2: w = 2u, H = 2E
    H, spec = oracle.helicity(inputs.abc_state(16, k=2))
    assert abs(H - 3.0) < 1e-14 and abs(spec[2] - 3.0) < 1e-14


def test_helicity_matches_grid_average():
    n = 16
    a = inputs.turbulence_state(n, 12, rms=0.9)
    H, spec = oracle.helicity(a)
    u = np.fft.irfftn(a, s=(n, n, n), axes=(1, 2, 3)) * n ** 3
    w = np.fft.irfftn(oracle.curl(a), s=(n, n, n), axes=(1, 2, 3)) * n ** 3
    assert abs(0.5 * np.mean(np.sum(u * w, axis=0)) - H) < 1e-13
    assert abs(spec.sum() - H) < 1e-14
    # mirror image (u(x) -> -u(-x) is a reflection: H changes sign)
    b = np.conj(a) * -1.0   # coefficients of -u(-x)
    Hb, _ = oracle.helicity(b)
    assert abs(Hb + H) < 1e-14


@pytest.mark.parametrize("k", [(2, 1, 3), (1, -2, 1), (-3, 0, 2)])
@pytest.mark.parametrize("s", [1, -1])
def test_rotation_inertial_wave_is_exact(k, s):
    """A single helical mode in a frame rotating about z is an inertial wave
    (Sec. 5 lists rotation among the equations of the same code): u x w = 0,
    and the projected Coriolis force turns the mode at the inertial frequency
    2 rot kz/|k|, positive sense for positive helicity.  The nonlinear term
    is then linear, N = lam a with lam = 2 i s rot kz/|k|, and IF-Heun
    multiplies the mode by exp(-nu k^2 dt) (1 + z + z^2/2), z = lam dt, per
    step exactly."""
    n, nu, dt, rot, steps = 16, 0.01, 0.01, 2.5, 20
    a0 = helical_mode(n, k, s)
    kk = np.linalg.norm(k)
    z = 2j * s * rot * k[2] / kk * dt
    g = np.exp(-nu * kk ** 2 * dt) * (1 + z + z * z / 2)
    b = oracle.step(a0, oracle.Params(n=n, nu=nu, dt=dt, rot=rot), steps)
    assert np.abs(b - a0 * g ** steps).max() < 1e-14
    # and the continuous solution a0 exp((lam - nu k^2) t) to second order in dt
    lam = 2j * s * rot * k[2] / kk
    T = 0.2
    errs = []
    for m in (20, 40):
        b = oracle.step(a0, oracle.Params(n=n, nu=nu, dt=T / m, rot=rot), m)
        errs.append(np.abs(b - a0 * np.exp((lam - nu * kk ** 2) * T)).max())
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_rotation_leaves_z_independent_flows_alone():
    """Taylor-Proudman: for kz = 0 the projected Coriolis force vanishes
    (z x u is a gradient there), so a z-independent flow evolves the same
    with and without rotation."""
    n = 16
    a = inputs.random_solenoidal_state(n, lo=1, hi=5, rms=0.5, seed=21, dealias=0)
    a[..., 1:] = 0.0
    b0 = oracle.step(a, oracle.Params(n=n, nu=0.01, dt=0.01), 5)
    b1 = oracle.step(a, oracle.Params(n=n, nu=0.01, dt=0.01, rot=4.0), 5)
    assert np.abs(b1 - b0).max() < 1e-13 * np.abs(b0).max()
    # while a 3D flow does feel it
    c = inputs.random_solenoidal_state(n, lo=1, hi=5, rms=0.5, seed=21, dealias=0)
    d0 = oracle.step(c, oracle.Params(n=n, nu=0.01, dt=0.01), 5)
    d1 = oracle.step(c, oracle.Params(n=n, nu=0.01, dt=0.01, rot=4.0), 5)
    assert np.abs(d1 - d0).max() > 1e-3 * np.abs(d0).max()


@pytest.mark.parametrize("n", [8, 12, 16])
def test_phase_shift_dealiasing_equals_exact_triad_sum(n):
    """Phase-shift dealiasing (dealias = 2): the product on the grid and on
    the grid shifted by (pi/N)(1,1,1), averaged, with the sphere
    9|k|^2 < 2 N^2, equals the exact convolution over that sphere, which
    holds modes beyond the 2/3 cube (|k| up to 0.47 N)."""
    a = inputs.random_solenoidal_state(n, 1.0, 0.47 * n, 0.7, seed=n, dealias=2)
    k = np.array(np.meshgrid(*[np.fft.fftfreq(n, 1.0 / n)] * 2, np.arange(n // 2 + 1),
                             indexing="ij"))
    outside_cube = 3 * np.max(np.abs(k), axis=0) >= n
    assert np.abs(a[:, outside_cube]).max() > 0      # the input uses the larger sphere
    got = oracle.nonlinear(a, oracle.Params(n=n, dealias=2))
    want = triad_nonlinear(a, 2)
    assert np.abs(got - want).max() < 1e-13 * np.abs(want).max()


def test_phase_shift_run_keeps_beltrami_decay_and_energy_budget():
    n, nu, dt = 16, 0.02, 0.01
    b = oracle.step(inputs.abc_state(n), oracle.Params(n=n, nu=nu, dt=dt, dealias=2), 5)
    assert abs(oracle.diagnostics(b)[0] - 1.5 * math.exp(-2 * nu * dt * 5)) < 1e-13
    # inviscid and unforced, the phase-shifted N conserves energy, so one Heun
    # step changes |a|^2 by exactly (dt^2/4) |N(a) - N(a1)|^2, a1 = a + dt N(a)
    a0 = inputs.random_solenoidal_state(n, 1.0, 7.0, 0.6, seed=5, dealias=2)
    h = 1e-2
    p = oracle.Params(n=n, dt=h, dealias=2)
    N0 = oracle.nonlinear(a0, p)
    N1 = oracle.nonlinear(a0 + h * N0, p)
    want = h * h / 4 * energy_half(N0 - N1)
    e0 = oracle.diagnostics(a0)[0]
    got = oracle.diagnostics(oracle.step(a0, p, 1))[0] - e0
    assert want > 0 and abs(got - want) < 1e-5 * want + 4e-15 * e0
