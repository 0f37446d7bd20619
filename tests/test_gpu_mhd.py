"""MHD in the plain FP64 and the fused FP32 form, through the C ABI, against the
oracle (the magnetohydrodynamic equations of the same code, Sec. 5; Alfven
units, state [u; b]) and against exact solutions."""
import math

import numpy as np
import pytest

import oracle
from paper_1003_4322_gb300 import inputs
from tests.spectral_ref import helical_mode, rel_l2

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-5}


def _mhd_state(n, seed):
    u = inputs.turbulence_state(n, seed=seed)
    b = inputs.random_solenoidal_state(n, 1.0, 4.0, 0.7, seed=seed + 50)
    return u, b


def _run(prec, run, u0, b0, steps):
    from paper_1003_4322_gb300.solver import Solver
    with Solver([run], prec=prec) as s:
        s.set_field(0, u0)
        s.set_field(1, b0)
        s.step(steps)
        return s.get_field(0), s.get_field(1), s.field_spectrum(1)


def _oracle(run, u0, b0, steps):
    p = oracle.Params(n=run["n"], nu=run["nu"], dt=run["dt"], force_amp=run.get("force_amp", 0.0),
                      force_k=run.get("force_k", 0), rot=run.get("rot", 0.0), eta=run["eta"], mhd=1)
    out = oracle.step(np.concatenate([u0, b0]), p, steps)
    return out[:3], out[3:]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [32, 48])
def test_mhd_matches_oracle(ns, prec, n):
    run = dict(n=n, nu=0.01, eta=0.02, dt=1e-3, force_amp=0.5, force_k=3, rot=1.0, mhd=1)
    u0, b0 = _mhd_state(n, 41)
    u, b, (Eb, Jb, spec) = _run(prec, run, u0, b0, 4)
    ru, rb = _oracle(run, u0, b0, 4)
    assert rel_l2(u, ru) < TOL[prec] and rel_l2(b, rb) < TOL[prec]
    rE, rJ, rspec = oracle.diagnostics(rb)
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert abs(Eb - rE) < tol * rE and abs(Jb - rJ) < tol * rJ
    # the magnetic field matters: without it the velocity differs
    ru0, _ = _oracle(run, u0, 0 * b0, 4)
    assert rel_l2(ru, ru0) > 100 * TOL["fp32"]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_alfven_wave_exact_on_gpu(ns, prec):
    """Mean field B0 z and one helical mode in u and b: the Elsasser fields
    turn at +-kz B0 with the exact discrete IF-Heun factor."""
    from paper_1003_4322_gb300.solver import Solver
    n, nu, dt, B0, steps = 32, 0.01, 0.01, 1.7, 15
    k, s_ = (1, 2, 3), 1
    h = helical_mode(n, k, s_, amp=1.0)
    al, be = 0.3, -0.1 + 0.2j
    b0 = be * h
    b0[2, 0, 0, 0] = B0
    with Solver([dict(n=n, nu=nu, eta=nu, dt=dt, mhd=1)], prec=prec) as s:
        s.set_field(0, al * h)
        s.set_field(1, b0)
        s.step(steps)
        u, b = s.get_field(0), s.get_field(1)
    kk = np.linalg.norm(k)
    E = math.exp(-nu * kk ** 2 * dt)
    g = [E * (1 + z + z * z / 2) for z in (1j * k[2] * B0 * dt, -1j * k[2] * B0 * dt)]
    zp, zm = (al + be) * g[0] ** steps, (al - be) * g[1] ** steps
    want_b = 0.5 * (zp - zm) * h
    want_b[2, 0, 0, 0] = B0
    tol = 1e-14 if prec == "fp64" else 2e-6
    assert np.abs(u - 0.5 * (zp + zm) * h).max() < tol
    assert np.abs(b - want_b).max() < tol


def test_force_free_field_and_form(ns):
    """u = 0, b = ABC: exact decay exp(-eta t); FP64 runs the plain form and
    FP32 the fused form (velocity and magnetic blocks); field 1 of a
    Navier-Stokes run is an argument error."""
    from paper_1003_4322_gb300 import _native as nat
    from paper_1003_4322_gb300.solver import Solver
    n, eta, dt, steps = 32, 0.02, 0.05, 6
    # FP32: j x b of the force-free field is zero only to rounding, so u picks
    # up an energy of order (eps32 |b|^2 dt)^2
    for prec, tol, utol in (("fp64", 1e-14, 1e-28), ("fp32", 1e-6, 1e-14)):
        with Solver([dict(n=n, nu=0.01, eta=eta, dt=dt, mhd=1)], prec=prec) as s:
            d = nat.ns_describe_run(s.ctx, 0)
            assert d["equations"] == "MHD"
            assert d["form"] == ("plain FP64" if prec == "fp64" else "fused FP32")
            s.set_field(1, inputs.abc_state(n))
            s.step(steps)
            Eb, _, _ = s.field_spectrum(1)
            Eu, _, _ = s.field_spectrum(0)
        assert abs(Eb - 1.5 * math.exp(-2 * eta * dt * steps)) < tol and Eu < utol
    with Solver([dict(n=n, nu=0.01, dt=dt)], prec="fp64") as s:
        with pytest.raises(nat.NsError) as e:
            s.set_field(1, inputs.abc_state(n))
        assert e.value.status == nat.NS_ERR_ARG
        with pytest.raises(nat.NsError):
            s.field_spectrum(1)


def test_mhd_group_with_navier_stokes_run(ns):
    """One fused context: two MHD runs of one size with different eta (one
    group, one launch per pass on both blocks) and a Navier-Stokes run of the
    same size (its own group); every member matches its oracle run."""
    from paper_1003_4322_gb300.solver import Solver
    n = 32
    runs = [dict(n=n, nu=0.01, eta=0.01, dt=1e-3, mhd=1),
            dict(n=n, nu=0.01, eta=0.03, dt=1e-3, force_amp=0.5, force_k=3, mhd=1),
            dict(n=n, nu=0.01, dt=1e-3)]
    u0, b0 = _mhd_state(n, 61)
    with Solver(runs, prec="fp32") as s:
        for r in range(3):
            s.set_field(0, u0, run=r)
        for r in range(2):
            s.set_field(1, b0, run=r)
        s.step(3)
        got = [(s.get_field(0, run=r), s.get_field(1, run=r) if r < 2 else None) for r in range(3)]
    for r in range(2):
        ru, rb = _oracle(runs[r], u0, b0, 3)
        assert rel_l2(got[r][0], ru) < TOL["fp32"] and rel_l2(got[r][1], rb) < TOL["fp32"]
    ref = oracle.step(u0, oracle.Params(n=n, nu=0.01, dt=1e-3), 3)
    assert rel_l2(got[2][0], ref) < TOL["fp32"]
