"""The plain form's z passes in both of their forms, forced through
NS_PLAIN_Z: one real line per complex transform of length N/2 (even/odd
packing), or two real lines per complex transform of length N (the spectra
of lines 2p and 2p + 1 as the real and imaginary parts of one Hermitian pair).
Steps of the solver (Sec. 2, Eqs. 1-2) against the FP64 oracle: cubes with
radix-3 lengths, a grid on a box of other aspect ratio, MHD, and the plain
FP32 form with phase-shift dealiasing."""
import numpy as np
import pytest

import oracle
from paper_1003_4322_gb300 import inputs
from tests.spectral_ref import rel_l2

pytestmark = pytest.mark.gpu


def _check(ns, run, a0, prec, steps, mode, tol):
    from paper_1003_4322_gb300.solver import Solver
    ref = oracle.step(a0, oracle.Params(**{k: v for k, v in run.items()}), steps)
    with Solver([run], prec=prec) as s:
        d = ns.ns_describe_run(s.ctx, 0)
        assert d["form"].startswith("plain"), d
        assert d["z_c2r"]["lines_per_transform"] == mode, d
        assert d["z_r2c"]["lines_per_transform"] == mode, d
        if a0.shape[0] == 6:
            s.set_field(0, a0[:3])
            s.set_field(1, a0[3:])
        else:
            s.set_state(a0)
        s.step(steps)
        got = s.get_state() if a0.shape[0] == 3 else np.concatenate([s.get_field(0), s.get_field(1)])
    err = rel_l2(got, ref)
    assert err < tol, (run, mode, err)


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("n", [8, 12, 24, 48, 96])
def test_cubes(ns, n, mode, monkeypatch):
    monkeypatch.setenv("NS_PLAIN_Z", str(mode))
    run = dict(n=n, nu=0.02, dt=2e-3, force_amp=0.5, force_k=min(3, (n - 1) // 3))
    _check(ns, run, inputs.turbulence_state(n, seed=n + 3), "fp64", 3, mode, 1e-12)


@pytest.mark.parametrize("mode", [1, 2])
def test_grid_box(ns, mode, monkeypatch):
    monkeypatch.setenv("NS_PLAIN_Z", str(mode))
    run = dict(n=16, ny=24, nz=36, lx=1.0, ly=1.5, lz=2.0, nu=0.02, dt=2e-3, force_amp=0.5, force_k=2)
    a0 = inputs.random_solenoidal_grid((16, 24, 36), (1.0, 1.5, 2.0), 0.5, 4.0, 1.0, seed=11)
    _check(ns, run, a0, "fp64", 2, mode, 1e-12)


@pytest.mark.parametrize("mode", [1, 2])
def test_mhd(ns, mode, monkeypatch):
    monkeypatch.setenv("NS_PLAIN_Z", str(mode))
    n = 24
    run = dict(n=n, nu=0.02, eta=0.03, mhd=1, dt=2e-3, force_amp=0.5, force_k=3)
    u = inputs.turbulence_state(n, seed=21)
    b = inputs.random_solenoidal_state(n, 1.0, 4.0, 0.7, seed=22)
    _check(ns, run, np.concatenate([u, b]), "fp64", 2, mode, 1e-12)


@pytest.mark.parametrize("mode", [1, 2])
def test_fp32_phase_shift(ns, mode, monkeypatch):
    monkeypatch.setenv("NS_PLAIN_Z", str(mode))
    n = 24
    run = dict(n=n, nu=0.02, dt=2e-3, dealias=2)
    a0 = inputs.random_solenoidal_state(n, 1.0, 4.0, 1.0, seed=31, dealias=2)
    _check(ns, run, a0, "fp32", 2, mode, 2e-5)
