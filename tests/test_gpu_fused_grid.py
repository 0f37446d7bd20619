"""The fused FP32 form on grids of N_x x N_y x N_z points and boxes of sides
2 pi l_i (the domains of aspect ratio other than one, Sec. 5; Sec. 2, Eqs.
1-2 on each): per-axis compaction |m_i| <= (N_i - 1) / 3, wavenumbers m_i / l_i
in the curl, the projection and the enstrophy, per-axis factor tables, the
forcing at the grid indices k_f l_i and the sphere of the spherical rule in
grid indices.  Against the FP64 oracle: the state after three steps, E, Omega,
the energy and helicity spectra (the plain form's shells on the expanded
state), and the per-step series of the update's compensated partials against
an FP64 sum.  Runs of one grid in one context advance in one launch per pass
and equal the runs done alone, bit for bit."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1003_4322_gb300 import inputs
from tests.spectral_ref import rel_l2

pytestmark = pytest.mark.gpu

TOL = 2e-5

RUNS = [
    # axis lengths with compile-time kernels, unit box, forced
    dict(n=64, ny=96, nz=128, nu=0.01, dt=1e-3, force_amp=0.5, force_k=2),
    # a box, rotation and the spherical rule
    dict(n=128, ny=64, nz=96, lx=1.0, ly=0.5, lz=1.5, nu=0.01, dt=1e-3, rot=1.5, dealias=1),
    # the box (2 pi, 2 pi, pi) of the 512 x 512 x 256 workload, at 96 x 96 x 48
    dict(n=96, ny=96, nz=48, lz=0.5, nu=5e-3, dt=1e-3, force_amp=0.3, force_k=2),
    # lengths without compile-time kernels (the runtime-length passes)
    dict(n=48, ny=24, nz=36, lx=1.5, nu=0.02, dt=2e-3, force_amp=0.5, force_k=2),
]


def _dims(run):
    return (run["n"], run.get("ny", 0) or run["n"], run.get("nz", 0) or run["n"])


def _box(run):
    return tuple(run.get(k, 0.0) or 1.0 for k in ("lx", "ly", "lz"))


def _params(run):
    return oracle.Params(n=run["n"], ny=run.get("ny", 0), nz=run.get("nz", 0), lx=run.get("lx", 0.0),
                         ly=run.get("ly", 0.0), lz=run.get("lz", 0.0), nu=run.get("nu", 0.0),
                         dt=run["dt"], force_amp=run.get("force_amp", 0.0),
                         force_k=run.get("force_k", 0), dealias=run.get("dealias", 0),
                         rot=run.get("rot", 0.0))


@pytest.fixture(scope="module", autouse=True)
def _threads():
    oracle.set_threads(os.cpu_count() or 1)


@pytest.mark.parametrize("i", range(len(RUNS)))
def test_fused_grid_runs_against_oracle(ns, i):
    from paper_1003_4322_gb300 import _native as nat
    from paper_1003_4322_gb300.solver import Solver
    run = RUNS[i]
    a0 = inputs.random_solenoidal_grid(_dims(run), _box(run), 0.5, 4.0, 1.0, seed=200 + i,
                                       dealias=run.get("dealias", 0))
    steps = 3
    p = _params(run)
    ref = oracle.step(a0, p, steps)
    with Solver([run], prec="fp32") as s:
        desc = nat.ns_describe_run(s.ctx, 0)
        s.set_state(a0)
        s.step(steps)
        got = s.get_state()
        E, Om, spec = s.energy_spectrum()
        H, hspec = s.helicity()
        Es, Os = s.series(count=steps)
    assert desc["form"] == "fused FP32" and desc["grid"] == list(_dims(run)), desc
    assert desc["box"] == list(_box(run)), desc
    err = rel_l2(got, ref)
    print(f"fused grid {_dims(run)} box {_box(run)}: rel-L2 vs oracle after {steps} steps {err:.2e}")
    assert err < TOL
    e_ref, om_ref, spec_ref = oracle.diagnostics(ref, p)
    h_ref, hspec_ref = oracle.helicity(ref, p)
    tol = 5e-5
    assert abs(E - e_ref) < tol * e_ref and abs(Om - om_ref) < tol * om_ref
    assert len(spec) == len(spec_ref) == oracle.nbins(p)
    assert np.abs(spec - spec_ref).max() < tol * e_ref
    assert abs(H - h_ref) < tol * math.sqrt(e_ref * om_ref)
    assert np.abs(hspec - hspec_ref).max() < tol * math.sqrt(e_ref * om_ref)
    # the update's compensated FP32 partials against the FP64 sums of the state
    assert abs(Es[-1] - E) < 1e-12 * E and abs(Os[-1] - Om) < 1e-12 * Om


def test_fused_grid_group_equals_runs_alone(ns):
    """Three runs on one box with different viscosity, forcing and rotation
    form one group (one launch per pass, grid y = run); each equals the same
    run done alone, bit for bit."""
    from paper_1003_4322_gb300.solver import Solver
    base = dict(n=64, ny=48, nz=96, lx=1.0, ly=0.75, lz=1.5, dt=1e-3)
    runs = [dict(base, nu=0.01), dict(base, nu=0.02, force_amp=0.5, force_k=4), dict(base, nu=5e-3, rot=1.0)]
    starts = [inputs.random_solenoidal_grid(_dims(base), _box(base), 0.5, 4.0, 1.0, seed=300 + i)
              for i in range(len(runs))]
    alone = []
    for r, a in zip(runs, starts):
        with Solver([r], prec="fp32") as s:
            s.set_state(a)
            s.step(3)
            alone.append(s.get_state())
    with Solver(runs, prec="fp32") as s:
        for i, a in enumerate(starts):
            s.set_state(a, run=i)
        s.step(3)
        together = [s.get_state(run=i) for i in range(len(runs))]
    for i, (a, b) in enumerate(zip(alone, together)):
        assert np.array_equal(a, b), i


def test_fused_cube_and_grids_in_one_context(ns):
    """A cube and two grids in one FP32 context: three groups of the fused
    form on concurrent branches of one CUDA graph, each bitwise equal to its
    run done alone."""
    from paper_1003_4322_gb300 import _native as nat
    from paper_1003_4322_gb300.solver import Solver
    runs = [dict(n=64, nu=0.01, dt=1e-3, force_amp=0.5, force_k=2),
            dict(n=64, ny=48, nz=96, lx=1.0, ly=0.75, lz=1.5, nu=0.02, dt=1e-3, rot=0.5),
            dict(n=96, ny=96, nz=48, lz=0.5, nu=5e-3, dt=1e-3, force_amp=0.3, force_k=2, dealias=1)]
    starts = [inputs.random_solenoidal_grid(_dims(r), _box(r), 0.5, 4.0, 1.0, seed=400 + i,
                                           dealias=r.get("dealias", 0)) for i, r in enumerate(runs)]
    alone = []
    for r, a in zip(runs, starts):
        with Solver([r], prec="fp32") as s:
            s.set_state(a)
            s.step(3)
            alone.append(s.get_state())
    with Solver(runs, prec="fp32") as s:
        for i in range(len(runs)):
            d = nat.ns_describe_run(s.ctx, i)
            assert d["form"] == "fused FP32" and d["grid"] == list(_dims(runs[i])), d
        for i, a in enumerate(starts):
            s.set_state(a, run=i)
        s.step(3)
        together = [s.get_state(run=i) for i in range(len(runs))]
    for i, (a, b) in enumerate(zip(alone, together)):
        assert np.array_equal(a, b), i


def _passes(desc):
    return {k: v for k, v in desc["passes"].items() if k in ("A_x_inverse_curl", "B_y_inverse",
                                                             "D_y_forward", "E_x_forward")}


@pytest.mark.parametrize("dims,E,ct,steps,oracle_check", [((96, 96, 48), 12, 8, 3, True),
                                                        ((96, 96, 48), 12, 16, 3, True),
                                                        ((512, 512, 256), 16, 8, 2, False),
                                                        ((512, 512, 256), 32, 16, 2, False)])
def test_constant_geometry_grid_kernels(ns, dims, E, ct, steps, oracle_check, monkeypatch):
    """Passes A, B, D, E on the kernels with the grid's whole geometry fixed
    at compile time (the box (2 pi, 2 pi, pi) of the 512 x 512 x 256
    workload, and the same box at 96 x 96 x 48), forced through
    NS_FORCE_STRIDED, against the runtime-stride kernels of the same length
    and shape (the same FFT and curl arithmetic) and, on the small grid,
    against the FP64 oracle."""
    from paper_1003_4322_gb300 import _native as nat
    from paper_1003_4322_gb300.solver import Solver
    nx, ny, nz = dims
    run = dict(n=nx, ny=ny, nz=nz, lz=0.5, nu=5e-3, dt=1e-3, force_amp=0.3, force_k=2)
    a0 = inputs.random_solenoidal_grid(dims, _box(run), 0.5, 4.0, 1.0, seed=500)
    got = {}
    for kind, name in ((2, "constant geometry"), (1, "compile-time length")):
        monkeypatch.setenv("NS_FORCE_STRIDED", f"{kind},{E},{ct}")
        with Solver([run], prec="fp32") as s:
            passes = _passes(nat.ns_describe_run(s.ctx, 0))
            assert all(p["kernel"] == name and p["E"] == E and p["cols_per_cta"] == ct
                       for p in passes.values()), passes
            s.set_state(a0)
            s.step(steps)
            got[kind] = s.get_state()
    d = rel_l2(got[2], got[1])
    print(f"grid {dims} E={E} ct={ct}: constant geometry vs runtime strides rel-L2 {d:.2e}, "
          f"bitwise {np.array_equal(got[2], got[1])}")
    assert np.abs(got[2]).max() > 0 and d < 1e-6
    if oracle_check:
        ref = oracle.step(a0, _params(run), steps)
        assert rel_l2(got[2], ref) < TOL
