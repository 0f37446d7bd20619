"""GPU parity on grids of N_x x N_y x N_z points and boxes of sides 2 pi l_i
(the domains of aspect ratio other than one that the scheme handles, Sec. 5),
through the C ABI, against the FP64 oracle: the standalone grid transforms,
the solver step (plain FP64 to 1e-12 relative L2, plain FP32 to 2e-5) with
forcing, rotation, every dealiasing rule and MHD, the diagnostics, and the
embedding identity that ties a stretched box to the cube on the GPU itself."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1003_4322_gb300 import inputs
from tests.spectral_ref import rel_l2

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-5}


def _params(run):
    return oracle.Params(n=run["n"], ny=run.get("ny", 0), nz=run.get("nz", 0), lx=run.get("lx", 0.0),
                         ly=run.get("ly", 0.0), lz=run.get("lz", 0.0), nu=run.get("nu", 0.0),
                         dt=run["dt"], force_amp=run.get("force_amp", 0.0),
                         force_k=run.get("force_k", 0), dealias=run.get("dealias", 0),
                         rot=run.get("rot", 0.0), eta=run.get("eta", 0.0), mhd=run.get("mhd", 0))


def _dims(run):
    n = run["n"]
    return (n, run.get("ny", 0) or n, run.get("nz", 0) or n)


def _box(run):
    return tuple(run.get(k, 0.0) or 1.0 for k in ("lx", "ly", "lz"))


@pytest.fixture(scope="module", autouse=True)
def _threads():
    oracle.set_threads(os.cpu_count() or 1)


# ---------------------------------------------------------------- transforms

# (96, 128, 64) and (128, 64, 192): every axis has a compile-time FP32 kernel
GRIDS = [(8, 12, 16), (16, 8, 36), (24, 48, 8), (64, 32, 96), (96, 128, 64), (16, 256, 8),
         (128, 64, 192)]


@pytest.mark.parametrize("dims", GRIDS)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_grid_transforms_against_oracle(ns, dims, prec):
    """r2c and c2r of three components on non-cubic grids (ragged CTA column
    counts where an axis is short) against the oracle's transforms."""
    import torch
    from paper_1003_4322_gb300.solver import Solver
    nx, ny, nz = dims
    u = inputs.random_real_grid(dims, 3, seed=nx + ny + nz)
    ref = oracle.fft3_r2c(u)
    a = inputs.random_hermitian_half_grid(dims, 3, seed=nx * ny)
    back = oracle.fft3_c2r(a)
    rt, ct = (torch.float64, torch.complex128) if prec == "fp64" else (torch.float32, torch.complex64)
    tol = 1e-13 if prec == "fp64" else 1e-5
    with Solver([dict(n=8, dt=1e-3)], prec=prec) as s:
        ud = torch.from_numpy(u).to("cuda", rt)
        out = torch.empty((3, nx, ny, nz // 2 + 1), dtype=ct, device="cuda")
        s.fft_r2c_grid(ud, out)
        ad = torch.from_numpy(a).to("cuda", ct)
        phys = torch.empty((3, nx, ny, nz), dtype=rt, device="cuda")
        s.fft_c2r_grid(ad, phys)
        s.sync()
        got = out.cpu().numpy().astype(np.complex128)
        gotp = phys.cpu().numpy().astype(np.float64)
        assert np.abs(ad.cpu().numpy() - a.astype(ad.cpu().numpy().dtype)).max() == 0.0  # input kept
    assert np.abs(got - ref).max() < tol * np.abs(ref).max()
    assert np.abs(gotp - back).max() < tol * np.abs(back).max()


# ---------------------------------------------------------------- solver

RUNS = [
    dict(n=16, ny=24, nz=32, lx=1.0, ly=1.5, lz=2.0, nu=0.02, dt=2e-3, force_amp=0.5, force_k=2),
    dict(n=24, ny=16, nz=12, lx=1.5, ly=1.0, lz=0.75, nu=0.01, dt=2e-3, rot=1.5, dealias=1),
    dict(n=32, ny=32, nz=16, lz=0.5, nu=0.01, dt=2e-3, force_amp=0.3, force_k=2, dealias=2),
    dict(n=12, ny=36, nz=24, nu=0.02, dt=2e-3, force_amp=0.5, force_k=3),
    dict(n=16, ny=12, nz=24, lx=1.0, ly=0.75, lz=1.5, nu=0.02, eta=0.03, dt=2e-3, mhd=1, rot=0.5),
    dict(n=64, ny=48, nz=96, lx=1.0, ly=0.75, lz=1.5, nu=5e-3, dt=1e-3, force_amp=0.5, force_k=4),
]


def _state(run, seed):
    dims, box = _dims(run), _box(run)
    a = inputs.random_solenoidal_grid(dims, box, 0.5, 4.0, 1.0, seed=seed, dealias=run.get("dealias", 0))
    if run.get("mhd"):
        b = inputs.random_solenoidal_grid(dims, box, 0.5, 3.0, 0.6, seed=seed + 1)
        a = np.concatenate([a, b])
    return a


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("i", range(len(RUNS)))
def test_grid_runs_against_oracle(ns, prec, i):
    from paper_1003_4322_gb300 import _native as nat
    from paper_1003_4322_gb300.solver import Solver
    run = RUNS[i]
    a0 = _state(run, seed=100 + i)
    steps = 3
    ref = oracle.step(a0, _params(run), steps)
    with Solver([run], prec=prec) as s:
        if run.get("mhd"):
            s.set_field(0, a0[:3])
            s.set_field(1, a0[3:])
        else:
            s.set_state(a0)
        s.step(steps)
        got = s.get_state()
        if run.get("mhd"):
            got = np.concatenate([got, s.get_field(1)])
        E, Om, spec = s.energy_spectrum()
        H, hspec = s.helicity()
        Es, Os = s.series(count=steps)
        desc = nat.ns_describe_run(s.ctx, 0)
    # FP32 Navier-Stokes runs with the 2/3 rules take the fused form on grids and boxes
    fused = prec == "fp32" and not run.get("mhd") and run.get("dealias", 0) in (0, 1)
    assert desc["form"] == ("fused FP32" if fused else "plain FP64" if prec == "fp64" else "plain FP32"), desc
    assert desc["grid"] == list(_dims(run))
    assert rel_l2(got, ref) < TOL[prec], rel_l2(got, ref)
    p = _params(run)
    e_ref, om_ref, spec_ref = oracle.diagnostics(ref[:3], p)
    h_ref, hspec_ref = oracle.helicity(ref[:3], p)
    tol = 1e-12 if prec == "fp64" else 5e-5
    assert abs(E - e_ref) < tol * e_ref and abs(Om - om_ref) < tol * om_ref
    assert len(spec) == len(spec_ref) == oracle.nbins(p)
    assert np.abs(spec - spec_ref).max() < tol * e_ref
    assert abs(H - h_ref) < tol * math.sqrt(e_ref * om_ref)
    assert np.abs(hspec - hspec_ref).max() < tol * math.sqrt(e_ref * om_ref)
    assert abs(Es[-1] - E) < 1e-12 * E and abs(Os[-1] - Om) < 1e-12 * Om


def test_stretched_box_reproduces_the_cube_on_the_gpu(ns):
    """The 48^3 forced run equals the run on the (96, 48, 144) grid of the box
    (4pi, 2pi, 6pi) holding indices (2 m_x, m_y, 3 m_z) (FP64, 4 steps), and
    both agree with the oracle's cubic run."""
    from paper_1003_4322_gb300.solver import Solver
    n, mult = 48, (2, 1, 3)
    dims = tuple(n * k for k in mult)
    kw = dict(nu=5e-3, dt=2e-3, force_amp=0.5, force_k=2, rot=0.8)
    a = inputs.turbulence_state(n, seed=5)
    with Solver([dict(n=n, **kw)], prec="fp64") as s:
        s.set_state(a)
        s.step(4)
        ref = s.get_state()
        e_ref = s.energy_spectrum()[:2]
    assert rel_l2(ref, oracle.step(a, oracle.Params(n=n, **kw), 4)) < 1e-12
    b = np.zeros((3, dims[0], dims[1], dims[2] // 2 + 1), dtype=np.complex128)
    m = np.fft.fftfreq(n, 1.0 / n).astype(int)
    ix, iy, iz = (2 * m) % dims[0], m % dims[1], 3 * np.arange(n // 2 + 1)
    sel = (slice(None), ix[:, None, None], iy[None, :, None], iz[None, None, :])
    b[sel] = a
    with Solver([dict(n=dims[0], ny=dims[1], nz=dims[2], lx=2.0, ly=1.0, lz=3.0, **kw)], prec="fp64") as s:
        s.set_state(b)
        s.step(4)
        got = s.get_state()
        e_got = s.energy_spectrum()[:2]
    assert rel_l2(got[sel], ref) < 1e-13
    rest = got.copy()
    rest[sel] = 0
    assert np.abs(rest).max() < 1e-15 * np.abs(ref).max()
    assert abs(e_got[0] - e_ref[0]) < 1e-13 * e_ref[0] and abs(e_got[1] - e_ref[1]) < 1e-12 * e_ref[1]


def test_grid_state_round_trip_and_mask(ns):
    """set_state drops the modes outside the per-axis 2/3 rule; get_state
    returns the rest bit for bit (FP64) on a grid of three different sizes."""
    from paper_1003_4322_gb300.solver import Solver
    run = dict(n=16, ny=24, nz=36, lx=1.0, ly=2.0, lz=3.0, dt=1e-3)
    a = inputs.random_hermitian_half_grid((16, 24, 36), 3, seed=3)
    with Solver([run], prec="fp64") as s:
        s.set_state(a)
        got = s.get_state()
    mx = np.abs(np.fft.fftfreq(16, 1 / 16))[:, None, None]
    my = np.abs(np.fft.fftfreq(24, 1 / 24))[None, :, None]
    mz = np.arange(19)[None, None, :]
    keep = (3 * mx < 16) & (3 * my < 24) & (3 * mz < 36)
    assert np.array_equal(got, np.where(keep, a, 0))


def test_shape_checks_refuse_wrong_buffers(ns):
    from paper_1003_4322_gb300.solver import Solver
    with Solver([dict(n=16, ny=24, nz=8, dt=1e-3)], prec="fp64") as s:
        with pytest.raises(ValueError):
            s.set_state(np.zeros((3, 16, 16, 9), dtype=np.complex128))
        with pytest.raises(TypeError):
            s.get_state(out=np.zeros((3, 16, 24, 5), dtype=np.complex64))
        assert s.get_state().shape == (3, 16, 24, 5)


@pytest.mark.parametrize("family", ["smem", "reg", "pf"])
@pytest.mark.parametrize("dims", [(64, 64, 512), (64, 96, 384), (32, 64, 1024), (64, 32, 768),
                                  (96, 64, 256)])
def test_std_z_kernel_families_against_oracle(ns, dims, family, monkeypatch):
    """The compile-time FP32 transforms with the z pass restricted to one
    kernel family (shared-memory lines; register-resident lines with the
    even/odd packing through warp shuffles; the same with four line groups
    per warp and the next group's input prefetched), NS_FORCE_STD_Z, against
    the oracle on grids whose z lengths have register candidates (the line
    counts leave the last warp's groups partly empty)."""
    import torch
    from paper_1003_4322_gb300.solver import Solver
    monkeypatch.setenv("NS_FORCE_STD_Z", family)
    nx, ny, nz = dims
    u = inputs.random_real_grid(dims, 2, seed=nz)
    ref = oracle.fft3_r2c(u)
    a = inputs.random_hermitian_half_grid(dims, 2, seed=nz + 1)
    a[:, :, :, -1] += 0.5   # a real Nyquist plane of its own
    back = oracle.fft3_c2r(a)
    with Solver([dict(n=8, dt=1e-3)], prec="fp32") as s:
        out = torch.empty((2, nx, ny, nz // 2 + 1), dtype=torch.complex64, device="cuda")
        s.fft_r2c_grid(torch.from_numpy(u).to("cuda", torch.float32), out)
        phys = torch.empty((2, nx, ny, nz), dtype=torch.float32, device="cuda")
        s.fft_c2r_grid(torch.from_numpy(a).to("cuda", torch.complex64), phys)
        s.sync()
        got, gotp = out.cpu().numpy(), phys.cpu().numpy()
    assert np.abs(got - ref).max() < 1e-5 * np.abs(ref).max()
    assert np.abs(gotp - back).max() < 1e-5 * np.abs(back).max()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_mixed_grid_ensemble_equals_runs_alone(ns, prec):
    """Grid runs, a cubic run and a phase-shift run in one context (the plain
    form, the runs on concurrent branches of one CUDA graph) give, bit for
    bit, what each gives alone.  Runs of one context share the transform
    plans of an axis length, so no grid axis here has the cubic run's length;
    alone in FP32 every run but the phase-shift one takes the fused form, so
    those are compared to the FP32 tolerance."""
    from paper_1003_4322_gb300.solver import Solver
    runs = [dict(n=32, ny=48, nz=24, lz=2.0, nu=0.01, dt=1e-3, force_amp=0.4, force_k=2),
            dict(n=36, nu=0.01, dt=1e-3, rot=1.0),
            dict(n=24, ny=24, nz=64, lx=1.5, nu=0.02, dt=1e-3, dealias=2),
            dict(n=64, ny=32, nz=32, nu=0.01, dt=1e-3, dealias=1)]
    starts = [_state(r, seed=50 + i) for i, r in enumerate(runs)]
    alone = []
    for r, a in zip(runs, starts):
        with Solver([r], prec=prec) as s:
            s.set_state(a)
            s.step(3)
            alone.append(s.get_state())
    with Solver(runs, prec=prec) as s:
        for i, a in enumerate(starts):
            s.set_state(a, run=i)
        s.step(3)
        together = [s.get_state(run=i) for i in range(len(runs))]
    for i, (a, b) in enumerate(zip(alone, together)):
        if i != 2 and prec == "fp32":
            assert rel_l2(b, a) < TOL["fp32"]
        else:
            assert np.array_equal(a, b), i
