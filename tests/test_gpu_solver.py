"""GPU parity of the solver step (Sec. 2, Eqs. 1-2) against the FP64 oracle,
through the C ABI: FP64 (plain form) to 1e-12 relative L2, FP32 to 2e-5,
plus invariants the method fixes at any size (exact Beltrami decay,
divergence-free state, Taylor-Green energy and enstrophy, determinism)."""
import math

import numpy as np
import pytest

import oracle
from paper_1003_4322_gb300 import inputs
from tests.spectral_ref import helical_mode, rel_l2, shell_error_ratios, wavenumbers

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-5}


def _solver(ns, prec, **run):
    from paper_1003_4322_gb300.solver import Solver
    return Solver([run], prec=prec)


def _oracle_run(a0, run, steps):
    return oracle.step(a0, oracle.Params(n=run["n"], nu=run.get("nu", 0.0), dt=run["dt"],
                                         force_amp=run.get("force_amp", 0.0),
                                         force_k=run.get("force_k", 0),
                                         dealias=run.get("dealias", 0),
                                         rot=run.get("rot", 0.0)), steps)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_config1_32cubed_ten_steps(ns, prec):
    """ABC + random perturbation on 2 <= |k| <= 4 (rms 0.1), nu = 0.01,
    dt = 1e-3, 10 RK2 steps on 32^3."""
    run = dict(n=32, nu=0.01, dt=1e-3)
    a0 = inputs.config1_state(32, seed=1)
    ref = _oracle_run(a0, run, 10)
    with _solver(ns, prec, **run) as s:
        s.set_state(a0)
        s.step(10)
        got = s.get_state()
    assert rel_l2(got, ref) < TOL[prec]
    if prec == "fp32":
        assert shell_error_ratios(got, ref).max() < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n,dealias,forced", [(8, 0, False), (12, 0, True), (16, 1, False),
                                              (24, 0, True), (48, 1, True), (96, 0, True)])
def test_sizes_dealias_forcing(ns, prec, n, dealias, forced):
    run = dict(n=n, nu=0.02, dt=2e-3, dealias=dealias)
    if forced:
        run.update(force_amp=0.5, force_k=min(3, (n - 1) // 3))
    a0 = inputs.turbulence_state(n, seed=n + 7, dealias=dealias)
    steps = 3
    ref = _oracle_run(a0, run, steps)
    with _solver(ns, prec, **run) as s:
        s.set_state(a0)
        s.step(steps)
        got = s.get_state()
    assert rel_l2(got, ref) < TOL[prec]
    if prec == "fp32":
        assert shell_error_ratios(got, ref).max() < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_beltrami_decays_exactly(ns, prec):
    n, nu, dt, steps = 32, 0.05, 0.01, 20
    with _solver(ns, prec, n=n, nu=nu, dt=dt) as s:
        s.set_state(inputs.abc_state(n))
        s.step(steps)
        E, Om, spec = s.energy_spectrum()
    want = 1.5 * math.exp(-2 * nu * dt * steps)
    # FP32: the state is rounded to float at every stage (2 x 20 roundings of
    # relative size 6e-8, plus the float E table): a few 1e-6 relative
    tol = 1e-13 if prec == "fp64" else 5e-6
    assert abs(E - want) < tol and abs(Om - want) < tol
    assert abs(spec[1] - want) < tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_state_is_divergence_free_and_dealiased(ns, prec):
    """A solenoidal start with extra solenoidal modes outside the kept set:
    those are dropped on entry, and the state stays divergence-free."""
    n = 48
    a0 = inputs.turbulence_state(n, seed=11)
    # k = (20, 3, 5) and (-2, 17, 9): outside the 2/3-rule cube (3*20 >= 48)
    for (kx, ky, kz), e in (((20, 3, 5), (3.0, -20.0, 0.0)), ((-2, 17, 9), (17.0, 2.0, 0.0))):
        for c in range(3):
            a0[c, kx % n, ky % n, kz] += 0.05 * e[c]
    with _solver(ns, prec, n=n, nu=0.01, dt=1e-3, force_amp=0.5, force_k=3) as s:
        s.set_state(a0)
        s.step(2)
        a = s.get_state()
    k = wavenumbers(n).astype(float)
    KX, KY, KZ = np.meshgrid(k, k, np.arange(n // 2 + 1.0), indexing="ij")
    div = np.abs(KX * a[0] + KY * a[1] + KZ * a[2]).max() / np.abs(a).max()
    assert div < (1e-13 if prec == "fp64" else 1e-5)
    outside = 3 * np.maximum(np.maximum(abs(KX), abs(KY)), KZ) >= n
    assert np.abs(a[:, outside]).max() == 0.0


def test_set_get_round_trip_drops_modes_outside_the_kept_set(ns):
    n = 24
    a = inputs.random_hermitian_half(n, 3, 3)
    with _solver(ns, "fp64", n=n, nu=0.0, dt=1e-3) as s:
        s.set_state(a)
        b = s.get_state()
    k = wavenumbers(n)
    KX, KY, KZ = np.meshgrid(k, k, np.arange(n // 2 + 1), indexing="ij")
    keep = 3 * np.maximum(np.maximum(abs(KX), abs(KY)), KZ) < n
    assert np.array_equal(b[:, keep], a[:, keep])
    assert np.all(b[:, ~keep] == 0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_diagnostics_and_series_match_oracle(ns, prec):
    run = dict(n=32, nu=0.01, dt=1e-3, force_amp=0.5, force_k=3)
    a0 = inputs.turbulence_state(32, seed=9)
    with _solver(ns, prec, **run) as s:
        s.set_state(a0)
        s.step(4)
        E, Om, spec = s.energy_spectrum()
        Es, Os = s.series(count=10)
        st = s.get_state()
    tol = 1e-13 if prec == "fp64" else 1e-6
    rE, rO, rspec = oracle.diagnostics(st)
    assert abs(E - rE) < tol * rE and abs(Om - rO) < tol * rO
    assert np.abs(spec - rspec).max() < tol * rE
    assert len(Es) == 4
    ref = a0
    for i in range(4):
        ref = _oracle_run(ref, run, 1)
        e_i, o_i, _ = oracle.diagnostics(ref)
        assert abs(Es[i] - e_i) < 20 * TOL[prec] * e_i
        assert abs(Os[i] - o_i) < 20 * TOL[prec] * o_i


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_repeated_runs_are_bitwise_identical(ns, prec):
    run = dict(n=64, nu=0.01, dt=1e-3, force_amp=0.5, force_k=3)
    a0 = inputs.turbulence_state(64, seed=2)
    outs = []
    for _ in range(2):
        with _solver(ns, prec, **run) as s:
            s.set_state(a0)
            s.step(3)
            outs.append((s.get_state(), s.energy_spectrum()))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][1][0] == outs[1][1][0] and np.array_equal(outs[0][1][2], outs[1][1][2])


def test_taylor_green_256_against_oracle_on_the_64_sublattice(ns):
    """Config 2's flow at full size (256^3, nu = 1/1600, dt = 2e-3): the GPU
    FP64 state after 2 steps against the oracle, compared on the grid points
    of the 64^3 sub-lattice (every 4th point), and the initial invariants."""
    import torch
    n, steps = 256, 2
    run = dict(n=n, nu=1 / 1600, dt=2e-3)
    a0 = inputs.taylor_green_state(n)
    with _solver(ns, "fp64", **run) as s:
        s.set_state(a0)
        E0, Om0, _ = s.energy_spectrum()
        s.step(steps)
        got = s.get_state()
    assert abs(E0 - 0.125) < 1e-15 and abs(Om0 - 0.375) < 1e-14
    ref = _oracle_run(a0, run, steps)
    ug = np.fft.irfftn(got, s=(n, n, n), axes=(1, 2, 3))[:, ::4, ::4, ::4]
    ur = np.fft.irfftn(ref, s=(n, n, n), axes=(1, 2, 3))[:, ::4, ::4, ::4]
    assert np.linalg.norm(ug - ur) / np.linalg.norm(ur) < TOL["fp64"]
    assert rel_l2(got, ref) < TOL["fp64"]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_non_finite_state_is_reported(ns, prec):
    from paper_1003_4322_gb300 import _native as nat
    n = 16
    a = inputs.turbulence_state(n, seed=1)
    a[0, 1, 1, 1] = np.nan
    with _solver(ns, prec, n=n, nu=0.01, dt=1e-3) as s:
        s.set_state(a)
        s.step(1)
        with pytest.raises(nat.NsError) as ei:
            s.sync()
        assert ei.value.status == nat.NS_ERR_NONFINITE


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_resume_from_saved_state_is_bitwise_equal(ns, prec):
    run = dict(n=48, nu=0.01, dt=1e-3, force_amp=0.5, force_k=3)
    a0 = inputs.turbulence_state(48, seed=6)
    with _solver(ns, prec, **run) as s:
        s.set_state(a0)
        s.step(4)
        straight = s.get_state()
    with _solver(ns, prec, **run) as s:
        s.set_state(a0)
        s.step(2)
        saved = s.get_state()
    with _solver(ns, prec, **run) as s:
        s.set_state(saved)
        s.step(2)
        resumed = s.get_state()
    assert np.array_equal(resumed, straight)


def test_allocation_failure_is_reported_and_cleaned_up(ns):
    """Forty 768^3 plain-FP64 runs need far more than the GPU's memory: ns_init
    must return NS_ERR_OOM (no fault), free what it took, and later contexts
    must work."""
    from paper_1003_4322_gb300 import _native as nat
    import torch
    free0, _ = torch.cuda.mem_get_info()
    with pytest.raises(nat.NsError) as ei:
        nat.ns_init([dict(n=768, nu=1e-3, dt=1e-3)] * 40, nat.NS_FP64)
    assert ei.value.status == nat.NS_ERR_OOM
    free1, _ = torch.cuda.mem_get_info()
    assert free1 > free0 - (1 << 30)
    with _solver(ns, "fp64", n=16, nu=0.01, dt=1e-3) as s:
        s.set_state(inputs.abc_state(16))
        s.step(1)
        s.sync()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_helicity_matches_oracle(ns, prec):
    n = 48
    a0 = inputs.turbulence_state(n, seed=13)
    with _solver(ns, prec, n=n, nu=0.01, dt=1e-3, force_amp=0.5, force_k=3) as s:
        s.set_state(a0)
        s.step(2)
        H, spec = s.helicity()
        st = s.get_state()
    rH, rspec = oracle.helicity(st)
    scale = np.abs(rspec).sum()
    tol = 1e-13 if prec == "fp64" else 1e-6
    assert abs(H - rH) < tol * scale
    assert np.abs(spec - rspec).max() < tol * scale
    with _solver(ns, prec, n=32, nu=0.0, dt=1e-3) as s:
        s.set_state(inputs.abc_state(32))
        H, spec = s.helicity()
    assert abs(H - 1.5) < (1e-14 if prec == "fp64" else 1e-6)


@pytest.mark.parametrize("n", [64, 256])
def test_fused_series_accumulation_is_fp64_quality(ns, n):
    """The fused form's per-step (E, Omega) come from compensated FP32 partial
    sums inside the update kernel; against an FP64 sum of the very state the
    step stored they agree to ~1e-12 (a plain FP32 running sum would be off by
    ~1e-7)."""
    run = dict(n=n, nu=2e-3, dt=1e-3, force_amp=0.5, force_k=3)
    with _solver(ns, "fp32", **run) as s:
        s.set_state(inputs.turbulence_state(n, seed=3))
        s.step(2)
        Es, Os = s.series(count=10)
        E, Om, _ = s.energy_spectrum()
        st = s.get_state() if n <= 64 else None
    assert abs(Es[-1] - E) < 1e-12 * E and abs(Os[-1] - Om) < 1e-12 * Om
    if st is not None:
        rE, rO, _ = oracle.diagnostics(st)
        assert abs(Es[-1] - rE) < 1e-12 * rE and abs(Os[-1] - rO) < 1e-12 * rO


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [32, 48])
def test_rotating_turbulence_matches_oracle(ns, prec, n):
    """Forced turbulence in a frame rotating about z (Coriolis -2 rot z x u
    inside the projected nonlinear term), both forms against the oracle."""
    run = dict(n=n, nu=0.01, dt=1e-3, force_amp=0.5, force_k=3, rot=3.0)
    a0 = inputs.turbulence_state(n, seed=17)
    ref = _oracle_run(a0, run, 4)
    with _solver(ns, prec, **run) as s:
        s.set_state(a0)
        s.step(4)
        got = s.get_state()
    assert rel_l2(got, ref) < TOL[prec]
    assert rel_l2(ref, _oracle_run(a0, dict(run, rot=0.0), 4)) > 100 * TOL["fp32"]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_inertial_wave_exact_on_gpu(ns, prec):
    """One helical mode turns at the inertial frequency 2 rot kz/|k| with the
    exact discrete IF-Heun amplification (the oracle's pin, on the GPU)."""
    n, nu, dt, rot, steps = 32, 0.01, 0.01, 2.5, 20
    k = (2, 1, 3)
    a0 = helical_mode(n, k, 1)
    kk = np.linalg.norm(k)
    z = 2j * rot * k[2] / kk * dt
    g = np.exp(-nu * kk ** 2 * dt) * (1 + z + z * z / 2)
    with _solver(ns, prec, n=n, nu=nu, dt=dt, rot=rot) as s:
        s.set_state(a0)
        s.step(steps)
        got = s.get_state()
    want = a0 * g ** steps
    assert np.abs(got - want).max() < (1e-14 if prec == "fp64" else 1e-6)


def test_rotation_is_per_run_in_a_group(ns):
    """Two runs of one size in one fused group, rotating and not: one launch
    per pass advances both, each with its own rotation rate."""
    from paper_1003_4322_gb300.solver import Solver
    n = 32
    runs = [dict(n=n, nu=0.01, dt=1e-3, rot=4.0), dict(n=n, nu=0.01, dt=1e-3)]
    a0 = inputs.turbulence_state(n, seed=23)
    with Solver(runs, prec="fp32") as s:
        for r in range(2):
            s.set_state(a0, run=r)
        s.step(3)
        got = [s.get_state(run=r) for r in range(2)]
    for r in range(2):
        assert rel_l2(got[r], _oracle_run(a0, runs[r], 3)) < TOL["fp32"]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [16, 24, 48])
def test_phase_shift_dealiasing_matches_oracle(ns, prec, n):
    """dealias = 2: the product on the grid and on the grid shifted by
    (pi/N)(1,1,1), averaged, sphere 9|k|^2 < 2 N^2 (the plain form in both
    precisions), against the oracle, with a start that fills that sphere."""
    from paper_1003_4322_gb300 import _native as nat
    run = dict(n=n, nu=0.01, dt=1e-3, force_amp=0.5, force_k=3, dealias=2)
    a0 = inputs.random_solenoidal_state(n, 1.0, 0.47 * n, 0.7, seed=n + 1, dealias=2)
    ref = _oracle_run(a0, run, 3)
    with _solver(ns, prec, **run) as s:
        assert nat.ns_describe_run(s.ctx, 0)["form"].startswith("plain")
        s.set_state(a0)
        s.step(3)
        got = s.get_state()
    assert rel_l2(got, ref) < TOL[prec]
    # and it differs from the cubic 2/3 rule on the same start
    assert rel_l2(ref, _oracle_run(a0, dict(run, dealias=0), 3)) > 100 * TOL["fp32"]


def test_phase_shift_with_mhd_is_rejected(ns):
    from paper_1003_4322_gb300 import _native as nat
    from paper_1003_4322_gb300.solver import Solver
    with pytest.raises(nat.NsError) as e:
        Solver([dict(n=16, nu=0.01, eta=0.01, dt=1e-3, mhd=1, dealias=2)], prec="fp64")
    assert e.value.status == nat.NS_ERR_ARG


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_page_locked_host_buffers_match_pageable(ns, prec):
    """ns_set_state / ns_get_state read and write page-locked host memory
    directly (no staging copies), every element of the output (filled with
    NaN first). The results equal the staged path's bit for bit, for the
    velocity and the magnetic field of an MHD run, on cubes, every
    dealiasing rule and a grid of another shape."""
    import torch
    from paper_1003_4322_gb300.solver import Solver
    for run, mhd in ((dict(n=64, nu=0.01, dt=1e-3, force_amp=0.5, force_k=3), False),
                     (dict(n=192, nu=0.01, dt=1e-3, dealias=1), False),
                     (dict(n=36, nu=0.01, dt=1e-3, dealias=2), False),
                     (dict(n=32, nu=0.01, eta=0.02, dt=1e-3, mhd=1), True),
                     (dict(n=32, ny=48, nz=24, lz=2.0, nu=0.01, dt=1e-3), False)):
        dims = (run["n"], run.get("ny", run["n"]), run.get("nz", run["n"]))
        a0 = inputs.random_solenoidal_grid(dims, (1.0, 1.0, run.get("lz", 1.0)), 0.5, 4.0, 1.0, seed=3)
        outs = []
        for pinned in (False, True):
            with Solver([run], prec=prec) as s:
                if pinned:
                    buf = torch.empty(a0.shape, dtype=torch.complex128, pin_memory=True)
                    buf.numpy()[...] = a0
                    src = buf.numpy()
                else:
                    src = a0.copy()
                s.set_state(src)
                if mhd:
                    s.set_field(1, src)
                src[...] = 0          # the call was synchronous: the buffer may be reused
                s.step(2)
                if pinned:
                    o = torch.empty(a0.shape, dtype=torch.complex128, pin_memory=True).numpy()
                    ob = torch.empty(a0.shape, dtype=torch.complex128, pin_memory=True).numpy()
                else:
                    o, ob = np.empty_like(a0), np.empty_like(a0)
                o[...] = np.nan
                ob[...] = np.nan
                s.get_state(out=o)
                if mhd:
                    s.get_field(1, out=ob)
                outs.append((o.copy(), ob.copy() if mhd else None))
        assert np.array_equal(outs[0][0], outs[1][0])
        if mhd:
            assert np.array_equal(outs[0][1], outs[1][1])
        assert np.abs(outs[1][0]).max() > 0
