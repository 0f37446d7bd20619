"""Parity at the benchmark configurations, in the default GPU suite (short
runs; the long ones are opt-in in test_gpu_long.py):

* 256^3 decaying Taylor-Green vortex (nu = 1/1600, dt = 2e-3): a few RK2
  steps of both forms against the FP64 CPU oracle (Sec. 2, Eqs. 1-2), on the
  whole spectral state, on the velocity at the 64^3 sub-lattice (every 4th
  grid point), and in E and Omega;
* the 48-run ensemble (16 runs each at 64^3, 96^3 and 128^3): two members of
  each size against the oracle, in both precisions;
* 512^3 forced turbulence (the benchmark's headline configuration): one RK2
  step of both forms against the oracle on the whole state (about a minute
  of oracle time on the host cores);
* 1024^3 forced turbulence: the fused FP32 form (its N = 1024 pass kernels)
  against the plain FP64 form after a few steps, on the whole state.

Every FP32 comparison also bounds the error shell by shell
(tests.spectral_ref.shell_error_ratios)."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1003_4322_gb300 import inputs
from tests.spectral_ref import rel_l2, shell_error_ratios, shell_error_ratios_device

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-5}


def _sub_lattice_rel(got, ref, stride):
    ug = oracle.fft3_c2r(got)[:, ::stride, ::stride, ::stride]
    ur = oracle.fft3_c2r(ref)[:, ::stride, ::stride, ::stride]
    return math.sqrt(float(np.sum((ug - ur) ** 2)) / float(np.sum(ur ** 2)))


def test_tg256_short_against_oracle(ns):
    from paper_1003_4322_gb300.solver import Solver
    n, nu, dt, steps = 256, 1 / 1600, 2e-3, 4
    oracle.set_threads(os.cpu_count() or 1)
    a0 = inputs.taylor_green_state(n)
    ref = oracle.step(a0, oracle.Params(n=n, nu=nu, dt=dt), steps)
    Er, Or, _ = oracle.diagnostics(ref)
    for prec in ("fp64", "fp32"):
        with Solver([dict(n=n, nu=nu, dt=dt)], prec=prec) as s:
            s.set_state(a0)
            s.step(steps)
            got = s.get_state()
            Eg, Og, _ = s.energy_spectrum()
        tol = TOL[prec]
        spec, sub = rel_l2(got, ref), _sub_lattice_rel(got, ref, n // 64)
        dE, dO = abs(Eg - Er) / Er, abs(Og - Or) / Or
        print(f"TG 256^3 {prec} after {steps} steps: spectral {spec:.2e}, 64^3 sub-lattice "
              f"{sub:.2e}, dE/E {dE:.2e}, dOmega/Omega {dO:.2e}")
        assert spec < tol and sub < tol and dE < tol and dO < tol
        if prec == "fp32":
            assert shell_error_ratios(got, ref).max() < tol


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_config4_members_against_oracle(ns, prec):
    from paper_1003_4322_gb300.solver import Solver
    runs, ics = [], []
    for r in range(48):
        n = (64, 96, 128)[r // 16]
        runs.append(dict(n=n, nu=inputs.ensemble_nu(r), dt=1e-3))
        ics.append(inputs.turbulence_state(n, 4000 + r))
    steps = 3
    picked = (0, 11, 16, 29, 32, 47)
    with Solver(runs, prec=prec) as s:
        s.set_states(ics)
        s.step(steps)
        got = {i: s.get_state(run=i) for i in picked}
    oracle.set_threads(os.cpu_count() or 1)
    for i in picked:
        r = runs[i]
        ref = oracle.step(ics[i], oracle.Params(n=r["n"], nu=r["nu"], dt=r["dt"]), steps)
        err = rel_l2(got[i], ref)
        print(f"member {i} ({r['n']}^3, nu {r['nu']:.4f}) {prec}: rel-L2 vs oracle {err:.2e}")
        assert err < TOL[prec]
        if prec == "fp32":
            assert shell_error_ratios(got[i], ref).max() < TOL[prec]


def test_forced512_one_step_against_oracle(ns):
    """The 512^3 forced-turbulence configuration (nu = 2e-3, dt = 1e-3, ABC
    forcing k = 3, F = 0.5, seeded k^-2 start on 1 <= |k| <= 4), one RK2 step
    of the plain FP64 and the fused FP32 form against the oracle on the whole
    state (about a minute of oracle time on the host cores)."""
    from paper_1003_4322_gb300.solver import Solver
    n = 512
    run = dict(n=n, nu=2e-3, dt=1e-3, force_amp=0.5, force_k=3)
    oracle.set_threads(os.cpu_count() or 1)
    a0 = inputs.turbulence_state(n, seed=3)
    ref = oracle.step(a0, oracle.Params(n=n, nu=2e-3, dt=1e-3, force_amp=0.5, force_k=3), 1)
    for prec, tol in (("fp64", 1e-12), ("fp32", 2e-5)):
        with Solver([run], prec=prec) as s:
            s.set_state(a0)
            s.step(1)
            got = s.get_state()
        err = rel_l2(got, ref)
        print(f"512^3 {prec}: rel-L2 vs oracle after one step {err:.3e}")
        assert err < tol
        if prec == "fp32":
            assert shell_error_ratios(got, ref).max() < tol


def test_forced1024_fused_fp32_against_plain_fp64_short(ns):
    """Config 5's grid and parameters (nu = 5e-4, dt = 5e-4, ABC forcing
    k = 3, F = 0.5, seeded k^-2 start): two RK2 steps of each form; both
    states stay on the device (the plain FP64 run holds about 155 GB)."""
    import torch
    from paper_1003_4322_gb300.solver import Solver
    n, steps = 1024, 2
    run = dict(n=n, nu=5e-4, dt=5e-4, force_amp=0.5, force_k=3)
    stream = torch.cuda.current_stream()
    a0 = torch.from_numpy(inputs.turbulence_state(n, seed=5)).cuda()
    out = {}
    for prec in ("fp32", "fp64"):
        with Solver([run], prec=prec, stream=stream) as s:
            s.set_state(a0)
            if prec == "fp64":
                del a0
                torch.cuda.empty_cache()
            s.step(steps)
            E, Om, _ = s.energy_spectrum()
            res = torch.empty(s.half_shape(), dtype=torch.complex128, device="cuda")
            s.get_state(out=res)
            s.sync()
            desc = ns.ns_describe_run(s.ctx, 0)
        out[prec] = (res, E)
        if prec == "fp32":
            assert desc["form"] == "fused FP32" and desc["n"] == 1024
    got, ref = out["fp32"][0], out["fp64"][0]
    num = den = 0.0
    for c in range(3):
        for x0 in range(0, n, 64):
            d = (got[c, x0:x0 + 64] - ref[c, x0:x0 + 64]).abs().square()
            r = ref[c, x0:x0 + 64].abs().square()
            num += 2 * d.sum().item() - d[..., 0].sum().item() - d[..., -1].sum().item()
            den += 2 * r.sum().item() - r[..., 0].sum().item() - r[..., -1].sum().item()
    err = math.sqrt(num / den)
    dE = abs(out["fp32"][1] - out["fp64"][1]) / out["fp64"][1]
    ratios = shell_error_ratios_device(got, ref)
    print(f"1024^3 after {steps} steps: rel-L2 FP32 vs FP64 {err:.3e}, |dE|/E {dE:.3e}, "
          f"worst shell ratio {ratios.max():.3e}")
    # the forced, advanced state is not the start: the step did work
    assert err < TOL["fp32"] and dE < TOL["fp32"] and ratios.max() < TOL["fp32"]
    assert err > 0.0
