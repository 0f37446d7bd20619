"""Long parity runs, opt-in (NS_LONG_TESTS=1): minutes of oracle time on the
host, or a GPU run of about 155 GB.

* 256^3 decaying Taylor-Green vortex (nu = 1/1600, dt = 2e-3), 200 RK2 steps
  of the plain FP64 GPU form against the FP64 CPU oracle (Sec. 2, Eqs. 1-2):
  relative L2 distance of the velocity on the 64^3 sub-lattice (every 4th
  grid point), of the spectral state, and of E and Omega after 50, 100, 150
  and 200 steps;
* 1024^3 forced turbulence, 20 steps of the fused FP32 form against the
  plain FP64 form."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1003_4322_gb300 import inputs
from tests.spectral_ref import rel_l2

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not os.environ.get("NS_LONG_TESTS"),
                                 reason="long oracle run; set NS_LONG_TESTS=1")]


def test_tg256_200_steps_against_oracle(ns):
    from paper_1003_4322_gb300.solver import Solver
    n, nu, dt = 256, 1 / 1600, 2e-3
    oracle.set_threads(os.cpu_count() or 1)
    p = oracle.Params(n=n, nu=nu, dt=dt)
    a0 = inputs.taylor_green_state(n)
    ref = a0
    rows = []
    with Solver([dict(n=n, nu=nu, dt=dt)], prec="fp64") as s:
        s.set_state(a0)
        for k in range(4):
            s.step(50)
            got = s.get_state()
            ref = oracle.step(ref, p, 50)
            ug = oracle.fft3_c2r(got)[:, ::4, ::4, ::4]
            ur = oracle.fft3_c2r(ref)[:, ::4, ::4, ::4]
            sub = math.sqrt(float(np.sum((ug - ur) ** 2)) / float(np.sum(ur ** 2)))
            Eg, Og, _ = s.energy_spectrum()
            Er, Or, _ = oracle.diagnostics(ref)
            rows.append((50 * (k + 1), sub, rel_l2(got, ref), abs(Eg - Er) / Er, abs(Og - Or) / Or))
    for step, sub, spec, dE, dO in rows:
        print(f"step {step}: sub-lattice rel-L2 {sub:.3e}, spectral rel-L2 {spec:.3e}, "
              f"dE/E {dE:.3e}, dOmega/Omega {dO:.3e}")
        assert sub < 1e-12 and spec < 1e-12 and dE < 1e-12 and dO < 1e-12


def _weighted_rel_l2_device(got, ref, planes=64):
    """rel-L2 of two device half-layout states (weights 2, and 1 on the kz = 0
    and kz = N/2 planes), accumulated in FP64 over slabs of x planes."""
    num = den = 0.0
    for c in range(got.shape[0]):
        for x0 in range(0, got.shape[1], planes):
            d = (got[c, x0:x0 + planes] - ref[c, x0:x0 + planes]).abs().square()
            r = ref[c, x0:x0 + planes].abs().square()
            num += 2 * d.sum().item() - d[..., 0].sum().item() - d[..., -1].sum().item()
            den += 2 * r.sum().item() - r[..., 0].sum().item() - r[..., -1].sum().item()
    return math.sqrt(num / den)


def test_forced1024_fp32_against_fp64_gpu(ns):
    """The 1024^3 forced-turbulence configuration (nu = 5e-4, dt = 5e-4, ABC
    forcing k = 3, F = 0.5, seeded k^-2 start on 1 <= |k| <= 4, seed 5):
    20 RK2 steps of the fused FP32 form against the plain FP64 form, which
    the oracle pins at smaller sizes.  Both states stay on the device (the
    plain FP64 run alone holds about 155 GB); the distance is the weighted
    rel-L2 of the spectral states."""
    import torch
    from paper_1003_4322_gb300.solver import Solver
    n, steps = 1024, 20
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
            s.step(1)                       # the first call captures the step's graph
            s.sync()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(stream)
            s.step(steps - 1)
            ev[1].record(stream)
            s.sync()
            ms = ev[0].elapsed_time(ev[1]) / (steps - 1)
            E, Om, _ = s.energy_spectrum()
            res = torch.empty(s.half_shape(), dtype=torch.complex128, device="cuda")
            s.get_state(out=res)
            s.sync()
        out[prec] = (res, ms, E, Om)
        print(f"1024^3 {prec}: {ms:.2f} ms/step ({1e3 / ms:.3f} steps/s), E {E:.9e}, Omega {Om:.9e}")
    err = _weighted_rel_l2_device(out["fp32"][0], out["fp64"][0])
    dE = abs(out["fp32"][2] - out["fp64"][2]) / out["fp64"][2]
    print(f"1024^3 after {steps} steps: rel-L2 FP32 vs FP64 {err:.3e}, |dE|/E {dE:.3e}")
    assert err < 2e-5 and dE < 2e-5
