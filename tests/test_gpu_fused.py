"""The fused, pruned FP32 form (NS_FP32) at the benchmark sizes, where the
oracle is too slow to run step by step: against the plain FP64 form on the
same GPU (itself pinned to the oracle), and against properties that hold at
any size."""
import math

import numpy as np
import pytest

from paper_1003_4322_gb300 import inputs
from tests.spectral_ref import rel_l2, wavenumbers

pytestmark = pytest.mark.gpu


def _run(prec, run, a0, steps):
    from paper_1003_4322_gb300.solver import Solver
    with Solver([run], prec=prec) as s:
        s.set_state(a0)
        s.step(steps)
        return s.get_state(), s.energy_spectrum()


@pytest.mark.parametrize("n", [128, 256])
def test_fused_matches_plain_fp64_mid_sizes(ns, n):
    run = dict(n=n, nu=2e-3, dt=1e-3, force_amp=0.5, force_k=3)
    a0 = inputs.turbulence_state(n, seed=3)
    b32, d32 = _run("fp32", run, a0, 5)
    b64, d64 = _run("fp64", run, a0, 5)
    assert rel_l2(b32, b64) < 2e-5
    assert abs(d32[0] - d64[0]) < 2e-5 * d64[0]


def test_config3_512_fused_fp32_vs_plain_fp64(ns):
    """512^3 forced turbulence (nu = 2e-3, dt = 1e-3, ABC forcing k = 3,
    F = 0.5, seeded k^-2 start on 1 <= |k| <= 4): FP32 fused within 2e-5 of
    the plain FP64 form after 3 steps."""
    n = 512
    run = dict(n=n, nu=2e-3, dt=1e-3, force_amp=0.5, force_k=3)
    a0 = inputs.turbulence_state(n, seed=3)
    b32, _ = _run("fp32", run, a0, 3)
    b64, _ = _run("fp64", run, a0, 3)
    assert rel_l2(b32, b64) < 2e-5


def test_1024_beltrami_decay_and_forced_energy(ns):
    """At 1024^3: exact Beltrami decay, and a forced turbulent step that stays
    finite and changes the energy by a small amount."""
    from paper_1003_4322_gb300.solver import Solver
    n, nu, dt, steps = 1024, 5e-4, 5e-4, 4
    with Solver([dict(n=n, nu=nu, dt=dt)], prec="fp32") as s:
        s.set_state(inputs.abc_state(n))
        s.step(steps)
        E, Om, spec = s.energy_spectrum()
    want = 1.5 * math.exp(-2 * nu * dt * steps)
    assert abs(E - want) < 5e-6 and abs(Om - want) < 5e-6
    with Solver([dict(n=n, nu=nu, dt=dt, force_amp=0.5, force_k=3)], prec="fp32") as s:
        s.set_state(inputs.turbulence_state(n, seed=5))
        E0, O0, _ = s.energy_spectrum()
        s.step(1)
        E1, O1, _ = s.energy_spectrum()
    assert np.isfinite(E1) and np.isfinite(O1)
    assert abs(E1 - E0) < 1e-2 * E0
