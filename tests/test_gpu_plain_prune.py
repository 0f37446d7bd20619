"""The plain form's transforms skip the lines that the dealiasing rule leaves
zero (inverse passes) or whose result it discards (forward passes): the x
lines with |ky| > K_y or kz > K_z, the y lines with kz > K_z, the rows beyond
K_x (x) and K_y (y), and the z entries kz > K_z (Sec. 2: the 2/3 rule, or
the run's spherical or phase-shift rule).  Every skipped line is one that
the unpruned step either fills with zeros or throws away, so the state after
a few steps is the same bit for bit as with every line transformed
(NS_PLAIN_PRUNE=0), for every rule, MHD, rotation and grid, in both
precisions on the runtime-length kernels."""
import numpy as np
import pytest

from paper_1003_4322_gb300 import inputs

pytestmark = pytest.mark.gpu

CASES = [
    ("fp64", dict(n=32, nu=2e-3, dt=1e-3, force_amp=0.5, force_k=3)),
    ("fp64", dict(n=48, nu=2e-3, dt=1e-3, dealias=1, rot=1.5)),
    ("fp64", dict(n=36, nu=5e-3, dt=1e-3, dealias=2, force_amp=0.3, force_k=2)),
    ("fp64", dict(n=24, nu=0.02, eta=0.03, dt=2e-3, mhd=1)),
    ("fp64", dict(n=24, ny=16, nz=12, lx=1.5, ly=1.0, lz=0.75, nu=0.01, dt=2e-3, rot=1.5, dealias=1)),
    ("fp64", dict(n=12, ny=36, nz=24, nu=0.02, dt=2e-3, force_amp=0.5, force_k=3, dealias=2)),
    ("fp32", dict(n=12, ny=36, nz=24, nu=0.02, dt=2e-3, force_amp=0.5, force_k=3, dealias=2)),
    ("fp32", dict(n=16, ny=12, nz=24, lx=1.0, ly=0.75, lz=1.5, nu=0.02, eta=0.03, dt=2e-3, mhd=1)),
]


def _state(run, seed):
    dims = (run["n"], run.get("ny", 0) or run["n"], run.get("nz", 0) or run["n"])
    box = tuple(run.get(k, 0.0) or 1.0 for k in ("lx", "ly", "lz"))
    a = inputs.random_solenoidal_grid(dims, box, 0.5, 4.0, 1.0, seed=seed, dealias=run.get("dealias", 0))
    if run.get("mhd"):
        a = np.concatenate([a, inputs.random_solenoidal_grid(dims, box, 0.5, 3.0, 0.6, seed=seed + 1)])
    return a


def _run(run, prec, a0, steps):
    from paper_1003_4322_gb300 import _native as nat
    from paper_1003_4322_gb300.solver import Solver
    with Solver([run], prec=prec) as s:
        assert nat.ns_describe_run(s.ctx, 0)["form"].startswith("plain")
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
    return got, (E, Om, spec)


@pytest.mark.parametrize("i", range(len(CASES)))
def test_pruned_step_is_bitwise_the_full_step(ns, i, monkeypatch):
    prec, run = CASES[i]
    a0 = _state(run, seed=300 + i)
    monkeypatch.setenv("NS_PLAIN_PRUNE", "0")
    full, dfull = _run(run, prec, a0, 3)
    monkeypatch.delenv("NS_PLAIN_PRUNE")
    pruned, dpruned = _run(run, prec, a0, 3)
    assert np.abs(full).max() > 0
    assert np.array_equal(full, pruned), np.abs(full - pruned).max()
    assert dfull[0] == dpruned[0] and dfull[1] == dpruned[1]
    assert np.array_equal(dfull[2], dpruned[2])
