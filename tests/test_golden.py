"""The stored fixtures of tests/golden/ (oracle outputs written by
tests/golden/make_golden.py; the paper prints no worked example of the
solver): the oracle reproduces them (CPU), and so do the GPU forms through
the C ABI (plain FP64 to 1e-12, FP32 to the FP32 tolerance)."""
import os

import numpy as np
import pytest

import oracle
from paper_1003_4322_gb300 import inputs

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(HERE, name)) as f:
        return [l.split() for l in f if l.strip() and not l.startswith("#")]


def _config1():
    rows = _rows("config1_32.txt")
    series = np.array([[float(x) for x in r] for r in rows[:10]])
    modes = [(tuple(int(x) for x in r[:4]), complex(float(r[4]), float(r[5]))) for r in rows[10:]]
    return series, modes


def _box():
    return np.array([[float(x) for x in r] for r in _rows("box_12x18x24.txt")])


BOX = dict(n=12, ny=18, nz=24, lx=1.0, ly=1.5, lz=2.0, nu=0.02, dt=2e-3, force_amp=0.5, force_k=2,
           rot=0.8)


def _box_start():
    return inputs.random_solenoidal_grid((12, 18, 24), (1.0, 1.5, 2.0), 0.5, 3.0, 1.0, seed=9)


def test_oracle_reproduces_config1_fixture():
    series, modes = _config1()
    p = oracle.Params(n=32, nu=0.01, dt=1e-3)
    a = inputs.config1_state(32, seed=1)
    for i in range(10):
        a = oracle.step(a, p, 1)
        e, om, _ = oracle.diagnostics(a)
        assert abs(e - series[i, 0]) <= 1e-14 * series[i, 0]
        assert abs(om - series[i, 1]) <= 1e-14 * series[i, 1]
    for (c, x, y, z), v in modes:
        assert abs(a[c, x, y, z] - v) <= 1e-14
    assert modes[1][1] == 0    # u_y at k = (0, 1, 0): k . u = 0


def test_oracle_reproduces_box_fixture():
    want = _box()
    p = oracle.Params(**BOX)
    a = _box_start()
    for i in range(5):
        a = oracle.step(a, p, 1)
        e, om, _ = oracle.diagnostics(a, p)
        h, _ = oracle.helicity(a, p)
        assert np.allclose([e, om, h], want[i], rtol=1e-14, atol=0)


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_gpu_reproduces_fixtures(ns, prec, tol):
    from paper_1003_4322_gb300.solver import Solver
    series, modes = _config1()
    with Solver([dict(n=32, nu=0.01, dt=1e-3)], prec=prec) as s:
        s.set_state(inputs.config1_state(32, seed=1))
        s.step(10)
        E, O = s.series(count=10)
        a = s.get_state()
    assert np.allclose(E, series[:, 0], rtol=tol, atol=0) and np.allclose(O, series[:, 1], rtol=tol, atol=0)
    scale = max(abs(v) for _, v in modes)
    for (c, x, y, z), v in modes:
        assert abs(a[c, x, y, z] - v) <= tol * scale
    want = _box()
    with Solver([BOX], prec=prec) as s:
        s.set_state(_box_start())
        s.step(5)
        E, O = s.series(count=5)
        H, _ = s.helicity()
    assert np.allclose(E, want[:, 0], rtol=tol, atol=0) and np.allclose(O, want[:, 1], rtol=tol, atol=0)
    assert abs(H - want[-1, 2]) <= tol * abs(want[-1, 2]) * 10
