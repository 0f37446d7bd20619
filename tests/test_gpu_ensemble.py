"""Ensembles: independent runs of uneven grid sizes in one context (runs of
the same N are advanced together by one launch per pass).  Every member must
equal the same run done alone, bit for bit, and match the oracle."""
import numpy as np
import pytest

import oracle
from paper_1003_4322_gb300 import inputs
from tests.spectral_ref import rel_l2

pytestmark = pytest.mark.gpu


def _members():
    runs, ics = [], []
    for r, n in enumerate([32, 48, 32, 24, 48, 32]):
        runs.append(dict(n=n, nu=inputs.ensemble_nu(r), dt=1e-3,
                         force_amp=0.5 if r % 2 else 0.0, force_k=3 if r % 2 else 0,
                         dealias=r % 3 == 2 and 1 or 0))
        ics.append(inputs.random_solenoidal_state(n, 1.0, 4.0, 1.0, 4000 + r,
                                                  dealias=runs[-1]["dealias"]))
    return runs, ics


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_ensemble_members_equal_single_runs_and_oracle(ns, prec):
    from paper_1003_4322_gb300.solver import Solver
    runs, ics = _members()
    steps = 3
    with Solver(runs, prec=prec) as s:
        for i, a in enumerate(ics):
            s.set_state(a, run=i)
        s.step(steps)
        got = [s.get_state(run=i) for i in range(len(runs))]
        series = [s.series(run=i, count=steps) for i in range(len(runs))]
    tol = 1e-12 if prec == "fp64" else 2e-5
    for i, (run, a0) in enumerate(zip(runs, ics)):
        with Solver([run], prec=prec) as s1:
            s1.set_state(a0)
            s1.step(steps)
            alone = s1.get_state()
        assert np.array_equal(got[i], alone), f"member {i} differs from its single run"
        ref = oracle.step(a0, oracle.Params(n=run["n"], nu=run["nu"], dt=run["dt"],
                                            force_amp=run["force_amp"], force_k=run["force_k"],
                                            dealias=run["dealias"]), steps)
        assert rel_l2(got[i], ref) < tol
        assert len(series[i][0]) == steps
        assert abs(series[i][0][-1] - oracle.diagnostics(ref)[0]) < 20 * tol * series[i][0][-1]


def test_config4_ensemble_shapes(ns):
    """The 48-member ensemble of config 4 (16 runs each at 64^3, 96^3 and
    128^3, FP32) initialises, steps and stays finite; one member of each size
    matches its single run, and every member stays within the FP32 tolerance
    of the plain FP64 ensemble (itself pinned to the oracle member by member
    at smaller sizes)."""
    from paper_1003_4322_gb300.solver import Solver
    runs, ics = [], []
    for r in range(48):
        n = (64, 96, 128)[r // 16]
        runs.append(dict(n=n, nu=inputs.ensemble_nu(r), dt=1e-3))
        ics.append(inputs.turbulence_state(n, 4000 + r))
    steps = 2
    with Solver(runs, prec="fp32") as s:
        s.set_states(ics)
        s.step(steps)
        fp32 = [s.get_state(run=i) for i in range(48)]
        energies = [s.energy_spectrum(run=i)[0] for i in range(48)]
    assert all(np.isfinite(energies))
    for i in (3, 20, 40):
        with Solver([runs[i]], prec="fp32") as s1:
            s1.set_state(ics[i])
            s1.step(steps)
            assert np.array_equal(fp32[i], s1.get_state())
    with Solver(runs, prec="fp64") as s:
        s.set_states(ics)
        s.step(steps)
        errs = [rel_l2(fp32[i], s.get_state(run=i)) for i in range(48)]
    assert max(errs) < 2e-5, max(errs)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batched_state_and_spectra_calls_match_per_run_calls(ns, prec):
    """ns_set_states and ns_energy_spectra (one synchronisation for all runs)
    give bit for bit what ns_set_state and ns_energy_spectrum give run by run,
    from page-locked and from pageable host buffers."""
    import torch
    from paper_1003_4322_gb300.solver import Solver
    runs = [dict(n=n, nu=0.01, dt=1e-3) for n in (32, 48, 32, 64)]
    starts = [inputs.turbulence_state(r["n"], seed=70 + i) for i, r in enumerate(runs)]
    with Solver(runs, prec=prec) as s:
        for i, a in enumerate(starts):
            s.set_state(a, run=i)
        s.step(2)
        one = [s.get_state(run=i) for i in range(len(runs))]
        diag = [s.energy_spectrum(run=i) for i in range(len(runs))]
    for pinned in (False, True):
        if pinned:
            hosts = []
            for a in starts:
                t = torch.empty(a.shape, dtype=torch.complex128, pin_memory=True)
                t.numpy()[...] = a
                hosts.append(t.numpy())
        else:
            hosts = [a.copy() for a in starts]
        with Solver(runs, prec=prec) as s:
            s.set_states(hosts)
            for h in hosts:
                h[...] = 0
            s.step(2)
            E, O, spec = s.energy_spectra()
            for i in range(len(runs)):
                assert np.array_equal(s.get_state(run=i), one[i])
        for i, (e, om, sp) in enumerate(diag):
            assert E[i] == e and O[i] == om
            assert np.array_equal(spec[i, :len(sp)], sp) and not spec[i, len(sp):].any()


def test_batched_calls_reject_bad_ranges_and_null_buffers(ns):
    """Argument errors of ns_set_states / ns_energy_spectra come back as
    NS_ERR_ARG before any device work, and leave the context usable."""
    import ctypes

    from paper_1003_4322_gb300 import _native as nat
    from paper_1003_4322_gb300.solver import Solver
    runs = [dict(n=16, nu=0.01, dt=1e-3), dict(n=24, nu=0.02, dt=1e-3)]
    starts = [inputs.turbulence_state(r["n"], seed=90 + i) for i, r in enumerate(runs)]
    lib = nat.load()
    with Solver(runs, prec="fp64") as s:
        good = [a.ctypes.data for a in starts]
        P2 = ctypes.c_void_p * 2
        assert lib.ns_set_states(s.ctx, 1, 2, P2(*good), 0) == nat.NS_ERR_ARG     # past the last run
        assert lib.ns_set_states(s.ctx, -1, 1, P2(*good), 0) == nat.NS_ERR_ARG
        assert lib.ns_set_states(s.ctx, 0, 0, P2(*good), 0) == nat.NS_ERR_ARG
        assert lib.ns_set_states(s.ctx, 0, 2, P2(good[0], None), 0) == nat.NS_ERR_ARG
        assert lib.ns_set_states(s.ctx, 0, 2, None, 0) == nat.NS_ERR_ARG
        spec = np.zeros((3, 40))
        sp = spec.ctypes.data_as(ctypes.c_void_p)
        assert lib.ns_energy_spectra(s.ctx, 0, 3, sp, 40, None, None) == nat.NS_ERR_ARG
        assert lib.ns_energy_spectra(s.ctx, 2, 1, sp, 40, None, None) == nat.NS_ERR_ARG
        assert lib.ns_energy_spectra(s.ctx, 0, 1, None, 40, None, None) == nat.NS_ERR_ARG
        # the context still works, and nbins = 0 with no spectrum buffer is allowed
        s.set_states(starts)
        s.step(1)
        E, O, _ = s.energy_spectra()
        e0, o0, _ = s.energy_spectrum(run=0)
        assert E[0] == e0 and O[0] == o0 and np.all(np.isfinite(E))
        E2 = (ctypes.c_double * 2)()
        assert lib.ns_energy_spectra(s.ctx, 0, 2, None, 0, E2, None) == nat.NS_OK
        assert list(E2) == list(E)
