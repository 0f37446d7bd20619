"""Guard bands around every device buffer of the library (NS_GUARD=1): after
steps of both forms (Navier-Stokes, rotation, MHD, ensembles of uneven
sizes, a size with no compiled fused MHD kernel, grids and boxes other than
the cube) and the standalone transforms, no kernel has written outside its
buffers.  Runs in a child
process, since the guard mode is fixed at the library's first allocation."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = textwrap.dedent("""
    import numpy as np, torch
    from paper_1003_4322_gb300 import _native as nat, inputs
    from paper_1003_4322_gb300.solver import Solver
    assert nat.ns_guard_selftest() == 1
    for prec in ("fp64", "fp32"):
        for n in (32, 48, 64, 96):
            with Solver([dict(n=n, nu=0.01, dt=1e-3, force_amp=0.5, force_k=3, rot=1.0)], prec=prec) as s:
                s.set_state(inputs.turbulence_state(n, seed=1))
                s.step(2)
                s.get_state(); s.energy_spectrum(); s.helicity()
        for n in (32, 48):
            with Solver([dict(n=n, nu=0.01, eta=0.02, dt=1e-3, mhd=1)] * 2, prec=prec) as s:
                for r in range(2):
                    s.set_field(0, inputs.turbulence_state(n, seed=2), run=r)
                    s.set_field(1, inputs.turbulence_state(n, seed=3), run=r)
                s.step(2)
                s.get_field(1); s.field_spectrum(1)
        runs = [dict(n=n, nu=0.01, dt=1e-3) for n in (64, 96, 64, 128)]
        with Solver(runs, prec=prec) as s:
            for r, q in enumerate(runs):
                s.set_state(inputs.turbulence_state(q["n"], seed=4 + r), run=r)
            s.step(2)
        for grid in (dict(n=16, ny=24, nz=36, lx=1.0, ly=1.5, lz=3.0, dealias=2),
                     dict(n=24, ny=16, nz=8, lz=0.5, force_amp=0.5, force_k=2, dealias=1, rot=1.0)):
            dims = (grid["n"], grid["ny"], grid["nz"])
            box = tuple(grid.get(k, 1.0) for k in ("lx", "ly", "lz"))
            with Solver([dict(nu=0.01, dt=1e-3, **grid)], prec=prec) as s:
                s.set_state(inputs.random_solenoidal_grid(dims, box, 0.5, 3.0, 1.0, 6, grid["dealias"]))
                s.step(2)
                s.get_state(); s.energy_spectrum(); s.helicity()
            with Solver([dict(nu=0.01, eta=0.02, dt=1e-3, mhd=1, n=16, ny=12, nz=24, ly=0.75)],
                        prec=prec) as s:
                s.set_field(1, inputs.random_solenoidal_grid((16, 12, 24), (1, 0.75, 1), 0.5, 3.0, 1.0, 7))
                s.step(2)
                s.field_spectrum(1)
            rt = torch.float64 if prec == "fp64" else torch.float32
            ct = torch.complex128 if prec == "fp64" else torch.complex64
            for d in (dims, (64, 96, 128)):
                u = torch.randn((3,) + d, device="cuda", dtype=rt)
                uh = torch.empty((3, d[0], d[1], d[2] // 2 + 1), device="cuda", dtype=ct)
                with Solver([dict(n=8, dt=1e-3)], prec=prec) as s:
                    s.fft_r2c_grid(u, uh)
                    s.fft_c2r_grid(uh, u)
        for n in (48, 64):
            rt = torch.float64 if prec == "fp64" else torch.float32
            ct = torch.complex128 if prec == "fp64" else torch.complex64
            u = torch.randn((3, n, n, n), device="cuda", dtype=rt)
            uh = torch.empty((3, n, n, n // 2 + 1), device="cuda", dtype=ct)
            with Solver([dict(n=8, dt=1e-3)], prec=prec) as s:
                s.fft_r2c(u, uh)
                s.fft_c2r(uh, u)
    torch.cuda.synchronize()
    print("BAD", nat.ns_guard_check())
""")


def test_no_kernel_writes_outside_its_buffers(ns):
    env = dict(os.environ, NS_GUARD="1")
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    bad = [l for l in r.stdout.splitlines() if l.startswith("BAD")]
    assert bad and bad[-1] == "BAD 0", r.stdout[-2000:]
