"""The oracle's pins must catch plausible mistakes.  Each case below plants
one mistake in a private copy of the oracle source (on the CPU), compiles it,
and requires that at least one pin of a fast battery fails on it, while the
unmodified source passes every pin."""
import ctypes
import math
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from paper_1003_4322_gb300 import inputs
from tests.spectral_ref import helical_mode, rel_l2, triad_mhd, triad_nonlinear

SRC = open(os.path.join(os.path.dirname(oracle.__file__), "ns_oracle.c")).read()

MUTATIONS = {
    "cross product order (w x u)":
        ("c[i] = u[V + i] * w[2 * V + i] - u[2 * V + i] * w[V + i];",
         "c[i] = w[V + i] * u[2 * V + i] - w[2 * V + i] * u[V + i];"),
    "curl sign":
        ("w[m] = I * (ky * az - kz * ay);", "w[m] = I * (kz * ay - ky * az);"),
    "projection sign":
        ("v[m] -= kx * kv / k2;", "v[m] += kx * kv / k2;"),
    "2/3 rule replaced by 1/2 rule":
        ("if (3 * mm >= g->n[i]) cube_ok = 0;", "if (2 * mm >= g->n[i]) cube_ok = 0;"),
    "missing 1/N^3 on the nonlinear term":
        ("for (long i = 0; i < 3 * M; i++) out[i] /= (double)V;", ""),
    "Heun second-stage weight dropped":
        ("a[i] = 0.5 * Ei * a[i] + 0.5 * (a1[i] + p->dt * N0[i]);",
         "a[i] = 0.5 * Ei * a[i] + (a1[i] + p->dt * N0[i]);"),
    "integrating factor outside the Euler stage":
        ("a1[i] = Ei * (a[i] + p->dt * N0[i]);", "a1[i] = Ei * a[i] + p->dt * N0[i];"),
    "half viscous factor":
        ("exp(-p->nu * k2 * p->dt);", "exp(-0.5 * p->nu * k2 * p->dt);"),
    "forcing sin/cos swapped":
        ("f[i] = F * (sin(kf * z) + cos(kf * y));", "f[i] = F * (cos(kf * z) + sin(kf * y));"),
    "twiddle sign":
        ("w[t] = cos(a) + I * (sign * sin(a));", "w[t] = cos(a) - I * (sign * sin(a));"),
    "Hermitian completion without conjugate":
        ("v = conj(h[(((nx - x) % nx) * ny + (ny - y) % ny) * nh + (nz - z)]);",
         "v = h[(((nx - x) % nx) * ny + (ny - y) % ny) * nh + (nz - z)];"),
    "energy weight 2 on every plane":
        ("double w = (mi[2] == 0 || 2 * mi[2] == g->n[2]) ? 1.0 : 2.0;", "double w = 2.0;"),
    "shell binning by truncation":
        ("long K = (long)floor(sqrt(k2) * lmax + 0.5);", "long K = (long)floor(sqrt(k2) * lmax);"),
    "Coriolis sign of one component":
        ("out[i] += 2.0 * p->rot * a[M + i];", "out[i] -= 2.0 * p->rot * a[M + i];"),
    "Coriolis without the factor 2":
        ("out[i] += 2.0 * p->rot * a[M + i];\n        out[M + i] -= 2.0 * p->rot * a[i];",
         "out[i] += p->rot * a[M + i];\n        out[M + i] -= p->rot * a[i];"),
    "Lorentz force j x b written b x j (x component)":
        ("+ j[V + i] * b[2 * V + i] - j[2 * V + i] * b[V + i];",
         "+ b[V + i] * j[2 * V + i] - b[2 * V + i] * j[V + i];"),
    "electromotive force written b x u (x component)":
        ("c[3 * V + i] = u[V + i] * b[2 * V + i] - u[2 * V + i] * b[V + i];",
         "c[3 * V + i] = b[V + i] * u[2 * V + i] - b[2 * V + i] * u[V + i];"),
    "induction term without the curl":
        ("curl_g(&g, tb, out + 3 * M);", "memcpy(out + 3 * M, tb, sizeof(cplx) * 3 * (size_t)M);"),
    "magnetic field diffused with nu":
        ("E[M + m] = exp(-p->eta * k2 * p->dt);", "E[M + m] = exp(-p->nu * k2 * p->dt);"),
    "phase shift: shifted evaluation dropped":
        ("    if (p->dealias == 2) {                           /* and on the shifted grid */",
         "    if (0) {"),
    "phase shift: shifted back with the same sign":
        ("        phase_shift(&g, -1, o2);", "        phase_shift(&g, +1, o2);"),
    "Coriolis added after the projection":
        ("    project_g(&g, p->dealias, out);                  /* Pi, then P */\n",
         "    for (long i = 0; i < M; i++) {\n        out[i] -= 2.0 * p->rot * a[M + i];\n"
         "        out[M + i] += 2.0 * p->rot * a[i];\n    }\n"
         "    project_g(&g, p->dealias, out);\n"
         "    for (long i = 0; i < M; i++) {\n        out[i] += 2.0 * p->rot * a[M + i];\n"
         "        out[M + i] -= 2.0 * p->rot * a[i];\n    }\n"),
    # grids of N_x x N_y x N_z points on boxes of sides 2 pi l_i
    "wavenumber m * l instead of m / l":
        ("for (int i = 0; i < 3; i++) k[i] = mi[i] / g->l[i];",
         "for (int i = 0; i < 3; i++) k[i] = mi[i] * g->l[i];"),
    "forcing sampled without the box side along z":
        ("z = OR_TWO_PI * g.l[2] * iz / nz;", "z = OR_TWO_PI * iz / nz;"),
    "2/3 rule of N_x applied to every axis":
        ("if (3 * mm >= g->n[i]) cube_ok = 0;", "if (3 * mm >= g->n[0]) cube_ok = 0;"),
    "ellipsoid scaled by N_x on every axis":
        ("const long q = mm * (D / g->n[i]);", "const long q = mm * (D / g->n[0]);"),
    "phase shift with the x spacing along z":
        ("(double)mi[2] / g->n[2]", "(double)mi[2] / g->n[0]"),
    "shells one unit wide on every box":
        ("    const double lmax = 1.0 / kmin_of(g);\n    double e = 0.0, om = 0.0;",
         "    const double lmax = 1.0;\n    double e = 0.0, om = 0.0;"),
    "Nyquist plane weight from N_x":
        ("double w = (mi[2] == 0 || 2 * mi[2] == g->n[2]) ? 1.0 : 2.0;",
         "double w = (mi[2] == 0 || 2 * mi[2] == g->n[0]) ? 1.0 : 2.0;"),
}


def _pins():
    """A fast battery of independent pins; returns the names that fail."""
    failed = []
    # FFT against numpy
    u = inputs.random_real(12, 1, 0)[0]
    if np.abs(oracle.fft3_r2c(u) - np.fft.rfftn(u)).max() > 1e-9:
        failed.append("r2c")
    a = inputs.random_hermitian_half(12, 1, 1)[0]
    if np.abs(oracle.fft3_c2r(a) - np.fft.irfftn(a, s=(12, 12, 12), axes=(0, 1, 2)) * 12 ** 3).max() > 1e-9:
        failed.append("c2r")
    # nonlinear term against the triad sum
    s = inputs.random_solenoidal_state(8, 1.0, 4.0, 0.7, seed=8)
    if np.abs(oracle.nonlinear(s, oracle.Params(n=8)) - triad_nonlinear(s)).max() > 1e-12:
        failed.append("triad")
    # forcing closed form (one coefficient)
    fh = oracle.forcing(oracle.Params(n=16, force_amp=0.5, force_k=3))
    if abs(fh[0, 0, 0, 3] - 0.5 / 2j) > 1e-14:
        failed.append("forcing")
    # exact ABC decay
    b = oracle.step(inputs.abc_state(16), oracle.Params(n=16, nu=0.01, dt=0.05), 4)
    if abs(oracle.diagnostics(b)[0] - 1.5 * math.exp(-2 * 0.01 * 0.2)) > 1e-13:
        failed.append("abc")
    # second-order convergence on a nonlinear case (Richardson ratio)
    a0 = inputs.random_solenoidal_state(8, 1.0, 3.5, 1.5, seed=21)
    res = [oracle.step(a0, oracle.Params(n=8, nu=0.05, dt=0.2 / k), k) for k in (10, 20, 40)]
    ratio = rel_l2(res[0], res[1]) / rel_l2(res[1], res[2])
    if not 3.6 < ratio < 4.4:
        failed.append("order")
    # diagnostics: Parseval and shell of k = (3, 4, 0)
    t = inputs.turbulence_state(16, 4, rms=0.8)
    if abs(oracle.diagnostics(t)[0] - 1.5 * 0.64) > 1e-13:
        failed.append("parseval")
    c = np.zeros_like(t)
    c[2, 3, 4, 0] = c[2, 13, 12, 0] = 0.5
    if abs(oracle.diagnostics(c)[2][5] - 0.25) > 1e-15:
        failed.append("shell")
    if abs(oracle.diagnostics(inputs.taylor_green_state(8))[2][2] - 0.125) > 1e-15:
        failed.append("shell-round")     # |k| = sqrt3 rounds to shell 2
    # rotation: one helical mode is an inertial wave of frequency 2 rot kz/|k|
    h = helical_mode(8, (1, 1, 2), 1)
    z = 2j * 2.0 * 2 / math.sqrt(6) * 0.02
    g = math.exp(-0.01 * 6 * 0.02) * (1 + z + z * z / 2)
    if np.abs(oracle.step(h, oracle.Params(n=8, nu=0.01, dt=0.02, rot=2.0), 5) - h * g ** 5).max() > 1e-14:
        failed.append("inertial")
    # rotation leaves z-independent flows alone (Taylor-Proudman)
    q = inputs.random_solenoidal_state(8, 1.0, 3.0, 0.5, seed=5)
    q[..., 1:] = 0.0
    q0 = oracle.step(q, oracle.Params(n=8, nu=0.01, dt=0.02), 3)
    q1 = oracle.step(q, oracle.Params(n=8, nu=0.01, dt=0.02, rot=3.0), 3)
    if np.abs(q1 - q0).max() > 1e-13 * np.abs(q0).max():
        failed.append("taylor-proudman")
    # phase-shift dealiasing: exact triad sum on the sphere 9|k|^2 < 2 n^2
    ps = inputs.random_solenoidal_state(8, 1.0, 3.7, 0.7, seed=12, dealias=2)
    if np.abs(oracle.nonlinear(ps, oracle.Params(n=8, dealias=2)) - triad_nonlinear(ps, 2)).max() > 1e-12:
        failed.append("phase-shift-triad")
    # MHD: exact triad sums, and the force-free field's decay with eta
    mh = np.concatenate([inputs.random_solenoidal_state(8, 1.0, 2.7, 0.6, seed=31),
                         inputs.random_solenoidal_state(8, 1.0, 2.7, 0.5, seed=32)])
    if np.abs(oracle.nonlinear(mh, oracle.Params(n=8, mhd=1)) - triad_mhd(mh)).max() > 1e-12:
        failed.append("mhd-triad")
    ff = np.concatenate([np.zeros_like(inputs.abc_state(8)), inputs.abc_state(8)])
    fb = oracle.step(ff, oracle.Params(n=8, nu=0.01, eta=0.03, dt=0.05, mhd=1), 4)
    if np.abs(fb[3:] - ff[3:] * math.exp(-0.03 * 0.2)).max() > 1e-14:
        failed.append("force-free")
    # grids and boxes of other aspect ratios
    gp = dict(n=8, ny=12, nz=6, lx=1.0, ly=1.5, lz=0.75)
    ug = inputs.random_real_grid((6, 8, 4), 1, 3)[0]
    if np.abs(oracle.fft3_r2c(ug) - np.fft.rfftn(ug)).max() > 1e-9:
        failed.append("r2c-grid")
    for d in (0, 1, 2):
        ag = inputs.random_solenoidal_grid((8, 12, 6), (1.0, 1.5, 0.75), 0.5, 6.0, 0.8, seed=17, dealias=d)
        if np.abs(oracle.nonlinear(ag, oracle.Params(dealias=d, **gp)) - triad_nonlinear(ag, d, (1.0, 1.5, 0.75))).max() > 1e-12:
            failed.append(f"triad-grid-{d}")
    fg = oracle.forcing(oracle.Params(n=8, ny=16, nz=8, lx=1.0, ly=2.0, lz=0.5, force_amp=0.5, force_k=2))
    if abs(fg[0, 0, 0, 1] - 0.5 / 2j) > 1e-14 or abs(fg[0, 0, 4, 0] - 0.25) > 1e-14:
        failed.append("forcing-grid")
    pb = oracle.Params(n=8, ny=8, nz=16, lz=2.0)
    sg = np.zeros(pb.half_shape(), dtype=np.complex128)
    sg[0, 1, 0, 1] = 0.5
    sg[2, 0, 0, 4] = 1.0
    eg, _, spg = oracle.diagnostics(sg, pb)
    if abs(spg[2] - 0.25) > 1e-16 or abs(spg[4] - 1.0) > 1e-16 or abs(eg - 1.25) > 1e-16:
        failed.append("shell-grid")
    ce = inputs.random_solenoidal_state(12, 1.0, 3.5, 0.8, seed=23)
    kw = dict(nu=0.02, dt=0.01, force_amp=0.4, force_k=2, rot=0.7)
    ref = oracle.step(ce, oracle.Params(n=12, **kw), 2)
    emb = np.zeros((3, 24, 12, 19), dtype=np.complex128)
    m = np.fft.fftfreq(12, 1.0 / 12).astype(int)
    ix, iy, iz = (2 * m) % 24, m % 12, 3 * np.arange(7)
    emb[:, ix[:, None, None], iy[None, :, None], iz[None, None, :]] = ce
    got = oracle.step(emb, oracle.Params(n=24, ny=12, nz=36, lx=2.0, ly=1.0, lz=3.0, **kw), 2)
    if rel_l2(got[:, ix[:, None, None], iy[None, :, None], iz[None, None, :]], ref) > 1e-14:
        failed.append("embedding")
    return failed


def _with_source(src: str):
    d = tempfile.mkdtemp(prefix="oracle_mut_")
    c = os.path.join(d, "m.c")
    so = os.path.join(d, "m.so")
    with open(c, "w") as f:
        f.write(src)
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", c, "-o", so, "-lm"],
                   check=True)
    saved = oracle._lib
    oracle._lib = None
    real = oracle.build
    oracle.build = lambda force=False: so
    try:
        return _pins()
    finally:
        oracle.build = real
        oracle._lib = saved


def test_unmodified_oracle_passes_battery():
    assert _pins() == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name):
    old, new = MUTATIONS[name]
    assert SRC.count(old) == 1, "mutation anchor not found"
    failed = _with_source(SRC.replace(old, new))
    assert failed, f"no pin caught: {name}"
