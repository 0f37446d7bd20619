"""GPU parity of the standalone 3D transforms (ns_fft_r2c / ns_fft_c2r,
Sec. 2, Fig. 1) against the FP64 oracle, called through the C ABI.

Tolerances: FP64 relative L2 <= 1e-13.  FP32: inputs are rounded to float
first (the oracle gets the same rounded values), and a radix-R Stockham FFT
with correctly rounded twiddles has relative RMS error of order
eps32 * sqrt(log2 N^3) ~ 6e-8 * 5.5 = 3.3e-7 at N = 1024; the bound used is
2e-6 (six-fold margin)."""
import math

import numpy as np
import pytest

import oracle
from paper_1003_4322_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-13, "fp32": 2e-6}


def _ctx(ns, prec):
    return ns.ns_init([dict(n=8, dt=1e-3)], ns.NS_FP64 if prec == "fp64" else ns.NS_FP32)


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _types(prec):
    import torch
    return (torch.float64, torch.complex128) if prec == "fp64" else (torch.float32, torch.complex64)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [8, 12, 16, 24, 32, 48, 64, 96, 128])
def test_r2c_matches_oracle(ns, prec, n):
    import torch
    rt, ct = _types(prec)
    ncomp = 3 if n <= 64 else 1
    u = inputs.random_real(n, ncomp, 100 + n)
    ud = torch.from_numpy(u).to("cuda", rt)
    ref = oracle.fft3_r2c(ud.double().cpu().numpy())
    out = torch.empty((ncomp, n, n, n // 2 + 1), dtype=ct, device="cuda")
    ctx = _ctx(ns, prec)
    try:
        ns.ns_fft_r2c(ctx, n, ncomp, ud, out)
        ns.ns_sync(ctx)
    finally:
        ns.ns_destroy(ctx)
    assert _rel(out.cpu().numpy().astype(np.complex128), ref) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [8, 12, 16, 24, 32, 48, 64, 96, 128])
def test_c2r_matches_oracle(ns, prec, n):
    import torch
    rt, ct = _types(prec)
    ncomp = 2 if n <= 64 else 1
    a = inputs.random_hermitian_half(n, ncomp, 7 + n)
    ad = torch.from_numpy(a).to("cuda", ct)
    a_in = ad.cpu().numpy().astype(np.complex128)
    ref = oracle.fft3_c2r(a_in)
    out = torch.empty((ncomp, n, n, n), dtype=rt, device="cuda")
    ctx = _ctx(ns, prec)
    try:
        ns.ns_fft_c2r(ctx, n, ncomp, ad, out)
        ns.ns_sync(ctx)
    finally:
        ns.ns_destroy(ctx)
    assert _rel(out.cpu().numpy().astype(np.float64), ref) < TOL[prec]
    assert torch.equal(ad.cpu(), torch.from_numpy(a).to(ct)), "c2r modified its input"


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_256_matches_oracle(ns, prec):
    import torch
    n = 256
    rt, ct = _types(prec)
    u = inputs.random_real(n, 1, 5)
    ud = torch.from_numpy(u).to("cuda", rt)
    ref = oracle.fft3_r2c(ud.double().cpu().numpy())
    out = torch.empty((1, n, n, n // 2 + 1), dtype=ct, device="cuda")
    back = torch.empty((1, n, n, n), dtype=rt, device="cuda")
    ctx = _ctx(ns, prec)
    try:
        ns.ns_fft_r2c(ctx, n, 1, ud, out)
        ns.ns_fft_c2r(ctx, n, 1, out, back)
        ns.ns_sync(ctx)
    finally:
        ns.ns_destroy(ctx)
    assert _rel(out.cpu().numpy().astype(np.complex128), ref) < TOL[prec]
    assert _rel(back.cpu().numpy() / n ** 3, ud.cpu().numpy()) < 2 * TOL[prec]


def _plane_waves(n, waves, dtype):
    """sum_j A_j cos(k_j . x + phi_j) on the grid, built in torch on the GPU."""
    import torch
    g = torch.arange(n, device="cuda", dtype=torch.float64) * (2 * math.pi / n)
    X, Y, Z = g.view(n, 1, 1), g.view(1, n, 1), g.view(1, 1, n)
    u = torch.zeros((n, n, n), device="cuda", dtype=torch.float64)
    for (kx, ky, kz), A, phi in waves:
        u += A * torch.cos(kx * X + ky * Y + kz * Z + phi)
    return u.to(dtype)


@pytest.mark.parametrize("n,prec", [(512, "fp32"), (1024, "fp32"), (512, "fp64"), (768, "fp64"),
                                    (1024, "fp64")])
def test_full_size_plane_waves_and_round_trip(ns, n, prec):
    """At the benchmark sizes: exact peaks of known plane waves, zero
    elsewhere, and c2r(r2c(u)) = N^3 u (properties that hold at any size)."""
    import torch
    rt, ct = _types(prec)
    rng = np.random.default_rng(n)
    waves = []
    for _ in range(6):
        k = tuple(int(v) for v in rng.integers(-n // 2 + 1, n // 2, size=3))
        k = (k[0], k[1], abs(k[2]) if k[2] != 0 else 1)
        waves.append((k, float(rng.uniform(0.5, 2.0)), float(rng.uniform(0, 2 * math.pi))))
    u = _plane_waves(n, waves, rt)
    out = torch.empty((1, n, n, n // 2 + 1), dtype=ct, device="cuda")
    back = torch.empty((1, n, n, n), dtype=rt, device="cuda")
    ctx = _ctx(ns, prec)
    try:
        ns.ns_fft_r2c(ctx, n, 1, u, out)
        ns.ns_sync(ctx)
        peak_tol = (1e-6 if prec == "fp32" else 1e-11) * n ** 3
        for (kx, ky, kz), A, phi in waves:
            got = complex(out[0, kx % n, ky % n, kz].cpu())
            want = 0.5 * A * n ** 3 * complex(math.cos(phi), math.sin(phi))
            assert abs(got - want) < peak_tol + 2e-6 * abs(want) * (prec == "fp32")
            out[0, kx % n, ky % n, kz] = 0
        resid = out.abs().max().item() / n ** 3
        assert resid < (5e-6 if prec == "fp32" else 1e-12)
        # round trip on the original field
        ns.ns_fft_r2c(ctx, n, 1, u, out)
        ns.ns_fft_c2r(ctx, n, 1, out, back)
        ns.ns_sync(ctx)
        err = ((back.double() / n ** 3 - u.double()).norm() / u.double().norm()).item()
        assert err < 2 * TOL[prec] * 5
    finally:
        ns.ns_destroy(ctx)


def test_sizes_in_any_order_fp64(ns):
    """Launch sizes that need different amounts of shared memory, larger
    after smaller after larger, in one process (regression: the dynamic
    shared-memory opt-in of a kernel must cover every size it is used at)."""
    import torch
    for n in (32, 24, 32, 96, 24, 32):
        a = inputs.random_hermitian_half(n, 1, n)
        ad = torch.from_numpy(a).cuda()
        out = torch.empty((1, n, n, n), dtype=torch.float64, device="cuda")
        ctx = _ctx(ns, "fp64")
        try:
            ns.ns_fft_c2r(ctx, n, 1, ad, out)
            ns.ns_sync(ctx)
        finally:
            ns.ns_destroy(ctx)
        assert _rel(out.cpu().numpy(), oracle.fft3_c2r(a)) < TOL["fp64"]


@pytest.mark.parametrize("n,prec", [(512, "fp32"), (1024, "fp32"), (512, "fp64"), (768, "fp64"),
                                    (1024, "fp64")])
def test_full_size_random_input_sampled_dft(ns, n, prec):
    """At the benchmark sizes, a random input: sampled output modes against
    the DFT written out on the host in FP64 (the sum over z for two kz in one
    pass, then the sums over y and x per mode).  Tolerance relative to the
    RMS coefficient magnitude sqrt(N^3) * rms(u)."""
    import torch
    rt, ct = _types(prec)
    g = torch.Generator(device="cuda").manual_seed(n + 11)
    u = (torch.rand((n, n, n), device="cuda", dtype=torch.float32, generator=g) - 0.5).to(rt)
    out = torch.empty((1, n, n, n // 2 + 1), dtype=ct, device="cuda")
    ctx = _ctx(ns, prec)
    try:
        ns.ns_fft_r2c(ctx, n, 1, u, out)
        ns.ns_sync(ctx)
    finally:
        ns.ns_destroy(ctx)
    host = u.double().cpu().numpy().reshape(n * n, n)
    del u
    kzs = (1, n // 2 - 3)
    z = np.arange(n)
    # phases from k x mod N, so that the exponentials see arguments below 2 pi
    Ez = np.stack([np.exp(-2j * np.pi * ((kz * z) % n) / n) for kz in kzs], axis=1)   # (n, 2)
    S = host @ np.concatenate([Ez.real, Ez.imag], axis=1)                          # one pass
    S = (S[:, :2] + 1j * S[:, 2:]).reshape(n, n, 2)                                # [x, y, kz]
    scale = math.sqrt(n ** 3) * float(np.sqrt(np.mean(host ** 2)))
    del host
    rng = np.random.default_rng(n)
    x = np.arange(n)
    tol = (2e-6 if prec == "fp32" else 1e-13) * scale
    for i, kz in enumerate(kzs):
        for _ in range(4):
            kx, ky = (int(v) for v in rng.integers(0, n, size=2))
            want = (np.exp(-2j * np.pi * ((kx * x) % n) / n) @ S[:, :, i]
                    @ np.exp(-2j * np.pi * ((ky * x) % n) / n))
            got = complex(out[0, kx, ky, kz].cpu())
            assert abs(got - want) < tol, (kx, ky, kz, got, want, tol)
