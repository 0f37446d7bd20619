"""The benchmark's algorithmic byte model, against the arrays each kernel
reads and writes (sized here with numpy, independently of the model's
formulas), and the roofline arithmetic on a synthetic census."""
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _sizes(dims, prec):
    nx, ny, nz = dims
    ct = np.complex128 if prec == "fp64" else np.complex64
    rt = np.float64 if prec == "fp64" else np.float32
    half = np.empty((3, nx, ny, nz // 2 + 1), dtype=ct).nbytes   # one 3-vector, half layout
    real = np.empty((3, nx, ny, nz), dtype=rt).nbytes           # one 3-vector on the grid
    return half, real


def _kept_cubic(dims):
    """Modes of the half layout inside the cubic 2/3 rule, counted one by one."""
    nx, ny, nz = dims
    mx = [m if 2 * m < nx else m - nx for m in range(nx)]
    my = [m if 2 * m < ny else m - ny for m in range(ny)]
    cx = sum(1 for m in mx if 3 * abs(m) < nx)
    cy = sum(1 for m in my if 3 * abs(m) < ny)
    cz = sum(1 for m in range(nz // 2 + 1) if 3 * m < nz)
    return cx * cy * cz


@pytest.mark.parametrize("dims", [(64, 64, 64), (96, 96, 96), (256, 256, 256), (48, 64, 96)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_plain_kernel_bytes_are_the_arrays_they_move(dims, prec):
    half, real = _sizes(dims, prec)
    n = dims if len(set(dims)) > 1 else dims[0]
    want = {
        "fft_x_inverse": 2 * half, "fft_x_forward": 2 * half,     # read and write in place
        "fft_y_inverse": 2 * half, "fft_y_forward": 2 * half,
        "fft_z_c2r": half + real, "fft_z_r2c": half + real,
        "fft_c2r_std": (half + real) + 4 * half, "fft_r2c_std": (half + real) + 4 * half,
        "curl": 2 * half,                                          # read a, write w
        "cross": 3 * real,                                         # read u, w; write u x w
        "cross_mhd": 6 * real,                                     # read u, w, b, j; write 2
    }
    for name, b in want.items():
        got, flops = bench.kernel_model(name, n, prec)
        assert got == b, (name, got, b)
        assert flops > 0
    # the update writes every mode of three components and reads the
    # product, the state and (at stage 2) the stage-1 state at the kept modes
    cb = half // (3 * dims[0] * dims[1] * (dims[2] // 2 + 1))
    got, _ = bench.kernel_model("update", n, prec)
    assert got == (3 * dims[0] * dims[1] * (dims[2] // 2 + 1) + 7.5 * _kept_cubic(dims)) * cb


@pytest.mark.parametrize("n", [64, 96, 128, 256, 512])
def test_fused_pass_bytes_follow_the_pruned_shapes(n):
    """Passes of the fused FP32 form move complex64 fields of the pruned
    shapes: the compact state [3][2K+1][2K+1][K+1], pass A/D fields
    [.][2K+1][N][K+1], pass B/C fields [.][N][N][K+1], K the largest kept
    wavenumber (3K < N)."""
    K = max(k for k in range(n) if 3 * k < n)
    c64 = np.dtype(np.complex64).itemsize
    S = (2 * K + 1) ** 2 * (K + 1)
    Ax = (2 * K + 1) * n * (K + 1)
    Bx = n * n * (K + 1)
    want = {
        "fused_A_x_inverse_curl": 3 * S + 6 * Ax,   # reads a, writes u and w
        "fused_B_y_inverse": 6 * Ax + 6 * Bx,
        "fused_C_z_nonlinear": 6 * Bx + 3 * Bx,     # reads u, w; writes u x w transformed
        "fused_D_y_forward": 3 * Bx + 3 * Ax,
        "fused_E_x_forward": 3 * Ax + 3 * S,
    }
    for name, modes in want.items():
        got, _ = bench.kernel_model(name, n, "fp32")
        assert got == modes * c64, (name, got, modes * c64)


@pytest.mark.parametrize("dims", [(512, 512, 256), (64, 96, 128), (48, 24, 36)])
def test_fused_pass_bytes_on_grids(dims):
    """On a grid of N_x x N_y x N_z points the kept wavenumbers are per axis,
    K_i the largest with 3 K_i < N_i: the compact state [3][2K_x+1][2K_y+1][K_z+1],
    pass A/D fields [.][2K_y+1][N_x][K_z+1], pass B/C fields [.][N_y][N_x][K_z+1].
    The transforms run along x in passes A and E (2K_y+1 by K_z+1 columns)
    and along y in B and D (N_x by K_z+1 columns)."""
    nx, ny, nz = dims
    Kx, Ky, Kz = ((m - 1) // 3 for m in dims)
    assert all(3 * k < m <= 3 * k + 3 for k, m in zip((Kx, Ky, Kz), dims))
    c64 = np.dtype(np.complex64).itemsize
    S = (2 * Kx + 1) * (2 * Ky + 1) * (Kz + 1)
    Ax = (2 * Ky + 1) * nx * (Kz + 1)
    Bx = ny * nx * (Kz + 1)
    want = {
        "fused_A_x_inverse_curl": (3 * S + 6 * Ax, 6 * (2 * Ky + 1) * (Kz + 1), nx),
        "fused_B_y_inverse": (6 * Ax + 6 * Bx, 6 * nx * (Kz + 1), ny),
        "fused_D_y_forward": (3 * Bx + 3 * Ax, 3 * nx * (Kz + 1), ny),
        "fused_E_x_forward": (3 * Ax + 3 * S, 3 * (2 * Ky + 1) * (Kz + 1), nx),
        "fused_C_z_nonlinear": (9 * Bx, None, None),
    }
    for name, (modes, lines, length) in want.items():
        got, flops = bench.kernel_model(name, dims, "fp32")
        assert got == modes * c64, (name, got, modes * c64)
        if lines is not None:   # 5 L log2 L per complex line of length L
            assert flops == pytest.approx(lines * 5 * length * np.log2(length)), name
    # the 512 x 512 x 256 box: K = (170, 170, 85), pass C moves 1,623,195,648 bytes
    if dims == (512, 512, 256):
        assert (Kx, Ky, Kz) == (170, 170, 85)
        assert bench.kernel_model("fused_C_z_nonlinear", dims, "fp32")[0] == 1623195648


def test_roofline_arithmetic_on_a_synthetic_census():
    peaks = {"hbm_gbs": 6000.0, "sm_max_mhz": 2000.0, "source": "measured"}
    w = {"n": 256, "name": "none"}
    # FP64 z c2r: flop-bound by its model; achieved = flops / time, frac = achieved / peak
    census = [("fft_z_c2r", 4, 8.0), ("curl", 2, 1.0)]
    roof, total = bench.roofline_of(census, w, "fp64", 2, peaks, None)
    assert total == 9.0 and roof["kernel"] == "fft_z_c2r" and roof["launches_per_step"] == 2
    _, flops = bench.kernel_model("fft_z_c2r", 256, "fp64")
    assert roof["bound"] == "alu"
    assert math.isclose(roof["achieved"], flops / 2e-3 / 1e12)
    assert math.isclose(roof["peak"], 152 * 4.0 * 2000e6 / 1e12)
    assert math.isclose(roof["frac"], roof["achieved"] / roof["peak"])
    # FP32 fused pass: HBM-bound; achieved = bytes / time against the HBM peak
    census = [("fused_C_z_nonlinear", 2, 1.0)]
    roof, _ = bench.roofline_of(census, w, "fp32", 1, peaks, None)
    b, _ = bench.kernel_model("fused_C_z_nonlinear", 256, "fp32")
    assert roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    assert math.isclose(roof["achieved"], b / 0.5e-3 / 1e9)
    assert math.isclose(roof["frac"], roof["achieved"] / 6000.0)


def _kept_rule(m, dims, dealias):
    """The dealiasing rule on one index vector m (grid indices), written out:
    3 |m_i| < N_i on every axis (and the sphere sum (3 m_i / N_i)^2 < 1 for
    rule 1); rule 2: 2 |m_i| < N_i and sum (3 m_i / N_i)^2 < 2."""
    r = sum((3 * mi / ni) ** 2 for mi, ni in zip(m, dims))
    if dealias == 2:
        return all(2 * abs(mi) < ni for mi, ni in zip(m, dims)) and r < 2
    return all(3 * abs(mi) < ni for mi, ni in zip(m, dims)) and (dealias != 1 or r < 1)


@pytest.mark.parametrize("dims,dealias", [((64, 64, 64), 0), ((48, 64, 96), 0), ((96, 96, 96), 1),
                                          ((64, 64, 64), 2), ((36, 24, 48), 2)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_pruned_plain_transforms_move_the_kept_lines(dims, dealias, prec, monkeypatch):
    """With the lines beyond the kept indices skipped, the x passes do the
    (2K_y+1)(K_z+1) lines of every component, the y passes N_x (K_z+1), and
    each reads or writes only the 2K+1 kept rows of its axis; the z passes
    read (c2r) or write (r2c) K_z+1 entries per line.  K_i is the largest
    index the rule keeps on axis i, found here by testing the rule index by
    index."""
    monkeypatch.delenv("NS_PLAIN_PRUNE", raising=False)
    nx, ny, nz = dims
    K = []
    for a, n in enumerate(dims):
        kept = [m for m in range(n // 2 + 1) if _kept_rule(tuple(m if i == a else 0 for i in range(3)), dims, dealias)]
        K.append(max(kept))
    assert bench.plain_keep(dims, dealias) == tuple(K)
    es = 8 if prec == "fp64" else 4
    cx, cy = (2 * K[1] + 1) * (K[2] + 1), nx * (K[2] + 1)
    want = {
        "fft_x_inverse": 3 * cx * ((2 * K[0] + 1) + nx) * 2 * es,
        "fft_x_forward": 3 * cx * ((2 * K[0] + 1) + nx) * 2 * es,
        "fft_y_inverse": 3 * cy * ((2 * K[1] + 1) + ny) * 2 * es,
        "fft_y_forward": 3 * cy * ((2 * K[1] + 1) + ny) * 2 * es,
        "fft_z_c2r": 3 * nx * ny * ((K[2] + 1) * 2 * es + nz * es),
        "fft_z_r2c": 3 * nx * ny * ((K[2] + 1) * 2 * es + nz * es),
    }
    # the FP64 curl reads and writes, and the energy partials read, only the
    # rectangle (2K_x+1)(2K_y+1)(K_z+1) of every component
    rect = (2 * K[0] + 1) * (2 * K[1] + 1) * (K[2] + 1)
    want["curl"] = 2 * 3 * rect * 2 * es
    want["energy_partials"] = 3 * rect * 2 * es
    for name, b in want.items():
        got, flops = bench.kernel_model(name, dims, prec, bench.plain_keep(dims, dealias))
        assert got == b, (name, got, b)
    # every line of the full form is at least as much
    for name in want:
        full, ffull = bench.kernel_model(name, dims, prec)
        got, fl = bench.kernel_model(name, dims, prec, bench.plain_keep(dims, dealias))
        assert got < full and fl <= ffull
    monkeypatch.setenv("NS_PLAIN_PRUNE", "0")
    assert bench.plain_keep(dims, dealias) is None
