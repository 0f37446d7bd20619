"""Pins of the oracle on grids of N_x x N_y x N_z points and boxes of sides
2 pi l_i (the domains of aspect ratio other than one that the scheme handles,
Sec. 5), against references that do not use the oracle: brute-force DFTs,
exact triad convolutions with non-integer wavenumbers, closed forms, and the
embedding identity that ties a stretched box to the pinned cubic case."""
import math

import numpy as np
import pytest

import oracle
from paper_1003_4322_gb300 import inputs
from tests.spectral_ref import brute_dft3, energy_half, half_to_full, kept_modes, rel_l2, triad_nonlinear

pytestmark = pytest.mark.filterwarnings("ignore")


def P(dims, box=(1.0, 1.0, 1.0), **kw):
    return oracle.Params(n=dims[0], ny=dims[1], nz=dims[2], lx=box[0], ly=box[1], lz=box[2], **kw)


@pytest.mark.parametrize("dims", [(6, 8, 4), (4, 6, 12), (8, 4, 6)])
def test_r2c_c2r_match_brute_force_dft(dims):
    u = inputs.random_real_grid(dims, 1, 3)[0]
    ref = brute_dft3(u, -1)[:, :, : dims[2] // 2 + 1]
    assert np.abs(oracle.fft3_r2c(u) - ref).max() < 1e-11 * np.abs(ref).max()
    a = inputs.random_hermitian_half_grid(dims, 1, 4)[0]
    back = brute_dft3(half_to_full(a[None])[0], +1)
    assert np.abs(back.imag).max() < 1e-10
    assert np.abs(oracle.fft3_c2r(a) - back.real).max() < 1e-11 * np.abs(back).max()


def test_r2c_matches_numpy_rfftn_on_a_larger_grid():
    u = inputs.random_real_grid((24, 12, 18), 2, 5)
    assert np.abs(oracle.fft3_r2c(u) - np.fft.rfftn(u, axes=(1, 2, 3))).max() < 1e-9


BOXES = [((8, 12, 8), (1.0, 1.5, 0.75)), ((12, 6, 8), (2.0, 1.0, 1.0)), ((6, 8, 12), (0.5, 1.0, 2.5))]


@pytest.mark.parametrize("dims,box", BOXES)
@pytest.mark.parametrize("dealias", [0, 1, 2])
def test_nonlinear_term_equals_exact_triad_sum(dims, box, dealias):
    """N(k) = P(k) sum_{p+q=k} a(p) x (i q x a(q)) with k = m / l, the
    convolution over grid indices: no transform, no aliasing.  Holds on the
    per-axis cube (dealias 0), the ellipsoid (1), and with phase shifts on the
    ellipsoid sum (3 m_i / N_i)^2 < 2 (2)."""
    hi = 1.0 + max(n / 3.0 / b for n, b in zip(dims, box))
    a = inputs.random_solenoidal_grid(dims, box, 0.5, hi, 0.8, seed=17, dealias=dealias)
    got = oracle.nonlinear(a, P(dims, box, dealias=dealias))
    ref = triad_nonlinear(a, dealias, box)
    assert np.abs(ref).max() > 1e-3
    assert np.abs(got - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())


def test_curl_and_projection_use_physical_wavenumbers():
    dims, box = (8, 12, 8), (1.0, 1.5, 0.75)
    p = P(dims, box)
    a = inputs.random_hermitian_half_grid(dims, 3, 9)
    w = oracle.curl(a, p)
    mx, my, mz = np.meshgrid(np.fft.fftfreq(8, 1 / 8), np.fft.fftfreq(12, 1 / 12), np.arange(5), indexing="ij")
    kx, ky, kz = mx / 1.0, my / 1.5, mz / 0.75
    assert np.abs(w[0] - 1j * (ky * a[2] - kz * a[1])).max() < 1e-13
    v = oracle.project(a, p=p)
    div = kx * v[0] + ky * v[1] + kz * v[2]
    assert np.abs(div).max() < 1e-13
    assert np.abs(oracle.project(v, p=p) - v).max() < 1e-13     # P^2 = P


def test_abc_forcing_coefficients_on_a_stretched_box():
    """f = F (sin kf z + cos kf y, ...) on sides (2pi, 4pi, pi): sin kf z sits
    at index kf l_z, cos kf y at kf l_y, with the closed-form amplitudes."""
    p = P((8, 16, 8), (1.0, 2.0, 0.5), force_amp=0.5, force_k=2)
    fh = oracle.forcing(p)
    assert abs(fh[0, 0, 0, 1] - 0.5 / 2j) < 1e-14        # sin(2 z), z-index 1
    assert abs(fh[0, 0, 4, 0] - 0.25) < 1e-14            # cos(2 y), y-index 4
    assert abs(fh[1, 2, 0, 0] - 0.5 / 2j) < 1e-14        # sin(2 x), x-index 2
    # six terms; a term with kz > 0 fills one entry, one on the kz = 0 plane
    # fills k and -k: 3 + 3 + 4 entries
    assert np.sum(np.abs(fh) > 1e-12) == 10
    with pytest.raises(RuntimeError):                    # sin(3 z) is not periodic on a side of pi
        oracle.forcing(P((8, 16, 8), (1.0, 2.0, 0.5), force_amp=0.5, force_k=3))


def test_shells_and_weights_on_a_stretched_box():
    """k_min = 1 / max l: on sides (2pi, 2pi, 4pi) the shells are half a unit
    wide; index (1, 0, 1) is k = (1, 0, 1/2), |k| / k_min = sqrt 5 -> shell 2;
    (0, 0, 3) -> k_z = 3/2 -> shell 3; the Nyquist plane kz index 8 has
    weight 1, index 4 weight 2."""
    p = P((8, 8, 16), (1.0, 1.0, 2.0))
    a = np.zeros(p.half_shape(), dtype=np.complex128)
    a[0, 1, 0, 1] = 0.5
    e, om, spec = oracle.diagnostics(a, p)
    assert abs(spec[2] - 0.25) < 1e-16 and abs(e - 0.25) < 1e-16 and abs(om - 0.25 * 1.25) < 1e-16
    a[:] = 0
    a[1, 0, 0, 3] = 0.5
    e, om, spec = oracle.diagnostics(a, p)
    assert abs(spec[3] - 0.25) < 1e-16 and abs(om - 0.25 * 2.25) < 1e-16
    a[:] = 0
    a[2, 0, 0, 8] = 1.0
    a[2, 0, 0, 4] = 1.0
    e, _, spec = oracle.diagnostics(a, p)
    assert abs(e - 1.5) < 1e-16                          # 1/2 * 1 + 1/2 * 2
    assert len(spec) == oracle.nbins(p) == math.ceil(math.sqrt(4 ** 2 + 4 ** 2 + 4 ** 2) * 2) + 1


def test_helicity_of_a_helical_mode_on_a_stretched_box():
    """One helical mode with curl eigenvalue s |k|: H = s |k| E, in its shell."""
    p = P((8, 12, 8), (1.0, 1.5, 0.75))
    kv = np.array([1 / 1.0, 2 / 1.5, 1 / 0.75])
    cross = np.array([[0.0, -kv[2], kv[1]], [kv[2], 0.0, -kv[0]], [-kv[1], kv[0], 0.0]])
    ev, V = np.linalg.eig(1j * cross)
    h = V[:, np.argmax(ev.real)]
    a = np.zeros(p.half_shape(), dtype=np.complex128)
    a[:, 1, 2, 1] = 0.3 * h / np.linalg.norm(h)
    H, spec = oracle.helicity(a, p)
    E = oracle.diagnostics(a, p)[0]
    assert abs(H - np.linalg.norm(kv) * E) < 1e-14
    K = int(math.floor(np.linalg.norm(kv) * 1.5 + 0.5))
    assert abs(spec[K] - H) < 1e-15


def _embed(a, dims, mult):
    """Place the cube state a (indices m) at indices mult * m of a grid."""
    n = a.shape[1]
    out = np.zeros((a.shape[0], dims[0], dims[1], dims[2] // 2 + 1), dtype=np.complex128)
    m = np.fft.fftfreq(n, 1.0 / n).astype(int)
    ix = (mult[0] * m) % dims[0]
    iy = (mult[1] * m) % dims[1]
    iz = mult[2] * np.arange(n // 2 + 1)
    out[:, ix[:, None, None], iy[None, :, None], iz[None, None, :]] = a
    return out, (ix, iy, iz)


@pytest.mark.parametrize("dealias", [0, 1, 2])
def test_stretched_box_reproduces_the_cube(dealias):
    """A field on the (2pi)^3 box is also a field on the box of sides
    (4pi, 2pi, 6pi) holding only indices (2 m_x, m_y, 3 m_z); with (2N, N, 3N)
    points the masks, wavenumbers, forcing (index kf l_i), phase shifts and
    products coincide, so the stretched run equals the cubic run (itself
    pinned) to rounding, and the other indices stay zero to rounding."""
    n, mult = 12, (2, 1, 3)
    dims = tuple(n * k for k in mult)
    a = inputs.random_solenoidal_state(n, 1.0, 3.5, 0.8, seed=23, dealias=dealias)
    kw = dict(nu=0.02, dt=0.01, force_amp=0.4, force_k=2, rot=0.7, dealias=dealias)
    ref = oracle.step(a, oracle.Params(n=n, **kw), 3)
    b, (ix, iy, iz) = _embed(a, dims, mult)
    got = oracle.step(b, P(dims, mult, **kw), 3)
    sub = got[:, ix[:, None, None], iy[None, :, None], iz[None, None, :]]
    assert rel_l2(sub, ref) < 1e-14
    rest = got.copy()
    rest[:, ix[:, None, None], iy[None, :, None], iz[None, None, :]] = 0
    assert np.abs(rest).max() < 1e-15 * np.abs(ref).max()
    e_ref = oracle.diagnostics(ref)[:2]
    e_got = oracle.diagnostics(got, P(dims, mult))[:2]
    assert abs(e_got[0] - e_ref[0]) < 1e-14 * e_ref[0] and abs(e_got[1] - e_ref[1]) < 1e-13 * e_ref[1]


def test_stretched_box_mhd_reproduces_the_cube():
    n, mult = 8, (1, 3, 2)
    dims = tuple(n * k for k in mult)
    a = np.concatenate([inputs.random_solenoidal_state(n, 1.0, 2.7, 0.6, seed=41),
                        inputs.random_solenoidal_state(n, 1.0, 2.7, 0.5, seed=42)])
    kw = dict(nu=0.02, eta=0.03, dt=0.01, mhd=1)
    ref = oracle.step(a, oracle.Params(n=n, **kw), 2)
    b, (ix, iy, iz) = _embed(a, dims, mult)
    got = oracle.step(b, P(dims, mult, **kw), 2)
    sub = got[:, ix[:, None, None], iy[None, :, None], iz[None, None, :]]
    assert rel_l2(sub, ref) < 1e-14


def test_single_mode_decays_exactly_on_a_stretched_box():
    """A single-wavevector solenoidal mode: u x w is a gradient, so the mode
    decays as exp(-nu |k|^2 t) with the physical |k| (k = m / l)."""
    dims, box = (8, 12, 8), (1.0, 1.5, 0.75)
    p = P(dims, box, nu=0.05, dt=0.03)
    kv = np.array([1 / 1.0, 1 / 1.5, 2 / 0.75])
    e1 = np.cross(kv, [0.0, 0.0, 1.0])
    a = np.zeros(p.half_shape(), dtype=np.complex128)
    a[:, 1, 1, 2] = 0.4 * e1 / np.linalg.norm(e1)
    got = oracle.step(a, p, 5)
    assert np.abs(got - a * math.exp(-0.05 * float(kv @ kv) * 0.15)).max() < 1e-15


def test_inviscid_energy_drift_is_third_order_and_positive_on_a_stretched_box():
    """With nu = 0 and no forcing <a, N(a)> = 0 on any box, so one Heun step
    changes |a|^2 by (dt^2/4)|N(a) - N(a1)|^2 >= 0: the drift over a fixed
    time is positive and O(dt^3)."""
    dims, box = (8, 12, 6), (1.0, 1.5, 0.75)
    a = inputs.random_solenoidal_grid(dims, box, 0.5, 3.0, 1.0, seed=29)
    p0 = P(dims, box)
    e0 = oracle.diagnostics(a, p0)[0]
    drift = []
    for k in (8, 16, 32):
        b = oracle.step(a, P(dims, box, dt=0.16 / k), k)
        drift.append(oracle.diagnostics(b, p0)[0] - e0)
    assert all(d > 0 for d in drift)
    assert 7.5 < drift[0] / drift[1] < 8.5 and 7.5 < drift[1] / drift[2] < 8.5, drift


def test_grid_generator_is_solenoidal_with_the_requested_rms():
    dims, box = (12, 8, 16), (1.5, 1.0, 2.0)
    a = inputs.random_solenoidal_grid(dims, box, 1.0, 3.0, 0.7, seed=2)
    assert abs(energy_half(a) - 1.5 * 0.49) < 1e-14
    m = np.meshgrid(np.fft.fftfreq(12, 1 / 12), np.fft.fftfreq(8, 1 / 8), np.arange(9), indexing="ij")
    div = sum(mi / b * a[i] for i, (mi, b) in enumerate(zip(m, box)))
    assert np.abs(div).max() < 1e-15
    assert len(kept_modes(dims)) == 7 * 5 * 11
