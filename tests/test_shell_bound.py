"""The per-shell error bound used beside the global relative L2 distance in
the FP32 parity tests: FP32-sized perturbations (relative to each mode, or
spread evenly over the modes) pass it, and an error confined to one shell of
small energy fails it although the global distance passes."""
import numpy as np

from paper_1003_4322_gb300 import inputs
from tests.spectral_ref import rel_l2, shell_error_ratios, wavenumbers

TOL = 2e-5


def _state():
    # energy on 1 <= |k| <= 4 plus a k^-2 tail of small amplitude up to the mask
    n = 48
    a = inputs.turbulence_state(n, seed=3)
    b = inputs.random_solenoidal_state(n, 5.0, 15.0, 1e-4, seed=4)
    return a + b


def test_fp32_sized_perturbations_pass():
    a = _state()
    rng = np.random.default_rng(1)
    rel = a * (1 + 6e-8 * (rng.standard_normal(a.shape) + 1j * rng.standard_normal(a.shape)))
    assert shell_error_ratios(rel, a).max() < 1e-6
    scale = 1e-7 * np.sqrt(np.sum(np.abs(a) ** 2) / a.size)
    white = a + scale * (rng.standard_normal(a.shape) + 1j * rng.standard_normal(a.shape))
    assert shell_error_ratios(white, a).max() < 1e-6


def test_error_confined_to_a_weak_shell_fails_the_bound_not_the_global_norm():
    a = _state()
    n = a.shape[1]
    k = wavenumbers(n).astype(float)
    KX, KY, KZ = np.meshgrid(k, k, np.arange(n // 2 + 1.0), indexing="ij")
    shell = np.floor(np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2) + 0.5)
    bad = a.copy()
    bad[:, shell == 12] *= 0.5          # half of one tail shell lost
    assert rel_l2(bad, a) < TOL         # the global distance does not see it
    # the shell holds ~6 % of the kept modes, so the bound is about four times
    # tighter there than the global distance (sqrt(n / n_K))
    assert shell_error_ratios(bad, a).max() > 2 * TOL
