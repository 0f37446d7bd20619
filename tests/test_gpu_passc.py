"""Every compiled pass-C kernel of the fused FP32 form (z c2r of u and w,
u x w on the grid, z r2c of the product; Sec. 2, Eqs. 1-2), forced in turn
through NS_FORCE_PASS_C, against the plain FP64 form on the same GPU (itself
pinned to the oracle).  The autotuner picks one kernel per N; this checks the
ones it did not pick as well, at sizes that span several lines per CTA, the
ragged last CTA and both families of N (powers of two, factor 3)."""
import pytest

from paper_1003_4322_gb300 import inputs
from tests.spectral_ref import rel_l2

pytestmark = pytest.mark.gpu

# (kind, E, tile) triples as the plan cache writes them: kind 2 =
# register-resident (tile = warps per CTA + 8 x parked fields, + 32 for the
# form with per-lane asynchronous copies two fields ahead, + 64 for the form
# with one bulk copy per warp and field), kind 1 = shared-memory line kernel
# (tile = warps per CTA).
LOADS = {0: "registers, one field ahead", 1: "per-lane asynchronous copies, two fields ahead",
         2: "bulk copies, two fields ahead"}
CANDIDATES = ([(2, E, t + a) for E in (16, 12, 8, 6, 4) for t in (1, 2, 9, 10, 17, 18)
               for a in (0, 32, 64)]
              + [(1, E, w) for E in (16, 12, 8, 6) for w in (1, 2, 4)])


def _matches(desc, kind, E, tile):
    c = desc["C_z_nonlinear"]
    if c.get("E") != E:
        return False
    if kind == 2:
        t = tile % 32
        return (c.get("kernel") == "register-resident" and c["warps_per_cta"] == t % 8
                and c["parked_fields"] == t // 8 and c["loads"] == LOADS[tile // 32])
    return c.get("kernel") == "compile-time length" and c["warps_per_cta"] == tile


def _find_c(desc):
    if "C_z_nonlinear" in desc:
        return desc
    for v in desc.values():
        if isinstance(v, dict):
            r = _find_c(v)
            if r is not None:
                return r
    return None


@pytest.mark.parametrize("n", [32, 64, 96, 128, 192, 256])
def test_every_pass_c_kernel(ns, n, monkeypatch):
    from paper_1003_4322_gb300 import _native as nat
    from paper_1003_4322_gb300.solver import Solver
    run = dict(n=n, nu=2e-3, dt=1e-3, force_amp=0.5, force_k=3)
    a0 = inputs.turbulence_state(n, seed=3)
    steps = 2
    with Solver([run], prec="fp64") as s:
        s.set_state(a0)
        s.step(steps)
        ref = s.get_state()
    tried = []
    for kind, E, tile in CANDIDATES:
        monkeypatch.setenv("NS_FORCE_PASS_C", f"{kind},{E},{tile}")
        with Solver([run], prec="fp32") as s:
            desc = _find_c(nat.ns_describe_run(s.ctx, 0))
            if desc is None or not _matches(desc, kind, E, tile):
                continue
            s.set_state(a0)
            s.step(steps)
            got = s.get_state()
        err = rel_l2(got, ref)
        assert err < 2e-5, (kind, E, tile, err)
        tried.append((kind, E, tile))
    # at least one register-resident and one shared-memory kernel per N, and
    # the asynchronous-copy form where it is compiled
    assert any(t[0] == 2 for t in tried) and any(t[0] == 1 for t in tried), tried
    if n in (256, 512, 1024):
        for mode in (1, 2):
            assert any(t[0] == 2 and t[2] // 32 == mode for t in tried), tried


STRIDED = [(k, E, ct) for k in (2, 1) for E in (8, 12, 16, 32) for ct in (8, 16)]


@pytest.mark.parametrize("n", [64, 96, 128, 256])
def test_every_strided_pass_kernel(ns, n, monkeypatch):
    """Passes A, B, D, E (x/y transforms with the curl, the pruning of rows
    and the dealiased output rows) on every compiled compile-time kernel,
    forced through NS_FORCE_STRIDED, against the plain FP64 form."""
    from paper_1003_4322_gb300 import _native as nat
    from paper_1003_4322_gb300.solver import Solver
    run = dict(n=n, nu=2e-3, dt=1e-3, force_amp=0.5, force_k=3)
    a0 = inputs.turbulence_state(n, seed=4)
    with Solver([run], prec="fp64") as s:
        s.set_state(a0)
        s.step(2)
        ref = s.get_state()
    names = {1: "compile-time length", 2: "constant geometry"}
    tried = []
    for kind, E, ct in STRIDED:
        monkeypatch.setenv("NS_FORCE_STRIDED", f"{kind},{E},{ct}")
        with Solver([run], prec="fp32") as s:
            passes = _find_c(nat.ns_describe_run(s.ctx, 0))
            forced = [p for p in ("A_x_inverse_curl", "B_y_inverse", "D_y_forward", "E_x_forward")
                      if passes[p]["kernel"] == names[kind] and passes[p]["E"] == E
                      and passes[p]["cols_per_cta"] == ct]
            if not forced:
                continue
            s.set_state(a0)
            s.step(2)
            got = s.get_state()
        err = rel_l2(got, ref)
        assert err < 2e-5, (kind, E, ct, forced, err)
        tried.append((kind, E, ct))
    assert any(t[0] == 2 for t in tried) and any(t[0] == 1 for t in tried), tried


EU = [(E, ct) for E in (8, 12, 16, 32) for ct in (8, 16)]


@pytest.mark.parametrize("n", [64, 96, 128, 256])
def test_pass_e_fused_with_update(ns, n, monkeypatch):
    """Pass E fused with the update (x forward FFT, then 1/N^3, Coriolis,
    projection, forcing, IF-RK2 and the energy partials per mode in
    registers), forced through NS_FORCE_EU for every compiled shape and off,
    against the plain FP64 form; the per-step (E, Omega) from its partials
    agree with an FP64 sum over the stored state."""
    from paper_1003_4322_gb300 import _native as nat
    from paper_1003_4322_gb300.solver import Solver
    run = dict(n=n, nu=2e-3, dt=1e-3, force_amp=0.5, force_k=3, rot=1.5)
    a0 = inputs.turbulence_state(n, seed=6)
    with Solver([run], prec="fp64") as s:
        s.set_state(a0)
        s.step(2)
        ref = s.get_state()
    tried = []
    for cfg in ["off"] + [f"{E},{ct}" for E, ct in EU]:
        monkeypatch.setenv("NS_FORCE_EU", cfg)
        with Solver([run], prec="fp32") as s:
            eu = _find_c(nat.ns_describe_run(s.ctx, 0))["E_fused_with_update"]
            if cfg == "off":
                assert eu is None
            elif eu is None or f"{eu['E']},{eu['cols_per_cta']}" != cfg:
                continue
            s.set_state(a0)
            s.step(2)
            got = s.get_state()
            Es, Os = s.series(count=4)
            E, Om, _ = s.energy_spectrum()
        assert rel_l2(got, ref) < 2e-5, cfg
        assert abs(Es[-1] - E) < 1e-12 * E and abs(Os[-1] - Om) < 1e-12 * Om, cfg
        tried.append(cfg)
    assert len(tried) >= 2, tried


def test_bulk_copy_wait_runs_out_and_reports(ns, monkeypatch):
    """The bulk-copy pass C waits for each copy with a bounded mbarrier wait.
    NS_TEST_ZR_SKIP_COPY=1 leaves every warp's first copy unissued, so that
    wait runs out (after about a millisecond). The kernel then raises the
    context's timeout bit and still waits for the copies it did issue before
    it exits. ns_sync reports NS_ERR_TIMEOUT, and the device stays usable: a
    fresh context runs the same kernel to the plain FP64 result."""
    from paper_1003_4322_gb300 import _native as nat
    from paper_1003_4322_gb300.solver import Solver
    n = 256
    run = dict(n=n, nu=2e-3, dt=1e-3, force_amp=0.5, force_k=3)
    a0 = inputs.turbulence_state(n, seed=8)
    with Solver([run], prec="fp64") as s:
        s.set_state(a0)
        s.step(1)
        ref = s.get_state()
    monkeypatch.setenv("NS_FORCE_PASS_C", "2,16,81")   # E = 16, one warp, two fields parked, bulk
    monkeypatch.setenv("NS_TEST_ZR_SKIP_COPY", "1")
    with Solver([run], prec="fp32") as s:
        c = _find_c(nat.ns_describe_run(s.ctx, 0))["C_z_nonlinear"]
        assert c["loads"] == "bulk copies, two fields ahead", c
        s.set_state(a0)
        s.step(1)
        with pytest.raises(nat.NsError) as err:
            s.sync()
        assert err.value.status == 5   # NS_ERR_TIMEOUT
    monkeypatch.delenv("NS_TEST_ZR_SKIP_COPY")
    with Solver([run], prec="fp32") as s:
        s.set_state(a0)
        s.step(1)
        got = s.get_state()
    assert rel_l2(got, ref) < 2e-5
