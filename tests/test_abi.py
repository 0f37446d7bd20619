"""The C-ABI library: it loads, exports every symbol include/ns.h declares,
and its host-side argument checks work without a GPU (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ns.h")


def declared_symbols():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ns_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1003_4322_gb300 import _native
    if not os.path.exists(_native.LIB_PATH):
        from paper_1003_4322_gb300 import build
        build.build()
    return _native.load()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("ns_init", "ns_set_state", "ns_get_state", "ns_step", "ns_fft_r2c", "ns_fft_c2r",
              "ns_energy_spectrum", "ns_sync", "ns_status_str", "ns_destroy"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    from paper_1003_4322_gb300 import _native
    for s in declared_symbols():
        assert hasattr(lib, s), f"{s} not exported"
    assert sorted(_native.SYMBOLS) == declared_symbols()


def test_status_strings_and_bins(lib):
    from paper_1003_4322_gb300 import _native as nat
    assert nat.ns_status_str(0) == "ok"
    assert "grid" in nat.ns_status_str(4)
    assert nat.ns_nbins(32) == 29          # ceil(sqrt3 * 16) + 1
    assert nat.ns_nbins(1024) == 888
    assert nat.ns_series_capacity() >= 1000
    # shells of other grids and boxes agree with the oracle's count
    import oracle
    for kw in (dict(n=32), dict(n=32, ny=64, nz=16), dict(n=32, nz=64, lz=2.0),
               dict(n=24, ny=36, nz=48, lx=1.0, ly=1.5, lz=0.75)):
        want = oracle.nbins(oracle.Params(**kw))
        assert nat.ns_run_nbins(dict(dt=1e-3, **kw)) == want, kw


@pytest.mark.parametrize("bad", [dict(n=30), dict(n=14), dict(n=7), dict(n=2048), dict(n=1536),
                                 dict(n=32, ny=30), dict(n=32, nz=2048), dict(n=1024, ny=1024, nz=1536),
                                 dict(n=1024, ny=1024, nz=1024 * 3 // 2 // 3 * 3)])
def test_unsupported_sizes_rejected_before_any_device_call(lib, bad):
    from paper_1003_4322_gb300 import _native as nat
    p = dict(dt=1e-3, nu=0.01)
    p.update(bad)
    with pytest.raises(nat.NsError) as ei:
        nat.ns_init([p], nat.NS_FP32)
    assert ei.value.status == nat.NS_ERR_UNSUPPORTED_N


@pytest.mark.parametrize("bad", [dict(dt=0.0), dict(nu=-1.0), dict(dealias=3), dict(force_k=-1),
                                 dict(dt=float("nan")), dict(mhd=2), dict(mhd=1, eta=-1.0),
                                 dict(mhd=1, dealias=2), dict(rot=float("inf")), dict(ny=-8),
                                 dict(lz=-1.0), dict(lx=float("nan")), dict(ly=1e7),
                                 dict(lz=0.5, force_k=3, force_amp=0.5),
                                 dict(ly=1.25, force_k=2, force_amp=0.5)])
def test_bad_parameters_rejected(lib, bad):
    from paper_1003_4322_gb300 import _native as nat
    p = dict(n=32, dt=1e-3, nu=0.01)
    p.update(bad)
    with pytest.raises(nat.NsError) as ei:
        nat.ns_init([p], nat.NS_FP64)
    assert ei.value.status == nat.NS_ERR_ARG


def test_null_arguments_rejected(lib):
    from paper_1003_4322_gb300 import _native as nat
    out = ctypes.c_void_p()
    assert lib.ns_init(None, 1, 0, None, ctypes.byref(out)) == nat.NS_ERR_ARG
    assert lib.ns_step(None, 1) == nat.NS_ERR_ARG
    assert lib.ns_sync(None) == nat.NS_ERR_ARG
    assert lib.ns_fft_r2c(None, 32, 1, None, None) == nat.NS_ERR_ARG
    assert lib.ns_set_states(None, 0, 1, None, 0) == nat.NS_ERR_ARG
    assert lib.ns_energy_spectra(None, 0, 1, None, 0, None, None) == nat.NS_ERR_ARG
    lib.ns_destroy(None)


def test_alu_peak_rejects_bad_arguments_before_any_device_call(lib):
    from paper_1003_4322_gb300 import _native as nat
    out = ctypes.c_double()
    assert lib.ns_alu_peak(nat.NS_FP64, 100.0, None, None) == nat.NS_ERR_ARG
    assert lib.ns_alu_peak(nat.NS_FP64, 0.0, ctypes.byref(out), None) == nat.NS_ERR_ARG
    assert lib.ns_alu_peak(nat.NS_FP64, 2e4, ctypes.byref(out), None) == nat.NS_ERR_ARG
    assert lib.ns_alu_peak(7, 100.0, ctypes.byref(out), None) == nat.NS_ERR_ARG
