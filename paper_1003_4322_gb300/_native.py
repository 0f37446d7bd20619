"""ctypes binding of libns (include/ns.h): argument marshalling only.

Every function here forwards to the C entry point of the same name; all
computation happens in the CUDA kernels of libns.  Loading fails loudly (an
exception) when libns.so is missing or cannot be opened: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libns.so")

NS_OK, NS_ERR_ARG, NS_ERR_CUDA, NS_ERR_OOM, NS_ERR_UNSUPPORTED_N, NS_ERR_TIMEOUT, \
    NS_ERR_NONFINITE = range(7)
NS_FP64, NS_FP32 = 0, 1

# every symbol include/ns.h declares
SYMBOLS = ("ns_init", "ns_set_state", "ns_get_state", "ns_step", "ns_fft_r2c", "ns_fft_c2r",
           "ns_energy_spectrum", "ns_nbins", "ns_series", "ns_series_capacity",
           "ns_kernel_census", "ns_sync", "ns_last_error", "ns_status_str", "ns_destroy",
           "ns_fft_c2r_noalloc", "ns_describe_run", "ns_helicity", "ns_set_field",
           "ns_get_field", "ns_field_spectrum", "ns_guard_check", "ns_guard_selftest",
           "ns_fft_r2c_grid", "ns_fft_c2r_grid", "ns_run_nbins", "ns_set_states",
           "ns_energy_spectra", "ns_alu_peak")


class NsError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str = ""):
        self.status = status
        msg = f"{what}: {ns_status_str(status)} (status {status})"
        super().__init__(msg + (f" [{detail}]" if detail else ""))


class ns_run_params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("nu", ctypes.c_double), ("dt", ctypes.c_double),
                ("force_amp", ctypes.c_double), ("force_k", ctypes.c_int),
                ("dealias", ctypes.c_int), ("rot", ctypes.c_double), ("eta", ctypes.c_double),
                ("mhd", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double)]


class ns_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int),
                ("total_ms", ctypes.c_double)]


_lib = None


def load(path: str = LIB_PATH):
    """Open libns.so and declare its signatures (raises if it is absent)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libns.so not found at {path}: build it with "
                          "paper_1003_4322_gb300.build.build() (needs nvcc)")
    L = ctypes.CDLL(path)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "ns_init": ([ctypes.POINTER(ns_run_params), I, I, P, ctypes.POINTER(P)], I),
        "ns_set_state": ([P, I, P, I], I),
        "ns_set_field": ([P, I, I, P, I], I),
        "ns_get_field": ([P, I, I, P, I], I),
        "ns_field_spectrum": ([P, I, I, P, I, ctypes.POINTER(D), ctypes.POINTER(D)], I),
        "ns_get_state": ([P, I, P, I], I),
        "ns_step": ([P, I], I),
        "ns_fft_r2c": ([P, I, I, P, P], I),
        "ns_fft_c2r": ([P, I, I, P, P], I),
        "ns_fft_c2r_noalloc": ([I, I, P, P, P], I),
        "ns_alu_peak": ([I, D, ctypes.POINTER(D), P], I),
        "ns_fft_r2c_grid": ([P, I, I, I, I, P, P], I),
        "ns_fft_c2r_grid": ([P, I, I, I, I, P, P], I),
        "ns_run_nbins": ([ctypes.POINTER(ns_run_params)], I),
        "ns_set_states": ([P, I, I, ctypes.POINTER(P), I], I),
        "ns_energy_spectra": ([P, I, I, P, I, P, P], I),
        "ns_energy_spectrum": ([P, I, P, I, ctypes.POINTER(D), ctypes.POINTER(D)], I),
        "ns_nbins": ([I], I),
        "ns_helicity": ([P, I, P, I, ctypes.POINTER(D)], I),
        "ns_series": ([P, I, I, P, P, ctypes.POINTER(I)], I),
        "ns_series_capacity": ([], I),
        "ns_kernel_census": ([P, I, ctypes.POINTER(ns_kernel_time), I, ctypes.POINTER(I)], I),
        "ns_sync": ([P], I),
        "ns_status_str": ([I], ctypes.c_char_p),
        "ns_last_error": ([P], ctypes.c_char_p),
        "ns_describe_run": ([P, I, ctypes.c_char_p, I], I),
        "ns_destroy": ([P], None),
        "ns_guard_check": ([ctypes.POINTER(ctypes.c_longlong)], I),
        "ns_guard_selftest": ([ctypes.POINTER(ctypes.c_longlong)], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _check(st: int, what: str, ctx=None) -> None:
    if st != NS_OK:
        detail = load().ns_last_error(ctx).decode() if ctx is not None else ""
        raise NsError(st, what, detail)


def _ptr(x):
    """Raw address of a torch tensor or numpy array (must be contiguous)."""
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data_as(ctypes.c_void_p)
    raise TypeError(f"unsupported buffer type {type(x)}")


def _on_device(x) -> int:
    return int(hasattr(x, "is_cuda") and x.is_cuda)


def ns_status_str(st: int) -> str:
    return load().ns_status_str(st).decode()


def ns_nbins(n: int) -> int:
    return load().ns_nbins(n)


def run_params(r) -> ns_run_params:
    """ns_run_params from a dict with keys n, dt and optionally nu,
    force_amp, force_k, dealias, rot, eta, mhd, ny, nz, lx, ly, lz."""
    if isinstance(r, ns_run_params):
        return r
    return ns_run_params(int(r["n"]), float(r.get("nu", 0.0)), float(r["dt"]),
                         float(r.get("force_amp", 0.0)), int(r.get("force_k", 0)),
                         int(r.get("dealias", 0)), float(r.get("rot", 0.0)),
                         float(r.get("eta", 0.0)), int(r.get("mhd", 0)), int(r.get("ny", 0)),
                         int(r.get("nz", 0)), float(r.get("lx", 0.0)), float(r.get("ly", 0.0)),
                         float(r.get("lz", 0.0)))


def ns_run_nbins(r) -> int:
    p = run_params(r)
    return load().ns_run_nbins(ctypes.byref(p))


def ns_series_capacity() -> int:
    return load().ns_series_capacity()


def ns_init(runs, prec: int, stream=None):
    """runs: list of dicts or ns_run_params; stream: torch.cuda.Stream, a raw
    cudaStream_t integer, or None (legacy default stream)."""
    arr = (ns_run_params * len(runs))()
    for i, r in enumerate(runs):
        arr[i] = run_params(r)
    if stream is None:
        s = None
    elif hasattr(stream, "cuda_stream"):
        s = ctypes.c_void_p(stream.cuda_stream)
    else:
        s = ctypes.c_void_p(int(stream))
    ctx = ctypes.c_void_p()
    _check(load().ns_init(arr, len(runs), prec, s, ctypes.byref(ctx)), "ns_init")
    return ctx


def ns_destroy(ctx) -> None:
    load().ns_destroy(ctx)


def ns_set_state(ctx, run: int, uhat) -> None:
    """uhat: complex128 [3][N][N][N/2+1], numpy (host) or torch (host/device)."""
    _check(load().ns_set_state(ctx, run, _ptr(uhat), _on_device(uhat)), "ns_set_state", ctx)


def ns_get_state(ctx, run: int, out) -> None:
    _check(load().ns_get_state(ctx, run, _ptr(out), _on_device(out)), "ns_get_state", ctx)


def ns_set_states(ctx, first: int, uhats) -> None:
    """uhats: complex128 half-layout states of runs first, first + 1, ...
    (all numpy / host torch, or all device torch)."""
    n = len(uhats)
    ptrs = (ctypes.c_void_p * n)(*[_ptr(u).value for u in uhats])
    dev = {_on_device(u) for u in uhats}
    if len(dev) != 1:
        raise ValueError("the buffers must all be on the host or all on the device")
    _check(load().ns_set_states(ctx, first, n, ptrs, dev.pop()), "ns_set_states", ctx)


def ns_energy_spectra(ctx, first: int, count: int, nbins: int):
    """Returns (E[count], Omega[count], spectra[count][nbins]) of runs first ..
    first + count - 1 (rows zero-padded past each run's shells)."""
    spec = np.zeros((count, max(nbins, 0)), dtype=np.float64)
    e = np.zeros(count, dtype=np.float64)
    om = np.zeros(count, dtype=np.float64)
    _check(load().ns_energy_spectra(ctx, first, count, _ptr(spec), nbins, _ptr(e), _ptr(om)),
           "ns_energy_spectra", ctx)
    return e, om, spec


def ns_set_field(ctx, run: int, field: int, uhat) -> None:
    """field 0: velocity, 1: magnetic field (MHD runs); layout as ns_set_state."""
    _check(load().ns_set_field(ctx, run, field, _ptr(uhat), _on_device(uhat)), "ns_set_field", ctx)


def ns_get_field(ctx, run: int, field: int, out) -> None:
    _check(load().ns_get_field(ctx, run, field, _ptr(out), _on_device(out)), "ns_get_field", ctx)


def _shells(n) -> int:
    """Shell count of N (an int: the cube) or of a run (dict or ns_run_params)."""
    return ns_nbins(n) if isinstance(n, int) else ns_run_nbins(n)


def ns_field_spectrum(ctx, run: int, field: int, n):
    """Returns (E, Omega, spectrum) of field 0 (velocity) or 1 (magnetic);
    n is N of a cubic run, or the run's parameters."""
    nb = _shells(n)
    spec = np.zeros(nb, dtype=np.float64)
    e, om = ctypes.c_double(), ctypes.c_double()
    _check(load().ns_field_spectrum(ctx, run, field, _ptr(spec), nb, ctypes.byref(e),
                                    ctypes.byref(om)), "ns_field_spectrum", ctx)
    return e.value, om.value, spec


def ns_guard_check() -> int:
    """Corrupted guard bytes of all live library buffers (-1: guards off)."""
    v = ctypes.c_longlong()
    _check(load().ns_guard_check(ctypes.byref(v)), "ns_guard_check")
    return v.value


def ns_guard_selftest() -> int:
    v = ctypes.c_longlong()
    _check(load().ns_guard_selftest(ctypes.byref(v)), "ns_guard_selftest")
    return v.value


def ns_step(ctx, nsteps: int) -> None:
    _check(load().ns_step(ctx, nsteps), "ns_step", ctx)


def ns_fft_r2c(ctx, n: int, ncomp: int, inp, out) -> None:
    _check(load().ns_fft_r2c(ctx, n, ncomp, _ptr(inp), _ptr(out)), "ns_fft_r2c", ctx)


def ns_fft_c2r(ctx, n: int, ncomp: int, inp, out) -> None:
    _check(load().ns_fft_c2r(ctx, n, ncomp, _ptr(inp), _ptr(out)), "ns_fft_c2r", ctx)


def ns_fft_r2c_grid(ctx, nx: int, ny: int, nz: int, ncomp: int, inp, out) -> None:
    _check(load().ns_fft_r2c_grid(ctx, nx, ny, nz, ncomp, _ptr(inp), _ptr(out)), "ns_fft_r2c_grid", ctx)


def ns_fft_c2r_grid(ctx, nx: int, ny: int, nz: int, ncomp: int, inp, out) -> None:
    _check(load().ns_fft_c2r_grid(ctx, nx, ny, nz, ncomp, _ptr(inp), _ptr(out)), "ns_fft_c2r_grid", ctx)


def ns_fft_c2r_noalloc(n: int, ncomp: int, inp, out, stream=None) -> None:
    """FP32 c2r that allocates nothing (fixed in-library scratch, n <= 128)."""
    if stream is None:
        s = None
    elif hasattr(stream, "cuda_stream"):
        s = ctypes.c_void_p(stream.cuda_stream)
    else:
        s = ctypes.c_void_p(int(stream))
    _check(load().ns_fft_c2r_noalloc(n, ncomp, _ptr(inp), _ptr(out), s), "ns_fft_c2r_noalloc")


def ns_energy_spectrum(ctx, run: int, n):
    """Returns (E, Omega, spectrum as a numpy array of the run's shells); n is
    N of a cubic run, or the run's parameters."""
    nb = _shells(n)
    spec = np.zeros(nb, dtype=np.float64)
    e, om = ctypes.c_double(), ctypes.c_double()
    _check(load().ns_energy_spectrum(ctx, run, _ptr(spec), nb, ctypes.byref(e), ctypes.byref(om)),
           "ns_energy_spectrum", ctx)
    return e.value, om.value, spec


def ns_helicity(ctx, run: int, n):
    """Returns (H, helicity spectrum as a numpy array of the run's shells)."""
    nb = _shells(n)
    spec = np.zeros(nb, dtype=np.float64)
    h = ctypes.c_double()
    _check(load().ns_helicity(ctx, run, _ptr(spec), nb, ctypes.byref(h)), "ns_helicity", ctx)
    return h.value, spec


def ns_series(ctx, run: int, count: int):
    E = np.zeros(max(count, 1), dtype=np.float64)
    O = np.zeros(max(count, 1), dtype=np.float64)
    w = ctypes.c_int()
    _check(load().ns_series(ctx, run, count, _ptr(E), _ptr(O), ctypes.byref(w)), "ns_series", ctx)
    return E[: w.value].copy(), O[: w.value].copy()


def ns_kernel_census(ctx, nsteps: int):
    """Per-kernel launches and device time over nsteps un-graphed steps:
    list of (name, launches, total_ms)."""
    arr = (ns_kernel_time * 64)()
    cnt = ctypes.c_int()
    _check(load().ns_kernel_census(ctx, nsteps, arr, 64, ctypes.byref(cnt)), "ns_kernel_census", ctx)
    return [(arr[i].name.decode(), arr[i].launches, arr[i].total_ms)
            for i in range(min(cnt.value, 64))]


def _stream_ptr(stream):
    """cudaStream_t of a torch.cuda.Stream, a raw integer, or None."""
    if stream is None:
        return ctypes.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def ns_alu_peak(prec: int, ms: float = 200.0, stream=None) -> float:
    """Measured FMA rate of the current device in flop/s (NS_FP64 or NS_FP32)."""
    out = ctypes.c_double()
    _check(load().ns_alu_peak(prec, float(ms), ctypes.byref(out), _stream_ptr(stream)),
           "ns_alu_peak")
    return out.value


def ns_describe_run(ctx, run: int = 0) -> dict:
    """How a run is executed (form, sizes, autotuned per-pass configuration)."""
    import json
    buf = ctypes.create_string_buffer(2048)
    _check(load().ns_describe_run(ctx, run, buf, 2048), "ns_describe_run", ctx)
    return json.loads(buf.value.decode())


def ns_sync(ctx) -> None:
    _check(load().ns_sync(ctx), "ns_sync", ctx)
