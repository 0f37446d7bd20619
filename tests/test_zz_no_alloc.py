"""ns_fft_c2r_noalloc: the FP32 inverse transform for callers that cannot
allocate device memory (a caching pool allocator owns it, or a real-time loop
forbids allocation after start-up).  It must give the same result as the
context-based ns_fft_c2r, call after call, although every call reuses the same
fixed scratch arrays inside the library.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_1003_4322_gb300 import _native as nat
from paper_1003_4322_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 2e-6   # the FP32 transform tolerance of the other GPU tests


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("n,ncomp", [(12, 2), (32, 3), (128, 1)])
def test_noalloc_c2r_matches_context_c2r_twice(ns, n, ncomp):
    import torch
    a = inputs.random_hermitian_half(n, ncomp, 40 + n)
    ad = torch.from_numpy(a).to("cuda", torch.complex64)
    ref = torch.empty((ncomp, n, n, n), dtype=torch.float32, device="cuda")
    ctx = nat.ns_init([dict(n=8, dt=1e-3)], nat.NS_FP32)
    try:
        nat.ns_fft_c2r(ctx, n, ncomp, ad, ref)
        nat.ns_sync(ctx)
    finally:
        nat.ns_destroy(ctx)
    lib = nat.load()
    stream = torch.cuda.current_stream()
    for _ in range(2):
        out = torch.full((ncomp, n, n, n), float("nan"), dtype=torch.float32, device="cuda")
        st = lib.ns_fft_c2r_noalloc(n, ncomp, ctypes.c_void_p(ad.data_ptr()),
                                    ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_void_p(stream.cuda_stream))
        assert st == nat.NS_OK, nat.ns_status_str(st)
        torch.cuda.synchronize()
        assert _rel(out.cpu().numpy(), ref.cpu().numpy()) < TOL


def test_noalloc_rejects_sizes_beyond_its_scratch(ns):
    import torch
    lib = nat.load()
    x = torch.zeros(16, dtype=torch.float32, device="cuda")
    assert lib.ns_fft_c2r_noalloc(256, 1, ctypes.c_void_p(x.data_ptr()),
                                  ctypes.c_void_p(x.data_ptr()), None) == nat.NS_ERR_UNSUPPORTED_N
    assert lib.ns_fft_c2r_noalloc(30, 1, ctypes.c_void_p(x.data_ptr()),
                                  ctypes.c_void_p(x.data_ptr()), None) == nat.NS_ERR_UNSUPPORTED_N
    assert lib.ns_fft_c2r_noalloc(32, 1, None, None, None) == nat.NS_ERR_ARG
