"""ns_fft_c2r_noalloc: the FP32 inverse transform for callers that cannot
allocate device memory (a caching pool allocator owns it, or a real-time loop
forbids allocation after start-up).  It must give the same result as the
context-based ns_fft_c2r, call after call, although every call reuses the same
fixed scratch arrays inside the library.  Collected last on purpose."""
import ctypes
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1003_4322_gb300 import _native as nat
from paper_1003_4322_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 2e-6   # the FP32 transform tolerance of the other GPU tests
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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


# Run in a fresh interpreter: the entry point is called before any libns
# context exists on the device (the situation of a caller that never makes
# one), free device memory is read after the first call and again after two
# more, and only then does a context compute the expected result.
_FRESH = r"""
import ctypes, json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_1003_4322_gb300 import _native as nat, inputs
n, ncomp = 48, 3
lib = nat.load()
a = inputs.random_hermitian_half(n, ncomp, 4848)
ad = torch.from_numpy(a).to("cuda", torch.complex64)
outs = [torch.full((ncomp, n, n, n), float("nan"), dtype=torch.float32, device="cuda")
        for _ in range(3)]
torch.cuda.synchronize()
stream = torch.cuda.current_stream()
def call(o):
    return lib.ns_fft_c2r_noalloc(n, ncomp, ctypes.c_void_p(ad.data_ptr()),
                                  ctypes.c_void_p(o.data_ptr()),
                                  ctypes.c_void_p(stream.cuda_stream))
st = [call(outs[0])]
torch.cuda.synchronize()
free1 = torch.cuda.mem_get_info()[0]
st += [call(outs[1]), call(outs[2])]
torch.cuda.synchronize()
free2 = torch.cuda.mem_get_info()[0]
ref = torch.empty_like(outs[0])
ctx = nat.ns_init([dict(n=8, dt=1e-3)], nat.NS_FP32)
nat.ns_fft_c2r(ctx, n, ncomp, ad, ref)
nat.ns_sync(ctx)
nat.ns_destroy(ctx)
r = ref.cpu().numpy()
errs = [float(np.linalg.norm((o.cpu().numpy() - r).ravel()) / np.linalg.norm(r.ravel()))
        for o in outs]
print(json.dumps(dict(status=st, free1=free1, free2=free2, errs=errs)))
"""


def test_noalloc_first_call_without_a_context_allocates_nothing_later(ns):
    r = subprocess.run([sys.executable, "-c", _FRESH, ROOT], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["status"] == [nat.NS_OK] * 3, res
    assert res["free2"] == res["free1"], res
    assert max(res["errs"]) < TOL, res


def test_noalloc_rejects_sizes_beyond_its_scratch(ns):
    import torch
    lib = nat.load()
    x = torch.zeros(16, dtype=torch.float32, device="cuda")
    assert lib.ns_fft_c2r_noalloc(256, 1, ctypes.c_void_p(x.data_ptr()),
                                  ctypes.c_void_p(x.data_ptr()), None) == nat.NS_ERR_UNSUPPORTED_N
    assert lib.ns_fft_c2r_noalloc(30, 1, ctypes.c_void_p(x.data_ptr()),
                                  ctypes.c_void_p(x.data_ptr()), None) == nat.NS_ERR_UNSUPPORTED_N
    assert lib.ns_fft_c2r_noalloc(32, 1, None, None, None) == nat.NS_ERR_ARG
