"""The allocation-free gradient entry point (mihs_gradient_noalloc).

Some callers cannot allocate device memory when they need a gradient (inside
a stream capture that forbids allocation, inside an allocator callback, or
under a fixed memory budget); this entry point keeps its scratch in a fixed
array inside the library instead.  The test calls it directly through the C
ABI, twice in a row on different inputs (the array keeps the previous call's
contents), and checks each result against mihs_gradient, the allocating entry
point, within the gradient tolerance the other tests use.  It lives in its
own file, collected last, and holds whether it runs alone or after the rest.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1912_03514_gb300 import mihs
from paper_1912_03514_gb300 import workloads as W
from tests._tol import apass_depths, gradient_bound

pytestmark = pytest.mark.gpu


def _entry():
    fn = mihs.lib().mihs_gradient_noalloc
    v, i64 = ctypes.c_void_p, ctypes.c_int64
    fn.restype = ctypes.c_int
    fn.argtypes = [v, i64, i64, i64, v, v, ctypes.c_double, v, v]
    return fn


@pytest.mark.parametrize("n,d,lda", [(65536, 1024, 1024), (3001, 129, 132), (5000, 2048, 2048)])
def test_noalloc_gradient_matches_allocating_entry_point(n, d, lda):
    fn = _entry()
    A = W.padded_matrix(n, d, lda, seed=40 + d).cuda().as_strided((n, d), (lda, 1))
    b = W.randn((n,), seed=41).cuda()
    xs = [W.randn((d,), seed=42 + k, scale=0.2 * (k + 1)).cuda() for k in range(2)]
    lam = 0.25
    stream = torch.cuda.current_stream().cuda_stream
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    dr, da = apass_depths(n, d, sms)
    An = A.cpu().numpy()
    for x in xs:  # two calls in a row, different inputs
        g = torch.full((d,), float("nan"), device="cuda")
        rc = fn(A.data_ptr(), n, d, lda, b.data_ptr(), x.data_ptr(), lam, g.data_ptr(), stream)
        assert rc == 0, mihs.lib().mihs_last_error()
        g_ref = mihs.gradient(A, b, x, lam)
        torch.cuda.synchronize()
        bound = gradient_bound(An, b.cpu().numpy(), x.cpu().numpy(), lam, dr, da)
        diff = np.abs(g.double().cpu().numpy() - g_ref.double().cpu().numpy())
        assert np.all(np.isfinite(g.cpu().numpy()))
        assert np.all(diff <= bound), f"max diff/bound {np.max(diff / bound)}"


def test_noalloc_rejects_bad_arguments():
    fn = _entry()
    A = torch.zeros(16, 8, device="cuda")
    v = torch.zeros(16, device="cuda")
    assert fn(A.data_ptr(), 16, 8, 6, v.data_ptr(), v.data_ptr(), 1.0, v.data_ptr(), None) == -1
    assert fn(A.data_ptr(), 16, 4096, 4096, v.data_ptr(), v.data_ptr(), 1.0, v.data_ptr(), None) == -1
