"""The allocation-free gradient entry point (mihs_gradient_noalloc).

Some callers cannot allocate device memory when they need a gradient (code
inside an allocator or memory-pool callback that must not re-enter the
allocator, code that may allocate only at start-up, or a process with a fixed
memory budget); this entry point keeps its scratch in a fixed array inside
the library instead.  The test calls it directly through the C ABI, twice in
a row on different inputs (the array keeps the previous call's contents),
and checks each result against mihs_gradient, the allocating entry point
(the same kernels in the same order: bit-identical), and against the
oracle's fp64 gradient within the fp32 rounding bound the other gradient
tests use.  After a first call, which looks the array's address up, a call
must leave the device's free memory unchanged.  The file is collected last
and holds whether it runs alone or after the rest.
"""
import ctypes
import gc

import numpy as np
import pytest
import torch

from oracle import mihs_oracle as o
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
    An = A.cpu().numpy().astype(np.float64)
    bn = b.cpu().numpy()
    for x in xs:  # two calls in a row, different inputs
        g = torch.full((d,), float("nan"), device="cuda")
        rc = fn(A.data_ptr(), n, d, lda, b.data_ptr(), x.data_ptr(), lam, g.data_ptr(), stream)
        assert rc == 0, mihs.lib().mihs_last_error()
        g_ref = mihs.gradient(A, b, x, lam)
        torch.cuda.synchronize()
        assert torch.equal(g, g_ref)
        xn = x.cpu().numpy()
        bound = gradient_bound(An, bn, xn, lam, dr, da)
        diff = np.abs(g.double().cpu().numpy() - o.gradient(An, bn, xn, lam))
        assert np.all(np.isfinite(g.cpu().numpy()))
        assert np.all(diff <= bound), f"max diff/bound {np.max(diff / bound)}"


def test_noalloc_allocates_nothing():
    fn = _entry()
    n, d = 20000, 512
    A = W.randn((n, d), seed=50, scale=0.05).cuda()
    b = W.randn((n,), seed=51).cuda()
    x = W.randn((d,), seed=52).cuda()
    g = torch.empty(d, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    assert fn(A.data_ptr(), n, d, d, b.data_ptr(), x.data_ptr(), 0.5, g.data_ptr(), stream) == 0
    # no garbage collection inside the measured window (it would release
    # tensors of earlier tests and move torch's counter)
    gc.collect()
    gc.disable()
    try:
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        torch_bytes = torch.cuda.memory_allocated()
        for _ in range(3):
            assert fn(A.data_ptr(), n, d, d, b.data_ptr(), x.data_ptr(), 0.5, g.data_ptr(), stream) == 0
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        torch_bytes1 = torch.cuda.memory_allocated()
    finally:
        gc.enable()
    assert free1 == free0 and torch_bytes1 == torch_bytes
    assert torch.equal(g, mihs.gradient(A, b, x, 0.5))


def test_noalloc_rejects_bad_arguments():
    fn = _entry()
    A = torch.zeros(16, 8, device="cuda")
    v = torch.zeros(16, device="cuda")
    assert fn(A.data_ptr(), 16, 8, 6, v.data_ptr(), v.data_ptr(), 1.0, v.data_ptr(), None) == -1
    assert fn(A.data_ptr(), 16, 4096, 4096, v.data_ptr(), v.data_ptr(), 1.0, v.data_ptr(), None) == -1
    # λ beyond fp32's range would turn into inf inside the kernel
    assert fn(A.data_ptr(), 16, 8, 8, v.data_ptr(), v.data_ptr(), 1e39, v.data_ptr(), None) == -1
    assert fn(A.data_ptr(), 16, 8, 8, v.data_ptr(), v.data_ptr(), float("nan"), v.data_ptr(), None) == -1
