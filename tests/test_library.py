"""The C-ABI library builds for sm_103a, loads, exports every entry point the
header declares, and rejects bad arguments on the host (no GPU needed: these
calls return before any CUDA call)."""
import ctypes
import os
import re

import pytest

from paper_1912_03514_gb300 import _build, mihs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    _build.build()
    return mihs.lib()


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"^[A-Za-z_][\w \*]*?\b(mihs_\w+)\s*\(", txt, re.M))
    return names


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert {"mihs_sketch", "mihs_solve", "mihs_gradient", "mihs_aab_solve"} <= names
    for n in sorted(names):
        assert hasattr(L, n), n


def test_strerror_and_defaults(L):
    for code in (0, 1, -1, -2, -3, -4, -5, -6):
        assert L.mihs_strerror(code)
    o = L.mihs_default_opts()
    assert (o.tol, o.max_outer, o.eps_sub, o.max_inner, o.warm_start) == (1e-6, 100, 0.1, 0, 0)


FAKE = ctypes.c_void_p(1 << 20)   # aligned, never dereferenced: rejected first


def test_host_side_argument_checks(L):
    EINVAL = -1
    assert L.mihs_gradient(None, 10, 4, 4, FAKE, FAKE, 1.0, FAKE, None) == EINVAL
    assert L.mihs_gradient(FAKE, 10, 4, 6, FAKE, FAKE, 1.0, FAKE, None) == EINVAL  # lda % 4
    assert L.mihs_gradient(FAKE, 10, 4096, 4096, FAKE, FAKE, 1.0, FAKE, None) == EINVAL  # d
    assert L.mihs_gradient(FAKE, 10, 4, 4, FAKE, FAKE, -1.0, FAKE, None) == EINVAL
    assert L.mihs_sketch_apply(FAKE, 10, 4, 4, 7, 5, 0, FAKE, 4, None) == EINVAL  # family
    assert L.mihs_sketch_apply(FAKE, 10, 4, 4, 0, 11, 0, FAKE, 4, None) == EINVAL  # m > n
    assert L.mihs_aab_solve(FAKE, 8, 4, 4, FAKE, 0.0, 0.1, 0, FAKE, None, None) == EINVAL
    assert L.mihs_aab_solve(FAKE, 8, 4, 4, FAKE, 1.0, -0.1, 0, FAKE, None, None) == EINVAL
    assert L.mihs_aab_solve(FAKE, 8, 4, 3, FAKE, 1.0, 0.1, 0, FAKE, None, None) == EINVAL  # ldsa < d
    o = L.mihs_default_opts()
    assert L.mihs_solve(None, FAKE, 4, FAKE, 1.0, ctypes.byref(o), FAKE, None, None) == EINVAL
    assert b"lambda" in L.mihs_last_error() or b"null" in L.mihs_last_error()
    assert L.mihs_sketch_set_aab(None, 0, 0) == EINVAL
    st = ctypes.c_int()
    assert L.mihs_selftest_wait(2, 50_000_000, ctypes.byref(st), None) == EINVAL  # which
    assert L.mihs_selftest_wait(0, 10, ctypes.byref(st), None) == EINVAL  # limit below 1 ms
    assert L.mihs_selftest_wait(0, 50_000_000, None, None) == EINVAL
    assert L.mihs_copy_to_device(FAKE, FAKE, -1, None) == EINVAL
    assert L.mihs_copy_to_device(None, FAKE, 16, None) == EINVAL
    assert L.mihs_copy_to_device(FAKE, FAKE, 0, None) == 0  # nothing to copy
    assert L.mihs_copy_to_device_dma(FAKE, FAKE, -1, None) == EINVAL
    assert L.mihs_copy_to_device_dma(FAKE, None, 16, None) == EINVAL
    assert L.mihs_copy_to_device_dma(FAKE, FAKE, 0, None) == 0
    assert L.mihs_sketch_destroy(None) == 0


def test_binding_rejects_host_tensors_before_any_cuda_call():
    """The binding marshals arguments only: it refuses what the C ABI could
    not take (host tensors, wrong dtype or layout) before calling into the
    library, so no CPU path can stand in for the kernels."""
    import torch
    A = torch.zeros(16, 4)
    v4, v16 = torch.zeros(4), torch.zeros(16)
    with pytest.raises(ValueError):
        mihs.gradient(A, v16, v4, 1.0)
    with pytest.raises(ValueError):
        mihs._mat(torch.zeros(16, 4, dtype=torch.float64), "A")
    with pytest.raises(ValueError):
        mihs._mat(torch.zeros(4, 16).t(), "A")  # column stride 4
    with pytest.raises(ValueError):
        mihs._vec(torch.zeros(8)[::2], 4, "x")  # not contiguous
    with pytest.raises(ValueError):
        mihs.copy_to_device(torch.zeros(4), torch.zeros(4))  # destination on the host
    with pytest.raises(ValueError):
        mihs._prec("fp4")
    assert mihs.family_id("srht") == 2 and mihs.AAB_FORMS["grid"] == 2
