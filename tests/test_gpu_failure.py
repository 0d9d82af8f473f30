"""Failure detection without a GPU fault: the library's bounded waits, run on
conditions that nothing satisfies with a short limit, return and report
MIHS_ERR_TIMEOUT; the device stays usable afterwards (a solve that follows is
checked against the oracle) and the device error word is untouched."""
import time

import pytest
import torch

from oracle import mihs_oracle as o
from paper_1912_03514_gb300 import mihs
from paper_1912_03514_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.mark.parametrize("which", [0, 1], ids=["mbarrier", "grid-barrier"])
def test_bounded_wait_times_out_and_device_stays_usable(which):
    torch.cuda.synchronize()
    assert mihs.device_status() == 0
    limit = 0.05
    t0 = time.perf_counter()
    st = mihs.selftest_wait(which, limit)
    dt = time.perf_counter() - t0
    assert st == mihs.ERR_TIMEOUT
    assert limit <= dt < limit + 5.0
    assert mihs.device_status() == 0
    # the context is intact: a solve after the timeout reaches the solution
    p = W.problem_scaled(8192, 128, seed=23)
    x, info = mihs.solve(p.A.to(DEV), p.b.to(DEV), p.lam, "countsketch", p.m, p.sd, seed=5, tol=1e-6,
                         max_outer=200)
    xs = o.exact_solve(p.A.numpy(), p.b.numpy(), p.lam)
    assert info.converged and o.rel_error(x.cpu().double().numpy(), xs) <= 1e-5
