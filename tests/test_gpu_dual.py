"""Parity of Dual M-IHS (Algorithm 2, n ≤ d) with the oracle: the sketch of
Aᵀ against the oracle's sketch of the transposed matrix, the dual gradient
and the recovery x = Aᵀν element by element against fp64, and the solves
against the oracle's solution through the dual closed form."""
import math

import numpy as np
import pytest
import torch

from oracle import mihs_oracle as o
from paper_1912_03514_gb300 import mihs
from paper_1912_03514_gb300 import workloads as W
from tests._tol import gamma
from tests.test_gpu_parity import _sketch_bound

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _wide(n, d, seed, decades=2.0):
    """A wide problem: A = Q diag(σ) Vᵀ-like rows via the problem generator on
    the transposed shape (d × n), transposed; b = A x0 + noise."""
    q = W.make_problem(d, n, W.profile_exponential(n, decades), 1e-3, 30.0, seed)
    At = q.A  # d × n with singular values σ
    A = At.t().contiguous()
    g = torch.Generator().manual_seed(seed + 1)
    x0 = torch.randn(d, generator=g, dtype=torch.float64)
    b = (A.double() @ x0)
    b = (b + 0.01 * b.norm() / math.sqrt(n) * torch.randn(n, generator=g, dtype=torch.float64)).float()
    return A, b, q.sigma


@pytest.mark.parametrize("n,d", [(256, 4096), (100, 3000), (7, 33), (1024, 65536)])
def test_gradient_dual_and_recover_elementwise(n, d):
    A = W.randn((n, d), 60 + n, scale=1.0 / math.sqrt(d))
    b = W.randn((n,), 61)
    nu = W.randn((n,), 62)
    lam = 0.3
    lda = (d + 3) // 4 * 4
    Ap = torch.zeros(n, lda)
    Ap[:, :d] = A
    Ad = Ap.to(DEV).as_strided((n, d), (lda, 1))
    g = mihs.gradient_dual(Ad, b.to(DEV), nu.to(DEV), lam).cpu().double().numpy()
    x = mihs.dual_recover(Ad, nu.to(DEV)).cpu().double().numpy()
    An, bn, nn = A.double().numpy(), b.double().numpy(), nu.double().numpy()
    u = An.T @ nn
    e_u = gamma(n + 1) * (np.abs(An.T) @ np.abs(nn))
    assert np.all(np.abs(x - u) <= e_u)
    ref = bn - An @ u - lam * nn
    # |A||û − u| + rounding of the row dot (≤ d terms, any order) and of b − · − λν
    e_g = np.abs(An) @ e_u + gamma(d + 3) * (np.abs(bn) + np.abs(An) @ np.abs(u) + lam * np.abs(nn))
    assert np.all(np.abs(g - ref) <= e_g)


@pytest.mark.parametrize("family", ["gaussian", "countsketch", "srht"])
def test_dual_sketch_matches_oracle(family):
    n, d, m = 96, 3000, 160
    A = W.randn((n, d), 70, scale=0.1)
    fam = mihs.family_id(family)
    with mihs.DualSketch(A.to(DEV), family, m, seed=17) as dk:
        SAt = dk.sat().cpu().double().numpy()
    At = A.numpy().T.astype(np.float64)
    ref = o.sketch_apply(fam, At, m, 17)
    bound = _sketch_bound(fam, At, m, 17, d)  # the sketch kernels' bound, on Aᵀ
    assert np.all(np.abs(SAt - ref) <= bound)


@pytest.mark.parametrize("family", ["gaussian", "countsketch", "srht"])
def test_dual_solve_matches_oracle(family):
    n, d, lam = 256, 16384, 1e-3
    A, b, sigma = _wide(n, d, seed=80)
    sd = W.nominal_sd(sigma, lam)
    m = int(math.ceil(4 * sd / 4)) * 4
    xs, nus = o.exact_solve_dual(A.numpy(), b.numpy(), lam)
    with mihs.DualSketch(A.to(DEV), family, m, seed=19) as dk:
        x, nu, info = dk.solve(A.to(DEV), b.to(DEV), lam, sd, tol=1e-6, max_outer=200)
    assert info.converged, info
    assert o.rel_error(nu.cpu().double().numpy(), nus) <= 1e-4
    assert o.rel_error(x.cpu().double().numpy(), xs) <= 1e-4
    # the oracle's own Algorithm 2 on the same SAᵀ converges to the same point
    SAt = o.sketch_apply(mihs.family_id(family), A.numpy().T.astype(np.float64), m, 19)
    xo, _, _ = o.dual_mihs(A.numpy(), b.numpy(), lam, SAt, sd, N=200, tol=1e-10)
    assert o.rel_error(xo, xs) <= 1e-8


def test_dual_warm_start_and_estimated_sd():
    n, d, lam = 128, 8192, 1e-2
    A, b, sigma = _wide(n, d, seed=81)
    xs, _ = o.exact_solve_dual(A.numpy(), b.numpy(), lam)
    m = 4 * 64
    with mihs.DualSketch(A.to(DEV), "countsketch", m, seed=3) as dk:
        x, nu, info = dk.solve(A.to(DEV), b.to(DEV), lam, 0.0, tol=1e-6, max_outer=300)  # sd from Algorithm 4
        x2, nu2, info2 = dk.solve(A.to(DEV), b.to(DEV), lam, 0.0, tol=2e-6, nu=nu.clone(), warm_start=True)
    assert info.converged and o.rel_error(x.cpu().double().numpy(), xs) <= 1e-4
    assert info2.converged and info2.outer_iters == 0 and torch.equal(nu2, nu)


def test_dual_invalid_arguments():
    A = W.randn((64, 32), 1).to(DEV)  # n > d: not the dual regime
    with pytest.raises(mihs.MihsError):
        mihs.DualSketch(A, "countsketch", 16, seed=1)
    A = W.randn((3000, 4000), 1).to(DEV)  # n > 2048
    with pytest.raises(mihs.MihsError):
        mihs.DualSketch(A, "countsketch", 16, seed=1)
