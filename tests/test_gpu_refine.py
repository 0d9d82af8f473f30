"""Parity of the compensated (refinement) path and of Algorithm 4 with the
oracle: the double-float gradient against an extended-precision gradient,
refined solves against the fp64 solution refined in extended precision, and
the Hutchinson estimate of sd against the oracle's on the same probes."""
import math

import numpy as np
import pytest
import torch

from oracle import mihs_oracle as o
from paper_1912_03514_gb300 import mihs
from paper_1912_03514_gb300 import workloads as W
from tests._tol import apass_depths, gradient_bound_refined

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.mark.parametrize("n,d,lda", [(4096, 256, 256), (3001, 129, 132), (20000, 640, 644), (5000, 2048, 2048),
                                     (33, 1, 4)])
def test_refined_gradient_matches_extended_precision(n, d, lda):
    A = W.padded_matrix(n, d, lda, seed=7 + d)
    b = W.randn((n,), seed=8)
    x = W.randn((d,), seed=9, scale=0.5, dtype=torch.float64)
    lam = 0.29
    Av = A.to(DEV).as_strided((n, d), (lda, 1))
    g = mihs.gradient_refined(Av, b.to(DEV), x.to(DEV), lam).cpu().numpy()
    An = A[:, :d].numpy().astype(np.float64)
    ref = o.gradient_extended(An, b.numpy(), x.numpy(), lam)
    dr, da = apass_depths(n, d, torch.cuda.get_device_properties(0).multi_processor_count)
    bound = gradient_bound_refined(An, b.numpy(), x.numpy(), lam, dr, da)
    err = np.abs(g - np.asarray(ref, dtype=np.float64))
    assert np.all(np.isfinite(g))
    assert np.all(err <= bound), f"max err/bound {np.max(err / bound)}"
    # and it is far more accurate than the plain fp32 gradient
    g32 = mihs.gradient(Av, b.to(DEV), x.float().to(DEV), lam).cpu().double().numpy()
    ref32 = o.gradient_extended(An, b.numpy(), x.float().double().numpy(), lam)
    e32 = np.max(np.abs(g32 - np.asarray(ref32, dtype=np.float64)))
    assert np.max(err) <= 1e-3 * max(e32, 1e-30) or np.max(err) < 1e-12


@pytest.mark.parametrize("family", ["gaussian", "countsketch", "srht"])
def test_refined_solve_reaches_1e10_on_small_problem(family):
    p = W.problem_small()
    A, b = p.A.to(DEV), p.b.to(DEV)
    xs = o.exact_solve(p.A.numpy(), p.b.numpy(), p.lam, refine=3, extended=True)
    with mihs.Sketch(A, family, p.m, seed=12) as sk:
        x, info = sk.solve_refined(A, b, p.lam, p.sd, tol=1e-13, max_outer=200)
    assert info.converged, info
    assert o.rel_error(x.cpu().numpy(), xs) <= 1e-10


def test_plain_fp32_gradient_never_stops_a_refined_solve():
    """A = [1; 1], b = [1, 2⁻³⁰], λ = 2: x* = (1 + 2⁻³⁰)/4 = ¼ + 2⁻³², and at
    the warm start x = ¼ (x*'s fp32 rounding) the plain fp32 gradient is
    exactly 0 (b₂ − x rounds to −¼, so Aᵀr = ½ = λx) while the true one is
    2⁻³⁰.  A refinement solve must not stop on that zero (a plain gradient
    certifies nothing below its own rounding floor): it goes on with
    compensated gradients and reaches x* to fp64 accuracy."""
    A = torch.zeros(2, 4)
    A[:, 0] = 1.0
    Ad = A.to(DEV).as_strided((2, 1), (4, 1))
    b = torch.tensor([1.0, 2.0 ** -30]).to(DEV)
    lam, xs = 2.0, 0.25 + 2.0 ** -32
    assert mihs.gradient(Ad, b, torch.tensor([0.25], device=DEV), lam).item() == 0.0  # the premise
    with mihs.Sketch(Ad, "gaussian", 2, seed=5) as sk:
        x = torch.tensor([0.25], dtype=torch.float64, device=DEV)
        x, info = sk.solve_refined(Ad, b, lam, 0.5, tol=1e-14, max_outer=50, x=x, warm_start=True)
    assert info.converged, info
    assert abs(x.item() - xs) <= 1e-13 * xs, (x.item(), xs)


def test_refined_solve_switches_phase_once():
    """Refinement solves take plain fp32 gradients until the relative residual
    is below 1e-7 or stops improving, then compensated ones.  The host-driven loop (per-kernel
    timing on) launches only the current variant; the graph launches both,
    gated on the device: the two must produce the same bytes."""
    p = W.problem_small()
    A, b = p.A.to(DEV), p.b.to(DEV)
    with mihs.Sketch(A, "gaussian", p.m, seed=12) as sk:
        xg, ig = sk.solve_refined(A, b, p.lam, p.sd, tol=1e-12, max_outer=200)
        mihs.timing(True)
        try:
            xt, it = sk.solve_refined(A, b, p.lam, p.sd, tol=1e-12, max_outer=200)
            _, n_plain = mihs.timing_read(mihs.TIMER_APASS)
            _, n_dd = mihs.timing_read(mihs.TIMER_APASS_DD)
            _, n_corr = mihs.timing_read(mihs.TIMER_APASS_CORR)
        finally:
            mihs.timing(False)
        hist = np.asarray(sk.history(), dtype=np.float64)
    assert ig.converged and it.converged
    assert torch.equal(xg, xt)
    assert ig.outer_iters == it.outer_iters
    assert n_plain >= 1 and n_dd >= 1
    # one gradient per step plus the final stop test (which is a refresh)
    assert n_plain + n_dd + n_corr == it.outer_iters + 1
    # the switch came at the first step whose plain residual was ≤ 1e-7·‖Aᵀb‖
    # or had set no new minimum for three steps
    gmin, stall, k_exp = np.inf, 0, None
    for k, h in enumerate(hist):
        stall = 0 if h < gmin else stall + 1
        gmin = min(gmin, h)
        if h <= 1e-7 * hist[0] or stall >= 3:
            k_exp = k
            break
    assert n_plain - 1 == k_exp


def test_refined_solve_ill_conditioned():
    """κ(H) ≈ 1e6 (eight decades of singular values, λ = 1e-6), the shape of
    the mixed-precision workload at a size the oracle refines quickly: the
    plain fp32 solve stalls near its floor, the refined one reaches 1e-10."""
    n, d = 65536, 512
    sigma = W.profile_exponential(d, 8.0)
    p = W.make_problem(n, d, sigma, 1e-6, 40.0, seed=21)
    A, b = p.A.to(DEV), p.b.to(DEV)
    xs = o.exact_solve(p.A.numpy(), p.b.numpy(), p.lam, refine=3, extended=True)
    with mihs.Sketch(A, "countsketch", p.m, seed=13) as sk:
        x, info = sk.solve_refined(A, b, p.lam, p.sd, tol=1e-14, max_outer=300)
        x32, i32 = sk.solve(A, b, p.lam, p.sd, tol=1e-14, max_outer=300)
    err = o.rel_error(x.cpu().numpy(), xs)
    err32 = o.rel_error(x32.cpu().double().numpy(), xs)
    assert err <= 1e-10, (err, info)
    assert err < 1e-2 * err32


def test_estimate_sd_matches_oracle():
    m, d, lam = 300, 200, 0.05
    SA = W.randn((m, d), 31, scale=1.0 / math.sqrt(m))
    SA[:, 100:] *= 0.01
    for T, eps in ((3, 1e-6), (2, 0.5)):
        sd_gpu = mihs.estimate_sd(SA.to(DEV), lam, T=T, eps_tr=eps, seed=77)
        sd_ref = o.hutchinson_sd(SA.numpy().astype(np.float64), lam, T, eps, seed=77)
        tol = 1e-4 if eps < 1e-3 else 0.05
        assert abs(sd_gpu - sd_ref) <= tol * sd_ref, (T, eps, sd_gpu, sd_ref)


def test_solve_with_estimated_sd():
    """sd ≤ 0 asks the solver to estimate it (Algorithm 4) before iterating."""
    p = W.problem_small()
    A, b = p.A.to(DEV), p.b.to(DEV)
    xs = o.exact_solve(p.A.numpy(), p.b.numpy(), p.lam)
    with mihs.Sketch(A, "gaussian", p.m, seed=5) as sk:
        x, info = sk.solve(A, b, p.lam, 0.0, tol=1e-6, max_outer=300)
    assert info.converged and o.rel_error(x.cpu().double().numpy(), xs) <= 1e-5


def test_refinement_corrections_between_refreshes():
    """κ(H) ≈ 1e4 (the 262144×1024 workload's conditioning at a size the
    oracle refines quickly): after the compensated refresh, fp32 corrections
    g(x_ref) − H(x − x_ref) carry most refinement steps, the solve still ends
    on a compensated gradient and reaches 1e-10 of the exact solution."""
    n, d = 32768, 256
    sigma = 1.0 / np.arange(1, d + 1, dtype=np.float64)
    p = W.make_problem(n, d, sigma, 1e-4, 40.0, seed=23)
    A, b = p.A.to(DEV), p.b.to(DEV)
    xs = o.exact_solve(p.A.numpy(), p.b.numpy(), p.lam, refine=3, extended=True)
    with mihs.Sketch(A, "countsketch", p.m, seed=14) as sk:
        xg, ig = sk.solve_refined(A, b, p.lam, p.sd, tol=1e-12, max_outer=300)
        mihs.timing(True)
        try:
            xt, it = sk.solve_refined(A, b, p.lam, p.sd, tol=1e-12, max_outer=300)
            _, n_plain = mihs.timing_read(mihs.TIMER_APASS)
            _, n_dd = mihs.timing_read(mihs.TIMER_APASS_DD)
            _, n_corr = mihs.timing_read(mihs.TIMER_APASS_CORR)
        finally:
            mihs.timing(False)
    assert ig.converged and it.converged, (ig, it)
    assert torch.equal(xg, xt)  # graph (gated launches) and host-driven steps agree
    assert n_plain + n_dd + n_corr == it.outer_iters + 1
    assert n_corr > n_dd >= 1, (n_plain, n_dd, n_corr)
    assert o.rel_error(xg.cpu().numpy(), xs) <= 1e-10
