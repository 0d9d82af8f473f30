"""Parity of the gradients of the solve with the oracle's adjoint formulas:
the fused pass (mihs_backward_grads) element by element against fp64 with
bounds from its fp32 arithmetic, the adjoint solve plus pass (mihs_backward)
against the oracle's exact gradients, and the autograd Function against
PyTorch's fp64 autograd through a dense solve."""
import numpy as np
import pytest
import torch

from oracle import mihs_oracle as o
from paper_1912_03514_gb300 import mihs
from paper_1912_03514_gb300 import workloads as W
from tests._tol import U32, gamma

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _grad_bounds(A, b, x, v):
    """Componentwise bounds for the fused pass: r̂ = b − A·x and q̂ = A·v are
    warp-reduced fp32 dot products (≤ d products per row in any order, γ_{d+1});
    each dA entry is fma(r̂, v_j, −fl(q̂·x_j)) (two more roundings)."""
    A = np.asarray(A, np.float64)
    Aa = np.abs(A)
    ax, av = np.abs(np.asarray(x, np.float64)), np.abs(np.asarray(v, np.float64))
    d = A.shape[1]
    e_r = gamma(d + 2) * (np.abs(np.asarray(b, np.float64)) + Aa @ ax)
    e_q = gamma(d + 1) * (Aa @ av)
    r = np.asarray(b, np.float64) - A @ np.asarray(x, np.float64)
    q = A @ np.asarray(v, np.float64)
    eA = (np.outer(e_r, av) + np.outer(e_q, ax)
          + 2 * U32 * (np.outer(np.abs(r) + e_r, av) + np.outer(np.abs(q) + e_q, ax)))
    return e_q, eA


@pytest.mark.parametrize("n,d,lda", [(4096, 256, 256), (3001, 1024, 1024), (777, 2048, 2048),
                                     (1000, 100, 100), (5000, 512, 516), (513, 129, 132),
                                     (33, 1, 4), (700, 2046, 2048), (1, 8, 8)])
def test_backward_grads_elementwise(n, d, lda):
    A = W.padded_matrix(n, d, lda, seed=40 + d)
    b = W.randn((n,), 41)
    x = W.randn((d,), 42, scale=0.3)
    v = W.randn((d,), 43, scale=0.7)
    Ad = A.to(DEV).as_strided((n, d), (lda, 1))
    dA, db, dl = mihs.backward_grads(Ad, b.to(DEV), x.to(DEV), v.to(DEV))
    An = A[:, :d].numpy().astype(np.float64)
    xn, vn, bn = x.double().numpy(), v.double().numpy(), b.double().numpy()
    rA = np.outer(bn - An @ xn, vn) - np.outer(An @ vn, xn)
    e_q, eA = _grad_bounds(An, bn, xn, vn)
    dA, db = dA.cpu().double().numpy(), db.cpu().double().numpy()
    assert np.all(np.isfinite(dA)) and np.all(np.isfinite(db))
    assert np.all(np.abs(db - An @ vn) <= e_q)
    assert np.all(np.abs(dA - rA) <= eA), np.max(np.abs(dA - rA) / eA)
    ref_l = -(xn @ vn)
    assert abs(dl.item() - ref_l) <= 4 * d * 2.0 ** -53 * (np.abs(xn) @ np.abs(vn)) + 1e-300


def test_backward_grads_optional_outputs():
    n, d = 2048, 256
    A = W.randn((n, d), 50).to(DEV)
    b = W.randn((n,), 51).to(DEV)
    x = W.randn((d,), 52).to(DEV)
    v = W.randn((d,), 53).to(DEV)
    full = mihs.backward_grads(A, b, x, v)
    dA, db, dl = mihs.backward_grads(A, None, x, v, want_dA=False)
    assert dA is None and torch.equal(db, full[1]) and torch.equal(dl, full[2])
    dA, db, dl = mihs.backward_grads(A, b, x, v, want_db=False, want_dlambda=False)
    assert db is None and dl is None and torch.equal(dA, full[0])
    _, _, dl = mihs.backward_grads(A, None, x, v, want_dA=False, want_db=False)
    assert torch.equal(dl, full[2])
    with pytest.raises(mihs.MihsError):  # dA needs r = b − Ax
        mihs.backward_grads(A, None, x, v)


def test_backward_grads_full_size_sampled_rows():
    """2²⁰ × 1024 (the differentiable workload's shape): rows sampled across
    the matrix against fp64, with the same bounds."""
    n, d = 1 << 20, 1024
    g = torch.Generator(device=DEV).manual_seed(60)
    A = torch.randn(n, d, device=DEV, generator=g)
    b = torch.randn(n, device=DEV, generator=g)
    x = torch.randn(d, device=DEV, generator=g) * 0.1
    v = torch.randn(d, device=DEV, generator=g) * 0.1
    dA, db, dl = mihs.backward_grads(A, b, x, v)
    rows = torch.cat([torch.arange(0, 64), torch.randint(0, n, (192,), generator=torch.Generator().manual_seed(61)),
                      torch.arange(n - 64, n)]).to(DEV)
    An = A[rows].cpu().double().numpy()
    bn = b[rows].cpu().double().numpy()
    xn, vn = x.cpu().double().numpy(), v.cpu().double().numpy()
    e_q, eA = _grad_bounds(An, bn, xn, vn)
    ref = np.outer(bn - An @ xn, vn) - np.outer(An @ vn, xn)
    assert np.all(np.abs(dA[rows].cpu().double().numpy() - ref) <= eA)
    assert np.all(np.abs(db[rows].cpu().double().numpy() - An @ vn) <= e_q)
    assert abs(dl.item() + xn @ vn) <= 1e-12 * (np.abs(xn) @ np.abs(vn))


def _problem():
    p = W.problem_small()
    rng = np.random.default_rng(70)
    w = rng.standard_normal(p.d).astype(np.float32)
    return p, w


@pytest.mark.parametrize("family", ["gaussian", "countsketch", "srht"])
def test_backward_matches_oracle(family):
    """mihs_backward (adjoint M-IHS solve with the forward sketch, then the
    fused pass) against the oracle's exact gradients.  H ⪰ λ_min(H)·I gives
    the certificates ‖x̂ − x*‖ ≤ ‖Aᵀb − Hx̂‖/λ_min and ‖v̂ − v*‖ ≤ ‖ḡ − Hv̂‖/λ_min
    (residuals in fp64); the gradients' differences are bounded through
    them plus the fused pass's fp32 rounding.  The adjoint's right-hand side
    ḡ is a generic vector, not Aᵀb, so its fp32 residual floor is higher
    (≈ κ(H)·u·‖ḡ‖ at worst, a few 1e-7 here): it is solved to 1e-6."""
    p, w = _problem()
    A, b = p.A.to(DEV), p.b.to(DEV)
    tol, tol_adj = 1e-7, 1e-6
    An, bn = p.A.double().numpy(), p.b.double().numpy()
    xs, vs, dAs, dbs, dls = o.ridge_backward(An, bn, p.lam, w.astype(np.float64))
    H = An.T @ An + p.lam * np.eye(p.d)
    ev = np.linalg.eigvalsh(H)
    smax = np.sqrt(max(ev[-1] - p.lam, 0.0))
    with mihs.Sketch(A, family, p.m, seed=5) as sk:
        x, ix = sk.solve(A, b, p.lam, p.sd, tol=tol, max_outer=300)
        dA, db, dl, v, iv = sk.backward(A, b, p.lam, p.sd, x, torch.from_numpy(w).to(DEV), tol=tol_adj,
                                        max_outer=300)
    assert ix.converged and iv.converged, (ix, iv)
    xn, vn = x.cpu().double().numpy(), v.cpu().double().numpy()
    rho_v = np.linalg.norm(w - H @ vn)
    assert rho_v <= 2 * tol_adj * np.linalg.norm(w)  # the adjoint solve did reach its tolerance
    ex = np.linalg.norm(An.T @ bn - H @ xn) / ev[0]
    ev_ = rho_v / ev[0]
    assert np.linalg.norm(vn - vs) <= ev_ * (1 + 1e-9)
    e_q, eA = _grad_bounds(An, bn, xn, vn)
    # db = Av
    assert np.linalg.norm(db.cpu().double().numpy() - dbs) <= smax * ev_ + np.linalg.norm(e_q) + 1e-300
    # dλ = −xᵀv
    assert abs(dl.item() - dls) <= ex * np.linalg.norm(vn) + np.linalg.norm(xs) * ev_ + 1e-12 * abs(dls)
    # dA = r vᵀ − (Av)xᵀ
    rs, qs = bn - An @ xs, An @ vs
    e_dA = (smax * ex * np.linalg.norm(vn) + np.linalg.norm(rs) * ev_
            + smax * ev_ * np.linalg.norm(xn) + np.linalg.norm(qs) * ex + np.linalg.norm(eA))
    assert np.linalg.norm(dA.cpu().double().numpy() - dAs) <= e_dA


def test_backward_padded_lda_and_warm_start():
    p, w = _problem()
    n, d, lda = p.n, p.d, p.d + 4
    Ap = torch.full((n, lda), float("nan"))
    Ap[:, :d] = p.A
    A = Ap.to(DEV).as_strided((n, d), (lda, 1))
    b = p.b.to(DEV)
    wt = torch.from_numpy(w).to(DEV)
    with mihs.Sketch(A, "countsketch", p.m, seed=6) as sk:
        x, _ = sk.solve(A, b, p.lam, p.sd, tol=1e-7)
        dA, db, dl, v, iv = sk.backward(A, b, p.lam, p.sd, x, wt, tol=1e-6)
        # warm start from the converged adjoint: stops at the first test
        _, _, _, v2, iv2 = sk.backward(A, b, p.lam, p.sd, x, wt, tol=2e-6, v=v.clone(), warm_start=True)
    assert torch.isfinite(dA).all() and iv.converged
    assert iv2.converged and iv2.outer_iters == 0
    assert torch.equal(v2, v)
    _, vs, dAs, _, _ = o.ridge_backward(p.A.numpy(), p.b.numpy(), p.lam, w.astype(np.float64))
    assert o.rel_error(v.cpu().double().numpy(), vs) <= 1e-4


def test_backward_deterministic_and_graphs_coexist():
    """Forward and adjoint solves on one handle alternate without
    disturbing each other; repeated calls give identical bytes."""
    p, w = _problem()
    A, b = p.A.to(DEV), p.b.to(DEV)
    wt = torch.from_numpy(w).to(DEV)
    outs = []
    with mihs.Sketch(A, "gaussian", p.m, seed=7) as sk:
        for _ in range(3):
            x, _ = sk.solve(A, b, p.lam, p.sd, tol=1e-7)
            dA, db, dl, v, _ = sk.backward(A, b, p.lam, p.sd, x, wt, tol=1e-6)
            outs.append((x.clone(), dA.clone(), db.clone(), dl.clone(), v.clone()))
    for t in outs[1:]:
        for a, c in zip(outs[0], t):
            assert torch.equal(a, c)


def test_ridge_solve_autograd_matches_torch_fp64():
    """RidgeSolve against PyTorch's own fp64 autograd through a dense solve
    of the normal equations (a plain reference independent of the oracle)."""
    p, w = _problem()
    wt = torch.from_numpy(w)
    A = p.A.to(DEV).requires_grad_(True)
    b = p.b.to(DEV).requires_grad_(True)
    lam = torch.tensor(p.lam, dtype=torch.float64, device=DEV, requires_grad=True)
    x = mihs.ridge_solve(A, b, lam, family="countsketch", m=p.m, sd=p.sd, seed=3, tol=1e-7, max_outer=100)
    (x * wt.to(DEV)).sum().backward()

    A64 = p.A.double().requires_grad_(True)
    b64 = p.b.double().requires_grad_(True)
    l64 = torch.tensor(p.lam, dtype=torch.float64, requires_grad=True)
    H = A64.T @ A64 + l64 * torch.eye(p.d, dtype=torch.float64)
    x64 = torch.linalg.solve(H, A64.T @ b64)
    (x64 * wt.double()).sum().backward()

    def rel(a, r):
        return (a.detach().cpu().double() - r).norm().item() / r.norm().item()

    # residual ≤ 1e-7 (the adjoint stops at its fp32 floor, a few 1e-7) and
    # κ(H) ≈ 98 put every relative error below ~1e-4
    assert rel(x, x64.detach()) <= 1e-4
    assert rel(A.grad, A64.grad) <= 1e-4
    assert rel(b.grad, b64.grad) <= 1e-4
    assert abs(lam.grad.item() - l64.grad.item()) <= 1e-4 * abs(l64.grad.item())


def _ill_conditioned():
    """σᵢ = i^(−1.5), λ = 1e-4 (κ(H) ≈ 1e4): the differentiable workload's
    profile at a size the oracle solves quickly."""
    n, d = 65536, 512
    p = W.make_problem(n, d, W.profile_polynomial(d, 1.5), 1e-4, 40.0, seed=80)
    w = np.random.default_rng(81).standard_normal(d).astype(np.float32)
    return p, w


def test_backward_refined_matches_oracle():
    """mihs_backward_refined: the adjoint reaches 1e-10 (the fp32 adjoint
    stalls orders of magnitude above); every gradient within its rigorous
    bound: x and v errors (fp64 vs the oracle, then rounded to fp32) pushed
    through the formulas componentwise, plus the fused pass's rounding."""
    p, w = _ill_conditioned()
    A, b = p.A.to(DEV), p.b.to(DEV)
    An, bn = p.A.double().numpy(), p.b.double().numpy()
    wt = torch.from_numpy(w).to(DEV)
    xs, vs, dAs, dbs, dls = o.ridge_backward(An, bn, p.lam, w.astype(np.float64))
    with mihs.Sketch(A, "countsketch", p.m, seed=9) as sk:
        x64, ix = sk.solve_refined(A, b, p.lam, p.sd, tol=1e-11, max_outer=300)
        dA, db, dl, v64, iv = sk.backward_refined(A, b, p.lam, p.sd, x64, wt, tol=1e-10, max_outer=300)
        x32, _ = sk.solve(A, b, p.lam, p.sd, tol=1e-10, max_outer=300)
        _, _, _, v32p, iv32 = sk.backward(A, b, p.lam, p.sd, x32, wt, tol=1e-10, max_outer=300)
    assert ix.converged and iv.converged, (ix, iv)
    vn = v64.cpu().numpy()
    err_v = o.rel_error(vn, vs)
    assert err_v <= 1e-8, err_v
    assert err_v < 1e-2 * o.rel_error(v32p.cpu().double().numpy(), vs)
    x32n = x64.cpu().float().double().numpy()
    v32n = v64.cpu().float().double().numpy()
    Aa = np.abs(An)
    ex, ev_ = np.abs(x32n - xs), np.abs(v32n - vs)
    e_q, eA = _grad_bounds(An, bn, x32n, v32n)
    assert np.all(np.abs(db.cpu().double().numpy() - dbs) <= Aa @ ev_ + e_q)
    rs, qs = bn - An @ xs, An @ vs
    bound_A = (np.outer(Aa @ ex, np.abs(v32n)) + np.outer(np.abs(rs), ev_)
               + np.outer(Aa @ ev_, np.abs(x32n)) + np.outer(np.abs(qs), ex) + eA)
    assert np.all(np.abs(dA.cpu().double().numpy() - dAs) <= bound_A)
    bound_l = ex @ np.abs(v32n) + np.abs(xs) @ ev_ + 4 * p.d * 2.0 ** -53 * (np.abs(x32n) @ np.abs(v32n))
    assert abs(dl.item() - dls) <= bound_l


def test_ridge_solve_refined_autograd_matches_torch_fp64():
    p, w = _ill_conditioned()
    wt = torch.from_numpy(w)
    A = p.A.to(DEV).requires_grad_(True)
    b = p.b.to(DEV).requires_grad_(True)
    lam = torch.tensor(p.lam, dtype=torch.float64, device=DEV, requires_grad=True)
    x = mihs.ridge_solve(A, b, lam, family="countsketch", m=p.m, sd=p.sd, seed=4, tol=1e-10, max_outer=300,
                         refine=True)
    assert x.dtype == torch.float64
    (x * wt.to(DEV).double()).sum().backward()
    A64 = p.A.double().requires_grad_(True)
    b64 = p.b.double().requires_grad_(True)
    l64 = torch.tensor(p.lam, dtype=torch.float64, requires_grad=True)
    x64 = torch.linalg.solve(A64.T @ A64 + l64 * torch.eye(p.d, dtype=torch.float64), A64.T @ b64)
    (x64 * wt.double()).sum().backward()

    def rel(a, r):
        return (a.detach().cpu().double() - r).norm().item() / r.norm().item()

    # fp64 solves to 1e-10 with κ(H) ≈ 1e4: x within ~1e-6 (dense fp64 solve
    # of the normal equations itself errs by ~κ²·u₆₄); gradients are fp32
    assert rel(x, x64.detach()) <= 1e-6
    assert rel(A.grad, A64.grad) <= 1e-5
    assert rel(b.grad, b64.grad) <= 1e-5
    assert abs(lam.grad.item() - l64.grad.item()) <= 1e-5 * abs(l64.grad.item())
