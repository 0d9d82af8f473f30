"""Parity of the λ-path and batched solves with the oracle: the fused
multi-iterate gradient pass element by element against fp64 within its
rounding bound, and every λ of a path against the oracle's exact x*(λ)
through the certificate ‖x − x*‖ ≤ ‖g(x)‖/λ_min(H)."""
import math

import numpy as np
import pytest
import torch

from oracle import mihs_oracle as o
from paper_1912_03514_gb300 import mihs
from paper_1912_03514_gb300 import workloads as W
from tests._tol import gradient_bound

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _path_depths(n, d, num_sms):
    """Rounding depths of the path pass: a row residual is ≤ 4⌈d/128⌉ chained
    products per thread, 2 shuffle levels, 8 warp partials and b − ·; a
    column sum is the rows of one block in sequence, the row subsets, the
    ≤ P/8 + 8 partial sums of the finalize and − λx."""
    ch = max(1, math.ceil(d / 128))
    depth_r = 4 * ch + 2 + 8 + 2
    P = min(num_sms, max(1, math.ceil(n / 16)))
    rows = math.ceil(math.ceil(n / P) / 16) * 16
    depth_acc = rows + 16 + math.ceil(P / 8) + 8 + 2
    return depth_r, depth_acc


@pytest.mark.parametrize("n,d,lda,nl", [(4096, 256, 256, 16), (3001, 1024, 1024, 16), (2000, 129, 132, 5),
                                        (17, 64, 64, 1), (5000, 512, 516, 16), (40, 1, 4, 3),
                                        (1000, 100, 100, 16), (333, 1000, 1000, 7)])
def test_gradient_path_elementwise(n, d, lda, nl):
    A = W.padded_matrix(n, d, lda, seed=90 + d)
    b = W.randn((n,), 91)
    X = W.randn((nl, d), 92, scale=0.3)
    lams = list(np.logspace(-3, 0, nl))
    Ad = A.to(DEV).as_strided((n, d), (lda, 1))
    G = mihs.gradient_path(Ad, b.to(DEV), X.to(DEV), lams).cpu().double().numpy()
    An = A[:, :d].numpy().astype(np.float64)
    dr, da = _path_depths(n, d, torch.cuda.get_device_properties(0).multi_processor_count)
    assert np.all(np.isfinite(G))
    for l in range(nl):
        x = X[l].double().numpy()
        ref = o.gradient(An, b.double().numpy(), x, lams[l])
        bound = gradient_bound(An, b.numpy(), x, lams[l], dr, da)
        err = np.abs(G[l] - ref)
        assert np.all(err <= bound), (l, float(np.max(err / bound)))


def _certified(A, b, lam, x, xs):
    """‖x − x*‖ ≤ ‖Aᵀb − Hx‖/λ_min(H) with λ_min(H) ≥ λ (fp64 residual)."""
    An = np.asarray(A, np.float64)
    r = An.T @ (np.asarray(b, np.float64) - An @ x) - lam * x
    return np.linalg.norm(x - xs) <= np.linalg.norm(r) / lam * (1 + 1e-9) + 1e-300, np.linalg.norm(r)


@pytest.fixture(params=["grid", "cluster"])
def aab_form(request, monkeypatch):
    """Both AAb forms of a path step: one thread-block cluster per λ (default)
    and all λ in one cooperative grid."""
    monkeypatch.setenv("MIHS_PATH_AAB", request.param)
    return request.param


@pytest.mark.parametrize("family", ["gaussian", "countsketch", "srht"])
def test_path_solve_matches_oracle(family, aab_form):
    p = W.problem_small()
    A, b = p.A.to(DEV), p.b.to(DEV)
    lams = list(np.logspace(-3, -1, 16))
    sds = [W.nominal_sd(p.sigma, l) for l in lams]
    tol = 1e-6
    with mihs.Sketch(A, family, p.m, seed=21) as sk:
        X, infos = sk.solve_path(A, b, lams, sds=sds, tol=tol, max_outer=200)
        x5, i5 = sk.solve(A, b, lams[5], sds[5], tol=tol, max_outer=200)
    An, bn = p.A.double().numpy(), p.b.double().numpy()
    XS = o.ridge_path(An, bn, lams)
    atb = np.linalg.norm(An.T @ bn)
    Xn = X.cpu().double().numpy()
    for l, (inf, lam) in enumerate(zip(infos, lams)):
        assert inf.converged, (l, inf)
        ok, rnorm = _certified(An, bn, lam, Xn[l], XS[l])
        assert ok
        assert rnorm <= 4 * tol * atb, (l, rnorm / atb)  # the fp32 stop test is honest in fp64
        assert o.rel_error(Xn[l], XS[l]) <= 1e-4
    # the same λ solved alone with the same sketch reaches the same point
    assert o.rel_error(x5.cpu().double().numpy(), XS[5]) <= 1e-4
    assert np.linalg.norm(Xn[5] - x5.cpu().double().numpy()) <= 2e-4 * np.linalg.norm(XS[5])


def test_path_estimated_sd_and_groups_of_16(aab_form):
    """sd from Algorithm 4 per λ, and 20 λ (two groups of the path loop)."""
    p = W.problem_scaled(8192, 128, seed=31)
    A, b = p.A.to(DEV), p.b.to(DEV)
    lams = list(np.logspace(-4, 0, 20))
    m = 4 * 128
    with mihs.Sketch(A, "countsketch", m, seed=3) as sk:
        X, infos = sk.solve_path(A, b, lams, sds=None, tol=1e-6, max_outer=300)
    An, bn = p.A.double().numpy(), p.b.double().numpy()
    XS = o.ridge_path(An, bn, lams)
    Xn = X.cpu().double().numpy()
    for l, inf in enumerate(infos):
        assert inf.converged, (l, inf)
        assert _certified(An, bn, lams[l], Xn[l], XS[l])[0]


def test_path_warm_start_and_determinism(aab_form):
    p = W.problem_small()
    A, b = p.A.to(DEV), p.b.to(DEV)
    lams = list(np.logspace(-2.5, -1, 8))
    sds = [W.nominal_sd(p.sigma, l) for l in lams]
    with mihs.Sketch(A, "gaussian", p.m, seed=5) as sk:
        X1, _ = sk.solve_path(A, b, lams, sds=sds, tol=1e-6)
        X2, _ = sk.solve_path(A, b, lams, sds=sds, tol=1e-6)
        X3, inf3 = sk.solve_path(A, b, lams, sds=sds, tol=2e-6, X=X1.clone(), warm_start=True)
    assert torch.equal(X1, X2)
    assert all(i.converged and i.outer_iters == 0 for i in inf3)
    assert torch.equal(X3, X1)


def test_solve_batched_matches_oracle(aab_form):
    probs = [W.problem_small(seed=1000),
             W.problem_scaled(3000, 100, seed=41),
             W.problem_scaled(16384, 512, seed=42, sd_frac=0.1)]
    fams = ["gaussian", "countsketch", "srht"]
    lams = list(np.logspace(-3, -1, 8))
    handles, entries, sds = [], [], []
    for pr, fam in zip(probs, fams):
        A, b = pr.A.to(DEV), pr.b.to(DEV)
        sd_row = [W.nominal_sd(pr.sigma, l) for l in lams]
        m = min(pr.n, int(math.ceil(4 * max(sd_row) / 4)) * 4 + 4)
        sk = mihs.Sketch(A, fam, m, seed=7)
        handles.append(sk)
        entries.append((sk, A, b, torch.empty(len(lams), pr.d, device=DEV)))
        sds.append(sd_row)
    infos = mihs.solve_batched(entries, lams, sds=sds, tol=1e-6, max_outer=300)
    for pr, (sk, A, b, X), inf in zip(probs, entries, infos):
        An, bn = pr.A.double().numpy(), pr.b.double().numpy()
        XS = o.ridge_path(An, bn, lams)
        Xn = X.cpu().double().numpy()
        for l in range(len(lams)):
            assert inf[l].converged, (pr.name, l, inf[l])
            assert _certified(An, bn, lams[l], Xn[l], XS[l])[0]
    for sk in handles:
        sk.close()


def test_path_invalid_arguments():
    A = W.randn((512, 1028), 1).to(DEV)
    b = W.randn((512,), 2).to(DEV)
    with mihs.Sketch(A, "countsketch", 64, seed=1) as sk:
        with pytest.raises(mihs.MihsError) as e:
            sk.solve_path(A, b, [0.1, 0.2], sds=[4.0, 4.0])
        assert e.value.code == mihs.UNSUPPORTED
    A = W.randn((512, 64), 1).to(DEV)
    with mihs.Sketch(A, "countsketch", 64, seed=1) as sk:
        with pytest.raises(mihs.MihsError):
            sk.solve_path(A, b, [0.1, -1.0], sds=[4.0, 4.0])
        with pytest.raises(mihs.MihsError):
            sk.solve_path(A, b, [0.1], sds=[64.0])  # sd must be < m
        X = torch.empty(1, 64, device=DEV)
        with pytest.raises(mihs.MihsError):
            mihs.solve_batched([(sk, A, b, X), (sk, A, b, X)], [0.1], sds=[[4.0], [4.0]])


def test_path_wide_sketch_grid_matches_cluster():
    """A sketch too large for one cluster (m = 2048, d = 1024: 8 MB of SA):
    the cooperative grid form and the cluster form reach the same solutions
    (both within the oracle's certificate)."""
    import os
    q = W.problem_scaled(16384, 1024, seed=55, decades=3.0, sd_frac=0.5)
    A, b = q.A.to(DEV), q.b.to(DEV)
    lams = list(np.logspace(-3, -1, 16))
    sds = [W.nominal_sd(q.sigma, l) for l in lams]
    m = 2048
    out = {}
    for form in ("grid", "cluster"):
        os.environ["MIHS_PATH_AAB"] = form
        try:
            with mihs.Sketch(A, "countsketch", m, seed=8) as sk:
                X, infos = sk.solve_path(A, b, lams, sds=sds, tol=1e-6, max_outer=200)
        finally:
            os.environ.pop("MIHS_PATH_AAB", None)
        assert all(i.converged for i in infos), (form, infos)
        out[form] = X.cpu().double().numpy()
    An, bn = q.A.double().numpy(), q.b.double().numpy()
    XS = o.ridge_path(An, bn, lams)
    for form, Xn in out.items():
        for l in range(len(lams)):
            assert _certified(An, bn, lams[l], Xn[l], XS[l])[0], (form, l)
