"""Parity of the grid form of AAb_Solver (SA spread over the shared memory of
up to every SM, grid-wide barriers) with the oracle.

The grid form is what a solve takes when SA does not fit in the shared memory
of one 16-block cluster; MIHS_AAB_FORM=grid forces it at any size, so the same
cases as the cluster kernel's parity tests run through it: fixed pass counts
against the oracle's fp64 Algorithm 5 (yardstick: the oracle's own fp32-vs-fp64
difference), the forcing-term stop, quantised SA, the heavy ball, and whole
solves (plain and refined) against the exact solution.  One case is large
enough (SA of 3076 × 2048, 25 MB) that the grid form is chosen without the
override, as in the mixed-precision workload.
"""
import math

import numpy as np
import pytest
import torch

from oracle import mihs_oracle as o
from paper_1912_03514_gb300 import mihs
from paper_1912_03514_gb300 import workloads as W

from tests._tol import U32

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _np(t):
    return t.detach().double().cpu().numpy()


@pytest.fixture
def grid_form(monkeypatch):
    monkeypatch.setenv("MIHS_AAB_FORM", "grid")


def _sa_case(m, d, seed):
    SA = W.randn((m, d), seed, scale=1.0 / math.sqrt(m))
    g = W.randn((d,), seed + 1)
    return SA, g


def _amp(SA, g, lam, k):
    x64, _ = o.aab_solve(SA, g, lam, 0.0, max_iter=k)
    x32, _ = o.aab_solve(SA.astype(np.float32), g.astype(np.float32), lam, 0.0, max_iter=k, dtype=np.float32)
    return o.rel_error(x32, x64), x64


GRID_CASES = [  # m, d, lam: ragged widths, fewer rows than blocks, wide slices, several rows per block
    (40, 30, 0.3), (588, 1024, 1e-4), (1000, 64, 1e-2), (7, 5, 0.5), (3, 2048, 1.0),
    (2048, 2048, 0.5), (1500, 300, 1e-3), (155, 129, 0.05),
]


@pytest.mark.parametrize("m,d,lam", GRID_CASES)
@pytest.mark.parametrize("k", [1, 4, 25])
def test_grid_aab_fixed_passes_matches_oracle(grid_form, m, d, lam, k):
    SA, g = _sa_case(m, d, 100 * m + d)
    SAn, gn = SA.numpy().astype(np.float64), g.numpy().astype(np.float64)
    amp, ref = _amp(SAn, gn, lam, k)
    passes = torch.zeros(1, dtype=torch.int32, device=DEV)
    delta = mihs.aab_solve(SA.to(DEV), g.to(DEV), lam, eps_sub=0.0, max_inner=k, passes=passes)
    delta2 = mihs.aab_solve(SA.to(DEV), g.to(DEV), lam, eps_sub=0.0, max_inner=k)
    torch.cuda.synchronize()
    assert int(passes.item()) == min(k, m, d)
    err = o.rel_error(_np(delta), ref)
    assert err <= 20 * max(amp, 4 * U32 * math.sqrt(d)), (err, amp)
    assert torch.equal(delta, delta2), "the grid form is not deterministic"


def test_grid_chosen_for_large_sa_matches_oracle_and_cluster(monkeypatch):
    """SA of 3076 × 2048 (25 MB) does not fit one cluster: without an
    override the grid form runs; the cluster form (SA read from L2) on the
    same input agrees within the same yardstick."""
    m, d, lam, k = 3076, 2048, 1e-3, 12
    SA, g = _sa_case(m, d, 4242)
    SAn, gn = SA.numpy().astype(np.float64), g.numpy().astype(np.float64)
    amp, ref = _amp(SAn, gn, lam, k)
    monkeypatch.delenv("MIHS_AAB_FORM", raising=False)
    dg = mihs.aab_solve(SA.to(DEV), g.to(DEV), lam, eps_sub=0.0, max_inner=k)
    monkeypatch.setenv("MIHS_AAB_FORM", "cluster")
    dc = mihs.aab_solve(SA.to(DEV), g.to(DEV), lam, eps_sub=0.0, max_inner=k)
    tol = 20 * max(amp, 4 * U32 * math.sqrt(d))
    assert o.rel_error(_np(dg), ref) <= tol
    assert o.rel_error(_np(dc), ref) <= tol


@pytest.mark.parametrize("m,d,lam", [(588, 1024, 1e-4), (1500, 300, 1e-3)])
@pytest.mark.parametrize("eps", [0.5, 0.1, 1e-3])
def test_grid_aab_forcing_term(grid_form, m, d, lam, eps):
    SA, g = _sa_case(m, d, 7 * m + d)
    SAn, gn = SA.numpy().astype(np.float64), g.numpy().astype(np.float64)
    x32, k32 = o.aab_solve(SAn.astype(np.float32), gn.astype(np.float32), lam, eps, dtype=np.float32)
    _, k64 = o.aab_solve(SAn, gn, lam, eps)
    passes = torch.zeros(1, dtype=torch.int32, device=DEV)
    delta = mihs.aab_solve(SA.to(DEV), g.to(DEV), lam, eps_sub=eps, passes=passes)
    kg = int(passes.item())
    slack = max(2, int(0.1 * max(k32, k64)))
    assert min(k32, k64) - slack <= kg <= max(k32, k64) + slack, (kg, k32, k64)
    H = SAn.T @ SAn + lam * np.eye(d)
    res = np.linalg.norm(H @ _np(delta) - gn) / np.linalg.norm(gn)
    res32 = np.linalg.norm(H @ x32.astype(np.float64) - gn) / np.linalg.norm(gn)
    assert res < max(eps * (1 + 1e-3), 10 * res32), (res, res32)


def test_grid_aab_zero_rhs(grid_form):
    SA, _ = _sa_case(50, 40, 1)
    passes = torch.full((1,), -1, dtype=torch.int32, device=DEV)
    delta = mihs.aab_solve(SA.to(DEV), torch.zeros(40, device=DEV), 0.1, passes=passes)
    assert int(passes.item()) == 0 and not torch.any(delta)


def _decoded(q, sc, prec, m, d):
    if prec == "bf16":
        return q[:, :d].to(torch.float64).cpu().numpy()
    dec = q[:, :d].cpu().view(torch.float8_e4m3fn).to(torch.float64).numpy()
    S = np.repeat(np.repeat(sc.cpu().numpy().astype(np.float64), 128, axis=0), 128, axis=1)[:m, :d]
    return dec * S


@pytest.mark.parametrize("m,d,lam", [(588, 1024, 1e-4), (300, 2000, 1e-2), (64, 48, 0.1)])
@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_grid_aab_quantised_sa(grid_form, m, d, lam, prec):
    k = 8
    SA = W.randn((m, d), 5 * m + d, scale=1.0 / math.sqrt(m))
    g = W.randn((d,), 3 * d)
    q, sc = mihs.quantize_sa(SA.to(DEV), prec)
    SAd = _decoded(q, sc, prec, m, d)
    gn = g.numpy().astype(np.float64)
    amp, x64 = _amp(SAd, gn, lam, k)
    delta = mihs.aab_solve_q(q, prec, sc, d, g.to(DEV), lam, eps_sub=0.0, max_inner=k)
    err = o.rel_error(_np(delta), x64)
    assert err <= 20 * max(amp, 4 * U32 * math.sqrt(d)), (err, amp)


def test_grid_aab_heavy_ball(grid_form):
    m, d, lam, k = 588, 1024, 1e-3, 6
    sd = 0.3 * min(m, d)
    SA, g = _sa_case(m, d, 3 * m)
    x = W.randn((d,), 91)
    xp = W.randn((d,), 92)
    alpha, beta = o.momentum_params(sd, m)
    amp, delta_ref = _amp(SA.numpy().astype(np.float64), g.numpy().astype(np.float64), lam, k)
    xr, _ = o.heavy_ball(x.numpy().astype(np.float64), xp.numpy().astype(np.float64), delta_ref, alpha, beta)
    xd, xpd = x.to(DEV), xp.to(DEV)
    mihs.aab_heavy_ball(SA.to(DEV), g.to(DEV), lam, 0.0, k, alpha, beta, xd, xpd)
    assert torch.equal(xpd.cpu(), x)
    tol = 20 * max(amp, 1e-6) * np.linalg.norm(alpha * delta_ref) + \
        8 * U32 * np.linalg.norm(np.abs(xr) + 2 * np.abs(x.numpy()))
    assert np.linalg.norm(_np(xd) - xr) <= tol


@pytest.mark.parametrize("family", ["gaussian", "countsketch", "srht"])
def test_grid_solves_reach_the_solution(grid_form, family):
    """Algorithm 1 end to end with the grid form inside the device-side loop:
    plain solves to 1e-5, refined solves to 1e-10 of the exact solution, and
    a repeated solve on the same handle gives the same bytes."""
    p = W.problem_small()
    A, b = p.A.to(DEV), p.b.to(DEV)
    xs = o.exact_solve(p.A.numpy(), p.b.numpy(), p.lam, refine=3, extended=True)
    with mihs.Sketch(A, family, p.m, seed=12) as sk:
        x, info = sk.solve(A, b, p.lam, p.sd, tol=1e-6, max_outer=200)
        x2, _ = sk.solve(A, b, p.lam, p.sd, tol=1e-6, max_outer=200)
        xr, ir = sk.solve_refined(A, b, p.lam, p.sd, tol=1e-13, max_outer=300)
        sk.set_precision("bf16")
        xq, iq = sk.solve_refined(A, b, p.lam, p.sd, tol=1e-13, max_outer=300)
    assert info.converged and ir.converged and iq.converged, (info, ir, iq)
    assert o.rel_error(_np(x), xs) <= 1e-5
    assert torch.equal(x, x2)
    assert o.rel_error(xr.cpu().numpy(), xs) <= 1e-10
    assert o.rel_error(xq.cpu().numpy(), xs) <= 1e-10
    assert mihs.device_status() == 0


# ---------------- one cluster reading SA from global memory (L2)
@pytest.mark.parametrize("m,d,lam,k", [(4096, 1024, 1e-3, 12), (3000, 700, 1e-2, 25), (5000, 512, 0.05, 7)])
def test_cluster_global_sa_matches_oracle(monkeypatch, m, d, lam, k):
    """SA too large for one cluster's shared memory, cluster form forced (the
    form the λ-path solves use for such sketches): its blocks read their rows
    of SA from global memory every pass; k passes against the oracle's
    Algorithm 5, repeatable."""
    monkeypatch.setenv("MIHS_AAB_FORM", "cluster")
    SA, g = _sa_case(m, d, 11 * m + d)
    dp = (d + 3) // 4 * 4
    SAp = torch.zeros(m, dp)
    SAp[:, :d] = SA
    SAd = SAp.to(DEV).as_strided((m, d), (dp, 1))
    SAn, gn = SA.numpy().astype(np.float64), g.numpy().astype(np.float64)
    amp, ref = _amp(SAn, gn, lam, k)
    passes = torch.zeros(1, dtype=torch.int32, device=DEV)
    delta = mihs.aab_solve(SAd, g.to(DEV), lam, eps_sub=0.0, max_inner=k, passes=passes)
    delta2 = mihs.aab_solve(SAd, g.to(DEV), lam, eps_sub=0.0, max_inner=k)
    assert int(passes.item()) == min(k, m, d)
    assert o.rel_error(_np(delta), ref) <= 20 * max(amp, 4 * U32 * math.sqrt(d))
    assert torch.equal(delta, delta2)
    assert mihs.device_status() == 0


def test_cluster_global_quantised_sa(monkeypatch):
    monkeypatch.setenv("MIHS_AAB_FORM", "cluster")
    m, d, lam, k = 8192, 1024, 1e-3, 9
    SA = W.randn((m, d), 77, scale=1.0 / math.sqrt(m))
    g = W.randn((d,), 78)
    q, sc = mihs.quantize_sa(SA.to(DEV), "bf16")
    SAd = _decoded(q, sc, "bf16", m, d)
    amp, x64 = _amp(SAd, g.numpy().astype(np.float64), lam, k)
    delta = mihs.aab_solve_q(q, "bf16", sc, d, g.to(DEV), lam, eps_sub=0.0, max_inner=k)
    assert o.rel_error(_np(delta), x64) <= 20 * max(amp, 4 * U32 * math.sqrt(d))


# ---------------- the form chosen per handle (mihs_sketch_set_aab)
@pytest.mark.parametrize("shape", ["small", "scaled"])
def test_handle_aab_form_reaches_the_solution(shape):
    """Every form of AAb_Solver a handle can be set to, inside the device-side
    loop of Algorithm 1: the cluster form, the grid form over all SMs, and
    small grids whose requested block count is too few to hold SA in shared
    memory (raised to the fewest that do).  Plain solves reach 1e-5 and
    refined solves 1e-10 of the exact solution; a repeated solve on the same
    form gives the same bytes, and switching forms rebuilds the solve graph."""
    p = W.problem_small() if shape == "small" else W.problem_scaled(16384, 512, seed=41)
    A, b = p.A.to(DEV), p.b.to(DEV)
    xs = o.exact_solve(p.A.numpy(), p.b.numpy(), p.lam, refine=3, extended=True)
    forms = [("auto", 0), ("cluster", 0), ("grid", 0), ("grid", 1), ("grid", 3), ("grid", 24), ("auto", 0)]
    with mihs.Sketch(A, "gaussian", p.m, seed=13) as sk:
        for form, blocks in forms:
            sk.set_aab(form, blocks)
            x, info = sk.solve(A, b, p.lam, p.sd, tol=1e-6, max_outer=200)
            x2, _ = sk.solve(A, b, p.lam, p.sd, tol=1e-6, max_outer=200)
            xr, ir = sk.solve_refined(A, b, p.lam, p.sd, tol=1e-13, max_outer=300)
            assert info.converged and ir.converged, (form, blocks, info, ir)
            assert o.rel_error(_np(x), xs) <= 1e-5, (form, blocks)
            assert torch.equal(x, x2), (form, blocks)
            assert o.rel_error(xr.cpu().numpy(), xs) <= 1e-10, (form, blocks)
    assert mihs.device_status() == 0


def test_handle_aab_form_arguments():
    p = W.problem_small()
    with mihs.Sketch(p.A.to(DEV), "gaussian", p.m, seed=13) as sk:
        for bad in [(3, 0), (-1, 0), (2, -5)]:
            with pytest.raises(mihs.MihsError):
                sk.set_aab(*bad)
        with pytest.raises(ValueError):
            sk.set_aab("persistent")
        sk.set_aab("grid", 10_000)  # more blocks than SMs: one per SM
        x, info = sk.solve(p.A.to(DEV), p.b.to(DEV), p.lam, p.sd, tol=1e-6, max_outer=200)
    assert info.converged
