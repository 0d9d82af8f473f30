"""Pins of the oracle against facts fixed by the paper and by mathematics.

None of these re-types an oracle formula: each compares the oracle with a
library routine, a closed form, an invariant, a printed number or brute force
chosen so that a dropped term, a wrong sign or a transposed operand fails.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.stats

from oracle import mihs_oracle as o
from paper_1912_03514_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- Philox
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        out = o.philox4x32_10(*v[:4], *v[4:6])
        assert [int(w) for w in out] == v[6:10]


def test_philox_vectorised_equals_scalar():
    c0 = np.arange(17, dtype=np.uint64)
    vec = o.philox4x32_10(c0, 5, 1, 0, 123, 456)
    for i in range(17):
        sc = o.philox4x32_10(i, 5, 1, 0, 123, 456)
        assert [int(w[i]) for w in vec] == [int(w) for w in sc]


# ------------------------------------------------------------ Box-Muller
def test_box_muller_closed_forms():
    # u1 = 1 exactly -> radius 0
    z0, z1 = o.box_muller(np.uint64(0xFFFFFFFF), np.uint64(12345 << 8))
    assert z0 == 0.0 and z1 == 0.0
    # u1 = 2^-24 (smallest), u2 = 1/4 -> (0, sqrt(2*24*ln 2))
    z0, z1 = o.box_muller(np.uint64(0), np.uint64(1 << 30))
    r = math.sqrt(2.0 * 24.0 * math.log(2.0))
    assert abs(z0) < 1e-12 and abs(z1 - r) < 1e-12


def test_box_muller_is_standard_normal():
    w0, w1, w2, w3 = o.philox4x32_10(np.arange(1 << 16, dtype=np.uint64), 0, 0, 0, 7, 9)
    z = np.concatenate(o.box_muller(w0, w1) + o.box_muller(w2, w3))
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1) < 5 * math.sqrt(2 / z.size)
    assert scipy.stats.kstest(z, "norm").pvalue > 1e-4


# ---------------------------------------------------------------- sketches
def _mc_isotropy(make_S, n, seeds):
    acc = np.zeros((n, n))
    for s in seeds:
        S = make_S(s)
        acc += S.T @ S
    return acc / len(seeds)


@pytest.mark.parametrize("family", [o.GAUSSIAN, o.COUNTSKETCH, o.SRHT])
def test_sketch_expectation_identity(family):
    """E[SᵀS] = I (text after Algorithm 1): Monte-Carlo mean over seeds."""
    n, m, T = 24, 8, 600
    mk = {o.GAUSSIAN: lambda s: o.gaussian_sketch_matrix(m, n, s),
          o.COUNTSKETCH: lambda s: o.countsketch_matrix(m, n, s),
          o.SRHT: lambda s: o.srht_matrix(m, n, s)}[family]
    E = _mc_isotropy(mk, n, range(T))
    assert np.max(np.abs(np.diag(E) - 1)) < 0.25
    off = E - np.diag(np.diag(E))
    assert np.max(np.abs(off)) < 0.25
    # a scaling mistake (e.g. 1/m instead of 1/sqrt(m)) moves the diagonal far
    assert abs(np.mean(np.diag(E)) - 1) < 0.05


def test_gaussian_entries_variance_and_independence():
    m, n = 64, 4096
    S = o.gaussian_sketch_matrix(m, n, 2024)
    z = S.ravel() * math.sqrt(m)
    assert scipy.stats.kstest(z, "norm").pvalue > 1e-4
    # each of the four counter slots is a standard normal on its own
    for t in range(4):
        zt = (S[:, t::4] * math.sqrt(m)).ravel()
        assert abs(zt.var() - 1) < 0.05
    C = np.corrcoef(S)
    assert np.max(np.abs(C - np.eye(m))) < 0.1


def test_countsketch_structure_and_exact_sum():
    n, m, d = 5000, 37, 6
    S = o.countsketch_matrix(m, n, 11)
    assert np.all(np.sum(S != 0, axis=0) == 1)
    assert set(np.unique(S[S != 0])) <= {-1.0, 1.0}
    h, s = o.countsketch_hash(n, m, 11)
    assert h.min() >= 0 and h.max() < m
    counts = np.bincount(h, minlength=m)
    assert scipy.stats.chisquare(counts).pvalue > 1e-4
    A = W.randint_matrix((n, d), 3).numpy().astype(np.float64)
    SA = o.sketch_apply(o.COUNTSKETCH, A, m, 11)
    brute = np.zeros((m, d))
    for j in range(n):                       # SA[h(j)] += s(j) A[j]
        brute[h[j]] += s[j] * A[j]
    assert np.array_equal(SA, brute)


def test_hadamard_matches_scipy():
    for L in range(0, 8):
        Hs = scipy.linalg.hadamard(1 << L)
        r = np.arange(1 << L)
        assert np.array_equal(o.hadamard_entry(r[:, None], r[None, :]), Hs)


def test_srht_definition():
    n, m = 100, 16                       # n not a power of two -> n_p = 128
    n_p, D, rows = o.srht_params(n, m, 5)
    assert n_p == 128 and rows.min() >= 0 and rows.max() < 128
    H = scipy.linalg.hadamard(n_p)
    Dfull = np.concatenate([D, np.ones(n_p - n)])
    Sfull = math.sqrt(n_p / m) * (H[rows] / math.sqrt(n_p)) * Dfull[None, :]
    assert np.allclose(o.srht_matrix(m, n, 5), Sfull[:, :n], atol=0, rtol=1e-15)
    rr = o.srht_params(1 << 12, 20000, 1)[2]
    assert scipy.stats.chisquare(np.bincount(rr >> 6, minlength=64)).pvalue > 1e-4


@pytest.mark.parametrize("family", [o.GAUSSIAN, o.COUNTSKETCH, o.SRHT])
def test_sketch_rows_equal_full_product(family):
    n, d, m = 300, 7, 12
    A = W.randn((n, d), 4).numpy()
    S = {o.GAUSSIAN: o.gaussian_sketch_matrix, o.COUNTSKETCH: o.countsketch_matrix,
         o.SRHT: o.srht_matrix}[family](m, n, 99)
    SA = o.sketch_apply(family, A, m, 99, row_block=5)
    assert np.allclose(SA, S @ A.astype(np.float64), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("family", [o.GAUSSIAN, o.COUNTSKETCH, o.SRHT])
def test_sketch_rows_in_any_order_are_rows_of_the_full_sketch(family):
    """The row-sampled form (used for sampled checks at full size) returns
    exactly the requested rows of S·A, in the order asked, repeats allowed."""
    n, d, m = 257, 5, 16
    A = W.randn((n, d), 8).numpy().astype(np.float64)
    S = {o.GAUSSIAN: o.gaussian_sketch_matrix, o.COUNTSKETCH: o.countsketch_matrix,
         o.SRHT: o.srht_matrix}[family](m, n, 31)
    rows = [11, 0, 15, 3, 11]
    got = o.sketch_rows(family, rows, A, m, 31)
    want = np.stack([sum(S[i, j] * A[j] for j in range(n)) for i in rows])  # brute force
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12)


# ----------------------------------------------------------- ridge solution
def _small(n=400, d=40, lam=1e-2, seed=0):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((n, d)))
    V, _ = np.linalg.qr(rng.standard_normal((d, d)))
    s = np.logspace(0, -3, d)
    A = (U * s) @ V.T
    b = rng.standard_normal(n)
    return A, b, lam, s


def test_exact_solve_matches_lstsq_and_svd():
    A, b, lam, _ = _small()
    x = o.exact_solve(A, b, lam)
    n, d = A.shape
    Aug = np.vstack([A, math.sqrt(lam) * np.eye(d)])
    x_ls = np.linalg.lstsq(Aug, np.concatenate([b, np.zeros(d)]), rcond=None)[0]
    assert o.rel_error(x, x_ls) < 1e-11
    assert o.rel_error(o.svd_solve(A, b, lam), x_ls) < 1e-11
    # first-order optimality
    assert np.linalg.norm(o.gradient(A, b, x, lam)) < 1e-11 * np.linalg.norm(A.T @ b)


def test_exact_solve_blocked_rows_same_result():
    A, b, lam, _ = _small(n=1000, d=20)
    assert o.rel_error(o.exact_solve(A, b, lam, row_block=37), o.exact_solve(A, b, lam)) < 1e-13


def test_stat_dim_identities():
    A, b, lam, s = _small()
    n, d = A.shape
    sd = o.stat_dim_of(A, lam)
    assert abs(sd - o.stat_dim(s, lam)) < 1e-9
    # definition tr(A (AᵀA+λI)⁻¹ Aᵀ)
    tr = np.trace(A @ np.linalg.solve(A.T @ A + lam * np.eye(d), A.T))
    assert abs(sd - tr) < 1e-9
    # ‖U1‖_F² with U1 the first n rows of an orthonormal basis of [A; √λ I]
    Q, _ = np.linalg.qr(np.vstack([A, math.sqrt(lam) * np.eye(d)]))
    assert abs(sd - np.sum(Q[:n] ** 2)) < 1e-9
    # λ → 0: the rank
    assert abs(o.stat_dim(s, 0.0) - d) < 1e-12


def test_gradient_brute_force():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((5, 3)); b = rng.standard_normal(5); x = rng.standard_normal(3)
    lam = 0.7
    g = np.zeros(3)
    for j in range(3):
        acc = 0.0
        for i in range(5):
            ri = b[i] - sum(A[i, k] * x[k] for k in range(3))
            acc += A[i, j] * ri
        g[j] = acc - lam * x[j]
    assert np.allclose(o.gradient(A, b, x, lam), g, rtol=1e-14, atol=1e-14)
    # g is minus the derivative of f (central differences)
    f = lambda z: 0.5 * np.sum((A @ z - b) ** 2) + 0.5 * lam * np.sum(z ** 2)
    num = np.array([(f(x + 1e-6 * e) - f(x - 1e-6 * e)) / 2e-6 for e in np.eye(3)])
    assert np.allclose(-num, g, atol=1e-7)


# -------------------------------------------------------------- AAb_Solver
def _aab_case(m=40, d=30, lam=0.3, seed=0):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((m, d)), rng.standard_normal(d), lam


def test_aab_residual_identity():
    """Section 3.6: the loop's t equals ‖(SAᵀSA+λI)x − g‖/‖g‖ of the iterate
    held before the pass (the unsquared norm)."""
    SA, g, lam = _aab_case()
    d = SA.shape[1]
    H = SA.T @ SA + lam * np.eye(d)
    _, _, ts = o.aab_solve(SA, g, lam, 0.0, max_iter=12, history=True)
    for k in range(12):
        xk, _ = o.aab_solve(SA, g, lam, 0.0, max_iter=k)
        true = np.linalg.norm(H @ xk - g) / np.linalg.norm(g)
        assert abs(ts[k] - true) <= 1e-10 * true


def test_aab_garbled_initial_sine_breaks_identity():
    """The printed initial sine √(λ/ρ̄) violates the residual identity, which is
    how the reading s = √λ/ρ̄ is pinned."""
    SA, g, lam = _aab_case()
    d = SA.shape[1]
    H = SA.T @ SA + lam * np.eye(d)
    _, _, ts = o.aab_solve(SA, g, lam, 0.0, max_iter=6, history=True, s_init="garbled")
    x5, _ = o.aab_solve(SA, g, lam, 0.0, max_iter=5, s_init="garbled")
    true = np.linalg.norm(H @ x5 - g) / np.linalg.norm(g)
    assert abs(ts[5] - true) > 1e-6 * true


def test_aab_finite_termination_and_stop_rule():
    SA, g, lam = _aab_case(m=25, d=18, lam=0.5)
    d = SA.shape[1]
    H = SA.T @ SA + lam * np.eye(d)
    x_direct = np.linalg.solve(H, g)
    x, k = o.aab_solve(SA, g, lam, 0.0)
    assert k <= min(SA.shape)
    assert o.rel_error(x, x_direct) < 1e-9
    # forcing term: the pass that stops has t < eps, and that t certifies the
    # previous iterate, so the returned one is at least as good in practice
    for eps in (0.5, 0.1, 1e-3):
        x, k, ts = o.aab_solve(SA, g, lam, eps, history=True)
        assert ts[-1] < eps and all(t >= eps for t in ts[:-1])
        assert np.linalg.norm(H @ x - g) / np.linalg.norm(g) < eps


def test_aab_zero_rhs_and_fp32_mode():
    SA, g, lam = _aab_case()
    x, k = o.aab_solve(SA, np.zeros_like(g), lam, 0.1)
    assert k == 0 and not np.any(x)
    x32, _ = o.aab_solve(SA, g, lam, 1e-4, dtype=np.float32)
    x64, _ = o.aab_solve(SA, g, lam, 1e-4)
    assert x32.dtype == np.float32 and o.rel_error(x32, x64) < 1e-4


# ------------------------------------------------------- momentum & rates
@pytest.mark.parametrize("eps", [0.05, 0.3, 0.5, 0.9])
def test_theorem1_parameters(eps):
    alpha, beta, rate = o.theorem1_params(eps)
    assert abs(alpha - o.theorem1_alpha_alt(eps)) < 1e-12
    # rate = min over α of max{1 − √α/√(1+ε), √α/√(1−ε) − 1} (brute force)
    a = np.linspace(1e-6, 2.0, 400001)
    worst = np.maximum(1 - np.sqrt(a) / math.sqrt(1 + eps), np.sqrt(a) / math.sqrt(1 - eps) - 1)
    i = np.argmin(worst)
    assert abs(worst[i] - rate) < 1e-5
    assert abs(a[i] - alpha) < 1e-4
    assert abs(math.sqrt(beta) - rate) < 1e-15
    # with μ spanning [1/(1+ε), 1/(1−ε)] every mode is under-damped
    mu = np.linspace(1 / (1 + eps), 1 / (1 - eps), 101)
    assert np.all(o.underdamped(mu, alpha, beta + 1e-12))
    assert abs(o.characteristic_rate(mu, alpha, beta) - rate) < 1e-6


@pytest.mark.parametrize("ratio", [0.1, 0.25, 0.5])
def test_corollary3_marchenko_pastur_edges(ratio):
    """With α = (1−β)², β = sd/m, both MP edges (1 ± √β)⁻² sit exactly on the
    under-damped boundary, so every μ between them has root modulus √β."""
    alpha, beta = o.momentum_params(ratio * 400, 400)
    lo, hi = o.mp_edges(ratio * 400, 400)
    for mu in (lo, hi):
        assert abs((1 - math.sqrt(alpha * mu)) ** 2 - beta) < 1e-12
    mu = np.linspace(lo, hi, 57)
    assert abs(o.characteristic_rate(mu, alpha, beta) - math.sqrt(beta)) < 1e-6
    # outside the edges the rate is strictly worse (over-damped mode)
    assert o.characteristic_rate([hi * 1.5], alpha, beta) > math.sqrt(beta) + 1e-3


def test_worked_number_no_reg_caption():
    rows = [l.split("|") for l in open(os.path.join(GOLDEN, "paper_worked_numbers.txt"))
            if l.strip() and not l.startswith("#")]
    (name, inputs, printed, _), = rows
    kv = dict(t.split("=") for t in inputs.split())
    d, m, N, kappa = int(kv["d"]), int(kv["m"]), int(kv["N"]), float(kv["kappa"])
    sd = o.stat_dim(np.ones(d), 0.0)                 # λ = 0 → rank
    _, beta = o.momentum_params(sd, m)
    val = o.predicted_error(kappa, beta, N)
    assert float(f"{val:.0e}") == float(printed)


def test_corollary2_reading_is_consistent_with_theorem1():
    eps, C, eta = 0.4, 50.0, 1e-8
    N = o.corollary2_iters(eta, C, eps)
    rate = o.theorem1_params(eps)[2]
    assert C * rate ** N <= eta < C * rate ** (N - 1)


# ------------------------------------------------------------- Algorithm 1
def _problem(n=3000, d=60, seed=5, sd_frac=0.2):
    p = W.problem_scaled(n, d, seed, decades=3.0, sd_frac=sd_frac)
    return p.A.numpy().astype(np.float64), p.b.numpy().astype(np.float64), p


def test_exact_inner_rate_equals_characteristic_rate():
    """Exact M-IHS error decays at the spectral radius of the heavy-ball
    transition computed from μ = eig((SAᵀSA+λI)⁻¹(AᵀA+λI))."""
    A, b, p = _problem()
    SA = o.sketch_apply(o.GAUSSIAN, A, p.m, 77)
    xs = o.exact_solve(A, b, p.lam)
    alpha, beta = o.momentum_params(p.sd, p.m)
    mu = o.sketched_hessian_eigs(A, SA, p.lam)
    pred = o.characteristic_rate(mu, alpha, beta)
    _, info = o.mihs(A, b, p.lam, SA, p.sd, 45, inner="exact", record=True)
    errs = np.array([np.linalg.norm(h[0] - xs) for h in info["history"]])
    k0, k1 = 10, 40
    obs = (errs[k1] / errs[k0]) ** (1.0 / (k1 - k0))
    assert abs(obs - pred) < 0.08 * pred
    # and a wrong β (momentum dropped) predicts a visibly different rate
    assert abs(o.characteristic_rate(mu, alpha, 0.0) - obs) > 0.05


def test_rate_is_sqrt_sd_over_m_statistically():
    """Corollary 3: rate √(sd/m), averaged over 8 Gaussian sketches."""
    A, b, p = _problem(n=4000, d=80, seed=6)
    xs = o.exact_solve(A, b, p.lam)
    sd = o.stat_dim_of(A, p.lam)
    rates = []
    for seed in range(8):
        SA = o.sketch_apply(o.GAUSSIAN, A, p.m, 100 + seed)
        _, info = o.mihs(A, b, p.lam, SA, sd, 30, inner="exact", record=True)
        e = np.array([np.linalg.norm(h[0] - xs) for h in info["history"]])
        rates.append((e[25] / e[5]) ** (1 / 20))
    assert abs(np.mean(rates) - math.sqrt(sd / p.m)) < 0.2 * math.sqrt(sd / p.m)


@pytest.mark.parametrize("family", [o.GAUSSIAN, o.COUNTSKETCH, o.SRHT])
def test_inexact_mihs_reaches_exact_solution(family):
    p = W.problem_small()
    A = p.A.numpy().astype(np.float64)
    b = p.b.numpy().astype(np.float64)
    xs = o.exact_solve(A, b, p.lam)
    x, info = o.mihs_solve(A, b, p.lam, family, p.m, p.sd, seed=31, N=120, tol=1e-13)
    assert o.rel_error(x, xs) < 1e-10
    assert info["outer"] < 80
    assert o.certify(A, b, x, p.lam) < 1e-9 * np.linalg.norm(xs)


def test_fp32_mode_floor_on_small_problem():
    p = W.problem_small()
    A = p.A.numpy()
    b = p.b.numpy()
    xs = o.exact_solve(A, b, p.lam)
    SA = o.sketch_apply(o.GAUSSIAN, A, p.m, 31).astype(np.float32)
    x, info = o.mihs(A, b, p.lam, SA, p.sd, 100, tol=1e-6, dtype=np.float32)
    assert info["resid"] <= 1e-6
    assert o.rel_error(x, xs) < 1e-5


def test_nominal_sd_close_to_actual():
    p = W.problem_small()
    sd = o.stat_dim_of(p.A.numpy(), p.lam)
    assert abs(sd - 64.0) < 2.0 and abs(p.sd - 64.0) < 1e-9


# ---------------------------------------------------------------- Algorithm 4
def test_hutchinson_probe_is_rademacher():
    v = o.rademacher_probe(20000, 3, 5)
    assert set(np.unique(v)) == {-1.0, 1.0}
    assert abs(v.mean()) < 5 / math.sqrt(v.size)
    assert not np.array_equal(v, o.rademacher_probe(20000, 4, 5))


def test_hutchinson_is_unbiased_for_the_sketched_trace():
    """With exact inner solves, the mean over many probes approaches
    d − λ·tr((SAᵀSA+λI)⁻¹), the statistical dimension of SA itself."""
    rng = np.random.default_rng(2)
    m, d, lam = 60, 40, 0.05
    SA = rng.standard_normal((m, d)) * np.logspace(0, -2, d)[None, :]
    exact = o.stat_dim_of(SA, lam)
    T = 3000
    est = o.hutchinson_sd(SA, lam, T, 0.0, seed=9)
    # per-probe variance of vᵀMv for Rademacher v is 2·Σ_{i≠j} M_ij²
    M = lam * np.linalg.inv(SA.T @ SA + lam * np.eye(d))
    var = 2 * (np.sum(M ** 2) - np.sum(np.diag(M) ** 2))
    assert abs(est - exact) < 5 * math.sqrt(var / T) + 1e-9


def test_hutchinson_inexact_overestimates_little():
    """ε_tr = 0.5 and T = 2 (the paper's setting) land within a few percent
    of the exact statistical dimension on a sketched problem."""
    p = W.problem_small()
    A = p.A.numpy().astype(np.float64)
    SA = o.sketch_apply(o.GAUSSIAN, A, p.m, 3)
    exact = o.stat_dim_of(A, p.lam)
    est = o.hutchinson_sd(SA, p.lam, 2, 0.5, seed=4)
    assert 0.7 * exact < est < 1.5 * exact


# ------------------------------------------------------ extended precision
def test_extended_gradient_agrees_and_is_more_accurate():
    rng = np.random.default_rng(11)
    A = rng.standard_normal((300, 20)).astype(np.float32).astype(np.float64)
    b = rng.standard_normal(300)
    x = rng.standard_normal(20)
    ge = o.gradient_extended(A, b, x, 0.3)
    g = o.gradient(A, b, x, 0.3)
    assert np.allclose(np.asarray(ge, dtype=np.float64), g, rtol=1e-12, atol=1e-12)
    # exact rational check on integer data: every operation is exact
    Ai = rng.integers(-5, 6, (50, 7)).astype(np.float64)
    bi = rng.integers(-5, 6, 50).astype(np.float64)
    xi = rng.integers(-5, 6, 7).astype(np.float64)
    ref = [sum(Ai[i, j] * (bi[i] - sum(Ai[i, k] * xi[k] for k in range(7))) for i in range(50)) - 2 * xi[j]
           for j in range(7)]
    assert np.array_equal(np.asarray(o.gradient_extended(Ai, bi, xi, 2.0), dtype=np.float64), np.array(ref))


def test_exact_solve_extended_on_ill_conditioned_problem():
    """κ(H) ≈ 1e6: the extended-precision refinement drives the certified
    error (‖g‖/λ against ‖x*‖) to ~1e-12, the fp64 one only to ~κ·u₆₄."""
    p = W.make_problem(4096, 64, W.profile_exponential(64, 8.0), 1e-6, 40.0, seed=3)
    A = p.A.numpy().astype(np.float64)
    b = p.b.numpy().astype(np.float64)
    x = o.exact_solve(A, b, p.lam, refine=3, extended=True)
    g = np.asarray(o.gradient_extended(A, b, x, p.lam), dtype=np.float64)
    assert np.linalg.norm(g) / p.lam <= 1e-11 * np.linalg.norm(x)
    assert o.rel_error(o.svd_solve(A, b, p.lam), x) < 1e-8


# ------------------------------------------------------ gradients of the solve
def _ridge_loss(A, b, lam, w):
    """L = wᵀ x*(A, b, λ) through LAPACK's general solver (not the oracle)."""
    return float(w @ scipy.linalg.solve(A.T @ A + lam * np.eye(A.shape[1]), A.T @ b))


def test_ridge_backward_matches_central_differences():
    """Every entry of ∂L/∂A, ∂L/∂b and ∂L/∂λ against fp64 central differences
    (truncation O(h²), rounding O(u/h)): a dropped term of the adjoint
    formula, a sign or a transposed outer product fails by orders."""
    rng = np.random.default_rng(5)
    n, d, lam = 9, 4, 0.37
    A = rng.standard_normal((n, d))
    b = rng.standard_normal(n)
    w = rng.standard_normal(d)
    _, _, dA, db, dlam = o.ridge_backward(A, b, lam, w)
    h = 1e-5
    fd = np.zeros_like(A)
    for i in range(n):
        for j in range(d):
            Ap, Am = A.copy(), A.copy()
            Ap[i, j] += h
            Am[i, j] -= h
            fd[i, j] = (_ridge_loss(Ap, b, lam, w) - _ridge_loss(Am, b, lam, w)) / (2 * h)
    assert np.max(np.abs(fd - dA)) <= 1e-7 * max(1.0, np.max(np.abs(dA)))
    fdb = np.array([(_ridge_loss(A, b + h * e, lam, w) - _ridge_loss(A, b - h * e, lam, w)) / (2 * h)
                    for e in np.eye(n)])
    assert np.max(np.abs(fdb - db)) <= 1e-7 * max(1.0, np.max(np.abs(db)))
    fdl = (_ridge_loss(A, b, lam + h, w) - _ridge_loss(A, b, lam - h, w)) / (2 * h)
    assert abs(fdl - dlam) <= 1e-7 * max(1.0, abs(dlam))


def test_ridge_backward_orthonormal_columns_closed_form():
    """AᵀA = I ⇒ x* = Aᵀb/(1+λ), so for L = wᵀx*: ∂L/∂b = A w/(1+λ) and
    ∂L/∂λ = −wᵀAᵀb/(1+λ)²; along A(t) = (1+t)Q the chain rule gives
    dL/dt = Σ_ij (∂L/∂A)_ij Q_ij."""
    rng = np.random.default_rng(6)
    Q, _ = np.linalg.qr(rng.standard_normal((20, 6)))
    b = rng.standard_normal(20)
    w = rng.standard_normal(6)
    lam = 0.8
    x, v, dA, db, dlam = o.ridge_backward(Q, b, lam, w)
    np.testing.assert_allclose(x, Q.T @ b / (1 + lam), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(db, Q @ w / (1 + lam), rtol=1e-12, atol=1e-14)
    assert abs(dlam - (-(w @ (Q.T @ b)) / (1 + lam) ** 2)) <= 1e-12
    # x*((1+t)Q) = (1+t)Qᵀb/((1+t)² + λ) in closed form
    def L(t):
        return (1 + t) * (w @ (Q.T @ b)) / ((1 + t) ** 2 + lam)
    t = 1e-6
    fd = (L(t) - L(-t)) / (2 * t)
    assert abs(fd - np.sum(dA * Q)) <= 1e-8


# ------------------------------------------------------------------ λ-paths
def test_ridge_path_against_svd_filter_factors_and_limits():
    """Each λ of a path against the SVD closed form (Eq. tsvdsol); ‖x*(λ)‖
    strictly decreasing in λ (the filter factors σ²/(σ²+λ) all decrease);
    λ·x*(λ) → Aᵀb as λ → ∞."""
    rng = np.random.default_rng(9)
    A = rng.standard_normal((60, 12)) @ np.diag(np.logspace(0, -3, 12))
    b = rng.standard_normal(60)
    lams = np.logspace(-6, 1, 16)
    X = o.ridge_path(A, b, lams)
    for lam, x in zip(lams, X):
        ref = o.svd_solve(A, b, lam)
        assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)
    norms = np.linalg.norm(X, axis=1)
    assert np.all(np.diff(norms) < 0)
    big = 1e8
    xb = o.ridge_path(A, b, [big])[0]
    assert np.linalg.norm(big * xb - A.T @ b) <= 1e-6 * np.linalg.norm(A.T @ b)


# ------------------------------------------------------ quantised SA storage
def test_quantize_sa_known_values():
    """bf16: 1 + 2⁻⁸ is a tie and rounds to even (1), 1 + 3·2⁻⁹ rounds up to
    1 + 2⁻⁷; fp8 e4m3: in a tile whose maximum is 448·s the scale is s, the
    maximum decodes exactly, 2⁻⁹·s (the smallest subnormal) survives and
    2⁻¹¹·s flushes to zero, 17·s is a tie between 16 and 18 (even: 16)."""
    SA = np.zeros((3, 5), np.float32)
    SA[0, 0] = 1 + 2.0 ** -8
    SA[0, 1] = 1 + 3 * 2.0 ** -9
    SA[0, 2] = -2.5
    q, sc, dec = o.quantize_sa(SA, "bf16")
    assert dec[0, 0] == 1.0 and dec[0, 1] == 1 + 2.0 ** -7 and dec[0, 2] == -2.5
    s = np.float32(0.75)
    SA = np.zeros((130, 131), np.float32)
    SA[0, 0] = 448 * s
    SA[1, 1] = 2.0 ** -9 * s
    SA[2, 2] = 2.0 ** -11 * s
    SA[3, 3] = 17 * s
    SA[129, 130] = -3.0  # second tile row and column: its own scale
    q, sc, dec = o.quantize_sa(SA, "fp8")
    assert sc.shape == (2, 2) and sc[0, 0] == np.float32(448 * s) / np.float32(448)
    assert sc[1, 1] == np.float32(3.0) / np.float32(448) and sc[0, 1] == 1.0
    assert dec[0, 0] == 448 * s and dec[1, 1] == 2.0 ** -9 * s and dec[2, 2] == 0.0
    assert dec[3, 3] == 16 * s
    assert abs(dec[129, 130] + 3.0) <= 3.0 * 2.0 ** -4  # 3 mantissa bits


# ------------------------------------------------------------ Dual M-IHS
def test_exact_solve_dual_push_through_identity():
    """Aᵀ(AAᵀ + λI)⁻¹b = (AᵀA + λI)⁻¹Aᵀb (push-through identity), and the
    dual solution satisfies ν* = (b − Ax*)/λ (Eq. dual_relation)."""
    rng = np.random.default_rng(12)
    A = rng.standard_normal((30, 80)) @ np.diag(np.logspace(0, -2, 80))
    b = rng.standard_normal(30)
    lam = 0.05
    x, nu = o.exact_solve_dual(A, b, lam)
    xp = np.linalg.lstsq(np.vstack([A, math.sqrt(lam) * np.eye(80)]), np.concatenate([b, np.zeros(80)]),
                         rcond=None)[0]
    assert np.linalg.norm(x - xp) <= 1e-10 * np.linalg.norm(xp)
    assert np.linalg.norm(nu - (b - A @ x) / lam) <= 1e-9 * np.linalg.norm(nu)


@pytest.mark.parametrize("family", [o.GAUSSIAN, o.COUNTSKETCH, o.SRHT])
def test_dual_mihs_reaches_the_solution(family):
    """Algorithm 2 on a wide problem (n = 64 ≪ d = 2000) with SAᵀ sketched
    along d: x = Aᵀν converges to the primal solution of the least squares
    formulation (not the oracle's own closed form)."""
    rng = np.random.default_rng(13 + family)
    n, d, lam = 64, 2000, 1e-3
    A = rng.standard_normal((n, d)) @ np.diag(np.logspace(0, -1, d)) / math.sqrt(d)
    b = rng.standard_normal(n)
    sd = o.stat_dim_of(A, lam)
    m = int(math.ceil(4 * sd / 4)) * 4 + 4
    SAt = o.sketch_apply(family, A.T, m, seed=21)
    x, nu, info = o.dual_mihs(A, b, lam, SAt, sd, N=200, tol=1e-12)
    # the minimiser of ½‖Ax − b‖² + (λ/2)‖x‖² from LAPACK's least squares
    xp = np.linalg.lstsq(np.vstack([A, math.sqrt(lam) * np.eye(d)]), np.concatenate([b, np.zeros(d)]),
                         rcond=None)[0]
    assert o.rel_error(x, xp) <= 1e-9, info
    assert info["outer"] < 60


# ------------------------------------------------- bf16-operand Gaussian sketch
def _bf16_rne_bits(x: float) -> float:
    """fp32 → bf16 by integer arithmetic on the fp32 bit pattern (round to
    nearest, ties to even), independent of torch's cast."""
    u = int(np.array(x, dtype=np.float32).view(np.uint32))
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return float(np.array(u, dtype=np.uint32).view(np.float32))


def test_gaussian_sketch_bf16_brute_force():
    """Entry by entry: Philox counter (⌊j/4⌋, i, tag, 0), the Box–Muller pair
    of the entry, both operands rounded by bit arithmetic, an exact sum over
    j and 1/√m — against the oracle's vectorised form.  Integer A is exact in
    bf16, so a wrong rounding of S, a wrong word pair or a transposed
    operand shows."""
    m, n, d, seed = 3, 9, 4, 0x1234ABCD
    A = W.randint_matrix((n, d), 17, -4, 4).numpy().astype(np.float64)
    A[0, 0] = 1 + 3 * 2.0 ** -9  # not a bf16 value: rounds up to 1 + 2⁻⁷
    k0, k1 = o.seed_key(seed)
    ref = np.zeros((m, d))
    for i in range(m):
        for j in range(n):
            w = o.philox4x32_10(np.uint64(j // 4), np.uint64(i), o.TAG_GAUSSIAN, 0, k0, k1)
            pa, pb = (w[0], w[1]) if j % 4 < 2 else (w[2], w[3])
            z = o.box_muller(pa, pb)[j % 2]
            zb = _bf16_rne_bits(float(z))
            for c in range(d):
                ref[i, c] += zb * _bf16_rne_bits(A[j, c])
    ref /= math.sqrt(m)
    got = o.gaussian_sketch_bf16(A, m, seed)
    assert np.allclose(got, ref, rtol=1e-14, atol=1e-14)
    assert _bf16_rne_bits(1 + 2.0 ** -8) == 1.0 and _bf16_rne_bits(1 + 3 * 2.0 ** -9) == 1 + 2.0 ** -7
    assert o.round_bf16(np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -9]))[1] == 1 + 2.0 ** -7


# ----------------------------------------------- double-double gradient (C)
def test_gradient_dd_against_exact_rationals():
    """Every entry of Aᵀ(b − Ax) − λx in exact rational arithmetic from the
    same fp32 / fp64 inputs: the double-double result agrees to ~2⁻¹⁰⁰ of
    the terms' magnitude, on generic data and on a row residual that cancels
    to far below fp64's resolution of b."""
    from fractions import Fraction as F
    rng = np.random.default_rng(5)
    n, d = 9, 6
    A = rng.standard_normal((n, d)).astype(np.float32)
    b = rng.standard_normal(n).astype(np.float32)
    x = rng.standard_normal(d)
    lam = 0.37
    # a row whose residual cancels: b_0 = fp32(A_0·x), x perturbed by 2⁻⁴⁰
    b[0] = np.float32(A[0].astype(np.float64) @ x)
    x[1] += 2.0 ** -40
    gh, gl = o.gradient_dd(A, b, x, lam, nthreads=3)
    Af = [[F(float(v)) for v in row] for row in A]
    r = [F(float(b[i])) - sum(Af[i][j] * F(float(x[j])) for j in range(d)) for i in range(n)]
    for j in range(d):
        exact = sum(Af[i][j] * r[i] for i in range(n)) - F(lam) * F(float(x[j]))
        scale = sum(abs(Af[i][j]) * (abs(F(float(b[i]))) + sum(abs(Af[i][k] * F(float(x[k]))) for k in range(d)))
                    for i in range(n)) + abs(F(lam) * F(float(x[j])))
        err = abs(F(float(gh[j])) + F(float(gl[j])) - exact)
        assert err <= scale * F(2) ** -100, (j, float(err), float(scale))
    # the thread split does not change the result beyond the last bits
    gh1, gl1 = o.gradient_dd(A, b, x, lam, nthreads=1)
    assert np.allclose(gh1 + gl1, gh + gl, rtol=0, atol=1e-28 * float(np.max(np.abs(gh))))


def test_exact_solve_dd_refinement_on_ill_conditioned_problem():
    """κ(H) ≈ 1e6: refining with the double-double residual drives the fp64
    residual of x to rounding level and agrees with the extended-precision
    refinement."""
    sigma = W.profile_exponential(128, 8.0)
    p = W.make_problem(2048, 128, sigma, 1e-6, 40.0, seed=31)
    A, b = p.A.numpy(), p.b.numpy()
    x = o.exact_solve(A, b, p.lam, refine=3, dd=True)
    xe = o.exact_solve(A, b, p.lam, refine=3, extended=True)
    assert o.rel_error(x, xe) <= 1e-12
    gh, gl = o.gradient_dd(A, b, x, p.lam)
    atb = np.abs(A.astype(np.float64)).T @ np.abs(b.astype(np.float64))
    assert np.linalg.norm(gh + gl) <= 1e-13 * np.linalg.norm(atb)


def test_gradient_blocked_is_blocking_independent_and_brute_force():
    rng = np.random.default_rng(5)
    n, d, lam = 37, 6, 0.3
    A, b, x = rng.standard_normal((n, d)), rng.standard_normal(n), rng.standard_normal(d)
    want = np.zeros(d)
    for i in range(n):  # row by row: a_i (b_i − a_i·x)
        want += A[i] * (b[i] - sum(A[i, j] * x[j] for j in range(d)))
    want -= lam * x
    for blk in (1, 5, 36, 37, 1000):
        assert np.allclose(o.gradient_blocked(A, b, x, lam, row_block=blk), want, rtol=1e-13, atol=1e-13)


def test_characteristic_roots_vieta_and_underdamped_modulus():
    """Roots of the heavy-ball characteristic polynomial (proof of Theorem 1):
    their sum is the trace 1 + β − αμ and their product β; when they are
    complex both have modulus √β."""
    rng = np.random.default_rng(6)
    for _ in range(50):
        beta = rng.uniform(0.01, 0.9)
        alpha = rng.uniform(0.05, 2.0)
        mu = rng.uniform(0.0, 3.0, size=7)
        r1, r2 = o.characteristic_roots(mu, alpha, beta)
        assert np.allclose(r1 + r2, 1 + beta - alpha * mu, atol=1e-12)
        assert np.allclose(r1 * r2, beta, atol=1e-12)
        cplx = (1 + beta - alpha * mu) ** 2 < 4 * beta
        assert np.allclose(np.abs(r1[cplx]), math.sqrt(beta)) and np.allclose(np.abs(r2[cplx]), math.sqrt(beta))


def test_corollary3_iteration_count_closed_form():
    """With β = 1/4 the rate √β is 1/2, so η = 2⁻¹⁰ needs exactly 10 steps;
    with β = 1/100, η = 1e-6 needs 6."""
    assert math.isclose(o.corollary3_iters(2.0 ** -10, 0.25), 10.0, rel_tol=1e-12)
    assert math.isclose(o.corollary3_iters(1e-6, 0.01), 6.0, rel_tol=1e-12)


def test_quantised_sa_spectrum_reading():
    """Reading of quantised SA storage (the sketch only preconditions, Section
    3.1; the heavy ball of Theorem 1 converges for eigenvalues μ of
    (SAᵀSA + λI)⁻¹(AᵀA + λI) with α·μ < 2(1 + β)).  At κ(AᵀA + λI) ≈ 1e6
    (8 decades, λ = 1e-6) bf16 rounding of SA keeps μ inside that region and
    fp8 e4m3 with 128 × 128 tile scales pushes it out, and the estimate
    ‖E‖_F²·(1/√m + 1/√d)² used by the library's guard tracks ‖E‖₂² of the
    actual rounding E = SA_q − SA within a factor 2 and sits on the same side
    of λ/2."""
    n, d, lam = 4096, 256, 1e-6
    sig = W.profile_exponential(d, 8.0)
    p = W.make_problem(n, d, sig, lam, 40.0, 77)
    A = p.A.numpy().astype(np.float64)
    m = min(n, W.round_up(4 * p.sd, 4))
    SA = o.sketch_apply(o.GAUSSIAN, p.A.numpy(), m, 5)
    alpha, beta = o.momentum_params(p.sd, m)
    edge = 2 * (1 + beta) / alpha
    out = {}
    for prec in ("bf16", "fp8"):
        dec = o.quantize_sa(SA.astype(np.float32), prec)[2]
        E = dec - SA.astype(np.float32).astype(np.float64)
        e2 = np.linalg.norm(E, 2) ** 2
        est = np.sum(E * E) * (1 / np.sqrt(m) + 1 / np.sqrt(d)) ** 2
        assert 0.5 * e2 <= est <= 2 * e2, (prec, est, e2)
        mu = o.sketched_hessian_eigs(A, dec, lam)
        out[prec] = (est / lam, mu.max())
    assert out["bf16"][0] <= 0.5 and out["bf16"][1] < edge, out
    assert out["fp8"][0] > 0.5 and out["fp8"][1] > edge, out


def test_round_e4m3_against_the_format():
    """e4m3: 3 mantissa bits, bias 7, largest finite 448, smallest subnormal
    2⁻⁹; ties to even; saturation at ±448."""
    cases = [(1.0, 1.0), (1.0625, 1.0), (1.1875, 1.25), (17.0, 16.0), (19.0, 20.0), (448.0, 448.0),
             (500.0, 448.0), (-1000.0, -448.0), (2.0 ** -9, 2.0 ** -9), (2.0 ** -10, 0.0),
             (3 * 2.0 ** -10, 2.0 ** -8), (0.3, 0.3125), (-2.2, -2.25), (240.0, 240.0), (232.0, 224.0)]
    got = o.round_e4m3([c[0] for c in cases])
    assert list(got) == [c[1] for c in cases], list(zip([c[0] for c in cases], got))


def test_gaussian_sketch_fp8_by_loops():
    """The fp8-operand sketch entry by entry: the N(0,1) entries of
    gaussian_sketch_rows rounded to e4m3, A scaled by the power of two that
    puts max|A| in [128, 256) and rounded to e4m3, products summed exactly
    (math.fsum), the scale and 1/√m undone."""
    rng = np.random.default_rng(3)
    n, d, m, seed = 37, 5, 3, 99
    A = (rng.standard_normal((n, d)) * 0.013).astype(np.float32)
    got = o.gaussian_sketch_fp8(A, m, seed)
    mx = float(np.max(np.abs(A)))
    k = 0
    while mx * 2.0 ** k < 128.0:
        k += 1
    assert 128.0 <= mx * 2.0 ** k < 256.0
    Z = o.gaussian_sketch_rows(np.arange(m), n, m, seed) * math.sqrt(m)
    for i in range(m):
        for j in range(d):
            terms = [float(o.round_e4m3(Z[i, kk])) * float(o.round_e4m3(A[kk, j] * 2.0 ** k)) for kk in range(n)]
            want = math.fsum(terms) * 2.0 ** -k / math.sqrt(m)
            assert got[i, j] == pytest.approx(want, rel=1e-14, abs=1e-18), (i, j)
    # the scale for A = 0, a power of two above 1, and a tiny maximum
    assert o.fp8_scale(np.zeros((2, 2))) == (1.0, 1.0)
    assert o.fp8_scale(np.array([[3.0]])) == (64.0, 1.0 / 64)
    assert o.fp8_scale(np.array([[256.0]])) == (0.5, 2.0)
    s, inv = o.fp8_scale(np.array([[1e-40]], dtype=np.float32))
    assert s == np.float32(2.0 ** 127) and inv == 2.0 ** -127
