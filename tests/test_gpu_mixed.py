"""Parity of the mixed-precision forms: the quantised storage of SA (bf16,
fp8 e4m3 with tile scales) byte for byte against the oracle's quantiser,
AAb_Solver on the quantised SA against the oracle's Algorithm 5 on the
decoded SA, the Gaussian sketch formed from bf16 operands against the
oracle's sum of the same rounded operands, and solves with a quantised SA
reaching the same solution."""
import math

import numpy as np
import pytest
import torch

from oracle import mihs_oracle as o
from paper_1912_03514_gb300 import mihs
from paper_1912_03514_gb300 import workloads as W
from tests._tol import U32, gamma

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _sa(m, d, seed):
    """Gaussian SA with column blocks of very different magnitudes, so that
    the fp8 tile scales differ."""
    SA = W.randn((m, d), seed, scale=1.0 / math.sqrt(m))
    col_scale = torch.from_numpy(np.logspace(0, -3, d).astype(np.float32))
    return SA * col_scale


@pytest.mark.parametrize("m,d", [(256, 256), (588, 1024), (300, 129), (130, 131), (3076, 2048), (1, 3)])
@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_quantize_sa_bytes_match_oracle(m, d, prec):
    SA = _sa(m, d, 11 + d)
    q, sc = mihs.quantize_sa(SA.to(DEV), prec)
    qr, scr, _ = o.quantize_sa(SA.numpy(), prec)
    q = q.cpu()
    ldq = q.shape[1]
    assert ldq % 16 == 0 and ldq >= d
    if prec == "bf16":
        assert torch.equal(q[:, :d].view(torch.int16), qr.view(torch.int16))
        assert not torch.any(q[:, d:].view(torch.int16))
    else:
        assert np.array_equal(sc.cpu().numpy(), scr)
        assert torch.equal(q[:, :d], qr.view(torch.uint8))
        assert not torch.any(q[:, d:])


def _decoded(q, sc, prec, m, d):
    if prec == "bf16":
        return q[:, :d].to(torch.float64).cpu().numpy()
    dec = q[:, :d].cpu().view(torch.float8_e4m3fn).to(torch.float64).numpy()
    S = np.repeat(np.repeat(sc.cpu().numpy().astype(np.float64), 128, axis=0), 128, axis=1)[:m, :d]
    return dec * S


@pytest.mark.parametrize("m,d,lam", [(588, 1024, 1e-4), (256, 256, 0.0103), (1500, 300, 1e-3), (64, 48, 0.1)])
@pytest.mark.parametrize("prec", ["bf16", "fp8"])
@pytest.mark.parametrize("k", [1, 4, 25])
def test_aab_on_quantised_sa_matches_oracle(m, d, lam, prec, k):
    """k passes of Algorithm 5 on the decoded SA: the kernel against the
    oracle in fp64, within 20× the oracle's own fp32-vs-fp64 difference."""
    SA = _sa(m, d, 5 * m + d)
    g = W.randn((d,), 3 * d)
    q, sc = mihs.quantize_sa(SA.to(DEV), prec)
    SAd = _decoded(q, sc, prec, m, d)
    gn = g.numpy().astype(np.float64)
    x64, _ = o.aab_solve(SAd, gn, lam, 0.0, max_iter=k)
    x32, _ = o.aab_solve(SAd.astype(np.float32), gn.astype(np.float32), lam, 0.0, max_iter=k, dtype=np.float32)
    amp = o.rel_error(x32, x64)
    passes = torch.zeros(1, dtype=torch.int32, device=DEV)
    delta = mihs.aab_solve_q(q, prec, sc, d, g.to(DEV), lam, eps_sub=0.0, max_inner=k, passes=passes)
    assert int(passes.item()) == min(k, m, d)
    err = o.rel_error(delta.cpu().double().numpy(), x64)
    assert err <= 20 * max(amp, 4 * U32 * math.sqrt(d)), (err, amp)


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
@pytest.mark.parametrize("family", ["gaussian", "countsketch"])
def test_solves_with_quantised_sa_reach_the_solution(prec, family):
    """The fixed point does not depend on SA: plain solves meet the same
    relative error as with fp32 SA, refined solves reach 1e-10."""
    p = W.problem_small()
    A, b = p.A.to(DEV), p.b.to(DEV)
    xs = o.exact_solve(p.A.numpy(), p.b.numpy(), p.lam, refine=3, extended=True)
    with mihs.Sketch(A, family, p.m, seed=12) as sk:
        x32, i32 = sk.solve(A, b, p.lam, p.sd, tol=1e-6, max_outer=200)
        sk.set_precision(prec)
        xq, iq = sk.solve(A, b, p.lam, p.sd, tol=1e-6, max_outer=200)
        xr, ir = sk.solve_refined(A, b, p.lam, p.sd, tol=1e-13, max_outer=300)
        sk.set_precision("fp32")
        x32b, _ = sk.solve(A, b, p.lam, p.sd, tol=1e-6, max_outer=200)
    assert iq.converged and ir.converged, (iq, ir)
    assert o.rel_error(xq.cpu().double().numpy(), xs) <= 1e-5
    assert o.rel_error(xr.cpu().numpy(), xs) <= 1e-10
    assert torch.equal(x32b, x32)  # back to fp32 storage: the same bytes as before
    # the rate may change a little, not the order of the step count
    assert iq.outer_iters <= 2 * i32.outer_iters + 5


def test_refined_solve_bf16_sa_ill_conditioned():
    """κ(H) ≈ 1e6 (the mixed-precision workload's conditioning at a size the
    oracle refines quickly): bf16 SA with refinement reaches 1e-10.  (fp8's
    2⁻⁴ relative rounding of every entry swamps the directions of A with
    σ_i ≪ 2⁻⁴·σ_1, so SAq stops preconditioning them: the library refuses
    that solve, test_fp8_refused_where_it_cannot_precondition.)"""
    n, d = 65536, 512
    sigma = W.profile_exponential(d, 8.0)
    p = W.make_problem(n, d, sigma, 1e-6, 40.0, seed=21)
    A, b = p.A.to(DEV), p.b.to(DEV)
    xs = o.exact_solve(p.A.numpy(), p.b.numpy(), p.lam, refine=3, extended=True)
    with mihs.Sketch(A, "countsketch", p.m, seed=13) as sk:
        sk.set_precision("bf16")
        x, info = sk.solve_refined(A, b, p.lam, p.sd, tol=1e-14, max_outer=400)
    err = o.rel_error(x.cpu().numpy(), xs)
    assert err <= 1e-10, (err, info)


def test_fp8_refused_where_it_cannot_precondition():
    """At κ(AᵀA + λI) ≈ 1e6 the fp8 rounding of SA is ≈ 75·λ in spectral norm
    (the oracle's test_quantised_sa_spectrum_reading): every solve on an fp8
    handle there returns MIHS_ERR_UNSUPPORTED with a message before launching
    anything, bf16 storage of the same sketch is accepted and reaches the
    oracle's solution, and fp8 at λ = 1e-3 (4 decades) is accepted too."""
    n, d = 16384, 512
    p = W.make_problem(n, d, W.profile_exponential(d, 8.0), 1e-6, 40.0, seed=1012)
    A, b = p.A.to(DEV), p.b.to(DEV)
    with mihs.Sketch(A, "gaussian", p.m, seed=3) as sk:
        sk.set_precision("fp8")
        for call in (lambda: sk.solve(A, b, p.lam, p.sd, tol=1e-6),
                     lambda: sk.solve_refined(A, b, p.lam, p.sd, tol=1e-12),
                     lambda: sk.solve_path(A, b, [1e-3, p.lam], sds=[10.0, p.sd], tol=1e-6)):
            with pytest.raises(mihs.MihsError) as e:
                call()
            assert e.value.code == mihs.UNSUPPORTED and "no longer preconditions" in str(e.value), str(e.value)
        sk.set_precision("bf16")
        x, info = sk.solve_refined(A, b, p.lam, p.sd, tol=1e-14, max_outer=400)
    xs = o.exact_solve(p.A.numpy(), p.b.numpy(), p.lam, refine=3, extended=True)
    assert info.converged and o.rel_error(x.cpu().numpy(), xs) <= 1e-10, info
    q = W.make_problem(n, d, W.profile_exponential(d, 4.0), 1e-3, 40.0, seed=1013)
    Aq, bq = q.A.to(DEV), q.b.to(DEV)
    with mihs.Sketch(Aq, "gaussian", q.m, seed=3) as sk:
        sk.set_precision("fp8")
        xq, iq = sk.solve_refined(Aq, bq, q.lam, q.sd, tol=1e-12, max_outer=300)
    xsq = o.exact_solve(q.A.numpy(), q.b.numpy(), q.lam, refine=3, extended=True)
    assert iq.converged and o.rel_error(xq.cpu().numpy(), xsq) <= 1e-10, iq


def test_path_with_bf16_sa():
    p = W.problem_small()
    A, b = p.A.to(DEV), p.b.to(DEV)
    lams = list(np.logspace(-3, -1, 8))
    sds = [W.nominal_sd(p.sigma, l) for l in lams]
    with mihs.Sketch(A, "gaussian", p.m, seed=4) as sk:
        sk.set_precision("bf16")
        X, infos = sk.solve_path(A, b, lams, sds=sds, tol=1e-6, max_outer=200)
    XS = o.ridge_path(p.A.double().numpy(), p.b.double().numpy(), lams)
    for l, inf in enumerate(infos):
        assert inf.converged, (l, inf)
        assert o.rel_error(X[l].cpu().double().numpy(), XS[l]) <= 1e-4


def test_quantised_arguments():
    SA = _sa(64, 48, 1).to(DEV)
    with pytest.raises(mihs.MihsError):
        mihs.quantize_sa(SA, 0)  # fp32 is not a quantised format
    with pytest.raises(ValueError):
        mihs.quantize_sa(SA, "fp16")


# ------------------------------------------- Gaussian sketch from bf16 operands
@pytest.mark.parametrize("n,d,m", [(4096, 256, 256), (5000, 700, 300), (2049, 1500, 129), (100, 520, 40),
                                   (12000, 2048, 260), (777, 33, 17)])
def test_gaussian_bf16_sketch_matches_oracle(n, d, m):
    """S·A from bf16-rounded operands on the tensor cores against the
    oracle's exact sum of the same rounded operands.  The kernel's S comes
    from fast fp32 transcendentals, so an entry may round to the neighbouring
    bf16 value (≤ 2⁻⁷ relative); products are exact in fp32, sums carry γ_K,
    the 1/√m scale 2u."""
    lda = (d + 3) // 4 * 4
    A = W.padded_matrix(n, d, lda, seed=n + 7 * d)
    seed = 0xBF16 + n
    Ad = A.to(DEV).as_strided((n, d), (lda, 1))
    SA = mihs.sketch_gaussian_bf16(Ad, m, seed)
    SA2 = mihs.sketch_gaussian_bf16(Ad, m, seed)
    torch.cuda.synchronize()
    An = A[:, :d].numpy().astype(np.float64)
    ref = o.gaussian_sketch_bf16(An, m, seed)
    S = np.abs(o.gaussian_sketch_matrix(m, n, seed))
    bound = (gamma(n + 16) + 2.0 ** -7 + 4 * U32) * (1 + 2.0 ** -7) * (S @ np.abs(o.round_bf16(An))) + 1e-30
    got = SA.double().cpu().numpy()
    assert np.all(np.isfinite(got))
    err = np.abs(got - ref)
    assert np.all(err <= bound), f"max err/bound {np.max(err / bound)}"
    assert torch.equal(SA, SA2), "not deterministic"


# -------------------------------------------- Gaussian sketch from fp8 operands
def _z_window(Z):
    """Half-width of the interval around the fp64 N(0,1) entry z that holds
    the kernel's fast-intrinsic Box–Muller value: CUDA documents the fast
    log's absolute error as 2⁻²¹·⁴¹ on [½, 2] (3 ulp elsewhere) and the fast
    sin/cos's as 2⁻²¹·⁴¹ on [−π, π], so t = −2 ln u₁ moves by ≤ 2⁻²⁰ and
    r = √t by ≤ min(√2⁻²⁰, 2⁻²⁰/r) ≤ min(2⁻¹⁰, 2⁻²⁰/|z|); 2⁻¹⁶(1 + |z|)
    covers the rest (angle, ulp roundings) with room."""
    a = np.abs(Z)
    return 2.0 ** -16 * (1.0 + a) + np.minimum(2.0 ** -10, 2.0 ** -20 / np.maximum(a, 2.0 ** -40))


@pytest.mark.parametrize("n,d,m", [(4096, 256, 256), (5000, 700, 300), (2049, 1500, 129), (100, 520, 40),
                                   (12000, 2048, 260), (777, 33, 17)])
def test_gaussian_fp8_sketch_matches_oracle(n, d, m):
    """S·A from e4m3 operands on the tensor cores (kind::f8f6f4) against
    the oracle's exact sum of the same rounded operands.  The scaled A is
    rounded identically on both sides (an exact power-of-two scale, then
    round-to-nearest-even); an entry of S within the fast intrinsics' error
    of an e4m3 rounding boundary may take either neighbour, which the bound
    carries entry by entry (ΔZ); products are exact in fp32, sums carry γ_K,
    the two scalings 3u."""
    lda = (d + 3) // 4 * 4
    A = W.padded_matrix(n, d, lda, seed=n + 7 * d + 8)
    seed = 0xF8 + n
    Ad = A.to(DEV).as_strided((n, d), (lda, 1))
    SA = mihs.sketch_gaussian_fp8(Ad, m, seed)
    SA2 = mihs.sketch_gaussian_fp8(Ad, m, seed)
    torch.cuda.synchronize()
    An = A[:, :d].numpy()
    ref = o.gaussian_sketch_fp8(An, m, seed)
    s, inv = o.fp8_scale(An)
    A8 = np.abs(o.round_e4m3(An * s))
    Z = o.gaussian_sketch_matrix(m, n, seed) * math.sqrt(m)
    h = _z_window(Z)
    lo, hi, mid = o.round_e4m3(Z - h), o.round_e4m3(Z + h), o.round_e4m3(Z)
    dz = np.maximum(np.abs(hi - mid), np.abs(mid - lo))
    zmax = np.maximum(np.abs(lo), np.abs(hi))
    c = inv / math.sqrt(m)
    bound = ((gamma(n + 16) + 4 * U32) * (zmax @ A8) + (1 + 4 * U32) * (dz @ A8)) * c + 1e-30
    got = SA.double().cpu().numpy()
    assert np.all(np.isfinite(got))
    err = np.abs(got - ref)
    assert np.all(err <= bound), f"max err/bound {np.max(err / bound)}"
    assert torch.equal(SA, SA2), "not deterministic"
    # the operands really are e4m3: SA differs from the bf16-operand sketch
    # by about 2⁻⁴ of |S|·|A|, far more than the bf16 rounding
    SAb = mihs.sketch_gaussian_bf16(Ad, m, seed).double().cpu().numpy()
    assert np.max(np.abs(got - SAb)) > 1e-3 * np.max(np.abs(SAb))


def test_gaussian_fp8_sketch_of_a_scaled_matrix_and_of_zero():
    """A power-of-two rescaling of A commutes with the fp8 sketch bit for
    bit (the scale is a power of two chosen from max|A|), and A = 0 gives
    SA = 0."""
    n, d, m = 3000, 96, 64
    A = W.randn((n, d), 5).to(DEV)
    SA = mihs.sketch_gaussian_fp8(A, m, 77)
    SA2 = mihs.sketch_gaussian_fp8(A * 2.0 ** -30, m, 77)
    SA0 = mihs.sketch_gaussian_fp8(torch.zeros_like(A), m, 77)
    torch.cuda.synchronize()
    assert torch.equal(SA * 2.0 ** -30, SA2)
    assert torch.count_nonzero(SA0).item() == 0


def test_gaussian_handle_with_fp8_storage_forms_sa_in_fp8():
    """A Gaussian handle stored in fp8 re-forms SA from e4m3 operands on
    resketch (its fp32 SA, which it then stores in fp8, is the row-level
    call's result byte for byte), and the refined solve reaches 1e-10."""
    p = W.problem_small()
    A, b = p.A.to(DEV), p.b.to(DEV)
    xs = o.exact_solve(p.A.numpy(), p.b.numpy(), p.lam, refine=3, extended=True)
    with mihs.Sketch(A, "gaussian", p.m, seed=23) as sk:
        sk.set_precision("fp8")
        sk.resketch(A, 23)
        sa8 = sk.sa().clone()
        x, info = sk.solve_refined(A, b, p.lam, p.sd, tol=1e-13, max_outer=300)
    assert torch.equal(sa8, mihs.sketch_gaussian_fp8(A, p.m, 23))
    assert info.converged and o.rel_error(x.cpu().numpy(), xs) <= 1e-10, info


def test_gaussian_handle_with_bf16_storage_forms_sa_in_bf16():
    """A Gaussian handle stored in bf16 re-forms SA from bf16 operands on
    resketch (the same bytes as the row-level call), and the refined solve
    on it still reaches 1e-10."""
    p = W.problem_small()
    A, b = p.A.to(DEV), p.b.to(DEV)
    xs = o.exact_solve(p.A.numpy(), p.b.numpy(), p.lam, refine=3, extended=True)
    with mihs.Sketch(A, "gaussian", p.m, seed=21) as sk:
        sa32 = sk.sa().clone()
        sk.set_precision("bf16")
        sk.resketch(A, 21)
        sab = sk.sa().clone()
        x, info = sk.solve_refined(A, b, p.lam, p.sd, tol=1e-13, max_outer=300)
    assert torch.equal(sab, mihs.sketch_gaussian_bf16(A, p.m, 21))
    assert not torch.equal(sab, sa32)
    assert info.converged and o.rel_error(x.cpu().numpy(), xs) <= 1e-10, info
