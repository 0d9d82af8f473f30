"""Seeded synthetic ridge problems shared by the CUDA path's tests, the oracle's
tests and the benchmark.

This module only draws random numbers and shapes them into inputs; it contains
none of the solver's arithmetic.  Every problem is `min ½‖Ax−b‖² + (λ/2)‖x‖²`
(Section 1, Eq. "intro") with a measurement model `b = A x0 + ω` (Eq. "setup").

Construction (stands in for the paper's RegTools-based generator of Section 4.1,
whose singular-value profiles and signals are not available here):

* ``A = G · diag(σ) · Vᵀ / √n`` with ``G`` an n×d standard Gaussian matrix and
  ``V`` Haar-orthogonal (QR of a d×d Gaussian with the sign of diag(R) fixed
  positive, Mezzadri 2007).  Since ``G/√n`` has nearly orthonormal columns for
  n ≫ d, the singular values of ``A`` are close to the profile ``σ``.
* ``x0 ~ N(0, I_d)``, ``ω`` Gaussian rescaled so that
  ``‖A x0‖ / ‖ω‖ = 10^(SNR/20)``.
* ``A`` and ``b`` are rounded to fp32; the problem *is* those fp32 bytes.

The nominal statistical dimension ``Σ σᵢ²/(σᵢ²+λ)`` of the profile is part of
the workload specification (it fixes λ for the 4096×256 case and the sketch
size m = 4·sd), so it is computed here from the profile, not from ``A``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch


# --------------------------------------------------------------------------
# singular-value profiles
# --------------------------------------------------------------------------
def profile_exponential(d: int, decades: float) -> np.ndarray:
    """σ_i = 10^(−decades·(i−1)/(d−1)), i = 1..d."""
    i = np.arange(d, dtype=np.float64)
    return 10.0 ** (-decades * i / max(d - 1, 1))


def profile_polynomial(d: int, power: float) -> np.ndarray:
    """σ_i = i^(−power), i = 1..d."""
    return np.arange(1, d + 1, dtype=np.float64) ** (-power)


def nominal_sd(sigma: np.ndarray, lam: float) -> float:
    """Statistical dimension of the nominal profile (workload specification)."""
    s2 = np.asarray(sigma, dtype=np.float64) ** 2
    return float(np.sum(s2 / (s2 + lam)))


def lambda_for_sd(sigma: np.ndarray, sd_target: float) -> float:
    """λ such that the nominal profile has statistical dimension sd_target
    (geometric bisection; sd is monotone decreasing in λ)."""
    lo, hi = 1e-300, 1e300
    for _ in range(400):
        mid = math.sqrt(lo * hi)
        if nominal_sd(sigma, mid) > sd_target:
            lo = mid
        else:
            hi = mid
    return math.sqrt(lo * hi)


def round_up(v: float, q: int) -> int:
    return int(math.ceil(v / q) * q)


# --------------------------------------------------------------------------
# problem container
# --------------------------------------------------------------------------
@dataclass
class RidgeProblem:
    name: str
    A: torch.Tensor          # n×d fp32, row-major, contiguous
    b: torch.Tensor          # n fp32
    lam: float
    sd: float                # nominal statistical dimension (solver input)
    m: int                   # sketch rows
    x0: torch.Tensor         # ground-truth signal (fp32, d)
    sigma: np.ndarray        # nominal singular values
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.A.shape[0])

    @property
    def d(self) -> int:
        return int(self.A.shape[1])


def _haar(d: int, gen: torch.Generator) -> torch.Tensor:
    Z = torch.randn(d, d, generator=gen, dtype=torch.float64)
    Q, R = torch.linalg.qr(Z)
    sgn = torch.sign(torch.diagonal(R))
    sgn[sgn == 0] = 1.0
    return Q * sgn.unsqueeze(0)


def make_problem(n: int, d: int, sigma: np.ndarray, lam: float, snr_db: float,
                 seed: int, m: int | None = None, sd_factor: float = 4.0,
                 name: str = "custom", device: str = "cpu",
                 chunk_rows: int = 1 << 15, device_rng: bool = False) -> RidgeProblem:
    """Build ``A = G diag(σ) Vᵀ/√n`` and ``b = A x0 + ω`` (see module doc).

    Random draws come from a CPU ``torch.Generator`` seeded with ``seed`` so the
    bytes do not depend on the device; the n×d×d product runs on ``device``
    (fp64 on CPU, fp32 without TF32 on CUDA) in row chunks.  Tensors are
    returned on ``device``.  With ``device_rng`` (CUDA only) the n×d Gaussian
    G is drawn by a CUDA generator seeded with ``seed`` instead (much faster
    for multi-GB batches; the bytes then depend on the torch build).
    """
    gen = torch.Generator(device="cpu").manual_seed(int(seed))
    dgen = torch.Generator(device=device).manual_seed(int(seed)) if device_rng else None
    sigma = np.asarray(sigma, dtype=np.float64)
    assert sigma.shape == (d,)
    V = _haar(d, gen)
    x0 = torch.randn(d, generator=gen, dtype=torch.float64)
    on_cuda = device.startswith("cuda")
    cdt = torch.float32 if on_cuda else torch.float64
    scale = torch.from_numpy(sigma / math.sqrt(n)).to(cdt)
    M = (scale.unsqueeze(1) * V.t().to(cdt)).to(device)          # diag(σ)Vᵀ/√n
    A = torch.empty(n, d, dtype=torch.float32, device=device)
    if on_cuda:
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for r0 in range(0, n, chunk_rows):
            r1 = min(n, r0 + chunk_rows)
            if dgen is not None:
                G = torch.randn(r1 - r0, d, generator=dgen, dtype=torch.float32, device=device)
            else:
                G = torch.randn(r1 - r0, d, generator=gen, dtype=torch.float32)
            A[r0:r1] = (G.to(device=device, dtype=cdt) @ M).to(torch.float32)
    finally:
        if on_cuda:
            torch.backends.cuda.matmul.allow_tf32 = prev
    omega = torch.randn(n, generator=gen, dtype=torch.float64)
    Ax0 = (A.to(cdt) @ x0.to(device=device, dtype=cdt)).to(torch.float64).cpu()
    omega = omega * (Ax0.norm() / omega.norm()) / (10.0 ** (snr_db / 20.0))
    b = (Ax0 + omega).to(torch.float32).to(device)
    sd = nominal_sd(sigma, lam)
    if m is None:
        m = min(n, round_up(sd_factor * sd, 4))
    return RidgeProblem(name=name, A=A, b=b, lam=float(lam), sd=sd, m=int(m),
                        x0=x0.to(torch.float32).to(device), sigma=sigma,
                        meta=dict(n=n, d=d, snr_db=snr_db, seed=seed))


# --------------------------------------------------------------------------
# the named workloads
# --------------------------------------------------------------------------
def problem_small(device: str = "cpu", seed: int = 1000) -> RidgeProblem:
    """4096×256, σ_i = 10^(−4(i−1)/255) (κ(A)=1e4), λ so that sd = 64,
    30 dB SNR, Gaussian sketch with m = 4·64 = 256."""
    n, d = 4096, 256
    sigma = profile_exponential(d, 4.0)
    lam = lambda_for_sd(sigma, 64.0)
    return make_problem(n, d, sigma, lam, 30.0, seed, m=256,
                        name="ridge-4096x256-exp4-sd64", device=device)


def problem_bandwidth(device: str = "cpu", seed: int = 1001,
                      n: int = 262144, d: int = 1024) -> RidgeProblem:
    """262144×1024, σ_i = 1/i, λ = 1e-4, 40 dB SNR, m = 4·sd rounded up to a
    multiple of 4 (sd ≈ 146.85 → m = 588)."""
    sigma = profile_polynomial(d, 1.0)
    return make_problem(n, d, sigma, 1e-4, 40.0, seed,
                        name=f"ridge-{n}x{d}-poly1-lam1e-4", device=device)


def problem_differentiable(device: str = "cpu", seed: int = 1004,
                           n: int = 1 << 20, d: int = 1024) -> RidgeProblem:
    """2²⁰×1024, σ_i = i^(−1.5), λ = 1e-4 (sd ≈ 25.5), 40 dB SNR, m = 4·sd
    rounded up to a multiple of 4: the workload of the differentiable solve."""
    sigma = profile_polynomial(d, 1.5)
    return make_problem(n, d, sigma, 1e-4, 40.0, seed,
                        name=f"ridge-{n}x{d}-poly1.5-lam1e-4", device=device)


def batch_lambda_path(device: str = "cpu", seed: int = 1003, count: int = 64, nlambda: int = 16,
                      n_range=(8192, 262144), d_choices=(64, 128, 256, 512, 1024),
                      device_rng: bool = False):
    """The batched λ-path workload: `count` matrices with n log-uniform in
    n_range (a multiple of 16), d uniform over d_choices, σ_i =
    10^(−r(i−1)/(d−1)) with r ~ U[2, 6], 30 dB SNR; one log-spaced path of
    `nlambda` values in [1e-6, 1e-1] shared by all; per matrix
    m = min(4·sd(λ_min), n) rounded up to a multiple of 4 and sd(λ_l) from
    the nominal profile.  Returns (problems, lambdas, sds) with sds[i][l]."""
    rng = np.random.default_rng(int(seed))
    lams = list(np.logspace(-6, -1, nlambda))
    probs, sds = [], []
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1]))) / 16.0)) * 16
        d = int(rng.choice(d_choices))
        r = float(rng.uniform(2.0, 6.0))
        sigma = profile_exponential(d, r)
        sd_row = [nominal_sd(sigma, l) for l in lams]
        m = min(n, round_up(4.0 * max(sd_row), 4))
        probs.append(make_problem(n, d, sigma, lams[0], 30.0, int(seed) * 1000 + i, m=m,
                                  name=f"path-{i}-{n}x{d}-exp{r:.2f}", device=device, device_rng=device_rng))
        sds.append(sd_row)
    return probs, lams, sds


def problem_scaled(n: int, d: int, seed: int, decades: float = 4.0,
                   sd_frac: float = 0.25, snr_db: float = 30.0,
                   device: str = "cpu") -> RidgeProblem:
    """Smaller members of the same family (test sizes): exponential decay,
    λ so that sd = sd_frac·d, m = 4·sd."""
    sigma = profile_exponential(d, decades)
    lam = lambda_for_sd(sigma, sd_frac * d)
    return make_problem(n, d, sigma, lam, snr_db, seed,
                        name=f"ridge-{n}x{d}-exp{decades:g}", device=device)


# --------------------------------------------------------------------------
# plain seeded tensors for kernel-level parity cases
# --------------------------------------------------------------------------
def randn(shape, seed: int, scale: float = 1.0, dtype=torch.float32) -> torch.Tensor:
    gen = torch.Generator(device="cpu").manual_seed(int(seed))
    return (torch.randn(*shape, generator=gen, dtype=torch.float64) * scale).to(dtype)


def randint_matrix(shape, seed: int, lo: int = -8, hi: int = 8) -> torch.Tensor:
    """Integer-valued fp32 matrix (sums of such entries are exact in fp32)."""
    gen = torch.Generator(device="cpu").manual_seed(int(seed))
    return torch.randint(lo, hi + 1, shape, generator=gen).to(torch.float32)


def padded_matrix(n: int, d: int, lda: int, seed: int) -> torch.Tensor:
    """n×lda storage whose first d columns hold N(0,1) values and whose
    padding holds NaN (so that any read of the padding shows up)."""
    M = torch.full((n, lda), float("nan"), dtype=torch.float32)
    M[:, :d] = randn((n, d), seed)
    return M
