"""Oracle for the Momentum Iterative Hessian Sketch (M-IHS) ridge solver.

TEST INFRASTRUCTURE ONLY: plain numpy, fp64 unless a function says otherwise,
no blocking or fusion beyond what the cited definition states.  Imported only
by the tests, by ``__graft_entry__.smoke()`` and by the benchmark's CPU
baseline / reference legs.  Shares no code with the CUDA path.

Problem (Section 1, Eq. "intro"):  x* = argmin ½‖Ax−b‖² + (λ/2)‖x‖²,
A ∈ R^{n×d}, n ≥ d, λ > 0  ⇒  x* = (AᵀA + λI)⁻¹ Aᵀ b, unique.

Contents and the passage each follows:
  philox4x32_10 ........ Salmon, Moraes, Dror, Shaw (SC'11), "Parallel random
                          numbers: as easy as 1, 2, 3", Philox-4x32 with 10 rounds.
  box_muller ........... Box & Muller (1958) on 24-bit uniforms.
  sketch_* ............. the three families of Lemma 3 used here: (i) sparse
                          embedding with one ±1 per column (CountSketch),
                          (iii) SRHT, (iv) Gaussian with entries N(0, 1/m)
                          (proof of Lemma 3), all with E[SᵀS] = I (Section 3.1,
                          text after Algorithm 1).
  exact_solve .......... the plain definition (Cholesky of AᵀA+λI, fp64),
                          refined with a residual in extended precision or
                          in double-double (gradient_dd, plain C in
                          resid_dd.c: TwoSum/TwoProduct, Ogita–Rump–Oishi 2005).
  svd_solve ............ closed form x* = Σ σᵢ²/(σᵢ²+λ)·(uᵢᵀb/σᵢ)·vᵢ (Eq. tsvdsol).
  stat_dim ............. sd_λ(A) = Σ σᵢ²/(σᵢ²+λ) (Section 1; proof of Lemma 3).
  gradient ............. g = Aᵀ(b − Ax) − λx (Algorithm 1, gradient step).
  aab_solve ............ AAb_Solver (Algorithm 5, Section 3.6).
  momentum_params ...... β = sd/m, α = (1−β)² (Corollary 3, Algorithm 1).
  theorem1_params ...... β*, α*, rate of Theorem 1.
  mihs ................. Algorithm 1 (M-IHS for n ≥ d).
  dual_mihs ............ Algorithm 2 (Dual M-IHS for n ≤ d) on the dual
                          problem of Eq. intro_dual, x = Aᵀν (Eq. dual_relation).
  exact_solve_dual ..... the plain definition through the dual:
                          x* = Aᵀ(AAᵀ + λI)⁻¹b.
  hutchinson_sd ........ Algorithm 4 (inexact Hutchinson estimate of sd).
  gaussian_sketch_bf16 . the Gaussian sketch from bf16-rounded S and A, summed
                          exactly (the operand format of the bf16 tensor-core
                          sketch; a format, not the paper's).
  gaussian_sketch_fp8 .. the same from e4m3-rounded S and scaled A (round_e4m3,
                          fp8_scale; the operand format of the fp8 sketch).
  quantize_sa .......... storage of SA in bf16, or fp8 e4m3 with one scale per
                          128 × 128 tile (a format, not the paper's: the
                          sketch only preconditions, Section 3.1); torch's
                          CPU casts are the rounding step.
  ridge_path ........... x*(λ) for every λ of a path (the plain definition
                          per λ; Algorithm 1 applied to each λ on its own).
  ridge_backward ....... gradients of x*(A, b, λ) through the normal equations
                          of Section 1 (not in the paper: the adjoint of the
                          linear solve; parity pinned by central differences).
  heavy_ball ........... x⁺ = x + αΔ + β(x − x⁻) (Eq. mihs1).
  characteristic_rate .. roots of u² − (1+β−αμ)u + β (proof of Theorem 1).

Readings of the paper taken where it is silent or garbled (each is listed in
the design notes with its justification):
  * Algorithm 5 initial rotation sine is s = √λ/ρ̄ (the text's s_k = λ̄_k/ρ̄_k
    with λ̄₁ = √λ), not √(λ/ρ̄).
  * The Eq. after Algorithm 5's derivation is the *unsquared* residual norm.
  * x⁰ = x¹ (no momentum on the first step).
  * SRHT: S = √(n_p/m)·P·(H/√n_p)·D with n_p = 2^⌈log₂ n⌉ (zero-padded rows),
    P sampling m rows uniformly with replacement.
"""
from __future__ import annotations

import math
import os

import numpy as np

# ---------------------------------------------------------------------------
# Philox4x32-10 (Salmon et al., SC'11).  Vectorised over numpy uint64 arrays
# that hold 32-bit words.
# ---------------------------------------------------------------------------
_MASK = np.uint64(0xFFFFFFFF)
_PHILOX_M0 = np.uint64(0xD2511F53)
_PHILOX_M1 = np.uint64(0xCD9E8D57)
_PHILOX_W0 = np.uint64(0x9E3779B9)
_PHILOX_W1 = np.uint64(0xBB67AE85)

# Counter word 2 tags the stream a family draws from, so that no two uses of
# one seed share a counter.
TAG_GAUSSIAN = 0
TAG_COUNTSKETCH = 1
TAG_SRHT_SIGNS = 2
TAG_SRHT_ROWS = 3
TAG_HUTCHINSON = 4

GAUSSIAN, COUNTSKETCH, SRHT = 0, 1, 2
FAMILY_NAMES = {GAUSSIAN: "gaussian", COUNTSKETCH: "countsketch", SRHT: "srht"}


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox-4x32 rounds.  Each round multiplies words 0 and 2 by the two
    round multipliers, and the new counter is (hi(M1·c2) ⊕ c1 ⊕ k0, lo(M1·c2),
    hi(M0·c0) ⊕ c3 ⊕ k1, lo(M0·c0)); the key is bumped by the Weyl constants
    before every round but the first."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & _MASK for c in (c0, c1, c2, c3))
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    for r in range(10):
        if r > 0:
            k0 = (k0 + _PHILOX_W0) & _MASK
            k1 = (k1 + _PHILOX_W1) & _MASK
        p0 = _PHILOX_M0 * c0
        p1 = _PHILOX_M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def seed_key(seed: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32


def box_muller(wa, wb):
    """Two N(0,1) values from two 32-bit words: u1 = (⌊wa/2⁸⌋+1)·2⁻²⁴ ∈ (0,1],
    u2 = ⌊wb/2⁸⌋·2⁻²⁴ ∈ [0,1) (both exact in fp32), r = √(−2 ln u1),
    z = (r cos 2πu2, r sin 2πu2)."""
    u1 = ((np.asarray(wa, dtype=np.uint64) >> np.uint64(8)).astype(np.float64) + 1.0) * 2.0 ** -24
    u2 = (np.asarray(wb, dtype=np.uint64) >> np.uint64(8)).astype(np.float64) * 2.0 ** -24
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)


# ---------------------------------------------------------------------------
# Sketch families (Lemma 3; E[SᵀS] = I after Algorithm 1)
# ---------------------------------------------------------------------------
def gaussian_sketch_rows(rows, n: int, m: int, seed: int) -> np.ndarray:
    """Rows `rows` of the Gaussian sketch S ∈ R^{m×n}, S_ij ~ N(0, 1/m).
    Entry (i, j) comes from Philox counter (⌊j/4⌋, i, TAG_GAUSSIAN, 0): the
    four words give two Box–Muller pairs, (w0,w1) → (cos, sin) for
    j ≡ 0, 1 (mod 4) and (w2,w3) → (cos, sin) for j ≡ 2, 3."""
    rows = np.atleast_1d(np.asarray(rows, dtype=np.int64))
    k0, k1 = seed_key(seed)
    q = np.arange((n + 3) // 4, dtype=np.uint64)
    out = np.empty((rows.size, 4 * q.size), dtype=np.float64)
    for t, i in enumerate(rows):
        w0, w1, w2, w3 = philox4x32_10(q, np.uint64(i), TAG_GAUSSIAN, 0, k0, k1)
        za, zb = box_muller(w0, w1)
        zc, zd = box_muller(w2, w3)
        out[t, 0::4], out[t, 1::4], out[t, 2::4], out[t, 3::4] = za, zb, zc, zd
    return out[:, :n] / math.sqrt(m)


def gaussian_sketch_matrix(m: int, n: int, seed: int) -> np.ndarray:
    return gaussian_sketch_rows(np.arange(m), n, m, seed)


def round_bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), through torch's CPU
    cast of the fp32 value; returned as fp64."""
    import torch
    t = torch.as_tensor(np.asarray(x, dtype=np.float32))
    return t.to(torch.bfloat16).to(torch.float64).numpy()


def gaussian_sketch_bf16(A: np.ndarray, m: int, seed: int) -> np.ndarray:
    """The Gaussian sketch formed from bf16 operands (a storage format for
    the preconditioner, not the paper's: the sketch only preconditions,
    Section 3.1): SA = (1/√m)·Z̃·Ã with Z̃ the N(0,1) matrix of
    gaussian_sketch_rows (before the 1/√m) and Ã = A, each entry rounded to
    bf16, the products summed exactly (fp64)."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    Z = gaussian_sketch_matrix(m, n, seed) * math.sqrt(m)
    return (round_bf16(Z) @ round_bf16(A)) / math.sqrt(m)


def round_e4m3(x) -> np.ndarray:
    """Round to the nearest fp8 e4m3 value (4 exponent bits with bias 7, 3
    mantissa bits, no infinities: largest finite ±448, smallest subnormal
    2⁻⁹), ties to even, magnitudes beyond 448 saturating to ±448 — through
    torch's CPU cast of the fp32 value (clamped first); returned as fp64."""
    import torch
    t = torch.as_tensor(np.asarray(x, dtype=np.float32)).clamp(-448.0, 448.0)
    return t.to(torch.float8_e4m3fn).to(torch.float64).numpy()


def fp8_scale(A) -> tuple:
    """The scale of A for e4m3 operands: the power of two s = 2^k with
    max|A|·s in [128, 256) (k = 8 − e for max|A| = f·2^e, f ∈ [½, 1), capped
    at 127; k = 0 for A = 0), so that scaling is exact and stays below e4m3's
    448; returns (s, 1/s)."""
    A32 = np.asarray(A, dtype=np.float32)
    mx = float(np.max(np.abs(A32))) if A32.size else 0.0
    k = min(8 - math.frexp(mx)[1], 127) if mx > 0 else 0
    return np.float32(2.0 ** k), 2.0 ** -k


def gaussian_sketch_fp8(A: np.ndarray, m: int, seed: int) -> np.ndarray:
    """The Gaussian sketch formed from fp8 e4m3 operands (a format of the
    preconditioner, not the paper's: the sketch only preconditions, Section
    3.1): SA = (1/√m)·(1/s)·Z̃·Ã with Z̃ the N(0,1) matrix of
    gaussian_sketch_rows (before the 1/√m) rounded to e4m3, Ã = e4m3(A·s)
    and s the power of two of fp8_scale, the products summed exactly
    (fp64)."""
    A32 = np.asarray(A, dtype=np.float32)
    n = A32.shape[0]
    s, inv = fp8_scale(A32)
    Z = gaussian_sketch_matrix(m, n, seed) * math.sqrt(m)
    At = round_e4m3((A32 * s).astype(np.float32))
    return (round_e4m3(Z) @ At) * inv / math.sqrt(m)


def countsketch_hash(n: int, m: int, seed: int):
    """Bucket h(j) ∈ [0, m) and sign s(j) = ±1 of column j of the one-nonzero-
    per-column sparse embedding: Philox counter (j, 0, TAG_COUNTSKETCH, 0),
    h = ⌊w0·m / 2³²⌋, s = +1 if w1 is even else −1."""
    k0, k1 = seed_key(seed)
    j = np.arange(n, dtype=np.uint64)
    w0, w1, _, _ = philox4x32_10(j, 0, TAG_COUNTSKETCH, 0, k0, k1)
    h = ((w0 * np.uint64(m)) >> np.uint64(32)).astype(np.int64)
    s = np.where((w1 & np.uint64(1)) == 0, 1.0, -1.0)
    return h, s


def countsketch_matrix(m: int, n: int, seed: int) -> np.ndarray:
    h, s = countsketch_hash(n, m, seed)
    S = np.zeros((m, n))
    S[h, np.arange(n)] = s
    return S


def srht_params(n: int, m: int, seed: int):
    """n_p = 2^⌈log₂ n⌉; D_j = ±1 from counter (j, 0, TAG_SRHT_SIGNS, 0)
    (w0 even → +1); sampled Hadamard rows r_i = ⌊w0 / 2^(32−L)⌋ from counter
    (i, 0, TAG_SRHT_ROWS, 0), n_p = 2^L (uniform, with replacement)."""
    L = max(0, int(math.ceil(math.log2(max(n, 1)))))
    n_p = 1 << L
    k0, k1 = seed_key(seed)
    w0, _, _, _ = philox4x32_10(np.arange(n, dtype=np.uint64), 0, TAG_SRHT_SIGNS, 0, k0, k1)
    D = np.where((w0 & np.uint64(1)) == 0, 1.0, -1.0)
    r0, _, _, _ = philox4x32_10(np.arange(m, dtype=np.uint64), 0, TAG_SRHT_ROWS, 0, k0, k1)
    rows = (r0 >> np.uint64(32 - L)).astype(np.int64) if L > 0 else np.zeros(m, np.int64)
    return n_p, D, rows


def hadamard_entry(r, j):
    """Sylvester–Hadamard entry H[r, j] = (−1)^popcount(r AND j), broadcast
    over r and j."""
    x = np.bitwise_and(np.asarray(r, dtype=np.int64), np.asarray(j, dtype=np.int64))
    pc = np.zeros(np.shape(x), dtype=np.int64)
    while np.any(x):
        pc += x & 1
        x = x >> 1
    return np.where(pc % 2 == 0, 1.0, -1.0)


def srht_rows(rows_idx, n: int, m: int, seed: int) -> np.ndarray:
    """Rows of S = √(n_p/m)·P·(H_{n_p}/√n_p)·D restricted to the n real
    columns (the padded columns multiply zero rows of A)."""
    n_p, D, rows = srht_params(n, m, seed)
    rows_idx = np.atleast_1d(np.asarray(rows_idx, dtype=np.int64))
    H = hadamard_entry(rows[rows_idx][:, None], np.arange(n)[None, :])
    return H * D[None, :] / math.sqrt(m)


def srht_matrix(m: int, n: int, seed: int) -> np.ndarray:
    return srht_rows(np.arange(m), n, m, seed)


def sketch_rows(family: int, rows, A: np.ndarray, m: int, seed: int,
                col_chunk: int | None = None) -> np.ndarray:
    """Rows `rows` of SA = S·A, by the definition of S, in fp64."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    rows = np.atleast_1d(np.asarray(rows, dtype=np.int64))
    if family == COUNTSKETCH:
        h, s = countsketch_hash(n, m, seed)
        out = np.zeros((rows.size, A.shape[1]))
        for t, i in enumerate(rows):
            sel = np.nonzero(h == i)[0]
            out[t] = s[sel] @ A[sel]
        return out
    if family == GAUSSIAN:
        S = gaussian_sketch_rows(rows, n, m, seed)
    elif family == SRHT:
        S = srht_rows(rows, n, m, seed)
    else:
        raise ValueError(f"unknown sketch family {family}")
    return S @ A


def sketch_apply(family: int, A: np.ndarray, m: int, seed: int, row_block: int = 64) -> np.ndarray:
    """SA = S·A for the whole sketch (row blocks keep S's memory bounded)."""
    out = np.empty((m, np.shape(A)[1]))
    for r0 in range(0, m, row_block):
        r1 = min(m, r0 + row_block)
        out[r0:r1] = sketch_rows(family, np.arange(r0, r1), A, m, seed)
    return out


# ---------------------------------------------------------------------------
# The ridge solution and its certificates
# ---------------------------------------------------------------------------
def gradient(A, b, x, lam):
    """g = Aᵀ(b − Ax) − λx in fp64 (Algorithm 1, gradient step)."""
    A = np.asarray(A, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    r = np.asarray(b, dtype=np.float64) - A @ x
    return A.T @ r - lam * x


def exact_solve(A, b, lam, refine: int = 2, row_block: int = 1 << 16, extended: bool = False,
                dd: bool = False):
    """x* = (AᵀA + λI)⁻¹Aᵀb: fp64 Gram matrix (row blocks summed in order),
    Cholesky, two triangular solves, then `refine` steps of iterative
    refinement x += H⁻¹(Aᵀ(b−Ax) − λx).  With `extended`, the refinement
    residual is formed in numpy's extended precision (np.longdouble: 64-bit
    significand on x86-64, IEEE quad on aarch64), which makes the result
    accurate to ~κ(H)·u_ext instead of ~κ(H)·u₆₄; with `dd`, in
    double-double by gradient_dd (fp32 A and b), which does the same at
    large sizes where software quad is too slow."""
    n, d = np.shape(A)
    H = np.zeros((d, d))
    Atb = np.zeros(d)
    for r0 in range(0, n, row_block):
        Ab = np.asarray(A[r0:r0 + row_block], dtype=np.float64)
        H += Ab.T @ Ab
        Atb += Ab.T @ np.asarray(b[r0:r0 + row_block], dtype=np.float64)
    H[np.diag_indices(d)] += lam
    L = np.linalg.cholesky(H)

    def hsolve(v):
        y = np.linalg.solve(L, v)          # forward substitution (L lower)
        return np.linalg.solve(L.T, y)     # back substitution

    x = hsolve(Atb)
    for _ in range(refine):
        if dd:
            gh, gl = gradient_dd(A, b, x, lam)
            r = gh + gl
        elif extended:
            r = gradient_extended(A, b, x, lam, row_block)
        else:
            r = gradient_blocked(A, b, x, lam, row_block)
        x = x + hsolve(np.asarray(r, dtype=np.float64))
    return x


def gradient_dd(A, b, x, lam, nthreads: int | None = None):
    """g = Aᵀ(b − Ax) − λx for fp32 A and b and fp64 x, every product and sum
    in double-double (Ogita, Rump & Oishi 2005), by the C helper
    oracle/resid_dd.c.  Returns (hi, lo) fp64 arrays, g = hi + lo."""
    from oracle import _c
    A = np.asarray(A)
    if A.dtype != np.float32:
        raise TypeError("gradient_dd takes the fp32 data itself")
    n, d = A.shape
    if A.strides[1] != 4 or A.strides[0] % 4:
        A = np.ascontiguousarray(A)
    lda = A.strides[0] // 4
    b32 = np.ascontiguousarray(b, dtype=np.float32)
    x64 = np.ascontiguousarray(x, dtype=np.float64)
    gh, gl = np.empty(d), np.empty(d)
    nt = nthreads or max(1, min(os.cpu_count() or 1, 64))
    rc = _c.lib().oracle_gradient_dd(A.ctypes.data, n, d, lda, b32.ctypes.data, x64.ctypes.data, float(lam),
                                     int(nt), gh.ctypes.data, gl.ctypes.data)
    if rc:
        raise MemoryError("oracle_gradient_dd failed")
    return gh, gl


def gradient_extended(A, b, x, lam, row_block: int = 1 << 14):
    """g = Aᵀ(b − Ax) − λx in np.longdouble (row blocks summed in order)."""
    n = np.shape(A)[0]
    xe = np.asarray(x, dtype=np.longdouble)
    g = -np.longdouble(lam) * xe
    for r0 in range(0, n, row_block):
        Ab = np.asarray(A[r0:r0 + row_block], dtype=np.longdouble)
        g += Ab.T @ (np.asarray(b[r0:r0 + row_block], dtype=np.longdouble) - Ab @ xe)
    return g


def gradient_blocked(A, b, x, lam, row_block: int = 1 << 16):
    n = np.shape(A)[0]
    g = -lam * np.asarray(x, dtype=np.float64)
    for r0 in range(0, n, row_block):
        Ab = np.asarray(A[r0:r0 + row_block], dtype=np.float64)
        g += Ab.T @ (np.asarray(b[r0:r0 + row_block], dtype=np.float64) - Ab @ x)
    return g


def svd_solve(A, b, lam):
    """Closed form of Eq. tsvdsol: x* = Σ σᵢ²/(σᵢ²+λ) (uᵢᵀb/σᵢ) vᵢ."""
    U, s, Vt = np.linalg.svd(np.asarray(A, dtype=np.float64), full_matrices=False)
    coef = (s ** 2 / (s ** 2 + lam)) * (U.T @ np.asarray(b, dtype=np.float64)) / s
    return Vt.T @ coef


def stat_dim(sigma, lam):
    """sd_λ(A) = Σ σᵢ²/(σᵢ²+λ)."""
    s2 = np.asarray(sigma, dtype=np.float64) ** 2
    return float(np.sum(s2 / (s2 + lam)))


def stat_dim_of(A, lam):
    return stat_dim(np.linalg.svd(np.asarray(A, dtype=np.float64), compute_uv=False), lam)


def quantize_sa(SA, prec: str):
    """Quantised SA and its decoded fp64 values.  'bf16': round to nearest
    even.  'fp8': per 128 × 128 tile, scale = max|SA|/448 in fp32 (1 for a zero
    tile), q = e4m3(SA/scale) (fp32 division, round to nearest even; the
    largest magnitude maps to 448 exactly or rounds to it).  Returns
    (q as a torch tensor, scales (fp32 array, tile rows × tile cols) or None,
    decoded fp64 array)."""
    import torch
    SA32 = torch.as_tensor(np.asarray(SA, dtype=np.float32))
    m, d = SA32.shape
    if prec == "bf16":
        q = SA32.to(torch.bfloat16)
        return q, None, q.to(torch.float64).numpy()
    if prec != "fp8":
        raise ValueError(prec)
    T = 128
    ntr, ntc = (m + T - 1) // T, (((d + 3) // 4) * 4 + T - 1) // T
    scales = np.ones((ntr, ntc), dtype=np.float32)
    for tr in range(ntr):
        for tc in range(ntc):
            amax = np.float32(np.max(np.abs(SA32[tr * T:(tr + 1) * T, tc * T:(tc + 1) * T].numpy()), initial=0.0))
            scales[tr, tc] = np.float32(amax / np.float32(448.0)) if amax > 0 else np.float32(1.0)
    S = torch.from_numpy(np.repeat(np.repeat(scales, T, axis=0), T, axis=1)[:m, :d].copy())
    q = (SA32 / S).to(torch.float8_e4m3fn)
    dec = q.to(torch.float64).numpy() * S.to(torch.float64).numpy()
    return q, scales, dec


def ridge_path(A, b, lambdas, refine: int = 2):
    """x*(λ_l) = (AᵀA + λ_l I)⁻¹Aᵀb for each λ_l: one fp64 Gram, then per λ a
    Cholesky, two triangular solves and `refine` refinement steps (as in
    exact_solve).  Returns an array of shape (len(lambdas), d)."""
    A64 = np.asarray(A, dtype=np.float64)
    b64 = np.asarray(b, dtype=np.float64)
    G = A64.T @ A64
    Atb = A64.T @ b64
    out = []
    for lam in lambdas:
        H = G + lam * np.eye(G.shape[0])
        L = np.linalg.cholesky(H)
        hsolve = lambda v: np.linalg.solve(L.T, np.linalg.solve(L, v))
        x = hsolve(Atb)
        for _ in range(refine):
            x = x + hsolve(A64.T @ (b64 - A64 @ x) - lam * x)
        out.append(x)
    return np.array(out)


def ridge_backward(A, b, lam, gbar, x=None):
    """Gradients of L = ḡᵀx* with respect to A, b and λ, where
    H x* = Aᵀb, H = AᵀA + λI.  Differentiating the normal equations:
    H dx = dAᵀ(b − Ax*) − AᵀdA x* + Aᵀdb − dλ x*, so with the adjoint
    v = H⁻¹ḡ and r = b − Ax*:
        ∂L/∂A = r vᵀ − (Av) x*ᵀ,  ∂L/∂b = Av,  ∂L/∂λ = −x*ᵀv.
    Returns (x, v, dA, db, dlam) in fp64; x defaults to the exact solution."""
    A64 = np.asarray(A, dtype=np.float64)
    b64 = np.asarray(b, dtype=np.float64)
    H = A64.T @ A64 + lam * np.eye(A64.shape[1])
    if x is None:
        x = np.linalg.solve(H, A64.T @ b64)
    x = np.asarray(x, dtype=np.float64)
    v = np.linalg.solve(H, np.asarray(gbar, dtype=np.float64))
    r = b64 - A64 @ x
    Av = A64 @ v
    dA = np.outer(r, v) - np.outer(Av, x)
    return x, v, dA, Av, float(-(x @ v))


def certify(A, b, x, lam):
    """Upper bound on ‖x − x*‖ from H ⪰ λI: ‖x − x*‖ ≤ ‖g(x)‖/λ."""
    return float(np.linalg.norm(gradient_blocked(A, b, x, lam)) / lam)


def rel_error(x, xstar):
    x = np.asarray(x, dtype=np.float64)
    xstar = np.asarray(xstar, dtype=np.float64)
    return float(np.linalg.norm(x - xstar) / np.linalg.norm(xstar))


# ---------------------------------------------------------------------------
# AAb_Solver (Algorithm 5): approximately solve (SAᵀSA + λI) x = g
# ---------------------------------------------------------------------------
def aab_solve(SA, g, lam, eps, max_iter=None, dtype=np.float64, history=False,
              s_init="sqrt_lam_over_rhobar"):
    """Upper bidiagonalisation of SA started at θ₁v = g, Eldén's Givens fold of
    √λ into the bidiagonal, the analytic φ recursion and the forward
    substitution update of Section 3.6.

    `max_iter` caps the number of loop passes (each pass = one product with
    SAᵀ and one with SA); the cap is also min(m, d) (finite termination).
    Returns (x, passes[, list of t]).  `dtype=np.float32` emulates fp32.
    `s_init` selects the reading of the initial sine (only for the test that
    shows the garbled form breaks the residual identity).
    """
    SA = np.asarray(SA, dtype=dtype)
    g = np.asarray(g, dtype=dtype)
    lam = dtype(lam)
    m, d = SA.shape
    cap = min(m, d) if max_iter is None else min(int(max_iter), min(m, d))
    theta1 = np.sqrt(np.sum(g * g, dtype=dtype))
    ts = []
    if theta1 == 0:
        return (np.zeros(d, dtype), 0, ts) if history else (np.zeros(d, dtype), 0)
    v = g / theta1                                   # θ₁ v = b
    w = SA @ v                                       # ρ p = A v
    rho = np.sqrt(np.sum(w * w, dtype=dtype))
    p = w / rho
    rhobar = np.sqrt(rho * rho + lam)
    c = rho / rhobar
    s = np.sqrt(lam) / rhobar if s_init == "sqrt_lam_over_rhobar" else np.sqrt(lam / rhobar)
    phi = theta1 / rhobar
    dv = v / rhobar
    x = phi * dv
    t = np.inf
    k = 0
    while t >= eps and k < cap:
        z = SA.T @ p - rho * v                       # θ v := Aᵀp − ρ v
        theta = np.sqrt(np.sum(z * z, dtype=dtype))
        if not theta > 0:
            break                                    # invariant subspace reached
        v = z / theta
        w = SA @ v - theta * p                       # ρ p := A v − θ p
        rho = np.sqrt(np.sum(w * w, dtype=dtype))
        lambar = np.sqrt(lam + (s * theta) ** 2)     # λ̄² = λ + (sθ)²
        thetabar = c * theta                         # θ̄ = cθ
        rhobar = np.sqrt(rho * rho + lambar * lambar)
        c = rho / rhobar
        s = lambar / rhobar
        dv = (v - thetabar * dv) / rhobar
        phi = -phi * thetabar / rhobar
        x = x + phi * dv
        t = abs(phi * rhobar) / theta1
        ts.append(float(t))
        k += 1
        if not rho > 0:
            break
        p = w / rho
    return (x, k, ts) if history else (x, k)


# ---------------------------------------------------------------------------
# Momentum parameters and convergence theory
# ---------------------------------------------------------------------------
def momentum_params(sd, m):
    """Corollary 3: β = sd/m, α = (1 − β)²."""
    beta = float(sd) / float(m)
    return (1.0 - beta) ** 2, beta


def theorem1_params(eps):
    """Theorem 1: β* = (ε/(1+√(1−ε²)))², α* = (1−β*)√(1−ε²), rate √β*."""
    rate = eps / (1.0 + math.sqrt(1.0 - eps * eps))
    beta = rate * rate
    alpha = (1.0 - beta) * math.sqrt(1.0 - eps * eps)
    return alpha, beta, rate


def theorem1_alpha_alt(eps):
    """Second form of α* in the proof of Theorem 1: 4(1−ε²)/(√(1+ε)+√(1−ε))²."""
    return 4.0 * (1.0 - eps * eps) / (math.sqrt(1.0 + eps) + math.sqrt(1.0 - eps)) ** 2


def corollary3_iters(eta, beta):
    """Corollary 3: at most log(η)/log(√β) iterations for an η-optimal x."""
    return math.log(eta) / math.log(math.sqrt(beta))


def corollary2_iters(eta, C, eps):
    """Corollary 2 under the reading ⌈log(η/C)/log(ε/(1+√(1−ε²)))⌉."""
    return int(math.ceil(math.log(eta / C) / math.log(eps / (1.0 + math.sqrt(1.0 - eps * eps)))))


def predicted_error(C, beta, N):
    """Corollary 3 applied to a start error of C (in units of the target
    norm): C·(√β)^N, the form used in the captions of Section 4."""
    return C * math.sqrt(beta) ** N


def characteristic_roots(mu, alpha, beta):
    """Roots of u² − (1 + β − αμ)u + β = 0 (proof of Theorem 1)."""
    mu = np.atleast_1d(np.asarray(mu, dtype=np.float64))
    tr = 1.0 + beta - alpha * mu
    disc = np.sqrt((tr * tr - 4.0 * beta).astype(np.complex128))
    return (tr + disc) / 2.0, (tr - disc) / 2.0


def characteristic_rate(mu, alpha, beta):
    """Spectral radius of the heavy-ball transition: max root modulus."""
    r1, r2 = characteristic_roots(mu, alpha, beta)
    return float(np.max(np.maximum(np.abs(r1), np.abs(r2))))


def underdamped(mu, alpha, beta):
    """Condition β ≥ (1 − √(αμ))² of the proof of Theorem 1."""
    mu = np.asarray(mu, dtype=np.float64)
    return beta >= (1.0 - np.sqrt(alpha * mu)) ** 2


def sketched_hessian_eigs(A, SA, lam):
    """μᵢ = eig((SAᵀSA + λI)⁻¹(AᵀA + λI)), the eigenvalues in the proof of
    Theorem 1 (similar to (ÂᵀŜᵀŜÂ)⁻¹)."""
    A = np.asarray(A, dtype=np.float64)
    SA = np.asarray(SA, dtype=np.float64)
    d = A.shape[1]
    H = A.T @ A + lam * np.eye(d)
    HS = SA.T @ SA + lam * np.eye(d)
    Lc = np.linalg.cholesky(HS)
    Li = np.linalg.inv(Lc)
    return np.sort(np.linalg.eigvalsh(Li @ H @ Li.T))


def mp_edges(sd, m):
    """Limits (1 ± √(sd/m))⁻² of the extreme μ (proof of Corollary 3)."""
    r = math.sqrt(sd / m)
    return (1.0 + r) ** -2, (1.0 - r) ** -2


# ---------------------------------------------------------------------------
# Algorithm 1: M-IHS for n ≥ d
# ---------------------------------------------------------------------------
def heavy_ball(x, x_prev, delta, alpha, beta):
    """x⁺ = x + αΔ + β(x − x⁻) (Eq. mihs1); returns (x⁺, new x⁻ = x)."""
    return x + alpha * delta + beta * (x - x_prev), x


def mihs(A, b, lam, SA, sd, N, x1=None, eps_sub=0.1, tol=None, inner="aab",
         max_inner=None, dtype=np.float64, record=False):
    """Algorithm 1 with the given SA.

    Each of at most N iterations: g = Aᵀ(b − Ax) − λx; stop if tol is set and
    ‖g‖ ≤ tol·‖Aᵀb‖; Δ from AAb_Solver(SA, g, λ, ε_sub) (or, with
    inner="exact", from a Cholesky solve of SAᵀSA + λI — the exact scheme);
    x ← x + αΔ + β(x − x⁻).  x⁰ = x¹.
    Returns (x, info) with info = {outer, inner_total, resid, history}.
    """
    A = np.asarray(A, dtype=dtype)
    b = np.asarray(b, dtype=dtype)
    SA = np.asarray(SA, dtype=dtype)
    m, d = SA.shape
    alpha, beta = momentum_params(sd, m)
    alpha, beta = dtype(alpha), dtype(beta)
    x = np.zeros(d, dtype) if x1 is None else np.asarray(x1, dtype=dtype).copy()
    x_prev = x.copy()
    gnorm0 = float(np.linalg.norm(A.T.astype(np.float64) @ b.astype(np.float64)))
    if inner == "exact":
        HS = SA.astype(np.float64).T @ SA.astype(np.float64) + lam * np.eye(d)
        Lc = np.linalg.cholesky(HS)
    hist = []
    inner_total = 0
    outer = 0
    resid = float("nan")
    for i in range(N):
        g = A.T @ (b - A @ x) - dtype(lam) * x
        resid = float(np.linalg.norm(g.astype(np.float64))) / gnorm0 if gnorm0 > 0 else 0.0
        if record:
            hist.append((x.astype(np.float64).copy(), resid))
        if tol is not None and resid <= tol:
            break
        if inner == "exact":
            delta = np.linalg.solve(Lc.T, np.linalg.solve(Lc, g.astype(np.float64))).astype(dtype)
            k = 0
        else:
            delta, k = aab_solve(SA, g, lam, eps_sub, max_iter=max_inner, dtype=dtype)
        inner_total += k
        x, x_prev = heavy_ball(x, x_prev, delta, alpha, beta)
        outer += 1
    info = dict(outer=outer, inner_total=inner_total, resid=resid, history=hist,
                alpha=float(alpha), beta=float(beta))
    return x.astype(np.float64), info


def exact_solve_dual(A, b, lam):
    """x* = Aᵀν*, ν* = (AAᵀ + λI)⁻¹b (Eq. dual_relation): an n × n Cholesky,
    the natural form when n ≤ d."""
    A64 = np.asarray(A, dtype=np.float64)
    K = A64 @ A64.T + lam * np.eye(A64.shape[0])
    L = np.linalg.cholesky(K)
    nu = np.linalg.solve(L.T, np.linalg.solve(L, np.asarray(b, dtype=np.float64)))
    return A64.T @ nu, nu


def dual_mihs(A, b, lam, SAt, sd, N, eps_sub=0.1, tol=None, max_inner=None, dtype=np.float64):
    """Algorithm 2 with the given sketch SAt = S·Aᵀ (m × n, S sketching the
    d coordinates).  Each of at most N iterations: g = b − AAᵀν − λν (the
    negative gradient of the dual objective of Eq. intro_dual); stop if tol
    is set and ‖g‖ ≤ tol·‖b‖ (= ‖g(0)‖); Δν = AAb_Solver(SAt, g, λ, ε_sub);
    ν ← ν + αΔν + β(ν − ν⁻) with β = sd/m, α = (1 − β)², ν¹ = ν⁰ = 0.  Then
    x = Aᵀν.  Returns (x, ν, info)."""
    A = np.asarray(A, dtype=dtype)
    b = np.asarray(b, dtype=dtype)
    SAt = np.asarray(SAt, dtype=dtype)
    m, n = SAt.shape
    alpha, beta = momentum_params(sd, m)
    alpha, beta = dtype(alpha), dtype(beta)
    nu = np.zeros(n, dtype)
    nu_prev = nu.copy()
    gnorm0 = float(np.linalg.norm(b.astype(np.float64)))
    inner_total, outer, resid = 0, 0, float("nan")
    for _ in range(N):
        g = b - A @ (A.T @ nu) - dtype(lam) * nu
        resid = float(np.linalg.norm(g.astype(np.float64))) / gnorm0 if gnorm0 > 0 else 0.0
        if tol is not None and resid <= tol:
            break
        delta, k = aab_solve(SAt, g, lam, eps_sub, max_iter=max_inner, dtype=dtype)
        inner_total += k
        nu, nu_prev = heavy_ball(nu, nu_prev, delta, alpha, beta)
        outer += 1
    x = A.T.astype(np.float64) @ nu.astype(np.float64)
    return x, nu.astype(np.float64), dict(outer=outer, inner_total=inner_total, resid=resid)


def mihs_solve(A, b, lam, family, m, sd, seed, N=200, tol=1e-6, eps_sub=0.1,
               max_inner=None, dtype=np.float64):
    """Sketch (RP_fun) then Algorithm 1: the whole path on the CPU."""
    SA = sketch_apply(family, A, m, seed)
    return mihs(A, b, lam, SA, sd, N, eps_sub=eps_sub, tol=tol,
                max_inner=max_inner, dtype=dtype)


# ---------------------------------------------------------------------------
# Algorithm 4: inexact Hutchinson trace estimator of the statistical dimension
# ---------------------------------------------------------------------------
def rademacher_probe(d: int, ell: int, seed: int) -> np.ndarray:
    """Probe v^ℓ ∈ {−1, +1}^d: entry j from Philox counter (j, ℓ,
    TAG_HUTCHINSON, 0), +1 when w0 is even."""
    k0, k1 = seed_key(seed)
    w0, _, _, _ = philox4x32_10(np.arange(d, dtype=np.uint64), np.uint64(ell), TAG_HUTCHINSON, 0, k0, k1)
    return np.where((w0 & np.uint64(1)) == 0, 1.0, -1.0)


def hutchinson_sd(SA, lam, T, eps_tr, seed, max_iter=None, dtype=np.float64):
    """sd ≈ d − (λ/T)·Σ_ℓ ⟨v^ℓ, z^ℓ⟩ with z^ℓ = AAb_Solver(SA, v^ℓ, λ, ε_tr):
    tr(A(AᵀA+λI)⁻¹Aᵀ) = d − λ·tr((AᵀA+λI)⁻¹) with SA standing in for A."""
    SA = np.asarray(SA, dtype=np.float64)
    d = SA.shape[1]
    tau = 0.0
    for ell in range(T):
        v = rademacher_probe(d, ell, seed)
        z, _ = aab_solve(SA, v, lam, eps_tr, max_iter=max_iter, dtype=dtype)
        tau += lam * float(np.dot(v, np.asarray(z, dtype=np.float64)))
    return d - tau / T
