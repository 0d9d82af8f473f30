"""Error bounds used by the parity tests, derived from the kernels' fp32
arithmetic (unit roundoff u = 2⁻²⁴; γ_k = k·u/(1 − k·u), Higham, Accuracy and
Stability of Numerical Algorithms, §3.1: a sum of k products computed in any
order errs by at most γ_k times the sum of the products' magnitudes)."""
import math

import numpy as np

U32 = 2.0 ** -24


def gamma(k: float) -> float:
    ku = k * U32
    return ku / (1.0 - ku)


def gradient_bound(A, b, x, lam, depth_r: int, depth_acc: int):
    """Componentwise bound on |ĝ − g| for g = Aᵀ(b − Ax) − λx when the row
    residual is a sum of `depth_r` terms and each column sum has `depth_acc`
    rounding levels."""
    A = np.abs(np.asarray(A, np.float64))
    rb = np.abs(np.asarray(b, np.float64)) + A @ np.abs(np.asarray(x, np.float64))
    return gamma(depth_r + depth_acc + 2) * (A.T @ rb) + 2 * U32 * lam * np.abs(np.asarray(x, np.float64))


def apass_depths(n: int, d: int, num_sms: int = 152):
    """Rounding depths of the A-pass: per lane ≤ 4·⌈d/128⌉ products + 5 shuffle
    levels for a row residual; per column ≤ rows/warp sequential adds, then the
    ≤ 16 warp partials, the ≤ P/8 + 8 partial sums."""
    ch = max(1, math.ceil(d / 128))
    depth_r = 4 * ch + 5 + 1
    rows_per_cta = math.ceil(n / min(num_sms, n))
    depth_acc = math.ceil(rows_per_cta / 8) + 16 + math.ceil(num_sms / 8) + 8 + 1
    return depth_r, depth_acc


def gradient_bound_refined(A, b, x, lam, depth_r: int, depth_acc: int):
    """Componentwise bound on |ĝ − g| for the compensated (double-float)
    gradient: each double-float sum of k terms errs by ≲ 2k·u² relative to the
    sum of magnitudes (TwoSum/TwoProduct, Ogita–Rump–Oishi 2005), plus the
    fp64 reductions and λx (≲ 4·u₆₄)."""
    Aa = np.abs(np.asarray(A, np.float64))
    M = Aa.T @ (np.abs(np.asarray(b, np.float64)) + Aa @ np.abs(np.asarray(x, np.float64)))
    u64 = 2.0 ** -53
    return (4 * (depth_r + depth_acc) * U32 * U32 + 16 * u64) * M + 4 * u64 * lam * np.abs(np.asarray(x, np.float64))
