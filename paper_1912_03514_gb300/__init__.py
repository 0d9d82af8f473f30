"""GB300-native M-IHS ridge solver (arXiv 1912.03514): C-ABI library libmihs.so
(CUDA, sm_103a) plus a thin ctypes binding.

    from paper_1912_03514_gb300 import mihs
    x, info = mihs.solve(A, b, lam, "countsketch", m, sd)

The library is loaded lazily on the first call; ``workloads`` (the seeded
problem generator) does not need it.
"""
__all__ = ["mihs", "workloads"]
