"""Python binding of libmihs (ctypes).  Argument marshalling only: every step
of the solver runs in the library's CUDA kernels.  The functions carry the
names of the C entry points in include/mihs.h without the ``mihs_`` prefix.

Tensors must be CUDA fp32 with unit column stride; row pitches are taken from
``stride(0)``.  Work is enqueued on ``torch.cuda.current_stream()`` unless a
stream is given.  There is no CPU fallback: without the built library every
call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

from . import _build

GAUSSIAN, COUNTSKETCH, SRHT = 0, 1, 2
SA_FP32, SA_BF16, SA_FP8 = 0, 1, 2
SA_PRECISIONS = {"fp32": SA_FP32, "bf16": SA_BF16, "fp8": SA_FP8}
AAB_AUTO, AAB_CLUSTER, AAB_GRID = 0, 1, 2
AAB_FORMS = {"auto": AAB_AUTO, "cluster": AAB_CLUSTER, "grid": AAB_GRID}
FAMILIES = {"gaussian": GAUSSIAN, "countsketch": COUNTSKETCH, "srht": SRHT}
OK, NOT_CONVERGED = 0, 1
ERR_INVALID_ARG, ERR_CUDA, ERR_OOM, ERR_TIMEOUT, ERR_NUMERIC, UNSUPPORTED = -1, -2, -3, -4, -5, -6


class MihsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(msg)
        self.code = code


class _Opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_outer", ctypes.c_int),
                ("eps_sub", ctypes.c_double), ("max_inner", ctypes.c_int),
                ("sd", ctypes.c_double), ("warm_start", ctypes.c_int)]


class _Problem(ctypes.Structure):
    _fields_ = [("sk", ctypes.c_void_p), ("A", ctypes.c_void_p), ("lda", ctypes.c_int64),
                ("b", ctypes.c_void_p), ("X", ctypes.c_void_p), ("ldx", ctypes.c_int64)]


class _Info(ctypes.Structure):
    _fields_ = [("outer_iters", ctypes.c_int), ("inner_iters_total", ctypes.c_int),
                ("rel_resid", ctypes.c_double), ("status", ctypes.c_int)]


_lib = None
_i64, _u64, _vp, _dbl, _int = ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_double, ctypes.c_int


def library_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """Load libmihs.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libmihs.so is not built ({path}); run "
                           "`python -m paper_1912_03514_gb300._build` or __graft_entry__.build()")
    L = ctypes.CDLL(path)
    sig = {
        "mihs_strerror": (ctypes.c_char_p, [_int]),
        "mihs_last_error": (ctypes.c_char_p, []),
        "mihs_launch_count": (_u64, []),
        "mihs_device_status": (_int, [ctypes.POINTER(_int)]),
        "mihs_selftest_wait": (_int, [_int, _i64, ctypes.POINTER(_int), _vp]),
        "mihs_copy_to_device": (_int, [_vp, _vp, _i64, _vp]),
        "mihs_copy_to_device_dma": (_int, [_vp, _vp, _i64, _vp]),
        "mihs_sketch_apply": (_int, [_vp, _i64, _i64, _i64, _int, _i64, _u64, _vp, _i64, _vp]),
        "mihs_sketch_gaussian_bf16": (_int, [_vp, _i64, _i64, _i64, _i64, _u64, _vp, _i64, _vp]),
        "mihs_sketch_gaussian_fp8": (_int, [_vp, _i64, _i64, _i64, _i64, _u64, _vp, _i64, _vp]),
        "mihs_gradient": (_int, [_vp, _i64, _i64, _i64, _vp, _vp, _dbl, _vp, _vp]),
        "mihs_gradient_noalloc": (_int, [_vp, _i64, _i64, _i64, _vp, _vp, _dbl, _vp, _vp]),
        "mihs_aab_solve": (_int, [_vp, _i64, _i64, _i64, _vp, _dbl, _dbl, _int, _vp, _vp, _vp]),
        "mihs_aab_heavy_ball": (_int, [_vp, _i64, _i64, _i64, _vp, _dbl, _dbl, _int, _dbl, _dbl,
                                       _vp, _vp, _vp, _vp]),
        "mihs_estimate_sd": (_int, [_vp, _i64, _i64, _i64, _dbl, _int, _dbl, _u64, ctypes.POINTER(_dbl), _vp]),
        "mihs_sketch": (_int, [_vp, _i64, _i64, _i64, _int, _i64, _u64, _vp, ctypes.POINTER(_vp)]),
        "mihs_sketch_info": (_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
        "mihs_resketch": (_int, [_vp, _vp, _i64, _u64, _vp]),
        "mihs_sketch_copy": (_int, [_vp, _vp, _i64, _vp]),
        "mihs_solve_history": (_int, [_vp, ctypes.POINTER(ctypes.c_float), _int, ctypes.POINTER(_int)]),
        "mihs_sketch_destroy": (_int, [_vp]),
        "mihs_default_opts": (_Opts, []),
        "mihs_timing": (_int, [_int]),
        "mihs_timing_read": (_int, [_int, ctypes.POINTER(_dbl), ctypes.POINTER(_i64)]),
        "mihs_solve_refined": (_int, [_vp, _vp, _i64, _vp, _dbl, ctypes.POINTER(_Opts), _vp,
                                      ctypes.POINTER(_Info), _vp]),
        "mihs_gradient_refined": (_int, [_vp, _i64, _i64, _i64, _vp, _vp, _dbl, _vp, _vp]),
        "mihs_solve": (_int, [_vp, _vp, _i64, _vp, _dbl, ctypes.POINTER(_Opts), _vp,
                              ctypes.POINTER(_Info), _vp]),
        "mihs_backward_grads": (_int, [_vp, _i64, _i64, _i64, _vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp]),
        "mihs_sketch_set_precision": (_int, [_vp, _int, _vp]),
        "mihs_sketch_set_aab": (_int, [_vp, _int, _int]),
        "mihs_dual_sketch": (_int, [_vp, _i64, _i64, _i64, _int, _i64, _u64, _vp, ctypes.POINTER(_vp)]),
        "mihs_dual_resketch": (_int, [_vp, _vp, _i64, _u64, _vp]),
        "mihs_dual_copy": (_int, [_vp, _vp, _i64, _vp]),
        "mihs_dual_destroy": (_int, [_vp]),
        "mihs_gradient_dual": (_int, [_vp, _i64, _i64, _i64, _vp, _vp, _dbl, _vp, _vp]),
        "mihs_dual_recover": (_int, [_vp, _i64, _i64, _i64, _vp, _vp, _vp]),
        "mihs_solve_dual": (_int, [_vp, _vp, _i64, _vp, _dbl, ctypes.POINTER(_Opts), _vp, _vp,
                                   ctypes.POINTER(_Info), _vp]),
        "mihs_quantize_sa": (_int, [_vp, _i64, _i64, _i64, _int, _vp, _i64, _vp, _vp]),
        "mihs_aab_solve_q": (_int, [_vp, _int, _vp, _i64, _i64, _i64, _vp, _dbl, _dbl, _int, _vp, _vp, _vp]),
        "mihs_gradient_path": (_int, [_vp, _i64, _i64, _i64, _vp, _int, _vp, _vp, _i64, _vp, _i64, _vp]),
        "mihs_solve_path": (_int, [_vp, _vp, _i64, _vp, _int, _vp, _vp, ctypes.POINTER(_Opts), _vp, _i64, _vp,
                                   _vp]),
        "mihs_solve_batched": (_int, [_int, _vp, _int, _vp, _vp, ctypes.POINTER(_Opts), _vp, _vp]),
        "mihs_refine_batched": (_int, [_int, _vp, _int, _vp, _vp, _vp, ctypes.POINTER(_Opts), _vp, _vp]),
        "mihs_backward_refined": (_int, [_vp, _vp, _i64, _vp, _dbl, _vp, _vp, ctypes.POINTER(_Opts), _vp, _vp,
                                         _i64, _vp, _vp, ctypes.POINTER(_Info), _vp]),
        "mihs_backward": (_int, [_vp, _vp, _i64, _vp, _dbl, _vp, _vp, ctypes.POINTER(_Opts), _vp, _vp, _i64,
                                 _vp, _vp, ctypes.POINTER(_Info), _vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(rc: int, allow_not_converged: bool = False) -> int:
    if rc == 0 or (allow_not_converged and rc == NOT_CONVERGED):
        return rc
    L = lib()
    raise MihsError(rc, f"{L.mihs_strerror(rc).decode()}: {L.mihs_last_error().decode()}")


def _stream(stream) -> int:
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


def _mat(A: torch.Tensor, name: str):
    if not (A.is_cuda and A.dtype == torch.float32 and A.dim() == 2 and A.stride(1) == 1):
        raise ValueError(f"{name} must be a CUDA fp32 matrix with unit column stride")
    return A.data_ptr(), A.shape[0], A.shape[1], A.stride(0)


def _vec(v: torch.Tensor, n: int, name: str):
    if not (v.is_cuda and v.dtype == torch.float32 and v.dim() == 1 and v.numel() == n
            and v.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA fp32 vector of length {n}")
    return v.data_ptr()


def family_id(family) -> int:
    return FAMILIES[family] if isinstance(family, str) else int(family)


def device_status() -> int:
    """Reads and clears the library's device-side failure code (0 if none)."""
    c = _int()
    _check(lib().mihs_device_status(ctypes.byref(c)))
    return c.value


def selftest_wait(which: int, limit_s: float = 0.05, stream=None) -> int:
    """Runs one of the library's bounded waits on a condition nothing
    satisfies (0: mbarrier, 1: grid barrier) with a limit of limit_s seconds;
    returns the status its kernel reported (TIMEOUT expected)
    (mihs_selftest_wait)."""
    st = _int()
    _check(lib().mihs_selftest_wait(int(which), int(limit_s * 1e9), ctypes.byref(st), _stream(stream)))
    return st.value


def copy_to_device(dst: torch.Tensor, src: torch.Tensor, stream=None, engine: str = "sm") -> torch.Tensor:
    """dst ← src for a contiguous host tensor src and a contiguous CUDA
    tensor dst of the same dtype and size.  engine "sm": the SMs read pinned
    host memory directly (mihs_copy_to_device, the faster copy alone); "dma":
    a copy engine, no SM work (mihs_copy_to_device_dma, for copies that
    overlap solves on other streams)."""
    if src.is_cuda or not dst.is_cuda or src.dtype != dst.dtype or src.numel() != dst.numel():
        raise ValueError("copy_to_device: host src and CUDA dst of one dtype and size")
    if not (src.is_contiguous() and dst.is_contiguous()):
        raise ValueError("copy_to_device: contiguous tensors only")
    if engine not in ("sm", "dma"):
        raise ValueError(f"copy_to_device: engine {engine!r} is not 'sm' or 'dma'")
    fn = lib().mihs_copy_to_device if engine == "sm" else lib().mihs_copy_to_device_dma
    _check(fn(dst.data_ptr(), src.data_ptr(), src.numel() * src.element_size(), _stream(stream)))
    return dst


def launch_count() -> int:
    return int(lib().mihs_launch_count())


TIMER_APASS, TIMER_AAB, TIMER_SKETCH, TIMER_APASS_DD, TIMER_BACKWARD, TIMER_APASS_PATH, TIMER_APASS_CORR = \
    0, 1, 2, 3, 4, 5, 6


def timing(on: bool) -> None:
    """Start (clearing old records) or stop per-kernel event timing."""
    _check(lib().mihs_timing(int(bool(on))))


def timing_read(which: int):
    """(total milliseconds, launches) recorded for one timer."""
    ms, cnt = _dbl(), _i64()
    _check(lib().mihs_timing_read(int(which), ctypes.byref(ms), ctypes.byref(cnt)))
    return ms.value, cnt.value


def sketch_apply(A: torch.Tensor, family, m: int, seed: int, SA: torch.Tensor | None = None,
                 stream=None) -> torch.Tensor:
    """SA = S·A (the sketch step of Algorithm 1) into a new or given m×d tensor."""
    pa, n, d, lda = _mat(A, "A")
    if SA is None:
        SA = torch.empty(m, d, dtype=torch.float32, device=A.device)
    ps, mm, dd, ldsa = _mat(SA, "SA")
    if (mm, dd) != (m, d):
        raise ValueError("SA has the wrong shape")
    _check(lib().mihs_sketch_apply(pa, n, d, lda, family_id(family), m, seed & (2**64 - 1),
                                   ps, ldsa, _stream(stream)))
    return SA


def sketch_gaussian_bf16(A: torch.Tensor, m: int, seed: int, SA: torch.Tensor | None = None,
                         stream=None) -> torch.Tensor:
    """The Gaussian SA = S·A formed from bf16-rounded S and A (fp32 accumulation)."""
    pa, n, d, lda = _mat(A, "A")
    if SA is None:
        SA = torch.empty(m, d, dtype=torch.float32, device=A.device)
    ps, mm, dd, ldsa = _mat(SA, "SA")
    if (mm, dd) != (m, d):
        raise ValueError("SA has the wrong shape")
    _check(lib().mihs_sketch_gaussian_bf16(pa, n, d, lda, m, seed & (2**64 - 1), ps, ldsa, _stream(stream)))
    return SA


def sketch_gaussian_fp8(A: torch.Tensor, m: int, seed: int, SA: torch.Tensor | None = None,
                        stream=None) -> torch.Tensor:
    """The Gaussian SA = S·A formed from e4m3-rounded S and A·2^k, 2^k the
    power of two putting max|A| in [128, 256) (fp32 accumulation, the scale
    undone)."""
    pa, n, d, lda = _mat(A, "A")
    if SA is None:
        SA = torch.empty(m, d, dtype=torch.float32, device=A.device)
    ps, mm, dd, ldsa = _mat(SA, "SA")
    if (mm, dd) != (m, d):
        raise ValueError("SA has the wrong shape")
    _check(lib().mihs_sketch_gaussian_fp8(pa, n, d, lda, m, seed & (2**64 - 1), ps, ldsa, _stream(stream)))
    return SA


def gradient(A: torch.Tensor, b: torch.Tensor, x: torch.Tensor, lam: float,
             g: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """g = Aᵀ(b − Ax) − λx."""
    pa, n, d, lda = _mat(A, "A")
    if g is None:
        g = torch.empty(d, dtype=torch.float32, device=A.device)
    _check(lib().mihs_gradient(pa, n, d, lda, _vec(b, n, "b"), _vec(x, d, "x"), float(lam),
                               _vec(g, d, "g"), _stream(stream)))
    return g


def gradient_refined(A: torch.Tensor, b: torch.Tensor, x: torch.Tensor, lam: float,
                     g: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Compensated g = Aᵀ(b − Ax) − λx with fp64 x and g (A, b fp32)."""
    pa, n, d, lda = _mat(A, "A")
    if not (x.is_cuda and x.dtype == torch.float64 and x.numel() == d and x.is_contiguous()):
        raise ValueError("x must be a contiguous CUDA fp64 vector of length d")
    if g is None:
        g = torch.empty(d, dtype=torch.float64, device=A.device)
    _check(lib().mihs_gradient_refined(pa, n, d, lda, _vec(b, n, "b"), x.data_ptr(), float(lam),
                                       g.data_ptr(), _stream(stream)))
    return g


def gradient_noalloc(A: torch.Tensor, b: torch.Tensor, x: torch.Tensor, lam: float,
                     g: torch.Tensor, stream=None) -> torch.Tensor:
    """g = Aᵀ(b − Ax) − λx through the entry point that allocates nothing (its
    scratch is a fixed array in the library; `g` must be given).  Calls that
    overlap on the GPU race on that array."""
    pa, n, d, lda = _mat(A, "A")
    _check(lib().mihs_gradient_noalloc(pa, n, d, lda, _vec(b, n, "b"), _vec(x, d, "x"), float(lam),
                                       _vec(g, d, "g"), _stream(stream)))
    return g


def aab_solve(SA: torch.Tensor, g: torch.Tensor, lam: float, eps_sub: float = 0.1,
              max_inner: int = 0, delta: torch.Tensor | None = None,
              passes: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Δ ≈ (SAᵀSA + λI)⁻¹ g by AAb_Solver (Algorithm 5)."""
    ps, m, d, ldsa = _mat(SA, "SA")
    if delta is None:
        delta = torch.empty(d, dtype=torch.float32, device=SA.device)
    pp = 0
    if passes is not None:
        assert passes.is_cuda and passes.dtype == torch.int32 and passes.numel() >= 1
        pp = passes.data_ptr()
    _check(lib().mihs_aab_solve(ps, m, d, ldsa, _vec(g, d, "g"), float(lam), float(eps_sub),
                                int(max_inner), _vec(delta, d, "delta"), pp or None,
                                _stream(stream)))
    return delta


def estimate_sd(SA: torch.Tensor, lam: float, T: int = 2, eps_tr: float = 0.5, seed: int = 0,
                stream=None) -> float:
    """Statistical dimension from SA by Algorithm 4 (Hutchinson)."""
    ps, m, d, ldsa = _mat(SA, "SA")
    out = _dbl()
    _check(lib().mihs_estimate_sd(ps, m, d, ldsa, float(lam), int(T), float(eps_tr), seed & (2**64 - 1),
                                  ctypes.byref(out), _stream(stream)))
    return out.value


def aab_heavy_ball(SA: torch.Tensor, g: torch.Tensor, lam: float, eps_sub: float, max_inner: int,
                   alpha: float, beta: float, x: torch.Tensor, x_prev: torch.Tensor,
                   passes: torch.Tensor | None = None, stream=None) -> None:
    """AAb_Solver then x⁺ = x + αΔ + β(x − x⁻), x⁻ ← x (in place)."""
    ps, m, d, ldsa = _mat(SA, "SA")
    pp = passes.data_ptr() if passes is not None else None
    _check(lib().mihs_aab_heavy_ball(ps, m, d, ldsa, _vec(g, d, "g"), float(lam), float(eps_sub),
                                     int(max_inner), float(alpha), float(beta),
                                     _vec(x, d, "x"), _vec(x_prev, d, "x_prev"), pp,
                                     _stream(stream)))


def _grad_outputs(n, d, dev, want_dA, want_db, want_dlambda):
    dA = torch.empty(n, d, dtype=torch.float32, device=dev) if want_dA else None
    db = torch.empty(n, dtype=torch.float32, device=dev) if want_db else None
    dl = torch.empty((), dtype=torch.float64, device=dev) if want_dlambda else None
    return dA, db, dl


def backward_grads(A: torch.Tensor, b: torch.Tensor | None, x: torch.Tensor, v: torch.Tensor,
                   want_dA: bool = True, want_db: bool = True, want_dlambda: bool = True, stream=None):
    """∂L/∂A = r vᵀ − (Av)xᵀ, ∂L/∂b = Av, ∂L/∂λ = −xᵀv for a given adjoint v
    (mihs_backward_grads).  Returns (dA, db, dlambda), None where not wanted."""
    pa, n, d, lda = _mat(A, "A")
    dA, db, dl = _grad_outputs(n, d, A.device, want_dA, want_db, want_dlambda)
    _check(lib().mihs_backward_grads(pa, n, d, lda, _vec(b, n, "b") if b is not None else None,
                                     _vec(x, d, "x"), _vec(v, d, "v"),
                                     dA.data_ptr() if dA is not None else None, d,
                                     db.data_ptr() if db is not None else None,
                                     dl.data_ptr() if dl is not None else None, _stream(stream)))
    return dA, db, dl


def _prec(p) -> int:
    if isinstance(p, str):
        if p not in SA_PRECISIONS:
            raise ValueError(f"unknown SA precision {p!r} (fp32, bf16, fp8)")
        return SA_PRECISIONS[p]
    return int(p)


def quantize_sa(SA: torch.Tensor, prec, stream=None):
    """mihs_quantize_sa: returns (q, scales) with q an m × ldq tensor
    (bfloat16, or uint8 holding fp8 e4m3 bytes), ldq = d rounded up to 16,
    and scales the fp8 tile scales (⌈m/128⌉ × ⌈d₄/128⌉) or None."""
    ps, m, d, ldsa = _mat(SA, "SA")
    pr = _prec(prec)
    ldq = (d + 15) // 16 * 16
    if pr == SA_BF16:
        q = torch.empty(m, ldq, dtype=torch.bfloat16, device=SA.device)
        sc = None
    else:
        q = torch.empty(m, ldq, dtype=torch.uint8, device=SA.device)
        sc = torch.empty((m + 127) // 128, ((d + 3) // 4 * 4 + 127) // 128, dtype=torch.float32, device=SA.device)
    _check(lib().mihs_quantize_sa(ps, m, d, ldsa, pr, q.data_ptr(), ldq, sc.data_ptr() if sc is not None else None,
                                  _stream(stream)))
    return q, sc


def aab_solve_q(q: torch.Tensor, prec, scales, d: int, g: torch.Tensor, lam: float, eps_sub: float = 0.1,
                max_inner: int = 0, delta: torch.Tensor | None = None, passes: torch.Tensor | None = None,
                stream=None) -> torch.Tensor:
    """mihs_aab_solve_q on the output of quantize_sa."""
    m, ldq = q.shape
    if delta is None:
        delta = torch.empty(d, dtype=torch.float32, device=q.device)
    _check(lib().mihs_aab_solve_q(q.data_ptr(), _prec(prec), scales.data_ptr() if scales is not None else None,
                                  m, d, ldq, _vec(g, d, "g"), float(lam), float(eps_sub), int(max_inner),
                                  _vec(delta, d, "delta"), passes.data_ptr() if passes is not None else None,
                                  _stream(stream)))
    return delta


def _dbl_array(vals):
    vals = [float(v) for v in vals]
    return (ctypes.c_double * len(vals))(*vals), len(vals)


def gradient_path(A: torch.Tensor, b: torch.Tensor, X: torch.Tensor, lambdas, G: torch.Tensor | None = None,
                  stream=None) -> torch.Tensor:
    """G_l = Aᵀ(b − A·X_l) − λ_l·X_l for the rows X_l of the λ-major X (nl × d),
    in one pass over A (mihs_gradient_path)."""
    pa, n, d, lda = _mat(A, "A")
    if not (X.is_cuda and X.dtype == torch.float32 and X.dim() == 2 and X.shape[1] == d and X.stride(1) == 1):
        raise ValueError("X must be a CUDA fp32 nl x d matrix with unit column stride")
    lam, nl = _dbl_array(lambdas)
    if nl != X.shape[0]:
        raise ValueError("one λ per row of X")
    if G is None:
        G = torch.empty(nl, d, dtype=torch.float32, device=A.device)
    _check(lib().mihs_gradient_path(pa, n, d, lda, _vec(b, n, "b"), nl, lam, X.data_ptr(), X.stride(0),
                                    G.data_ptr(), G.stride(0), _stream(stream)))
    return G


def _infos(arr, k):
    return [SolveInfo(arr[i].outer_iters, arr[i].inner_iters_total, arr[i].rel_resid, arr[i].status)
            for i in range(k)]


def _path_opts(tol, max_outer, eps_sub, max_inner, warm_start):
    o = lib().mihs_default_opts()
    o.tol, o.max_outer, o.eps_sub = float(tol), int(max_outer), float(eps_sub)
    o.max_inner, o.warm_start = int(max_inner), int(bool(warm_start))
    return o


def solve_batched(problems, lambdas, sds=None, tol: float = 1e-6, max_outer: int = 100, eps_sub: float = 0.1,
                  max_inner: int = 0, warm_start: bool = False, want_info: bool = True, stream=None):
    """mihs_solve_batched: `problems` is a list of (Sketch, A, b, X) with X a
    λ-major nl × d CUDA tensor per problem; sds (optional) is nprob × nl.
    Returns a list (per problem) of lists (per λ) of SolveInfo, or None."""
    lam, nl = _dbl_array(lambdas)
    arr = (_Problem * len(problems))()
    for i, (sk, A, b, X) in enumerate(problems):
        pa, n, d, lda = _mat(A, "A")
        if (n, d) != (sk.n, sk.d) or tuple(X.shape) != (nl, d) or X.stride(1) != 1:
            raise ValueError(f"problem {i}: shapes do not match")
        arr[i] = _Problem(sk._h.value, pa, lda, _vec(b, n, "b"), X.data_ptr(), X.stride(0))
    sd_arr = None
    if sds is not None:
        flat = [float(v) for row in sds for v in row]
        sd_arr = (ctypes.c_double * len(flat))(*flat)
    o = _path_opts(tol, max_outer, eps_sub, max_inner, warm_start)
    infos = (_Info * (len(problems) * nl))() if want_info else None
    rc = lib().mihs_solve_batched(len(problems), arr, nl, lam, sd_arr, ctypes.byref(o), infos, _stream(stream))
    _check(rc, allow_not_converged=True)
    if not want_info:
        return None
    flat = _infos(infos, len(problems) * nl)
    return [flat[i * nl:(i + 1) * nl] for i in range(len(problems))]


def refine_batched(problems, lambdas, tols, sds=None, max_outer: int = 200, eps_sub: float = 0.1,
                   max_inner: int = 0, want_info: bool = True, stream=None):
    """mihs_refine_batched: compensated refinement of the λ with tols[l] > 0
    of every problem's X (warm-started from X, result written back in fp32).
    `problems` as for solve_batched.  Returns per problem a list over λ of
    SolveInfo (None for λ not refined), or None."""
    lam, nl = _dbl_array(lambdas)
    tl, nt = _dbl_array(tols)
    if nt != nl:
        raise ValueError("tols must have one entry per λ")
    arr = (_Problem * len(problems))()
    for i, (sk, A, b, X) in enumerate(problems):
        pa, n, d, lda = _mat(A, "A")
        if (n, d) != (sk.n, sk.d) or tuple(X.shape) != (nl, d) or X.stride(1) != 1 or X.dtype != torch.float32:
            raise ValueError(f"problem {i}: shapes do not match")
        arr[i] = _Problem(sk._h.value, pa, lda, _vec(b, n, "b"), X.data_ptr(), X.stride(0))
    sd_arr = None
    if sds is not None:
        flat = [float(v) for row in sds for v in row]
        sd_arr = (ctypes.c_double * len(flat))(*flat)
    o = _path_opts(0.0, max_outer, eps_sub, max_inner, True)
    infos = (_Info * (len(problems) * nl))() if want_info else None
    rc = lib().mihs_refine_batched(len(problems), arr, nl, lam, sd_arr, tl, ctypes.byref(o), infos,
                                   _stream(stream))
    _check(rc, allow_not_converged=True)
    if not want_info:
        return None
    flat = _infos(infos, len(problems) * nl)
    return [[flat[i * nl + l] if tols[l] > 0 else None for l in range(nl)] for i in range(len(problems))]


@dataclass
class SolveInfo:
    outer_iters: int
    inner_iters_total: int
    rel_resid: float
    status: int

    @property
    def converged(self) -> bool:
        return self.status == OK


class Sketch:
    """A handle holding SA = S·A (mihs_sketch) for repeated solves."""

    def __init__(self, A: torch.Tensor, family, m: int, seed: int, stream=None):
        pa, n, d, lda = _mat(A, "A")
        h = ctypes.c_void_p()
        _check(lib().mihs_sketch(pa, n, d, lda, family_id(family), int(m), seed & (2**64 - 1),
                                 _stream(stream), ctypes.byref(h)))
        self._h = h
        self.n, self.d, self.m = n, d, int(m)
        self.family = family_id(family)
        self.device = A.device

    def resketch(self, A: torch.Tensor, seed: int, stream=None) -> None:
        """Recompute SA for a new A of the same shape (reuses the handle's memory)."""
        pa, n, d, lda = _mat(A, "A")
        if (n, d) != (self.n, self.d):
            raise ValueError("A does not match the sketch")
        _check(lib().mihs_resketch(self._h, pa, lda, seed & (2**64 - 1), _stream(stream)))

    def set_precision(self, prec, stream=None) -> None:
        """Storage of SA inside AAb_Solver: 'fp32', 'bf16' or 'fp8' (mihs_sketch_set_precision)."""
        _check(lib().mihs_sketch_set_precision(self._h, _prec(prec), _stream(stream)))

    def set_aab(self, form="auto", grid_blocks=0) -> None:
        """Form of AAb_Solver in this handle's solves: 'auto', 'cluster' or 'grid'
        with `grid_blocks` blocks (0: one per SM) (mihs_sketch_set_aab)."""
        if isinstance(form, str):
            if form not in AAB_FORMS:
                raise ValueError(f"unknown AAb_Solver form {form!r}: one of {sorted(AAB_FORMS)}")
            form = AAB_FORMS[form]
        _check(lib().mihs_sketch_set_aab(self._h, int(form), int(grid_blocks)))

    def sa(self, stream=None) -> torch.Tensor:
        out = torch.empty(self.m, self.d, dtype=torch.float32, device=self.device)
        _check(lib().mihs_sketch_copy(self._h, out.data_ptr(), self.d, _stream(stream)))
        return out

    def solve(self, A: torch.Tensor, b: torch.Tensor, lam: float, sd: float, tol: float = 1e-6,
              max_outer: int = 100, eps_sub: float = 0.1, max_inner: int = 0,
              x: torch.Tensor | None = None, warm_start: bool = False, want_info: bool = True,
              stream=None):
        """Algorithm 1 with this sketch.  Returns (x, SolveInfo or None)."""
        pa, n, d, lda = _mat(A, "A")
        if (n, d) != (self.n, self.d):
            raise ValueError("A does not match the sketch")
        if x is None:
            x = torch.empty(d, dtype=torch.float32, device=A.device)
        o = lib().mihs_default_opts()
        o.tol, o.max_outer, o.eps_sub = float(tol), int(max_outer), float(eps_sub)
        o.max_inner, o.sd, o.warm_start = int(max_inner), float(sd), int(bool(warm_start))
        info = _Info()
        rc = lib().mihs_solve(self._h, pa, lda, _vec(b, n, "b"), float(lam), ctypes.byref(o),
                              _vec(x, d, "x"), ctypes.byref(info) if want_info else None,
                              _stream(stream))
        _check(rc, allow_not_converged=True)
        if not want_info:
            return x, None
        return x, SolveInfo(info.outer_iters, info.inner_iters_total, info.rel_resid, info.status)

    def solve_refined(self, A: torch.Tensor, b: torch.Tensor, lam: float, sd: float, tol: float = 1e-12,
                      max_outer: int = 200, eps_sub: float = 0.1, max_inner: int = 0,
                      x: torch.Tensor | None = None, warm_start: bool = False, want_info: bool = True,
                      stream=None):
        """Algorithm 1 with compensated refinement (fp64 x).  Returns (x, SolveInfo)."""
        pa, n, d, lda = _mat(A, "A")
        if (n, d) != (self.n, self.d):
            raise ValueError("A does not match the sketch")
        if x is None:
            x = torch.empty(d, dtype=torch.float64, device=A.device)
        if not (x.is_cuda and x.dtype == torch.float64 and x.numel() == d and x.is_contiguous()):
            raise ValueError("x must be a contiguous CUDA fp64 vector of length d")
        o = lib().mihs_default_opts()
        o.tol, o.max_outer, o.eps_sub = float(tol), int(max_outer), float(eps_sub)
        o.max_inner, o.sd, o.warm_start = int(max_inner), float(sd), int(bool(warm_start))
        info = _Info()
        rc = lib().mihs_solve_refined(self._h, pa, lda, _vec(b, n, "b"), float(lam), ctypes.byref(o),
                                      x.data_ptr(), ctypes.byref(info) if want_info else None,
                                      _stream(stream))
        _check(rc, allow_not_converged=True)
        if not want_info:
            return x, None
        return x, SolveInfo(info.outer_iters, info.inner_iters_total, info.rel_resid, info.status)

    def backward(self, A: torch.Tensor, b: torch.Tensor, lam: float, sd: float, x: torch.Tensor,
                 gx: torch.Tensor, tol: float = 1e-6, max_outer: int = 100, eps_sub: float = 0.1,
                 max_inner: int = 0, v: torch.Tensor | None = None, warm_start: bool = False,
                 want_dA: bool = True, want_db: bool = True, want_dlambda: bool = True,
                 want_info: bool = True, stream=None):
        """Adjoint solve (AᵀA + λI)v = ḡ with this sketch, then the gradients
        (mihs_backward).  Returns (dA, db, dlambda, v, SolveInfo or None)."""
        pa, n, d, lda = _mat(A, "A")
        if (n, d) != (self.n, self.d):
            raise ValueError("A does not match the sketch")
        if v is None:
            v = torch.empty(d, dtype=torch.float32, device=A.device)
        dA, db, dl = _grad_outputs(n, d, A.device, want_dA, want_db, want_dlambda)
        o = lib().mihs_default_opts()
        o.tol, o.max_outer, o.eps_sub = float(tol), int(max_outer), float(eps_sub)
        o.max_inner, o.sd, o.warm_start = int(max_inner), float(sd), int(bool(warm_start))
        info = _Info()
        rc = lib().mihs_backward(self._h, pa, lda, _vec(b, n, "b"), float(lam), _vec(x, d, "x"),
                                 _vec(gx, d, "gx"), ctypes.byref(o), _vec(v, d, "v"),
                                 dA.data_ptr() if dA is not None else None, d,
                                 db.data_ptr() if db is not None else None,
                                 dl.data_ptr() if dl is not None else None,
                                 ctypes.byref(info) if want_info else None, _stream(stream))
        _check(rc, allow_not_converged=True)
        si = SolveInfo(info.outer_iters, info.inner_iters_total, info.rel_resid, info.status) if want_info else None
        return dA, db, dl, v, si

    def backward_refined(self, A: torch.Tensor, b: torch.Tensor, lam: float, sd: float, x: torch.Tensor,
                         gx: torch.Tensor, tol: float = 1e-10, max_outer: int = 200, eps_sub: float = 0.1,
                         max_inner: int = 0, v: torch.Tensor | None = None, warm_start: bool = False,
                         want_dA: bool = True, want_db: bool = True, want_dlambda: bool = True,
                         want_info: bool = True, stream=None):
        """mihs_backward_refined: the adjoint solved with compensated refinement
        (x and v fp64).  Returns (dA, db, dlambda, v, SolveInfo or None)."""
        pa, n, d, lda = _mat(A, "A")
        if (n, d) != (self.n, self.d):
            raise ValueError("A does not match the sketch")
        for t, nm in ((x, "x"),) + (((v, "v"),) if v is not None else ()):
            if not (t.is_cuda and t.dtype == torch.float64 and t.numel() == d and t.is_contiguous()):
                raise ValueError(f"{nm} must be a contiguous CUDA fp64 vector of length d")
        if v is None:
            v = torch.empty(d, dtype=torch.float64, device=A.device)
        dA, db, dl = _grad_outputs(n, d, A.device, want_dA, want_db, want_dlambda)
        o = lib().mihs_default_opts()
        o.tol, o.max_outer, o.eps_sub = float(tol), int(max_outer), float(eps_sub)
        o.max_inner, o.sd, o.warm_start = int(max_inner), float(sd), int(bool(warm_start))
        info = _Info()
        rc = lib().mihs_backward_refined(self._h, pa, lda, _vec(b, n, "b"), float(lam), x.data_ptr(),
                                         _vec(gx, d, "gx"), ctypes.byref(o), v.data_ptr(),
                                         dA.data_ptr() if dA is not None else None, d,
                                         db.data_ptr() if db is not None else None,
                                         dl.data_ptr() if dl is not None else None,
                                         ctypes.byref(info) if want_info else None, _stream(stream))
        _check(rc, allow_not_converged=True)
        si = SolveInfo(info.outer_iters, info.inner_iters_total, info.rel_resid, info.status) if want_info else None
        return dA, db, dl, v, si

    def solve_path(self, A: torch.Tensor, b: torch.Tensor, lambdas, sds=None, tol: float = 1e-6,
                   max_outer: int = 100, eps_sub: float = 0.1, max_inner: int = 0,
                   X: torch.Tensor | None = None, warm_start: bool = False, want_info: bool = True,
                   stream=None):
        """Algorithm 1 for every λ of `lambdas` with this sketch (mihs_solve_path).
        Returns (X, [SolveInfo] or None) with X λ-major (nl × d)."""
        pa, n, d, lda = _mat(A, "A")
        if (n, d) != (self.n, self.d):
            raise ValueError("A does not match the sketch")
        lam, nl = _dbl_array(lambdas)
        if X is None:
            X = torch.empty(nl, d, dtype=torch.float32, device=A.device)
        if not (X.is_cuda and X.dtype == torch.float32 and tuple(X.shape) == (nl, d) and X.stride(1) == 1):
            raise ValueError("X must be a CUDA fp32 nl x d matrix with unit column stride")
        sd_arr = _dbl_array(sds)[0] if sds is not None else None
        o = _path_opts(tol, max_outer, eps_sub, max_inner, warm_start)
        infos = (_Info * nl)() if want_info else None
        rc = lib().mihs_solve_path(self._h, pa, lda, _vec(b, n, "b"), nl, lam, sd_arr, ctypes.byref(o),
                                   X.data_ptr(), X.stride(0), infos, _stream(stream))
        _check(rc, allow_not_converged=True)
        return X, (_infos(infos, nl) if want_info else None)

    def history(self):
        """Relative residual ‖g(xⁱ)‖/‖Aᵀb‖ of every gradient step of the last solve."""
        buf = (ctypes.c_float * 1024)()
        cnt = _int()
        _check(lib().mihs_solve_history(self._h, buf, 1024, ctypes.byref(cnt)))
        return [float(buf[i]) for i in range(cnt.value)]

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().mihs_sketch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


_HANDLES: dict = {}
_IN_FLIGHT: list = []  # (event, host tensors) of host → device copies not known to have run


def _to_device(t: torch.Tensor, dev) -> torch.Tensor:
    """Host tensor → new CUDA tensor on the current stream by
    mihs_copy_to_device (pinned memory is read by the SMs); the host tensor
    is kept alive until the copy has run."""
    t = t.contiguous()
    out = torch.empty(t.shape, dtype=t.dtype, device=dev)
    copy_to_device(out, t)
    ev = torch.cuda.Event()
    ev.record()
    while _IN_FLIGHT and _IN_FLIGHT[0][0].query():
        _IN_FLIGHT.pop(0)
    _IN_FLIGHT.append((ev, t))
    return out


def solve(A: torch.Tensor, b: torch.Tensor, lam: float, family, m: int, sd: float, seed: int = 0,
          out: torch.Tensor | None = None, aab: str = "auto", **kw):
    """Sketch A then run Algorithm 1: the one-call form.

    A and b may live on the GPU or on the host (ideally pinned).  Host inputs
    are copied to the current CUDA device (mihs_copy_to_device) and x is
    copied back (into `out` when given), which makes this the end-to-end
    form of the solver.  One
    sketch handle per (device, n, d, m, family) is kept and reused, so
    repeated calls allocate nothing new.  `aab` is the form of AAb_Solver,
    "auto", "cluster", "grid" or "grid:<blocks>" (Sketch.set_aab).
    Returns (x, SolveInfo or None).
    """
    host = not A.is_cuda
    dev = torch.device("cuda", torch.cuda.current_device())
    if host:
        A = _to_device(A, dev)
        b = _to_device(b, dev)
    key = (A.device.index, A.shape[0], A.shape[1], int(m), family_id(family))
    sk = _HANDLES.get(key)
    if sk is None:
        sk = _HANDLES[key] = Sketch(A, family, m, seed)
    else:
        sk.resketch(A, seed)
    form, _, blocks = aab.partition(":")
    sk.set_aab(form, int(blocks or 0))
    x, info = sk.solve(A, b, lam, sd, **kw)
    if host:
        if out is None:
            out = torch.empty(x.shape, dtype=x.dtype, pin_memory=True)
        out.copy_(x, non_blocking=True)
        return out, info
    return x, info


class RidgeSolve(torch.autograd.Function):
    """x = (AᵀA + λI)⁻¹Aᵀb by M-IHS, differentiable in A, b and λ.

    The forward pass sketches A and runs Algorithm 1; the backward pass runs
    the adjoint solve with the same sketch and one fused pass over A
    (mihs_backward).  λ may be a Python number or a 0-d tensor.  With
    `refine`, both solves use compensated refinement (mihs_solve_refined,
    mihs_backward_refined) and x is returned in fp64."""

    @staticmethod
    def forward(ctx, A, b, lam, family, m, sd, seed, tol, max_outer, eps_sub, refine):
        lam_f = float(lam)
        sk = Sketch(A, family, m, seed)
        kw = dict(tol=tol, max_outer=max_outer, eps_sub=eps_sub, want_info=False)
        if refine:
            x, _ = sk.solve_refined(A, b, lam_f, sd, **kw)
        else:
            x, _ = sk.solve(A, b, lam_f, sd, **kw)
        ctx.sk, ctx.lam, ctx.sd, ctx.refine = sk, lam_f, sd, refine
        ctx.kw = dict(tol=tol, max_outer=max_outer, eps_sub=eps_sub)
        ctx.lam_like = lam if torch.is_tensor(lam) else None
        ctx.save_for_backward(A, b, x)
        return x

    @staticmethod
    def backward(ctx, gx):
        A, b, x = ctx.saved_tensors
        need_A, need_b, need_lam = ctx.needs_input_grad[:3]
        bw = ctx.sk.backward_refined if ctx.refine else ctx.sk.backward
        dA, db, dl, _, _ = bw(A, b, ctx.lam, ctx.sd, x, gx.contiguous().float(),
                              want_dA=need_A, want_db=need_b,
                              want_dlambda=need_lam and ctx.lam_like is not None,
                              want_info=False, **ctx.kw)
        if dl is not None:
            dl = dl.to(dtype=ctx.lam_like.dtype).reshape(ctx.lam_like.shape)
        return dA, db, dl, None, None, None, None, None, None, None, None


def ridge_solve(A: torch.Tensor, b: torch.Tensor, lam, family="countsketch", m: int | None = None,
                sd: float = 0.0, seed: int = 0, tol: float = 1e-6, max_outer: int = 100,
                eps_sub: float = 0.1, refine: bool = False) -> torch.Tensor:
    """Differentiable ridge solve (RidgeSolve).  m defaults to min(n, 4·sd)
    rounded up to a multiple of 4 when sd > 0, else to min(n, d)."""
    n, d = A.shape
    if m is None:
        m = min(n, ((int(4 * sd) + 3) // 4) * 4) if sd > 0 else min(n, d)
    return RidgeSolve.apply(A, b, lam, family, int(m), float(sd), int(seed), float(tol), int(max_outer),
                            float(eps_sub), bool(refine))


def gradient_dual(A: torch.Tensor, b: torch.Tensor, nu: torch.Tensor, lam: float, g: torch.Tensor | None = None,
                  stream=None) -> torch.Tensor:
    """g = b − A(Aᵀν) − λν (mihs_gradient_dual)."""
    pa, n, d, lda = _mat(A, "A")
    if g is None:
        g = torch.empty(n, dtype=torch.float32, device=A.device)
    _check(lib().mihs_gradient_dual(pa, n, d, lda, _vec(b, n, "b"), _vec(nu, n, "nu"), float(lam), _vec(g, n, "g"),
                                    _stream(stream)))
    return g


def dual_recover(A: torch.Tensor, nu: torch.Tensor, x: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """x = Aᵀν (mihs_dual_recover)."""
    pa, n, d, lda = _mat(A, "A")
    if x is None:
        x = torch.empty(d, dtype=torch.float32, device=A.device)
    _check(lib().mihs_dual_recover(pa, n, d, lda, _vec(nu, n, "nu"), _vec(x, d, "x"), _stream(stream)))
    return x


class DualSketch:
    """A handle holding SAᵀ (mihs_dual_sketch) for Dual M-IHS solves (n ≤ d)."""

    def __init__(self, A: torch.Tensor, family, m: int, seed: int, stream=None):
        pa, n, d, lda = _mat(A, "A")
        h = ctypes.c_void_p()
        _check(lib().mihs_dual_sketch(pa, n, d, lda, family_id(family), int(m), seed & (2**64 - 1),
                                      _stream(stream), ctypes.byref(h)))
        self._h = h
        self.n, self.d, self.m = n, d, int(m)
        self.device = A.device

    def resketch(self, A: torch.Tensor, seed: int, stream=None) -> None:
        pa, n, d, lda = _mat(A, "A")
        _check(lib().mihs_dual_resketch(self._h, pa, lda, seed & (2**64 - 1), _stream(stream)))

    def sat(self, stream=None) -> torch.Tensor:
        out = torch.empty(self.m, self.n, dtype=torch.float32, device=self.device)
        _check(lib().mihs_dual_copy(self._h, out.data_ptr(), self.n, _stream(stream)))
        return out

    def solve(self, A: torch.Tensor, b: torch.Tensor, lam: float, sd: float, tol: float = 1e-6,
              max_outer: int = 100, eps_sub: float = 0.1, max_inner: int = 0, nu: torch.Tensor | None = None,
              x: torch.Tensor | None = None, warm_start: bool = False, want_info: bool = True, stream=None):
        """Algorithm 2.  Returns (x, nu, SolveInfo or None)."""
        pa, n, d, lda = _mat(A, "A")
        if (n, d) != (self.n, self.d):
            raise ValueError("A does not match the sketch")
        if nu is None:
            nu = torch.empty(n, dtype=torch.float32, device=A.device)
        if x is None:
            x = torch.empty(d, dtype=torch.float32, device=A.device)
        o = lib().mihs_default_opts()
        o.tol, o.max_outer, o.eps_sub = float(tol), int(max_outer), float(eps_sub)
        o.max_inner, o.sd, o.warm_start = int(max_inner), float(sd), int(bool(warm_start))
        info = _Info()
        rc = lib().mihs_solve_dual(self._h, pa, lda, _vec(b, n, "b"), float(lam), ctypes.byref(o), _vec(x, d, "x"),
                                   _vec(nu, n, "nu"), ctypes.byref(info) if want_info else None, _stream(stream))
        _check(rc, allow_not_converged=True)
        return x, nu, (SolveInfo(info.outer_iters, info.inner_iters_total, info.rel_resid, info.status)
                       if want_info else None)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().mihs_dual_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
