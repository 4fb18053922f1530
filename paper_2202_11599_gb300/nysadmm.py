"""Thin Python binding of libnysadmm (include/nysadmm.h).

Argument marshalling only: every step of the solve runs in the CUDA library.
Tensors are torch CUDA tensors (PyTorch supplies device memory and the stream);
the library is required -- there is no CPU fallback, and a missing or
unloadable library raises at first use.
"""
from __future__ import annotations

import ctypes
import math
import os
from ctypes import POINTER, c_double, c_int32, c_int64, c_void_p

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnysadmm.so")

NYS_OK, NYS_EINVAL, NYS_ENOTSPD, NYS_EBREAKDOWN, NYS_ENOCONV, NYS_ETIMEOUT, NYS_ECUDA, NYS_ENOMEM = range(8)
NYS_LASSO, NYS_LOGISTIC, NYS_ELASTIC_NET = 0, 1, 2
NYS_F64, NYS_F32, NYS_BF16, NYS_FP8E4M3 = 0, 1, 2, 3
TOL_MODES = {"rel": 0, "abs": 1, "sqrt_rprd": 2, "rnorm_pow": 3}
_DTYPES = {torch.float64: NYS_F64, torch.float32: NYS_F32, torch.bfloat16: NYS_BF16,
           torch.float8_e4m3fn: NYS_FP8E4M3}
FP8_E4M3_MAX = 448.0
_LOSSES = {"lasso": NYS_LASSO, "logistic": NYS_LOGISTIC, "elastic_net": NYS_ELASTIC_NET}


class NysMatrixC(ctypes.Structure):
    _fields_ = [("data", c_void_p), ("dtype", c_int32), ("n", c_int64), ("d", c_int64), ("ld", c_int64),
                ("col_scale", c_void_p)]


class NysOptsC(ctypes.Structure):
    _fields_ = [("shift_scale", c_double), ("pcg_tol_mode", c_int32), ("pcg_maxit", c_int32),
                ("pcg_fixed_iters", POINTER(c_int32)), ("admm_maxit", c_int32),
                ("eps_abs", c_double), ("eps_rel", c_double), ("A_inner", POINTER(NysMatrixC)),
                ("refine", c_int32), ("z_trace", c_void_p), ("rank_max", c_int32),
                ("ada_tol", c_double), ("resketch_every", c_int32), ("stream", c_void_p),
                ("device_loop", c_int32), ("hx_refresh", c_int32), ("warm_model", c_void_p),
                ("warm_record", c_void_p), ("seed", ctypes.c_uint64), ("allreduce", c_void_p),
                ("allreduce_ctx", c_void_p), ("pcg_trace", POINTER(c_int32))]


class NysInfoC(ctypes.Structure):
    _fields_ = [("admm_iters", c_int32), ("pcg_iters_total", c_int32), ("final_rank", c_int32),
                ("status", c_int32), ("r_p", c_double), ("r_d", c_double), ("emp_cond", c_double),
                ("nu", c_double)]


class NysStatsC(ctypes.Structure):
    _fields_ = [("launches", c_int64), ("apass_launches", c_int64 * 4), ("apass_ms", c_double * 4),
                ("apass_bytes", c_double * 4), ("dev_launches", c_int64 * 4), ("dev_ms", c_double * 4),
                ("dev_bytes", c_double * 4)]


class NysInstanceC(ctypes.Structure):
    _fields_ = [("A", POINTER(NysMatrixC)), ("b", c_void_p), ("gamma", c_double), ("rank", c_int32),
                ("Omega", c_void_p), ("x_out", c_void_p), ("z_out", c_void_p)]


_ALLREDUCE_FN = ctypes.CFUNCTYPE(c_int32, c_void_p, c_int64, c_int32, c_void_p, c_void_p)


class _DeviceView:
    """Zero-copy view of a library-owned device buffer for torch (CUDA array interface)."""

    def __init__(self, ptr: int, count: int, dtype: int):
        self.__cuda_array_interface__ = {"data": (int(ptr), False), "shape": (int(count),),
                                         "typestr": "<f8" if dtype == NYS_F64 else "<f4", "strides": None,
                                         "version": 2}


def _allreduce_callback(fn):
    """Wrap fn(tensor) -- an in-place sum over the ranks -- as the library's nys_allreduce_fn.
    The tensor views the library's buffer; fn runs with the library's stream current."""
    def cb(buf, count, dtype, stream, ctx):
        try:
            t = torch.as_tensor(_DeviceView(buf, count, dtype), device="cuda")
            s = torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream()
            with torch.cuda.stream(s):
                fn(t)
            return NYS_OK
        except Exception:  # noqa: BLE001 -- reported to the library as a status, never raised through C
            return NYS_ECUDA
    return _ALLREDUCE_FN(cb)


def row_block(n: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous block of rows [r0, r1) of rank `rank` in a row-sharded solve (sizes differ by
    at most one row; the blocks cover 0..n-1 once, in rank order)."""
    if not (0 <= rank < world) or n < world:
        raise ValueError("need 0 <= rank < world <= n")
    return n * rank // world, n * (rank + 1) // world


def host_staged_allreduce(dist, group=None):
    """An allreduce for row-sharded solves over any torch.distributed backend (gloo included):
    the device buffer is copied to the host, summed over the ranks, and copied back on the
    library's stream."""
    def fn(t):
        c = t.cpu()
        dist.all_reduce(c, group=group)
        t.copy_(c)
    return fn


class NysError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {strerror(status)} (status {status})")


_lib = None


def lib() -> ctypes.CDLL:
    """Load libnysadmm.so (built by __graft_entry__.build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                           "(the CUDA library is required; there is no CPU path)")
    L = ctypes.CDLL(LIB_PATH)
    P = POINTER
    L.nys_opts_default.argtypes = [P(NysOptsC)]
    L.nys_opts_default.restype = None
    L.nys_strerror.argtypes = [c_int32]
    L.nys_strerror.restype = ctypes.c_char_p
    L.nys_hmatvec.argtypes = [P(NysMatrixC), c_void_p, c_double, c_void_p, c_void_p, c_void_p]
    L.nys_hmatvec_noalloc.argtypes = [P(NysMatrixC), c_void_p, c_double, c_void_p, c_void_p, c_void_p]
    L.nys_check_wait_bound.argtypes = [c_double, c_void_p]
    L.nys_sketch.argtypes = [P(NysMatrixC), c_void_p, c_double, c_int32, c_void_p, P(NysOptsC), P(c_void_p)]
    L.nys_gaussian_test_matrix.argtypes = [ctypes.c_uint64, c_int64, c_int32, c_void_p, c_void_p]
    L.nys_precond_get.argtypes = [c_void_p, c_void_p, P(c_double), P(c_int32), P(c_int64), P(c_double), c_void_p]
    L.nys_precond_apply.argtypes = [c_void_p, c_double, c_void_p, c_void_p, c_int64, c_int32, c_void_p]
    L.pcg_solve.argtypes = [P(NysMatrixC), c_void_p, c_double, c_void_p, c_void_p, c_void_p, c_double,
                            P(NysOptsC), P(c_int32), P(c_double)]
    L.nysadmm_solve.argtypes = [c_int32, P(NysMatrixC), c_void_p, c_double, c_double, c_int32, c_double,
                                c_void_p, P(NysOptsC), c_void_p, c_void_p, P(NysInfoC)]
    L.nysadmm_solve_path.argtypes = [P(NysMatrixC), c_void_p, P(c_double), c_int32, c_double, c_int32, c_double,
                                     c_void_p, P(NysOptsC), c_void_p, c_void_p, P(NysInfoC), P(c_int32)]
    L.nysadmm_solve_batch.argtypes = [c_int32, POINTER(NysInstanceC), c_double, c_double, P(NysOptsC),
                                      POINTER(NysInfoC)]
    L.nys_objective.argtypes = [c_int32, P(NysMatrixC), c_void_p, c_double, c_void_p, P(c_double), c_void_p]
    L.nys_stats_enable.argtypes = [c_int32]
    L.nys_stats_enable.restype = None
    L.nys_stats_read.argtypes = [POINTER(NysStatsC)]
    L.nys_mlp_create.argtypes = [c_int32, c_int32, c_int32, c_void_p, P(c_void_p)]
    L.nys_mlp_forward.argtypes = [c_void_p, c_void_p, c_int32, c_void_p, c_void_p]
    L.nys_mlp_grad.argtypes = [c_void_p, c_void_p, c_void_p, c_int32, c_void_p, P(ctypes.c_float), c_void_p]
    L.nys_mlp_train_step.argtypes = [c_void_p, c_void_p, c_void_p, c_int32, ctypes.c_float, P(ctypes.c_float),
                                     c_void_p]
    L.nys_mlp_get_params.argtypes = [c_void_p, c_void_p, P(c_int64), c_void_p]
    L.nys_mlp_destroy.argtypes = [c_void_p]
    L.nys_mlp_destroy.restype = None
    L.nys_autotune_apass.argtypes = [P(NysMatrixC), P(c_int32), P(c_double), c_void_p]
    L.nys_autotune_apass.restype = c_int32
    L.nys_precond_destroy.argtypes = [c_void_p]
    L.nys_precond_destroy.restype = None
    for name in ("nys_hmatvec", "nys_hmatvec_noalloc", "nys_gaussian_test_matrix", "nys_sketch", "nys_precond_get", "nys_precond_apply", "pcg_solve",
                 "nysadmm_solve", "nysadmm_solve_path", "nysadmm_solve_batch", "nys_objective",
                 "nys_stats_read", "nys_mlp_create", "nys_mlp_forward", "nys_mlp_grad", "nys_mlp_train_step",
                 "nys_mlp_get_params"):
        getattr(L, name).restype = c_int32
    _lib = L
    return L


def strerror(status: int) -> str:
    return lib().nys_strerror(int(status)).decode()


def _check(status: int, where: str, ok=(NYS_OK,)):
    if status not in ok:
        raise NysError(status, where)
    return status


def _stream_ptr(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _ptr(t):
    return None if t is None else c_void_p(t.data_ptr())


class Matrix:
    """Row-major device matrix (n x d, leading dimension ld >= d) for the C ABI."""

    def __init__(self, t: torch.Tensor, d: int | None = None, col_scale: torch.Tensor | None = None):
        if not t.is_cuda or t.dim() != 2 or t.stride(1) != 1:
            raise ValueError("Matrix needs a 2-D CUDA tensor with unit column stride")
        if t.dtype not in _DTYPES:
            raise ValueError(f"unsupported dtype {t.dtype}")
        self.tensor = t
        self.n = t.shape[0]
        self.d = t.shape[1] if d is None else d
        self.ld = t.stride(0)
        self.col_scale = None
        if t.dtype == torch.float8_e4m3fn:
            if col_scale is None or col_scale.dtype != torch.float32 or not col_scale.is_cuda:
                raise ValueError("an FP8 matrix needs FP32 per-column scales on the device")
            self.col_scale = col_scale.contiguous()
        self.c = NysMatrixC(c_void_p(t.data_ptr()), _DTYPES[t.dtype], self.n, self.d, self.ld,
                            c_void_p(self.col_scale.data_ptr() if self.col_scale is not None else 0))

    @property
    def compute_dtype(self):
        return torch.float64 if self.tensor.dtype == torch.float64 else torch.float32

    @staticmethod
    def padded(src: torch.Tensor, dtype=None) -> "Matrix":
        """Copy src (n x d) into a row-major buffer whose rows start on 16-byte boundaries."""
        dtype = dtype or src.dtype
        n, d = src.shape
        esz = torch.tensor([], dtype=dtype).element_size()
        vec = 16 // esz
        ld = (d + vec - 1) // vec * vec
        buf = torch.zeros(n, ld, dtype=dtype, device=src.device)
        buf[:, :d] = src.to(dtype)
        return Matrix(buf, d=d)

    @staticmethod
    def fp8(src: torch.Tensor) -> "Matrix":
        """FP8 E4M3 codes with one FP32 scale per column, A_ij ~ scale_j * q_ij (scale_j maps
        the column's largest magnitude to the E4M3 maximum), rows on 16-byte boundaries."""
        n, d = src.shape
        a = src.to(torch.float32)
        scale = (a.abs().amax(dim=0) / FP8_E4M3_MAX).clamp_min(torch.finfo(torch.float32).tiny)
        ld = (d + 15) // 16 * 16
        buf = torch.zeros(n, ld, dtype=torch.float8_e4m3fn, device=src.device)
        buf[:, :d] = (a / scale[None, :]).to(torch.float8_e4m3fn)
        return Matrix(buf, d=d, col_scale=scale)

    def dequantized(self) -> torch.Tensor:
        """The stored values as FP64 (FP8: scale_j * q_ij), n x d."""
        t = self.tensor[:, : self.d].to(torch.float64)
        return t * self.col_scale.to(torch.float64)[None, :] if self.col_scale is not None else t


def _opts(stream=None, **kw) -> NysOptsC:
    o = NysOptsC()
    lib().nys_opts_default(ctypes.byref(o))
    o.stream = c_void_p(_stream_ptr(stream))
    for k, v in kw.items():
        if v is not None:
            setattr(o, k, v)
    return o


def hmatvec(A: Matrix, p: torch.Tensor, rho: float = 0.0, D: torch.Tensor | None = None,
            stream=None) -> torch.Tensor:
    """y = A^T diag(D) A p + rho p (Table 1 T_mv), in A's compute precision."""
    y = torch.empty(A.d, dtype=A.compute_dtype, device=A.tensor.device)
    p = p.to(A.compute_dtype).contiguous()
    _check(lib().nys_hmatvec(ctypes.byref(A.c), _ptr(D), float(rho), _ptr(p), _ptr(y),
                             c_void_p(_stream_ptr(stream))), "nys_hmatvec")
    return y


def hmatvec_noalloc(A: Matrix, p: torch.Tensor, rho: float = 0.0, D: torch.Tensor | None = None,
                    stream=None) -> torch.Tensor:
    """hmatvec through the allocation-free entry point (fixed in-library scratch)."""
    y = torch.empty(A.d, dtype=A.compute_dtype, device=A.tensor.device)
    p = p.to(A.compute_dtype).contiguous()
    _check(lib().nys_hmatvec_noalloc(ctypes.byref(A.c), _ptr(D), float(rho), _ptr(p), _ptr(y),
                                     c_void_p(_stream_ptr(stream))), "nys_hmatvec_noalloc")
    return y


def autotune_apass(A: Matrix, stream=None):
    """Time the supported rows-per-stage choices of the fused pass on A, keep the best.
    Returns (rows, ms per pass)."""
    r = c_int32()
    ms = c_double()
    _check(lib().nys_autotune_apass(ctypes.byref(A.c), ctypes.byref(r), ctypes.byref(ms),
                                    c_void_p(_stream_ptr(stream))), "nys_autotune_apass")
    return r.value, ms.value


class Precond:
    """Randomized Nystrom preconditioner handle (App. B; Eq. Nystrom preconditioner)."""

    def __init__(self, handle: int):
        self.h = c_void_p(handle)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None and self.h.value:
            _lib.nys_precond_destroy(self.h)
            self.h = c_void_p(0)

    def info(self):
        s = c_int32()
        d = c_int64()
        nu = c_double()
        _check(lib().nys_precond_get(self.h, None, None, ctypes.byref(s), ctypes.byref(d), ctypes.byref(nu),
                                     c_void_p(_stream_ptr())), "nys_precond_get")
        return s.value, d.value, nu.value

    @property
    def lam(self) -> torch.Tensor:
        s, _, _ = self.info()
        out = (c_double * s)()
        _check(lib().nys_precond_get(self.h, None, out, None, None, None, c_void_p(_stream_ptr())),
               "nys_precond_get")
        return torch.tensor(list(out), dtype=torch.float64)

    @property
    def nu(self) -> float:
        return self.info()[2]

    @property
    def U(self) -> torch.Tensor:
        s, d, _ = self.info()
        U = torch.empty(s, d, dtype=torch.float64, device="cuda")      # column-major d x s
        _check(lib().nys_precond_get(self.h, _ptr(U), None, None, None, None, c_void_p(_stream_ptr())),
               "nys_precond_get")
        return U.T

    def apply(self, V: torch.Tensor, rho: float, stream=None) -> torch.Tensor:
        """P^{-1} V for V of shape (d,) or (d, k); FP64 or FP32."""
        squeeze = V.dim() == 1
        Vc = V.reshape(V.shape[0], -1).T.contiguous()                  # k x d == column-major d x k
        Y = torch.empty_like(Vc)
        dt = NYS_F64 if V.dtype == torch.float64 else NYS_F32
        _check(lib().nys_precond_apply(self.h, float(rho), _ptr(Vc), _ptr(Y), Vc.shape[0], dt,
                                       c_void_p(_stream_ptr(stream))), "nys_precond_apply")
        Y = Y.T
        return Y.reshape(-1) if squeeze else Y


def gaussian_test_matrix(seed: int, d: int, s: int, stream=None) -> torch.Tensor:
    """Omega (d x s, FP64, device) ~ N(0,1) drawn in the library (Philox-4x32-10 + Box-Muller)."""
    Om = torch.empty(s, d, dtype=torch.float64, device="cuda")          # column-major d x s
    _check(lib().nys_gaussian_test_matrix(int(seed) & (2**64 - 1), int(d), int(s), _ptr(Om),
                                          c_void_p(_stream_ptr(stream))), "nys_gaussian_test_matrix")
    return Om.T


def sketch(A: Matrix, Omega: torch.Tensor | None, D: torch.Tensor | None = None, diag_shift: float = 0.0,
           shift_scale: float | None = None, stream=None, s: int | None = None, seed: int = 0,
           allreduce=None) -> Precond:
    """Nystrom sketch of H = A^T diag(D) A + diag_shift I from the Gaussian Omega (d x s), or,
    with Omega None, from s columns drawn in the library from `seed`."""
    if Omega is None:
        Om = None
    else:
        s = Omega.shape[1]
        Om = Omega.to(torch.float64).T.contiguous()                    # column-major d x s
    h = c_void_p()
    cb = _allreduce_callback(allreduce) if allreduce is not None else None
    o = _opts(stream, shift_scale=shift_scale, seed=int(seed) & (2**64 - 1),
              allreduce=ctypes.cast(cb, c_void_p) if cb is not None else None)
    _check(lib().nys_sketch(ctypes.byref(A.c), _ptr(D), float(diag_shift), int(s), _ptr(Om), ctypes.byref(o),
                            ctypes.byref(h)), "nys_sketch")
    return Precond(h.value)


def pcg_solve(A: Matrix, r: torch.Tensor, rho: float, P: Precond | None = None, x0=None, tol: float = 1e-8,
              tol_mode: str = "rel", maxit: int | None = None, fixed_iters: int | None = None,
              D: torch.Tensor | None = None, stream=None, allow_noconv: bool = False, allreduce=None):
    """Nystrom PCG (App. B) for (A^T diag(D) A + rho I) x = r.  Returns (x, iters, ||w||)."""
    ct = A.compute_dtype
    r = r.to(ct).contiguous()
    x = torch.zeros(A.d, dtype=ct, device=r.device) if x0 is None else x0.to(ct).clone().contiguous()
    fixed = (c_int32 * 1)(fixed_iters) if fixed_iters is not None else None
    cb = _allreduce_callback(allreduce) if allreduce is not None else None
    o = _opts(stream, pcg_tol_mode=TOL_MODES[tol_mode], pcg_maxit=maxit or 0,
              pcg_fixed_iters=ctypes.cast(fixed, POINTER(c_int32)) if fixed is not None else None,
              allreduce=ctypes.cast(cb, c_void_p) if cb is not None else None)
    it = c_int32()
    rn = c_double()
    st = lib().pcg_solve(ctypes.byref(A.c), _ptr(D), float(rho), P.h if P is not None else None, _ptr(r),
                         _ptr(x), float(tol), ctypes.byref(o), ctypes.byref(it), ctypes.byref(rn))
    _check(st, "pcg_solve", ok=(NYS_OK, NYS_ENOCONV) if allow_noconv else (NYS_OK,))
    return x, it.value, rn.value


def nysadmm_solve(loss: str, A: Matrix, b: torch.Tensor, gamma: float, rho: float, rank: int, tol: float,
                  Omega: torch.Tensor, admm_iters: int = 200, A_inner: Matrix | None = None,
                  refine: bool = True, z_trace: bool = False, pcg_fixed=None, tol_mode: str = "rel",
                  pcg_maxit: int | None = None, eps_abs: float = 0.0, eps_rel: float = 0.0,
                  rank_max: int | None = None, ada_tol: float | None = None, resketch_every: int = 1,
                  shift_scale: float | None = None, stream=None, allow_noconv: bool = True,
                  device_loop: bool = True, hx_refresh: int = 0, warm_model=None,
                  warm_record: bool = False, seed: int = 0, pcg_trace: bool = False, allreduce=None) -> dict:
    """NysADMM (Alg. NysADMM / AdaNysADMM) through the C ABI.  Returns a dict with
    x, z (FP64 device tensors), info (dict) and, when requested, the z trace and the PCG
    iterations of each ADMM iteration.  Omega None: the test matrix is drawn in the library
    from `seed`.  allreduce: fn(tensor) summing a device tensor over the ranks in place, for a
    row-sharded solve (A, b: this rank's rows; host-driven loop)."""
    d = A.d
    Om = None if Omega is None else Omega.to(torch.float64).T.contiguous()   # column-major d x s
    x = torch.empty(d, dtype=torch.float64, device="cuda")
    z = torch.empty(d, dtype=torch.float64, device="cuda")
    zt = torch.empty(admm_iters, d, dtype=torch.float64, device="cuda") if z_trace else None
    rec = torch.zeros(admm_iters, 2 * int(rank) + 3, dtype=torch.float32, device="cuda") if warm_record else None
    fixed = None
    if pcg_fixed is not None:
        seq = [int(pcg_fixed)] * admm_iters if isinstance(pcg_fixed, int) else [int(v) for v in pcg_fixed]
        fixed = (c_int32 * len(seq))(*seq)
    ptrace = (c_int32 * admm_iters)() if pcg_trace else None
    cb = _allreduce_callback(allreduce) if allreduce is not None else None
    if cb is not None:
        device_loop = False
    o = _opts(stream, shift_scale=shift_scale, pcg_tol_mode=TOL_MODES[tol_mode], pcg_maxit=pcg_maxit or 0,
              pcg_fixed_iters=ctypes.cast(fixed, POINTER(c_int32)) if fixed is not None else None,
              pcg_trace=ctypes.cast(ptrace, POINTER(c_int32)) if ptrace is not None else None,
              allreduce=ctypes.cast(cb, c_void_p) if cb is not None else None,
              admm_maxit=admm_iters, eps_abs=eps_abs, eps_rel=eps_rel,
              A_inner=ctypes.pointer(A_inner.c) if A_inner is not None else None,
              refine=int(bool(refine)), z_trace=c_void_p(zt.data_ptr()) if zt is not None else None,
              rank_max=rank_max or 0, ada_tol=ada_tol, resketch_every=resketch_every,
              device_loop=int(bool(device_loop)), hx_refresh=int(hx_refresh),
              warm_model=warm_model.h if warm_model is not None else None,
              warm_record=c_void_p(rec.data_ptr()) if rec is not None else None,
              seed=int(seed) & (2**64 - 1))
    info = NysInfoC()
    st = lib().nysadmm_solve(_LOSSES[loss], ctypes.byref(A.c), _ptr(b.to(torch.float64).contiguous()),
                             float(gamma), float(rho), int(rank), float(tol), _ptr(Om), ctypes.byref(o),
                             _ptr(x), _ptr(z), ctypes.byref(info))
    _check(st, "nysadmm_solve", ok=(NYS_OK, NYS_ENOCONV) if allow_noconv else (NYS_OK,))
    inf = {f: getattr(info, f) for f, _ in NysInfoC._fields_}
    inf["status"] = st
    out = {"x": x, "z": z, "info": inf}
    if zt is not None:
        out["z_trace"] = zt[: inf["admm_iters"]]
    if rec is not None:
        out["warm_record"] = rec[: inf["admm_iters"]]
    if ptrace is not None:
        out["pcg_trace"] = list(ptrace)[: inf["admm_iters"]]
    return out


def nysadmm_solve_path(A: Matrix, b: torch.Tensor, gammas, rho: float, rank: int, tol: float,
                       Omega: torch.Tensor, admm_iters: int = 200, A_inner: Matrix | None = None,
                       tol_mode: str = "rel", pcg_maxit: int | None = None, pcg_fixed=None,
                       shift_scale: float | None = None, stream=None, allow_noconv: bool = True) -> dict:
    """k lasso solves along a regularisation path (one gamma per column) with shared
    multi-right-hand-side PCG.  Returns X, Z (d x k FP64), pcg iterations per column, info."""
    d = A.d
    k = len(gammas)
    Om = Omega.to(torch.float64).T.contiguous()
    X = torch.empty(k, d, dtype=torch.float64, device="cuda")           # column-major d x k
    Z = torch.empty(k, d, dtype=torch.float64, device="cuda")
    g = (c_double * k)(*[float(v) for v in gammas])
    its = (c_int32 * k)()
    fixed = None
    if pcg_fixed is not None:
        seq = [int(pcg_fixed)] * admm_iters if isinstance(pcg_fixed, int) else [int(v) for v in pcg_fixed]
        fixed = (c_int32 * len(seq))(*seq)
    o = _opts(stream, shift_scale=shift_scale, pcg_tol_mode=TOL_MODES[tol_mode], pcg_maxit=pcg_maxit or 0,
              admm_maxit=admm_iters, A_inner=ctypes.pointer(A_inner.c) if A_inner is not None else None,
              pcg_fixed_iters=ctypes.cast(fixed, POINTER(c_int32)) if fixed is not None else None)
    info = NysInfoC()
    st = lib().nysadmm_solve_path(ctypes.byref(A.c), _ptr(b.to(torch.float64).contiguous()), g, k, float(rho),
                                  int(rank), float(tol), _ptr(Om), ctypes.byref(o), _ptr(X), _ptr(Z),
                                  ctypes.byref(info), its)
    _check(st, "nysadmm_solve_path", ok=(NYS_OK, NYS_ENOCONV) if allow_noconv else (NYS_OK,))
    inf = {f: getattr(info, f) for f, _ in NysInfoC._fields_}
    inf["status"] = st
    return {"X": X.T, "Z": Z.T, "pcg_iters": list(its), "info": inf}


def nysadmm_solve_batch(problems, rho: float, tol: float, admm_iters: int = 200, tol_mode: str = "rel",
                        pcg_maxit: int | None = None, hx_refresh: int = 0, eps_abs: float = 0.0,
                        eps_rel: float = 0.0, stream=None, allow_noconv: bool = True) -> list:
    """Independent lasso instances, one graph launch.  problems: list of dicts with keys
    A (Matrix), b, gamma, rank, Omega (d x rank).  Returns a list of dicts (x, z, info)."""
    n = len(problems)
    arr = (NysInstanceC * n)()
    keep = []
    outs = []
    for i, pr in enumerate(problems):
        A = pr["A"]
        Om = pr["Omega"].to(torch.float64).T.contiguous()
        b = pr["b"].to(torch.float64).contiguous()
        x = torch.empty(A.d, dtype=torch.float64, device="cuda")
        z = torch.empty(A.d, dtype=torch.float64, device="cuda")
        keep += [Om, b, A]
        arr[i] = NysInstanceC(ctypes.pointer(A.c), c_void_p(b.data_ptr()), float(pr["gamma"]), int(pr["rank"]),
                              c_void_p(Om.data_ptr()), c_void_p(x.data_ptr()), c_void_p(z.data_ptr()))
        outs.append({"x": x, "z": z})
    o = _opts(stream, pcg_tol_mode=TOL_MODES[tol_mode], pcg_maxit=pcg_maxit or 0, admm_maxit=admm_iters,
              eps_abs=eps_abs, eps_rel=eps_rel, hx_refresh=int(hx_refresh))
    infos = (NysInfoC * n)()
    st = lib().nysadmm_solve_batch(n, arr, float(rho), float(tol), ctypes.byref(o), infos)
    _check(st, "nysadmm_solve_batch", ok=(NYS_OK, NYS_ENOCONV) if allow_noconv else (NYS_OK,))
    for i in range(n):
        outs[i]["info"] = {f: getattr(infos[i], f) for f, _ in NysInfoC._fields_}
    return outs


def objective(loss: str, A: Matrix, b: torch.Tensor, gamma: float, x: torch.Tensor, stream=None):
    """(objective, KKT measure, duality gap) at x: Eq. (2)/(31) for the lasso, Eq. (9) for logistic."""
    out = (c_double * 3)()
    _check(lib().nys_objective(_LOSSES[loss], ctypes.byref(A.c), _ptr(b.to(torch.float64).contiguous()),
                               float(gamma), _ptr(x.to(torch.float64).contiguous()), out,
                               c_void_p(_stream_ptr(stream))), "nys_objective")
    return out[0], out[1], out[2]


def stats_enable(on: bool = True) -> None:
    """Reset and (de)activate the library's launch counter and A-pass event timing."""
    lib().nys_stats_enable(int(bool(on)))


def stats_read() -> dict:
    """Kernel launches and A-pass device time / algorithmic bytes since stats_enable."""
    s = NysStatsC()
    _check(lib().nys_stats_read(ctypes.byref(s)), "nys_stats_read")
    names = {NYS_F64: "f64", NYS_F32: "f32", NYS_BF16: "bf16", NYS_FP8E4M3: "fp8"}
    return {"launches": s.launches,
            "apass": {names[k]: {"launches": s.apass_launches[k], "ms": s.apass_ms[k],
                                 "bytes": s.apass_bytes[k]} for k in range(4)},
            "apass_dev": {names[k]: {"launches": s.dev_launches[k], "ms": s.dev_ms[k],
                                     "bytes": s.dev_bytes[k]} for k in range(4)}}


def check_wait_bound(wait_us: float = 2000.0, stream=None) -> int:
    """Run the library's bounded device-side wait on a barrier nothing completes; returns
    the status (NYS_ETIMEOUT = 5 when the bound works)."""
    return lib().nys_check_wait_bound(float(wait_us), c_void_p(_stream_ptr(stream)))


class MLP:
    """Learned warm-start model (nys_mlp): n_in -> n_hid -> n_hid -> n_out, erf-GELU."""

    def __init__(self, n_in: int, n_hid: int, n_out: int, init_params):
        self.n_in, self.n_hid, self.n_out = n_in, n_hid, n_out
        p = torch.as_tensor(init_params, dtype=torch.float32).contiguous().cpu()
        h = c_void_p()
        _check(lib().nys_mlp_create(n_in, n_hid, n_out, c_void_p(p.data_ptr()), ctypes.byref(h)), "nys_mlp_create")
        self.h = h

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None and self.h.value:
            _lib.nys_mlp_destroy(self.h)
            self.h = c_void_p(0)

    def forward(self, X: torch.Tensor, stream=None) -> torch.Tensor:
        X = X.to(torch.float32).contiguous()
        Y = torch.empty(X.shape[0], self.n_out, dtype=torch.float32, device="cuda")
        _check(lib().nys_mlp_forward(self.h, _ptr(X), X.shape[0], _ptr(Y), c_void_p(_stream_ptr(stream))),
               "nys_mlp_forward")
        return Y

    def grad(self, X: torch.Tensor, T: torch.Tensor, stream=None):
        X = X.to(torch.float32).contiguous()
        T = T.to(torch.float32).contiguous()
        g = torch.empty(self.n_params(), dtype=torch.float32, device="cuda")
        loss = ctypes.c_float()
        _check(lib().nys_mlp_grad(self.h, _ptr(X), _ptr(T), X.shape[0], _ptr(g), ctypes.byref(loss),
                                  c_void_p(_stream_ptr(stream))), "nys_mlp_grad")
        return loss.value, g

    def train_step(self, X: torch.Tensor, T: torch.Tensor, lr: float = 1e-3, stream=None) -> float:
        X = X.to(torch.float32).contiguous()
        T = T.to(torch.float32).contiguous()
        loss = ctypes.c_float()
        _check(lib().nys_mlp_train_step(self.h, _ptr(X), _ptr(T), X.shape[0], float(lr), ctypes.byref(loss),
                                        c_void_p(_stream_ptr(stream))), "nys_mlp_train_step")
        return loss.value

    def n_params(self) -> int:
        n = c_int64()
        _check(lib().nys_mlp_get_params(self.h, None, ctypes.byref(n), None), "nys_mlp_get_params")
        return n.value

    def params(self) -> torch.Tensor:
        out = torch.empty(self.n_params(), dtype=torch.float32, device="cuda")
        _check(lib().nys_mlp_get_params(self.h, _ptr(out), None, c_void_p(_stream_ptr())), "nys_mlp_get_params")
        return out
