"""ctypes binding of libbec (include/bec.h): argument marshalling only.

Every numerical step runs in the CUDA kernels of libbec.so; this module only
checks tensor shapes/dtypes/devices and passes raw pointers and the current
CUDA stream.  If the library is missing it raises; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libbec.so")

BEC_OK, BEC_EINVAL, BEC_ENOMEM, BEC_ECUDA, BEC_ENOTCONV, BEC_ENUMERIC, BEC_ETIMEOUT, \
    BEC_EUNSUPPORTED = range(8)
BEC_ROUTE_FST, BEC_ROUTE_MG, BEC_ROUTE_LEARNED = 0, 1, 2
BEC_PC_FP64, BEC_PC_FP32 = 0, 1

#: every symbol include/bec.h declares
EXPORTED = (
    "bec_allocate_problem", "bec_set_eps", "bec_apply_A", "bec_apply_P", "bec_apply_Pinv",
    "bec_build_rhs", "bec_build_rhs_dirichlet", "bec_gmres_solve", "bec_gmres_solve_host",
    "bec_gmres_solve_host_many",
    "bec_true_relres",
    "bec_free_problem", "bec_problem_size", "bec_kernel_launches", "bec_status_string",
    "bec_last_error", "bec_profile_start", "bec_profile_stop", "bec_relres_noalloc",
    "bec_batch_create", "bec_batch_problem", "bec_batch_solve", "bec_batch_unknowns",
    "bec_batch_kernel_launches", "bec_batch_free", "bec_learned_num_weights",
    "bec_learned_get_weights", "bec_learned_set_weights", "bec_learned_train",
    "bec_learned_loss_grad", "bec_learned_fallbacks", "bec_learned_residual_ratios",
    "bec_learned_set_judge", "bec_learned_judge_radii",
    "bec_convert_to_float", "bec_convert_to_double", "bec_reciprocal_fp64", "bec_autotune",
    "bec_set_tiles",
    "bec_inject_fault",
)


class ProblemDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("N", ctypes.c_int), ("T", ctypes.c_double), ("a", ctypes.c_double),
                ("route", ctypes.c_int), ("precision", ctypes.c_int),
                ("max_restart", ctypes.c_int), ("flexible", ctypes.c_int),
                ("host_io", ctypes.c_int), ("a_nodes", ctypes.c_void_p),
                ("mg_pre", ctypes.c_int), ("mg_post", ctypes.c_int), ("mg_omega", ctypes.c_double),
                ("net_channels", ctypes.c_int), ("net_fp32", ctypes.c_int),
                ("space", ctypes.c_int), ("time_scheme", ctypes.c_int),
                ("wind", ctypes.c_void_p), ("side", ctypes.c_double), ("mg_smoother", ctypes.c_int)]


class GmresOpts(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int), ("maxit", ctypes.c_int), ("rtol", ctypes.c_double),
                ("flexible", ctypes.c_int), ("left_pc", ctypes.c_int), ("use_x0", ctypes.c_int)]


class GmresInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("restarts", ctypes.c_int), ("converged", ctypes.c_int),
                ("prec_relres", ctypes.c_double), ("true_relres", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_longlong), ("ms", ctypes.c_double)]


class TuneReport(ctypes.Structure):
    _fields_ = [("rows_warps", ctypes.c_int), ("cols_warps", ctypes.c_int),
                ("time_warps", ctypes.c_int), ("rows_ms", ctypes.c_float * 3),
                ("cols_ms", ctypes.c_float * 3), ("time_ms", ctypes.c_float * 3),
                ("cached", ctypes.c_int)]


class BecError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: {_lib().bec_status_string(status).decode()} ({detail})")
        self.status = status


_LIB = None


def _lib():
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2002_01108_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    D = ctypes.c_void_p
    sig = {
        "bec_allocate_problem": ([ctypes.POINTER(ProblemDesc), P, ctypes.POINTER(P)], ctypes.c_int),
        "bec_set_eps": ([P, ctypes.c_double], ctypes.c_int),
        "bec_apply_A": ([P, D, D], ctypes.c_int),
        "bec_apply_P": ([P, D, D], ctypes.c_int),
        "bec_apply_Pinv": ([P, D, D], ctypes.c_int),
        "bec_build_rhs": ([P, D, D, D], ctypes.c_int),
        "bec_build_rhs_dirichlet": ([P, D, D, D, D], ctypes.c_int),
        "bec_gmres_solve": ([P, D, D, ctypes.POINTER(GmresOpts), ctypes.POINTER(GmresInfo)],
                            ctypes.c_int),
        "bec_gmres_solve_host": ([P, D, D, ctypes.POINTER(GmresOpts), ctypes.POINTER(GmresInfo)],
                                 ctypes.c_int),
        "bec_gmres_solve_host_many": ([P, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.c_int,
                                       ctypes.POINTER(GmresOpts), ctypes.POINTER(GmresInfo)],
                                      ctypes.c_int),
        "bec_true_relres": ([P, D, D, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "bec_free_problem": ([P], ctypes.c_int),
        "bec_problem_size": ([P], ctypes.c_longlong),
        "bec_kernel_launches": ([P], ctypes.c_longlong),
        "bec_status_string": ([ctypes.c_int], ctypes.c_char_p),
        "bec_last_error": ([], ctypes.c_char_p),
        "bec_profile_start": ([P, ctypes.c_int], ctypes.c_int),
        "bec_batch_create": ([ctypes.POINTER(ProblemDesc), ctypes.POINTER(ctypes.c_double),
                              ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(P)],
                             ctypes.c_int),
        "bec_batch_problem": ([P, ctypes.c_int, ctypes.POINTER(P)], ctypes.c_int),
        "bec_batch_solve": ([P, ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(GmresOpts),
                             ctypes.POINTER(GmresInfo)], ctypes.c_int),
        "bec_batch_unknowns": ([P], ctypes.c_longlong),
        "bec_batch_kernel_launches": ([P], ctypes.c_longlong),
        "bec_batch_free": ([P], ctypes.c_int),
        "bec_learned_num_weights": ([P], ctypes.c_longlong),
        "bec_learned_get_weights": ([P, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
        "bec_learned_set_weights": ([P, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
        "bec_learned_train": ([P, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_ulonglong,
                               ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "bec_learned_loss_grad": ([P, ctypes.c_int, ctypes.POINTER(ctypes.c_int), D, D,
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float)],
                                  ctypes.c_int),
        "bec_learned_fallbacks": ([P], ctypes.c_longlong),
        "bec_learned_residual_ratios": ([P, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "bec_learned_set_judge": ([P, ctypes.c_int], ctypes.c_int),
        "bec_learned_judge_radii": ([P, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "bec_autotune": ([P, ctypes.c_int, ctypes.POINTER(TuneReport)], ctypes.c_int),
        "bec_inject_fault": ([ctypes.c_int], ctypes.c_int),
        "bec_set_tiles": ([P, ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "bec_convert_to_float": ([D, D, ctypes.c_longlong, P], ctypes.c_int),
        "bec_convert_to_double": ([D, D, ctypes.c_longlong, P], ctypes.c_int),
        "bec_reciprocal_fp64": ([D, D, ctypes.c_longlong, P], ctypes.c_int),
        "bec_relres_noalloc": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                ctypes.c_double, D, D, D, P], ctypes.c_int),
        "bec_profile_stop": ([P, ctypes.POINTER(KernelTime), ctypes.c_int,
                              ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _LIB = lib
    return lib


def load():
    """Load libbec.so (raises if it is not built)."""
    return _lib()


def _check(status: int, where: str, allow=(BEC_OK,)):
    if status not in allow:
        raise BecError(status, where, _lib().bec_last_error().decode())
    return status


def _dptr(t, U: int, name: str):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float64:
        raise TypeError(f"{name} must be float64")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() != U:
        raise ValueError(f"{name} has {t.numel()} elements, expected {U}")
    return ctypes.c_void_p(t.data_ptr())


def reciprocal_fp64(x, out=None):
    """1/x by the FP64 reciprocal of the multigrid smoother (a contiguous
    float64 CUDA tensor), on the current torch stream."""
    import torch
    if not isinstance(x, torch.Tensor) or not x.is_cuda or not x.is_contiguous() \
            or x.dtype != torch.float64:
        raise TypeError("x must be a contiguous float64 CUDA tensor")
    out = torch.empty_like(x) if out is None else out
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    _check(_lib().bec_reciprocal_fp64(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                      x.numel(), st), "bec_reciprocal_fp64")
    return out


def convert(x, out=None):
    """The library's FP64 <-> FP32 conversion of a contiguous CUDA tensor
    (float64 -> float32 rounds to nearest even, float32 -> float64 is exact),
    on the current torch stream."""
    import torch
    if not isinstance(x, torch.Tensor) or not x.is_cuda or not x.is_contiguous():
        raise TypeError("x must be a contiguous CUDA tensor")
    if x.dtype == torch.float64:
        to, fn = torch.float32, "bec_convert_to_float"
    elif x.dtype == torch.float32:
        to, fn = torch.float64, "bec_convert_to_double"
    else:
        raise TypeError("x must be float32 or float64")
    if out is None:
        out = torch.empty(x.shape, dtype=to, device=x.device)
    if out.dtype != to or not out.is_contiguous() or out.numel() != x.numel():
        raise ValueError("out must be a contiguous tensor of the other precision and the same size")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    _check(getattr(_lib(), fn)(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                               x.numel(), st), fn)
    return out


class Problem:
    """One all-at-once heat problem bound to a CUDA stream (include/bec.h)."""

    def __init__(self, dim: int, nx: int, N: int, T: float = 1.0, a: float = 1.0,
                 precision: str = "fp64", max_restart: int = 30, flexible: bool = False,
                 host_io: bool = False, stream=None, route: str = "fst", a_nodes=None,
                 mg_pre: int = 0, mg_post: int = 0, mg_omega: float = 0.0,
                 net_channels: int = 0, net_fp32: bool = False, space: str = "fd",
                 scheme: str = "bdf1", wind=None, side: float = 0.0, mg_smoother: str = "jacobi"):
        import torch
        self.dim, self.nx, self.N, self.T, self.a = dim, nx, N, T, a
        self.precision = precision
        self._a_nodes = None
        a_ptr = None
        if a_nodes is not None:
            self._a_nodes = np.ascontiguousarray(a_nodes, dtype=np.float64)
            if self._a_nodes.size != (nx + 2) ** 2:
                raise ValueError("a_nodes must hold (nx+2)^2 values")
            a_ptr = self._a_nodes.ctypes.data
        self._wind = None
        w_ptr = None
        if wind is not None:
            self._wind = np.ascontiguousarray(wind, dtype=np.float64)
            if self._wind.size != 2 * (nx + 2) ** 2:
                raise ValueError("wind must hold 2 (nx+2)^2 values")
            w_ptr = self._wind.ctypes.data
        routes = {"fst": BEC_ROUTE_FST, "mg": BEC_ROUTE_MG, "learned": BEC_ROUTE_LEARNED}
        desc = ProblemDesc(dim, nx, nx if dim >= 2 else 1, N, T, a, routes[route],
                           BEC_PC_FP32 if precision == "fp32" else BEC_PC_FP64,
                           max_restart, int(flexible), int(host_io), a_ptr,
                           int(mg_pre), int(mg_post), float(mg_omega), int(net_channels),
                           int(net_fp32), {"fd": 0, "q1": 1}[space],
                           {"bdf1": 0, "bdf2": 1}[scheme], w_ptr, float(side),
                           {"jacobi": 0, "ilu": 1}[mg_smoother])
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        handle = ctypes.c_void_p(stream.cuda_stream)
        out = ctypes.c_void_p()
        _check(_lib().bec_allocate_problem(ctypes.byref(desc), handle, ctypes.byref(out)),
               "bec_allocate_problem")
        self._p = out
        self.U = int(_lib().bec_problem_size(self._p))
        self.J = self.U // N
        self.shape = (N,) + (nx,) * dim

    # -- lifetime
    def close(self):
        if getattr(self, "_p", None):
            _lib().bec_free_problem(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def launches(self) -> int:
        return int(_lib().bec_kernel_launches(self._p))

    def _new(self):
        import torch
        return torch.empty(self.shape, dtype=torch.float64, device="cuda")

    # -- entry points
    def set_eps(self, eps: float):
        _check(_lib().bec_set_eps(self._p, float(eps)), "bec_set_eps")
        self.eps = float(eps)

    def apply_A(self, v, y=None):
        y = self._new() if y is None else y
        _check(_lib().bec_apply_A(self._p, _dptr(v, self.U, "v"), _dptr(y, self.U, "y")), "bec_apply_A")
        return y

    def apply_P(self, v, y=None):
        y = self._new() if y is None else y
        _check(_lib().bec_apply_P(self._p, _dptr(v, self.U, "v"), _dptr(y, self.U, "y")), "bec_apply_P")
        return y

    def apply_Pinv(self, y, z=None):
        z = self._new() if z is None else z
        _check(_lib().bec_apply_Pinv(self._p, _dptr(y, self.U, "y"), _dptr(z, self.U, "z")),
               "bec_apply_Pinv")
        return z

    def build_rhs(self, u0, fsrc, f=None):
        f = self._new() if f is None else f
        _check(_lib().bec_build_rhs(self._p, _dptr(u0, self.J, "u0"), _dptr(fsrc, self.U, "fsrc"),
                                    _dptr(f, self.U, "f")), "bec_build_rhs")
        return f

    def build_rhs_dirichlet(self, u0, fsrc, g, f=None):
        """f with Dirichlet node values g ([N][nx+2][nx+2] on the device)."""
        f = self._new() if f is None else f
        _check(_lib().bec_build_rhs_dirichlet(self._p, _dptr(u0, self.J, "u0"),
                                              _dptr(fsrc, self.U, "fsrc"),
                                              _dptr(g, self.N * (self.nx + 2) ** 2, "g"),
                                              _dptr(f, self.U, "f")), "bec_build_rhs_dirichlet")
        return f

    @staticmethod
    def _opts(restart, maxit, rtol, flexible, left_pc, use_x0):
        return GmresOpts(int(restart), int(maxit), float(rtol), int(flexible), int(left_pc), int(use_x0))

    def gmres_solve(self, f, u=None, restart: int = 30, maxit: int = 300, rtol: float = 1e-8,
                    flexible: bool = False, left_pc: bool = False, use_x0: bool = False):
        """Returns (u, info dict).  Raises BecError except on convergence or maxit."""
        u = self._new() if u is None else u
        opts = self._opts(restart, maxit, rtol, flexible, left_pc, use_x0)
        info = GmresInfo()
        _check(_lib().bec_gmres_solve(self._p, _dptr(f, self.U, "f"), _dptr(u, self.U, "u"),
                                      ctypes.byref(opts), ctypes.byref(info)),
               "bec_gmres_solve", allow=(BEC_OK, BEC_ENOTCONV))
        return u, info.as_dict()

    def gmres_solve_host(self, f_host, u_host=None, restart: int = 30, maxit: int = 300,
                         rtol: float = 1e-8, flexible: bool = False, left_pc: bool = False,
                         use_x0: bool = False):
        """Host-buffer solve: f_host/u_host are float64 CPU tensors or arrays of U
        elements (pinned CPU tensors give the fastest copies)."""
        f_ptr, u_ptr, u_out = self._host_ptrs(f_host, u_host)
        opts = self._opts(restart, maxit, rtol, flexible, left_pc, use_x0)
        info = GmresInfo()
        _check(_lib().bec_gmres_solve_host(self._p, f_ptr, u_ptr, ctypes.byref(opts),
                                           ctypes.byref(info)),
               "bec_gmres_solve_host", allow=(BEC_OK, BEC_ENOTCONV))
        return u_out, info.as_dict()

    def gmres_solve_host_many(self, f_list, u_list=None, restart: int = 30, maxit: int = 300,
                              rtol: float = 1e-8, flexible: bool = False, left_pc: bool = False):
        """Solves len(f_list) systems from host buffers, with the copies of
        one solve overlapping the compute of its neighbours
        (bec_gmres_solve_host_many).  Returns (u_list, list of info dicts)."""
        if len(f_list) == 0:
            raise ValueError("f_list is empty")
        if u_list is None:
            u_list = [None] * len(f_list)
        if len(u_list) != len(f_list):
            raise ValueError("u_list and f_list differ in length")
        fp, up, outs = [], [], []
        for f_host, u_host in zip(f_list, u_list):
            a, b, c = self._host_ptrs(f_host, u_host)
            fp.append(a)
            up.append(b)
            outs.append(c)
        count = len(fp)
        farr = (ctypes.c_void_p * count)(*fp)
        uarr = (ctypes.c_void_p * count)(*up)
        opts = self._opts(restart, maxit, rtol, flexible, left_pc, False)
        infos = (GmresInfo * count)()
        _check(_lib().bec_gmres_solve_host_many(self._p, farr, uarr, count, ctypes.byref(opts), infos),
               "bec_gmres_solve_host_many", allow=(BEC_OK, BEC_ENOTCONV))
        return outs, [i.as_dict() for i in infos]

    def _host_ptrs(self, f_host, u_host):
        import torch

        def ptr(x, name):
            if isinstance(x, torch.Tensor):
                if x.is_cuda or x.dtype != torch.float64 or not x.is_contiguous() or x.numel() != self.U:
                    raise ValueError(f"{name} must be a contiguous float64 CPU tensor of U elements")
                return ctypes.c_void_p(x.data_ptr())
            if isinstance(x, np.ndarray):
                if x.dtype != np.float64 or not x.flags.c_contiguous or x.size != self.U:
                    raise ValueError(f"{name} must be a contiguous float64 array of U elements")
                return ctypes.c_void_p(x.ctypes.data)
            raise TypeError(f"{name} must be a torch CPU tensor or a numpy array")

        if u_host is None:
            u_host = (torch.empty(self.shape, dtype=torch.float64) if isinstance(f_host, torch.Tensor)
                      else np.empty(self.shape))
        return ptr(f_host, "f_host"), ptr(u_host, "u_host"), u_host

    def profile_start(self, capacity: int = 65536):
        """Bracket every kernel launch with CUDA events (include/bec.h)."""
        _check(_lib().bec_profile_start(self._p, int(capacity)), "bec_profile_start")

    def profile_stop(self) -> dict:
        """Synchronise and return {kernel name: (launches, total ms)}."""
        cap = 64
        buf = (KernelTime * cap)()
        n = ctypes.c_int()
        _check(_lib().bec_profile_stop(self._p, buf, cap, ctypes.byref(n)), "bec_profile_stop")
        return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].ms))
                for i in range(min(n.value, cap))}

    # -- tile shapes of the preconditioner passes
    def autotune(self, force: bool = False) -> dict:
        """Times 4, 8 and 16 warps per block for each pass and keeps the fastest."""
        r = TuneReport()
        _check(_lib().bec_autotune(self._p, int(force), ctypes.byref(r)), "bec_autotune")
        return {"rows_warps": r.rows_warps, "cols_warps": r.cols_warps, "time_warps": r.time_warps,
                "rows_ms": list(r.rows_ms), "cols_ms": list(r.cols_ms), "time_ms": list(r.time_ms),
                "cached": bool(r.cached)}

    def set_tiles(self, rows: int = 0, cols: int = 0, time: int = 0):
        _check(_lib().bec_set_tiles(self._p, int(rows), int(cols), int(time)), "bec_set_tiles")

    # -- learned correction
    def learned_weights(self):
        n = int(_lib().bec_learned_num_weights(self._p))
        w = np.empty(n, dtype=np.float32)
        _check(_lib().bec_learned_get_weights(self._p, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
               "bec_learned_get_weights")
        return w

    def set_learned_weights(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        _check(_lib().bec_learned_set_weights(self._p, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
               "bec_learned_set_weights")

    def learned_train(self, steps: int, batch: int = 16, lr: float = 1e-3, seed: int = 0):
        hist = np.zeros(steps)
        _check(_lib().bec_learned_train(self._p, int(steps), int(batch), float(lr), int(seed),
                                        hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "bec_learned_train")
        return hist

    def learned_loss_grad(self, lam_idx, r, e_target):
        """r: complex128 CUDA tensor [B][nx][nx] (fine residuals); e_target:
        complex128 CUDA tensor [B][mc][mc], mc = (nx - 1) / 2 (coarse targets)."""
        import torch
        B = len(lam_idx)
        mc = (self.nx - 1) // 2
        if tuple(r.shape) != (B, self.nx, self.nx) or tuple(e_target.shape) != (B, mc, mc):
            raise ValueError("r must be [B][nx][nx] and e_target [B][mc][mc] complex128")
        idx = (ctypes.c_int * B)(*[int(k) for k in lam_idx])
        rr = torch.view_as_real(r).contiguous()
        et = torch.view_as_real(e_target).contiguous()
        loss = ctypes.c_double()
        g = np.empty(int(_lib().bec_learned_num_weights(self._p)), dtype=np.float32)
        _check(_lib().bec_learned_loss_grad(self._p, B, idx, ctypes.c_void_p(rr.data_ptr()),
                                            ctypes.c_void_p(et.data_ptr()), ctypes.byref(loss),
                                            g.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
               "bec_learned_loss_grad")
        return loss.value, g

    @property
    def learned_fallbacks(self) -> int:
        return int(_lib().bec_learned_fallbacks(self._p))

    def set_learned_judge(self, on: bool):
        _check(_lib().bec_learned_set_judge(self._p, 1 if on else 0), "bec_learned_set_judge")

    def learned_judge_radii(self):
        """(rho_vcycle[N/2+1], rho_corrected[N/2+1], max_vcycle, max_corrected)
        of the last calibration (NaN when the judge was off)."""
        K = self.N // 2 + 1
        out = np.empty(2 * K + 2)
        _check(_lib().bec_learned_judge_radii(self._p, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "bec_learned_judge_radii")
        return out[:K], out[K:2 * K], float(out[2 * K]), float(out[2 * K + 1])

    def learned_residual_ratios(self):
        """Per frequency k <= N/2, from the calibration apply: the residual after
        the corrected step over the V-cycle's residual."""
        out = np.empty(self.N // 2 + 1)
        _check(_lib().bec_learned_residual_ratios(self._p, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "bec_learned_residual_ratios")
        return out

    def true_relres(self, f, u) -> float:
        out = ctypes.c_double()
        _check(_lib().bec_true_relres(self._p, _dptr(f, self.U, "f"), _dptr(u, self.U, "u"),
                                      ctypes.byref(out)), "bec_true_relres")
        return out.value


class Batch:
    """Independent problems of uneven size solved together (bec_batch_*).
    `specs` is a list of dicts with keys dim, nx, N, eps and optionally T, a,
    precision, max_restart, route, a_nodes.  `mode` is "streams", "graphs" or
    "persistent" (BEC_BATCH_*); without it, use_graphs picks the first two."""

    MODES = {"streams": 0, "graphs": 1, "persistent": 2}

    def __init__(self, specs, nstreams: int = 8, use_graphs: bool = True, flexible: bool = True,
                 mode: str | None = None):
        n = len(specs)
        descs = (ProblemDesc * n)()
        eps = (ctypes.c_double * n)()
        self._keep = []
        self.shapes = []
        for i, sp in enumerate(specs):
            a_ptr = None
            if sp.get("a_nodes") is not None:
                arr = np.ascontiguousarray(sp["a_nodes"], dtype=np.float64)
                self._keep.append(arr)
                a_ptr = arr.ctypes.data
            dim, nx, N = sp["dim"], sp["nx"], sp["N"]
            descs[i] = ProblemDesc(dim, nx, nx if dim >= 2 else 1, N, sp.get("T", 1.0), sp.get("a", 1.0),
                                   BEC_ROUTE_MG if sp.get("route") == "mg" else BEC_ROUTE_FST,
                                   BEC_PC_FP32 if sp.get("precision", "fp32") == "fp32" else BEC_PC_FP64,
                                   sp.get("max_restart", 10), int(flexible), 0, a_ptr, 0, 0, 0.0,
                                   0, 0, {"fd": 0, "q1": 1}[sp.get("space", "fd")],
                                   {"bdf1": 0, "bdf2": 1}[sp.get("scheme", "bdf1")])
            eps[i] = sp["eps"]
            self.shapes.append((N,) + (nx,) * dim)
        out = ctypes.c_void_p()
        m = self.MODES[mode] if mode is not None else int(bool(use_graphs))
        _check(_lib().bec_batch_create(descs, eps, n, int(nstreams), m, ctypes.byref(out)),
               "bec_batch_create")
        self._b = out
        self.count = n

    @property
    def unknowns(self) -> int:
        return int(_lib().bec_batch_unknowns(self._b))

    @property
    def launches(self) -> int:
        return int(_lib().bec_batch_kernel_launches(self._b))

    def problem_handle(self, i: int):
        out = ctypes.c_void_p()
        _check(_lib().bec_batch_problem(self._b, int(i), ctypes.byref(out)), "bec_batch_problem")
        return out

    def build_rhs(self, i: int, u0, fsrc, f):
        U = f.numel()
        _check(_lib().bec_build_rhs(self.problem_handle(i), _dptr(u0, U // self.shapes[i][0], "u0"),
                                    _dptr(fsrc, U, "fsrc"), _dptr(f, U, "f")), "bec_build_rhs")
        return f

    def solve(self, fs, us, restart: int = 10, maxit: int = 300, rtol: float = 1e-8,
              flexible: bool = True):
        n = self.count
        fp = (ctypes.c_void_p * n)(*[ctypes.c_void_p(f.data_ptr()) for f in fs])
        up = (ctypes.c_void_p * n)(*[ctypes.c_void_p(u.data_ptr()) for u in us])
        for i in range(n):
            _dptr(fs[i], fs[i].numel(), "f")
            _dptr(us[i], us[i].numel(), "u")
        opts = GmresOpts(int(restart), int(maxit), float(rtol), int(flexible), 0, 0)
        infos = (GmresInfo * n)()
        _check(_lib().bec_batch_solve(self._b, fp, up, ctypes.byref(opts), infos),
               "bec_batch_solve", allow=(BEC_OK, BEC_ENOTCONV))
        return [infos[i].as_dict() for i in range(n)]

    def close(self):
        if getattr(self, "_b", None):
            _lib().bec_batch_free(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
