"""GB300-native primal-dual affine scaling (PDAS) Newton-direction solver.

Python binding of libpdas (include/pdas.h): argument marshalling only.  Every
step of the solve runs in the library's CUDA kernels; PyTorch supplies device
memory and the stream.  Method: N. Divakar, "Primal Dual Affine Scaling on
GPUs", arXiv:1502.03543 -- the Newton system Eq. (3) reduced to
(A D A') dy = A x by Eq. (4), ds = -A' dy, dx = D(-ds) - x, then the psi ratio
test and the alpha/psi step of the algorithm in Section III.
"""
from __future__ import annotations

import ctypes

import numpy as np

import torch

from . import _native as N

__all__ = ["Solver", "BatchSolver", "WoodburySolver", "PdasError", "FORMS", "A_DTYPES", "solve_lp"]

FORMS = {"fp64": N.FP64, "tf32_ir": N.TF32_IR, "bf16_ir": N.BF16_IR, "fp32_ir": N.FP32_IR}
A_DTYPES = {torch.float64: N.A_F64, torch.float32: N.A_F32, torch.bfloat16: N.A_BF16}
STATUS_NAMES = {
    N.OK: "ok", N.OPTIMAL: "optimal", N.OPTIMAL_EXACT: "optimal_exact", N.MAX_ITER: "max_iter",
    N.STALLED: "stalled", N.ZERO_DIRECTION: "zero_direction", N.ERR_ARG: "err_arg",
    N.ERR_NOT_INTERIOR: "err_not_interior", N.ERR_NOT_SPD: "err_not_spd", N.ERR_NONFINITE: "err_nonfinite",
    N.ERR_TIMEOUT: "err_timeout", N.ERR_CUDA: "err_cuda", N.ERR_UNSUPPORTED: "err_unsupported",
}


class PdasError(RuntimeError):
    def __init__(self, code, where, detail=""):
        self.code = int(code)
        msg = "%s: %s (%d)" % (where, N.status_str(code), code)
        if detail:
            msg += ": " + detail
        super().__init__(msg)


def _ptr(t, dtype=None, numel=None, name="tensor"):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if numel is not None and t.numel() != numel:
        raise ValueError("%s must have %d elements, got %d" % (name, numel, t.numel()))
    if t.data_ptr() % 16:
        raise ValueError("%s must be 16-byte aligned" % name)
    return ctypes.c_void_p(t.data_ptr())


class Solver:
    """A libpdas handle for m x n problems (1 <= m < n).

    form: "fp64" (plain FP64), "bf16_ir", "tf32_ir" or "fp32_ir" (mixed
    precision with FP64 refinement).  a_dtype: torch dtype A is stored in.
    stream: torch.cuda.Stream (default: the current stream at construction).
    Other keyword options map to pdas_options fields."""

    def __init__(self, m, n, form="fp64", a_dtype=torch.float64, stream=None, **opts):
        self.m, self.n = int(m), int(n)
        self.form = form
        self.a_dtype = a_dtype
        lib = N.lib()
        o = N.Options()
        lib.pdas_default_options(ctypes.byref(o))
        o.form = FORMS[form]
        o.a_dtype = A_DTYPES[a_dtype]
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        o.stream = ctypes.c_void_p(self.stream.cuda_stream)
        for k, v in opts.items():
            if not hasattr(o, k) or k in ("form", "a_dtype", "stream"):
                raise TypeError("unknown option %r" % k)
            setattr(o, k, v)
        self.options = o
        h = ctypes.c_void_p()
        st = lib.pdas_create(self.m, self.n, ctypes.byref(o), ctypes.byref(h))
        if st != N.OK:
            raise PdasError(st, "pdas_create")
        self._h = h

    # -- life cycle --------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            N.lib().pdas_destroy(self._h)
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

    def _check(self, st, where, ok=(N.OK,)):
        if st not in ok:
            detail = ""
            if st == N.ERR_CUDA:
                detail = N.lib().pdas_last_error_message(self._h).decode()
            elif st == N.ERR_NOT_SPD:
                detail = "pivot %d" % N.lib().pdas_last_error_index(self._h)
            raise PdasError(st, where, detail)
        return st

    def profile_enable(self, enable=True):
        """Start (clear) or stop per-stage CUDA-event timing on the handle's stream."""
        self._check(N.lib().pdas_profile_enable(self._h, int(bool(enable))), "pdas_profile_enable")

    def profile_read(self):
        """dict(ms={stage: ms}, calls={stage: n}, launches=kernels launched)."""
        p = N.Profile()
        self._check(N.lib().pdas_profile_read(self._h, ctypes.byref(p)), "pdas_profile_read")
        return p.as_dict()

    def last_error_index(self):
        return int(N.lib().pdas_last_error_index(self._h))

    def set_wait_limit(self, microseconds):
        """Limit of the handle's bounded inter-block waits (0: the 2 s default)."""
        self._check(N.lib().pdas_set_wait_limit(self._h, int(microseconds)), "pdas_set_wait_limit")

    # -- argument marshalling ----------------------------------------------
    def _A(self, A):
        return _ptr(A, self.a_dtype, self.m * self.n, "A")

    def _vn(self, v, name):
        return _ptr(v, torch.float64, self.n, name)

    def _vm(self, v, name):
        return _ptr(v, torch.float64, self.m, name)

    # -- the algorithm -------------------------------------------------------
    def step(self, A, b, c, x, y, s, alpha=0.95, raise_on_error=True):
        """One iteration in place on (x, y, s).  Returns (status, info dict)."""
        info = N.IterInfo()
        st = N.lib().pdas_step(self._h, self._A(A), self._vm(b, "b"), self._vn(c, "c"), self._vn(x, "x"),
                               self._vm(y, "y"), self._vn(s, "s"), float(alpha), ctypes.byref(info))
        if raise_on_error:
            self._check(st, "pdas_step", ok=(N.OK, N.OPTIMAL_EXACT))
        return st, info.as_dict()

    def solve(self, A, b, c, x, y, s, alpha=0.95, tol=1e-8):
        """Run to the stop test in place on (x, y, s).  Returns dict(status,
        status_name, iters, rel_gap); errors (status < 0) are returned, not raised."""
        iters = ctypes.c_int(0)
        gap = ctypes.c_double(0.0)
        st = N.lib().pdas_solve(self._h, self._A(A), self._vm(b, "b"), self._vn(c, "c"), self._vn(x, "x"),
                                self._vm(y, "y"), self._vn(s, "s"), float(alpha), float(tol),
                                ctypes.byref(iters), ctypes.byref(gap))
        return dict(status=st, status_name=STATUS_NAMES.get(st, str(st)), iters=iters.value, rel_gap=gap.value)

    def direction(self, A, x, s):
        """Newton direction at (x, s): returns (dx, dy, ds, info dict)."""
        dev = x.device
        dx = torch.empty(self.n, dtype=torch.float64, device=dev)
        ds = torch.empty(self.n, dtype=torch.float64, device=dev)
        dy = torch.empty(self.m, dtype=torch.float64, device=dev)
        info = N.IterInfo()
        st = N.lib().pdas_direction(self._h, self._A(A), self._vn(x, "x"), self._vn(s, "s"), _ptr(dx), _ptr(dy),
                                    _ptr(ds), ctypes.byref(info))
        self._check(st, "pdas_direction")
        return dx, dy, ds, info.as_dict()

    def direction_infeasible(self, A, b, c, x, y, s):
        """Newton direction of the infeasible-start variant at (x, y, s)
        (handle created with infeasible=1): returns (dx, dy, ds, info dict)."""
        dev = x.device
        dx = torch.empty(self.n, dtype=torch.float64, device=dev)
        ds = torch.empty(self.n, dtype=torch.float64, device=dev)
        dy = torch.empty(self.m, dtype=torch.float64, device=dev)
        info = N.IterInfo()
        st = N.lib().pdas_direction_infeasible(self._h, self._A(A), self._vm(b, "b"), self._vn(c, "c"),
                                               self._vn(x, "x"), self._vm(y, "y"), self._vn(s, "s"), _ptr(dx),
                                               _ptr(dy), _ptr(ds), ctypes.byref(info))
        self._check(st, "pdas_direction_infeasible")
        return dx, dy, ds, info.as_dict()

    def backward(self, A, x, y, s, dL_dx, want_dA=True):
        """Sensitivities of L(x*) at the final iterate (x, y, s): returns
        (dL/dA or None, dL/db, dL/dc), FP64 (pdas_backward)."""
        dev = dL_dx.device
        dA = torch.empty(self.m * self.n, dtype=torch.float64, device=dev) if want_dA else None
        db = torch.empty(self.m, dtype=torch.float64, device=dev)
        dc = torch.empty(self.n, dtype=torch.float64, device=dev)
        st = N.lib().pdas_backward(self._h, self._A(A), self._vn(x, "x"), self._vm(y, "y"), self._vn(s, "s"),
                                   self._vn(dL_dx, "dL_dx"), _ptr(dA) if want_dA else None, _ptr(db), _ptr(dc))
        self._check(st, "pdas_backward")
        return (dA.view(self.m, self.n) if want_dA else None), db, dc

    # -- components ----------------------------------------------------------
    def form_normal(self, A, x, s):
        self._check(N.lib().pdas_form_normal(self._h, self._A(A), self._vn(x, "x"), self._vn(s, "s")),
                    "pdas_form_normal")

    def copy_matrix(self, device="cuda"):
        """The workspace matrix (M or its factor L) as an m x m tensor."""
        out = torch.empty(self.m * self.m, dtype=torch.float64, device=device)
        dt = ctypes.c_int(0)
        self._check(N.lib().pdas_copy_matrix(self._h, _ptr(out), ctypes.byref(dt)), "pdas_copy_matrix")
        if dt.value == N.A_F32:
            out = out.view(torch.float32)[: self.m * self.m].clone()
        return out.view(self.m, self.m)

    def load_matrix(self, M):
        dtype = {torch.float64: N.A_F64, torch.float32: N.A_F32}[M.dtype]
        self._check(N.lib().pdas_load_matrix(self._h, _ptr(M, numel=self.m * self.m), dtype), "pdas_load_matrix")

    def factor(self, raise_on_error=True):
        st = N.lib().pdas_factor(self._h)
        if raise_on_error:
            self._check(st, "pdas_factor")
        return st

    def factor_solve(self, rhs):
        out = torch.empty_like(rhs)
        self._check(N.lib().pdas_factor_solve(self._h, self._vm(rhs, "rhs"), _ptr(out)), "pdas_factor_solve")
        return out

    def gemv(self, A, v):
        out = torch.empty(self.m, dtype=torch.float64, device=v.device)
        self._check(N.lib().pdas_gemv(self._h, self._A(A), self._vn(v, "v"), _ptr(out)), "pdas_gemv")
        return out

    def gemv_t(self, A, u):
        out = torch.empty(self.n, dtype=torch.float64, device=u.device)
        self._check(N.lib().pdas_gemv_t(self._h, self._A(A), self._vm(u, "u"), _ptr(out)), "pdas_gemv_t")
        return out


class _LPSolve(torch.autograd.Function):
    """x* = PDAS solution of min c'x s.t. Ax = b, x >= 0 from (x0, y0, s0);
    its backward is pdas_backward (implicit differentiation at the final
    iterate with x.*s held fixed)."""

    @staticmethod
    def forward(ctx, A, b, c, x0, y0, s0, solver, alpha, tol):
        x, y, s = x0.detach().clone(), y0.detach().clone(), s0.detach().clone()
        out = solver.solve(A.detach(), b.detach(), c.detach(), x, y, s, alpha=alpha, tol=tol)
        if out["status"] < 0:
            raise PdasError(out["status"], "pdas_solve")
        ctx.solver = solver
        ctx.save_for_backward(A, x, y, s)
        return x

    @staticmethod
    def backward(ctx, gx):
        A, x, y, s = ctx.saved_tensors
        dA, db, dc = ctx.solver.backward(A.detach(), x, y, s, gx.detach().contiguous().double(),
                                         want_dA=ctx.needs_input_grad[0])
        if dA is not None:
            dA = dA.to(A.dtype)
        return dA, db, dc, None, None, None, None, None, None


class BatchSolver:
    """A libpdas batch handle (pdas_batch.h): count small LPs solved together,
    one CTA per LP, replayed as one CUDA graph.

    A: packed float32 CUDA tensor (A_i row-major, in LP order); b, c, x, y, s:
    packed float64 CUDA tensors (lpgen.pack gives the layout).  The tensors
    are bound to the handle: it keeps references to them until close();
    (x, y, s) is updated in place by solve()."""

    def __init__(self, m, n, A, b, c, x, y, s, alpha=0.95, tol=1e-7, max_iter=500, refine_tol=1e-14,
                 refine_max=40, autotune=True, stream=None):
        lib = N.lib()
        self.m = np.ascontiguousarray(m, dtype=np.int32)
        self.n = np.ascontiguousarray(n, dtype=np.int32)
        self.count = int(self.m.size)
        mt, nt, at = int(self.m.sum()), int(self.n.sum()), int((self.m.astype(np.int64) * self.n).sum())
        self._bufs = (A, b, c, x, y, s)
        ptrs = [_ptr(A, torch.float32, at, "A"), _ptr(b, torch.float64, mt, "b"), _ptr(c, torch.float64, nt, "c"),
                _ptr(x, torch.float64, nt, "x"), _ptr(y, torch.float64, mt, "y"), _ptr(s, torch.float64, nt, "s")]
        o = N.BatchOptions()
        lib.pdas_batch_default_options(ctypes.byref(o))
        o.alpha, o.tol, o.max_iter, o.refine_tol, o.refine_max = alpha, tol, max_iter, refine_tol, refine_max
        o.autotune = 1 if autotune else 0
        self.stream = stream
        o.stream = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
        h = ctypes.c_void_p()
        st = lib.pdas_batch_create(self.count, self.m.ctypes.data_as(ctypes.c_void_p),
                                   self.n.ctypes.data_as(ctypes.c_void_p), *ptrs, ctypes.byref(o), ctypes.byref(h))
        if st != N.OK:
            raise PdasError(st, "pdas_batch_create")
        self._h = h

    def solve(self):
        """Runs every LP to its stop: dict of per-LP status, iters, gap, FP64-tier
        and unrefined iteration counts (numpy) and the device time in ms."""
        status = np.zeros(self.count, dtype=np.int32)
        iters = np.zeros(self.count, dtype=np.int32)
        gap = np.zeros(self.count, dtype=np.float64)
        cp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        st = N.lib().pdas_batch_solve(self._h, cp(status), cp(iters), cp(gap))
        if st != N.OK:
            raise PdasError(st, "pdas_batch_solve", N.lib().pdas_batch_last_error_message(self._h).decode())
        fp64 = np.zeros(self.count, dtype=np.int32)
        unrefined = np.zeros(self.count, dtype=np.int32)
        time_us = np.zeros(self.count, dtype=np.float32)
        N.lib().pdas_batch_diagnostics(self._h, cp(fp64), cp(unrefined), cp(time_us))
        return dict(status=status, iters=iters, gap=gap, fp64_iters=fp64, unrefined=unrefined, time_us=time_us,
                    ms=N.lib().pdas_batch_last_ms(self._h))

    def backward(self, dL_dx, want_dA=True):
        """Sensitivities at every LP's final iterate (pdas_batch_backward):
        dL_dx packed like x; returns (dL_dA packed like A in FP64 or None,
        dL_db packed like b, dL_dc packed like c, per-LP status array)."""
        mt, nt = int(self.m.sum()), int(self.n.sum())
        at = int((self.m.astype(np.int64) * self.n).sum())
        dev = dL_dx.device
        dA = torch.empty(at, dtype=torch.float64, device=dev) if want_dA else None
        db = torch.empty(mt, dtype=torch.float64, device=dev)
        dc = torch.empty(nt, dtype=torch.float64, device=dev)
        status = np.zeros(self.count, dtype=np.int32)
        st = N.lib().pdas_batch_backward(self._h, _ptr(dL_dx, torch.float64, nt, "dL_dx"),
                                         _ptr(dA) if want_dA else None, _ptr(db), _ptr(dc),
                                         status.ctypes.data_as(ctypes.c_void_p))
        if st != N.OK:
            raise PdasError(st, "pdas_batch_backward", N.lib().pdas_batch_last_error_message(self._h).decode())
        return dA, db, dc, status

    def config(self):
        """The buckets: list of (m bound, CTA threads, LP count)."""
        k = 8
        mb, th, ct = (np.zeros(k, dtype=np.int32) for _ in range(3))
        cp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        nb = N.lib().pdas_batch_config(self._h, cp(mb), cp(th), cp(ct), k)
        return [(int(mb[i]), int(th[i]), int(ct[i])) for i in range(min(nb, k))]

    def close(self):
        if getattr(self, "_h", None):
            N.lib().pdas_batch_destroy(self._h)
            self._h = None
            self._bufs = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_lp(A, b, c, x0, y0, s0, solver, alpha=0.95, tol=1e-8):
    """Differentiable LP solve through libpdas: returns x*; gradients with
    respect to A, b, c come from the adjoint at the final iterate."""
    return _LPSolve.apply(A, b, c, x0, y0, s0, solver, alpha, tol)


class WoodburySolver:
    """A libpdas Woodbury handle (pdas_woodbury.h): the paper's own solver of
    (A D A') x = r, the Egidi-Maponi rank-one recurrence from (A A')^{-1} A,
    for comparison with the Cholesky path.  prepare(A) once per A, then
    solve(A, D, r) -> (x, smallest |den_l|)."""

    def __init__(self, m, n, a_dtype=torch.float64, stream=None):
        self.m, self.n, self.a_dtype = int(m), int(n), a_dtype
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        st = N.lib().pdas_woodbury_create(self.m, self.n, A_DTYPES[a_dtype], ctypes.c_void_p(self.stream.cuda_stream),
                                          ctypes.byref(h))
        if st != N.OK:
            raise PdasError(st, "pdas_woodbury_create")
        self._h = h

    def _check(self, st, where):
        if st != N.OK:
            detail = N.lib().pdas_woodbury_last_error_message(self._h).decode() if st == N.ERR_CUDA else ""
            raise PdasError(st, where, detail)

    def prepare(self, A):
        self._check(N.lib().pdas_woodbury_prepare(self._h, _ptr(A, self.a_dtype, self.m * self.n, "A")),
                    "pdas_woodbury_prepare")

    def solve(self, A, D, r):
        x = torch.empty(self.m, dtype=torch.float64, device=r.device)
        den = ctypes.c_double(0.0)
        self._check(N.lib().pdas_woodbury_solve(self._h, _ptr(A, self.a_dtype, self.m * self.n, "A"),
                                                _ptr(D, torch.float64, self.n, "D"),
                                                _ptr(r, torch.float64, self.m, "r"), _ptr(x), ctypes.byref(den)),
                    "pdas_woodbury_solve")
        return x, den.value

    def close(self):
        if getattr(self, "_h", None):
            N.lib().pdas_woodbury_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
