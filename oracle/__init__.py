"""FP64 CPU oracle for the primal-dual affine scaling Newton solve.

TEST INFRASTRUCTURE ONLY: this package exists so the test suite, the smoke
check and the benchmark's CPU-baseline leg can check the GPU library against
a plain, slow, obviously correct statement of the method.  The product path
(``paper_1502_03543_gb300``) never imports it, and it never imports the
product path.

The arithmetic lives in ``pdas_oracle.c`` (plain C, FP64, sums left to right,
no fused multiply-add); this module compiles it with gcc on first use and
wraps each function with ctypes.  Every function cites the passage of
N. Divakar, "Primal Dual Affine Scaling on GPUs" (arXiv:1502.03543) it
follows; the readings of garbled or silent passages are listed at the top
of ``pdas_oracle.c``.

Pins (tests/test_oracle_pins.py) tie every function here to something other
than itself: brute-force basis enumeration, the m=1 closed form, a textbook
LP solved by hand, the Newton identities of Eq. (3), the Sherman-Morrison
recurrence of Section V-A as an independent solver, the exact gap
recurrence, and library routines for the special cases (SYRK, Cholesky,
triangular solves).  The same tests compile mutated copies of the C source
(``Oracle.from_source``) to show that a planted mistake fails a pin.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "pdas_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

OPTIMAL = 1
OPTIMAL_EXACT = 2
MAX_ITER = 3
STALLED = 4
ZERO_DIRECTION = 5
NOT_SPD = -3

_lock = threading.Lock()

_I64, _F64, _I32, _P = ctypes.c_int64, ctypes.c_double, ctypes.c_int, ctypes.c_void_p
_SIGNATURES = {
    "or_threads": ([], _I32),
    "or_scaling": ([_I64, _P, _P, _P], None),
    "or_gemv": ([_I64, _I64, _P, _P, _P], None),
    "or_gemv_t": ([_I64, _I64, _P, _P, _P], None),
    "or_normal_entry": ([_I64, _I64, _P, _P, _I64, _I64], _F64),
    "or_normal_rows": ([_I64, _I64, _P, _P, _I64, _I64, _P], None),
    "or_normal_matrix": ([_I64, _I64, _P, _P, _P], None),
    "or_cholesky": ([_I64, _P, _P], _I64),
    "or_forward": ([_I64, _P, _P, _P], None),
    "or_backward": ([_I64, _P, _P, _P], None),
    "or_direction": ([_I64, _I64] + [_P] * 10, _I64),
    "or_psi": ([_I64, _P, _P, _P, _P], _F64),
    "or_theta": ([_F64, _F64], _F64),
    "or_step": ([_I64, _I64, _F64] + [_P] * 6, None),
    "or_rel_gap": ([_I64, _I64, _P, _P, _P, _P], _F64),
    "or_solve": ([_I64, _I64] + [_P] * 6 + [_F64, _F64, _I32] + [_P] * 4 + [_I32, _P], _I32),
    "or_direction_infeasible": ([_I64, _I64] + [_P] * 12, _I64),
    "or_residuals": ([_I64, _I64] + [_P] * 7, None),
    "or_theta_infeasible": ([_F64, _F64], _F64),
}


def _compile(src: str, out: str) -> None:
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
    last = ""
    for extra in (["-fopenmp"], []):
        tmp = out + ".%d.tmp" % os.getpid()
        proc = subprocess.run(base + extra + [src, "-o", tmp, "-lm"], capture_output=True, text=True)
        if proc.returncode == 0:
            os.replace(tmp, out)
            return
        last = proc.stderr
    raise RuntimeError("oracle build failed:\n" + last)


def build(force: bool = False) -> str:
    """Compile pdas_oracle.c into _build/liboracle.so (OpenMP when available)."""
    with _lock:
        if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(SOURCE):
            os.makedirs(_OUT_DIR, exist_ok=True)
            _compile(SOURCE, _LIB_PATH)
    return _LIB_PATH


def _f64(a, shape=None):
    out = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and out.shape != shape:
        raise ValueError("expected shape %s, got %s" % (shape, out.shape))
    return out


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


class Oracle:
    """One compiled copy of pdas_oracle.c: the committed one by default, or a
    mutated copy (``from_source``) in the tests that check the pins."""

    def __init__(self, lib_path: str | None = None):
        self._path = lib_path
        self._lib = None

    @classmethod
    def from_source(cls, source_text: str) -> "Oracle":
        d = tempfile.mkdtemp(prefix="oracle_variant_")
        src = os.path.join(d, "variant.c")
        with open(src, "w") as f:
            f.write(source_text)
        out = os.path.join(d, "libvariant.so")
        _compile(src, out)
        return cls(out)

    @property
    def lib(self):
        if self._lib is None:
            lib = ctypes.CDLL(self._path or build())
            for name, (args, res) in _SIGNATURES.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            self._lib = lib
        return self._lib

    def threads(self) -> int:
        """OpenMP threads the oracle uses (1 without OpenMP)."""
        return int(self.lib.or_threads())

    def scaling(self, x, s):
        """D = S^{-1} X of Eq. (4), as the n-vector x/s."""
        x = _f64(x)
        s = _f64(s, x.shape)
        D = np.empty_like(x)
        self.lib.or_scaling(x.size, _p(x), _p(s), _p(D))
        return D

    def gemv(self, A, v):
        """A v (right-hand side A x of the normal equations, Section V)."""
        A = _f64(A)
        m, n = A.shape
        v = _f64(v, (n,))
        out = np.empty(m)
        self.lib.or_gemv(m, n, _p(A), _p(v), _p(out))
        return out

    def gemv_t(self, A, v):
        """A' v (ds = -A' dy, Section V)."""
        A = _f64(A)
        m, n = A.shape
        v = _f64(v, (m,))
        out = np.empty(n)
        self.lib.or_gemv_t(m, n, _p(A), _p(v), _p(out))
        return out

    def normal_entry(self, A, D, p, q):
        """One entry M_pq = sum_j A_pj D_j A_qj of M = A D A' (Section V)."""
        A = _f64(A)
        m, n = A.shape
        return float(self.lib.or_normal_entry(m, n, _p(A), _p(_f64(D, (n,))), int(p), int(q)))

    def normal_rows(self, A, D, p0, p1):
        """Rows [p0, p1) of the lower triangle of M = A D A' in an m x m array
        (entries outside those rows, and above the diagonal, are NaN)."""
        A = _f64(A)
        m, n = A.shape
        M = np.full((m, m), np.nan)
        self.lib.or_normal_rows(m, n, _p(A), _p(_f64(D, (n,))), int(p0), int(p1), _p(M))
        return M

    def normal_matrix(self, A, D):
        """The full symmetric normal matrix M = A D A' (Section V)."""
        A = _f64(A)
        m, n = A.shape
        M = np.empty((m, m))
        self.lib.or_normal_matrix(m, n, _p(A), _p(_f64(D, (n,))), _p(M))
        return M

    def cholesky(self, M):
        """(L, fail): M = L L' from the lower triangle of M (Section V-A).
        fail = -1 on success, else the first non-positive pivot index."""
        M = _f64(M)
        m = M.shape[0]
        L = np.empty((m, m))
        fail = int(self.lib.or_cholesky(m, _p(M), _p(L)))
        return L, fail

    def forward(self, L, v):
        """Solve L z = v by forward substitution."""
        L = _f64(L)
        m = L.shape[0]
        z = np.empty(m)
        self.lib.or_forward(m, _p(L), _p(_f64(v, (m,))), _p(z))
        return z

    def backward(self, L, z):
        """Solve L' y = z by back substitution."""
        L = _f64(L)
        m = L.shape[0]
        y = np.empty(m)
        self.lib.or_backward(m, _p(L), _p(_f64(z, (m,))), _p(y))
        return y

    def direction(self, A, x, s, want_matrices=False):
        """Newton direction of Eq. (3) via Eq. (4).

        Returns a dict with dx, dy, ds, D, r (= A x), fail (-1 or the failing
        pivot index) and, if want_matrices, M and L."""
        A = _f64(A)
        m, n = A.shape
        x, s = _f64(x, (n,)), _f64(s, (n,))
        dx, ds, D = np.empty(n), np.empty(n), np.empty(n)
        dy, r = np.empty(m), np.empty(m)
        M = np.empty((m, m)) if want_matrices else None
        L = np.empty((m, m)) if want_matrices else None
        fail = int(self.lib.or_direction(m, n, _p(A), _p(x), _p(s), _p(dx), _p(dy), _p(ds), _p(D), _p(r), _p(M),
                                         _p(L)))
        out = dict(dx=dx, dy=dy, ds=ds, D=D, r=r, fail=fail)
        if want_matrices:
            out.update(M=M, L=L)
        return out

    def direction_infeasible(self, A, b, c, x, y, s):
        """Newton direction of the infeasible-start variant: Eq. (3) with the
        residuals r_p = b - A x and r_d = c - A' y - s as right-hand sides of
        its first two rows, reduced as in Section V.

        Returns a dict with dx, dy, ds, D, r (= b + A D r_d), rd (= r_d) and
        fail (-1 or the failing pivot index)."""
        A = _f64(A)
        m, n = A.shape
        b, c = _f64(b, (m,)), _f64(c, (n,))
        x, y, s = _f64(x, (n,)), _f64(y, (m,)), _f64(s, (n,))
        dx, ds, D, rd = np.empty(n), np.empty(n), np.empty(n), np.empty(n)
        dy, r = np.empty(m), np.empty(m)
        fail = int(self.lib.or_direction_infeasible(m, n, _p(A), _p(b), _p(c), _p(x), _p(y), _p(s), _p(dx), _p(dy),
                                                    _p(ds), _p(D), _p(r), _p(rd)))
        return dict(dx=dx, dy=dy, ds=ds, D=D, r=r, rd=rd, fail=fail)

    def residuals(self, A, b, c, x, y, s):
        """(||b - A x||_inf / (1 + ||b||_inf), ||c - A' y - s||_inf / (1 + ||c||_inf))."""
        A = _f64(A)
        m, n = A.shape
        out = np.empty(2)
        self.lib.or_residuals(m, n, _p(A), _p(_f64(b, (m,))), _p(_f64(c, (n,))), _p(_f64(x, (n,))),
                              _p(_f64(y, (m,))), _p(_f64(s, (n,))), _p(out))
        return float(out[0]), float(out[1])

    def theta_infeasible(self, psi_value, alpha):
        """Step length of the infeasible-start variant: min(1, alpha / psi)."""
        return float(self.lib.or_theta_infeasible(float(psi_value), float(alpha)))

    def psi(self, x, s, dx, ds):
        """psi = max{phi(-X^{-1} dx), phi(-S^{-1} ds)}, phi(u) = max_j u_j (Section III)."""
        x = _f64(x)
        n = x.size
        return float(self.lib.or_psi(n, _p(x), _p(_f64(s, (n,))), _p(_f64(dx, (n,))), _p(_f64(ds, (n,)))))

    def theta(self, psi_value, alpha):
        """Step length: 1 if psi <= 1, else alpha / psi (Section III)."""
        return float(self.lib.or_theta(float(psi_value), float(alpha)))

    def step(self, x, y, s, dx, dy, ds, theta_value):
        """(x, y, s) + theta (dx, dy, ds), returned as new arrays (Section III)."""
        x, y, s = _f64(x).copy(), _f64(y).copy(), _f64(s).copy()
        n, m = x.size, y.size
        self.lib.or_step(m, n, float(theta_value), _p(x), _p(y), _p(s), _p(_f64(dx, (n,))), _p(_f64(dy, (m,))),
                         _p(_f64(ds, (n,))))
        return x, y, s

    def rel_gap(self, b, c, x, y):
        """(c'x - b'y) / (1 + |c'x|)."""
        b, c, x, y = _f64(b), _f64(c), _f64(x), _f64(y)
        return float(self.lib.or_rel_gap(b.size, c.size, _p(b), _p(c), _p(x), _p(y)))

    def solve(self, A, b, c, x0, y0, s0, alpha=0.95, tol=1e-8, max_iter=500, keep_iterates=False,
              infeasible=False):
        """Run the Primal-Dual Affine Scaling algorithm (Section III).

        Returns a dict: status (one of the codes above), iters, x, y, s,
        trace (iters x 4: psi, theta, rel_gap after the step, max D / min D),
        fail_index and, if keep_iterates, iterates (iters x (2n+m): x | y | s
        after each step).  infeasible=True runs the infeasible-start variant
        (direction_infeasible, theta_infeasible, stop on the gap and both
        relative residuals) and adds res_trace (iters x 2: the residuals of
        ``residuals`` after each step)."""
        A = _f64(A)
        m, n = A.shape
        x, y, s = _f64(x0, (n,)).copy(), _f64(y0, (m,)).copy(), _f64(s0, (n,)).copy()
        b, c = _f64(b, (m,)), _f64(c, (n,))
        trace = np.zeros((max_iter, 4))
        its = np.zeros((max_iter, 2 * n + m)) if keep_iterates else None
        res_trace = np.zeros((max_iter, 2))
        iters = ctypes.c_int(0)
        fail = ctypes.c_int64(-1)
        status = int(self.lib.or_solve(m, n, _p(A), _p(b), _p(c), _p(x), _p(y), _p(s), float(alpha), float(tol),
                                       int(max_iter), ctypes.addressof(iters), _p(trace), _p(its),
                                       ctypes.addressof(fail), int(bool(infeasible)), _p(res_trace)))
        k = iters.value
        out = dict(status=status, iters=k, x=x, y=y, s=s, trace=trace[:k], fail_index=fail.value)
        if infeasible:
            out["res_trace"] = res_trace[:k]
        if keep_iterates:
            out["iterates"] = its[:k]
        return out


default = Oracle()
threads = default.threads
scaling = default.scaling
gemv = default.gemv
gemv_t = default.gemv_t
normal_entry = default.normal_entry
normal_rows = default.normal_rows
normal_matrix = default.normal_matrix
cholesky = default.cholesky
forward = default.forward
backward = default.backward
direction = default.direction
direction_infeasible = default.direction_infeasible
residuals = default.residuals
theta_infeasible = default.theta_infeasible
psi = default.psi
theta = default.theta
step = default.step
rel_gap = default.rel_gap
solve = default.solve
