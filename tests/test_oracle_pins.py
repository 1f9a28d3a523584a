"""Pins for the FP64 CPU oracle: each check ties an oracle function to
something other than the oracle itself -- a hand-solved LP, brute-force basis
enumeration, the m=1 closed form, the identities that Eq. (3) fixes, the
Sherman-Morrison recurrence of Section V-A used as an independent solver, the
exact gap recurrence of a feasible step, the full Newton system of the
infeasible-start variant solved by LAPACK, and library routines for the
special cases.  ``test_planted_mistakes_fail_a_pin`` compiles mutated copies of the C
oracle and checks that each planted mistake trips at least one pin.
"""
import itertools
import os
import subprocess
import sys

import numpy as np
import pytest
import scipy.linalg as sl

import lpgen
import oracle
from conftest import ROOT, load_fixture

ALPHA = 0.95


# ---------------------------------------------------------------------------
# independent references (never call the oracle)
# ---------------------------------------------------------------------------

def brute_force_optimum(A, b, c):
    """Minimum of c'x over the basic feasible solutions of A x = b, x >= 0
    (the optimum of a bounded LP is attained at a vertex, Section II)."""
    m, n = A.shape
    best, best_basis = np.inf, None
    for basis in itertools.combinations(range(n), m):
        B = A[:, basis]
        if abs(np.linalg.det(B)) <= 1e-12:
            continue
        xB = np.linalg.solve(B, b)
        if np.all(xB >= -1e-12):
            val = float(c[list(basis)] @ xB)
            if val < best:
                best, best_basis = val, basis
    return best, best_basis


def sherman_morrison_dy(A, D, r):
    """(A D A') dy = r by the rank-one recurrence of Section V-A:
    A D A' = A A' + sum_l u_l v_l' with u_l = a_l (column l of A) and
    v_l = (D_l - 1) a_l, starting from Y = (A A')^{-1} A and x_0 = (A A')^{-1} r.
    Returns dy and the smallest |1 + v_l' y_{l-1,l}| seen."""
    m, n = A.shape
    G = A @ A.T
    Y = np.linalg.solve(G, A)
    xl = np.linalg.solve(G, r)
    min_den = np.inf
    for l in range(n):
        v = (D[l] - 1.0) * A[:, l]
        yl = Y[:, l].copy()
        den = 1.0 + v @ yl
        min_den = min(min_den, abs(den))
        xl = xl - (v @ xl) / den * yl
        if l + 1 < n:
            coef = (v @ Y[:, l + 1:]) / den
            Y[:, l + 1:] -= np.outer(yl, coef)
    return xl, min_den


# ---------------------------------------------------------------------------
# pins: each returns (ok, detail) for a given compiled oracle
# ---------------------------------------------------------------------------

def pin_textbook_lp(o):
    g = load_fixture("lp_2x4_hand.txt")
    m, n = int(g["m"][0]), int(g["n"][0])
    A = np.array(g["A"]).reshape(m, n)
    res = o.solve(A, g["b"], g["c"], g["x0"], g["y0"], g["s0"], alpha=ALPHA, tol=1e-10)
    obj = float(np.dot(g["c"], res["x"]))
    ok = (res["status"] in (oracle.OPTIMAL, oracle.OPTIMAL_EXACT)
          and abs(obj - g["objective"][0]) <= 1e-8 * (1 + abs(g["objective"][0]))
          and np.abs(res["x"] - g["x_opt"]).max() <= 1e-6
          and np.abs(res["y"] - g["y_opt"]).max() <= 1e-6
          and np.abs(res["s"] - g["s_opt"]).max() <= 1e-6)
    return ok, "status=%d obj=%.12g x=%s y=%s" % (res["status"], obj, res["x"], res["y"])


def pin_full_step_branch(o):
    """psi = 1 (Section III): step length 1, stop, and the iterate is the
    optimal vertex; the fixture's arithmetic is exact, so the check is too."""
    g = load_fixture("lp_2x4_one_step.txt")
    m, n = int(g["m"][0]), int(g["n"][0])
    A = np.array(g["A"]).reshape(m, n)
    res = o.solve(A, g["b"], g["c"], g["x0"], g["y0"], g["s0"], alpha=ALPHA, tol=1e-8)
    tr = res["trace"]
    ok = (res["status"] == oracle.OPTIMAL_EXACT and res["iters"] == int(g["iters"][0])
          and tr[0, 0] == g["psi"][0] and tr[0, 1] == 1.0
          and np.array_equal(res["x"], g["x_opt"]) and np.array_equal(res["y"], g["y_opt"])
          and np.array_equal(res["s"], g["s_opt"]))
    return ok, "status=%d iters=%d x=%s" % (res["status"], res["iters"], res["x"])


TINY = [(1, 3), (2, 5), (3, 7), (4, 8), (3, 6), (2, 8)]


def pin_brute_force(o, seeds=(0, 1, 2)):
    details = []
    ok = True
    for (m, n), seed in itertools.product(TINY, seeds):
        lp = lpgen.generate(m, n, seed=seed)
        res = o.solve(lp.A64, lp.b, lp.c, lp.x0, lp.y0, lp.s0, alpha=ALPHA, tol=1e-8)
        cx = float(lp.c @ res["x"])
        opt, basis = brute_force_optimum(lp.A64, lp.b, lp.c)
        # weak duality: c'x >= opt >= b'y, and c'x - b'y < tol (1 + |c'x|) at the stop
        good = (res["status"] in (oracle.OPTIMAL, oracle.OPTIMAL_EXACT)
                and abs(cx - opt) <= 1e-8 * (1 + abs(cx)) + 1e-12)
        # the oracle's final iterate sits at the optimal vertex
        xb = np.zeros(n)
        xb[list(basis)] = np.linalg.solve(lp.A64[:, basis], lp.b)
        good = good and np.abs(res["x"] - xb).max() <= 1e-5 * (1 + np.abs(xb).max())
        # and the optimal basis is dual feasible (reduced costs >= 0)
        yb = np.linalg.solve(lp.A64[:, basis].T, lp.c[list(basis)])
        good = good and (lp.c - lp.A64.T @ yb).min() >= -1e-10
        ok &= bool(good)
        if not good:
            details.append("m=%d n=%d seed=%d status=%d cx=%.12g opt=%.12g" % (m, n, seed, res["status"], cx, opt))
    return ok, "; ".join(details)


def pin_m1_closed_form(o):
    """m = 1: min c'x s.t. a'x = b, x >= 0 is attained at x = (b/a_j) e_j with
    the smallest c_j b / a_j over the j with a_j b > 0."""
    ok, det = True, []
    for n, seed in [(2, 0), (5, 1), (9, 2), (16, 3)]:
        lp = lpgen.generate(1, n, seed=seed)
        a, bb = lp.A64[0], lp.b[0]
        cand = [lp.c[j] * bb / a[j] for j in range(n) if a[j] * bb > 0]
        opt = min(cand)
        res = o.solve(lp.A64, lp.b, lp.c, lp.x0, lp.y0, lp.s0, alpha=ALPHA, tol=1e-10)
        cx = float(lp.c @ res["x"])
        good = abs(cx - opt) <= 1e-9 * (1 + abs(opt))
        ok &= good
        det.append("n=%d cx=%.12g opt=%.12g" % (n, cx, opt))
    return ok, "; ".join(det)


def _iterates_of(o, lp, k_max=None):
    res = o.solve(lp.A64, lp.b, lp.c, lp.x0, lp.y0, lp.s0, alpha=ALPHA, tol=1e-8, keep_iterates=True)
    m, n = lp.m, lp.n
    pts = [(lp.x0, lp.y0, lp.s0)]
    for row in res["iterates"]:
        pts.append((row[:n], row[n:n + m], row[n + m:]))
    return res, pts[:k_max] if k_max else pts


def pin_newton_identities(o, m=12, n=30, seed=4):
    """The direction solves Eq. (3): A dx = 0, A' dy + ds = 0, S dx + X ds = -Xs;
    hence dx_j/x_j + ds_j/s_j = -1 and dx'ds = 0."""
    lp = lpgen.generate(m, n, seed=seed)
    A = lp.A64
    res, pts = _iterates_of(o, lp)
    worst = dict(Adx=0.0, dual=0.0, comp=0.0, ratio=0.0, orth=0.0)
    for (x, y, s) in pts[:-1][:8]:
        d = o.direction(A, x, s)
        dx, dy, ds = d["dx"], d["dy"], d["ds"]
        worst["Adx"] = max(worst["Adx"], np.abs(A @ dx).max() / (np.abs(A).max() * np.abs(dx).max() * n))
        worst["dual"] = max(worst["dual"], np.abs(A.T @ dy + ds).max() / (np.abs(A).max() * np.abs(dy).max() * m))
        worst["comp"] = max(worst["comp"], np.abs(s * dx + x * ds + x * s).max() / np.abs(x * s).max())
        worst["ratio"] = max(worst["ratio"], np.abs(dx / x + ds / s + 1.0).max())
        worst["orth"] = max(worst["orth"], abs(dx @ ds) / (np.linalg.norm(dx) * np.linalg.norm(ds)))
    ok = (worst["Adx"] < 1e-10 and worst["dual"] < 1e-13 and worst["comp"] < 1e-12 and worst["ratio"] < 1e-10
          and worst["orth"] < 1e-10)
    return ok, str(worst)


def pin_sherman_morrison(o):
    """Section V-A's rank-one recurrence, run independently, gives the same dy
    at early, well-conditioned iterates."""
    ok, det = True, []
    for (m, n, seed) in [(4, 10, 0), (6, 15, 1), (8, 20, 2)]:
        lp = lpgen.generate(m, n, seed=seed)
        _, pts = _iterates_of(o, lp, k_max=3)
        for (x, y, s) in pts:
            d = o.direction(lp.A64, x, s)
            D = x / s
            dy_sm, min_den = sherman_morrison_dy(lp.A64, D, lp.A64 @ x)
            if min_den < 1e-3:  # an indefinite intermediate matrix: recurrence unreliable
                continue
            err = np.abs(d["dy"] - dy_sm).max() / np.abs(dy_sm).max()
            ok &= err < 1e-9
            det.append("%.1e" % err)
    return ok and len(det) >= 5, " ".join(det)


def pin_normal_matrix(o):
    """M = A D A' against a library matrix product, entry by entry; rows only."""
    rng = np.random.default_rng(7)
    ok, det = True, []
    for m, n in [(1, 3), (5, 17), (33, 70)]:
        A = rng.standard_normal((m, n))
        D = rng.uniform(0.01, 100.0, n)
        M = o.normal_matrix(A, D)
        ref = (A * D) @ A.T
        err = np.abs(M - ref).max() / np.abs(ref).max()
        sym = np.array_equal(M, M.T)
        e = o.normal_entry(A, D, m - 1, 0)
        rows = o.normal_rows(A, D, m // 2, m)
        rows_ok = (np.isnan(rows[: m // 2]).all()
                   and np.allclose(np.tril(rows[m // 2:]), np.tril(ref[m // 2:]), rtol=1e-12, atol=1e-12 * np.abs(ref).max()))
        ok &= err < 1e-13 and sym and abs(e - ref[m - 1, 0]) <= 1e-13 * np.abs(ref).max() and rows_ok
        det.append("m=%d err=%.1e sym=%s rows=%s" % (m, err, sym, rows_ok))
    return ok, "; ".join(det)


def pin_cholesky(o):
    """L L' = M against a library Cholesky; a planted non-positive pivot is
    reported at its index."""
    rng = np.random.default_rng(8)
    ok, det = True, []
    for m in (1, 7, 40):
        G = rng.standard_normal((m, 3 * m))
        M = G @ G.T
        L, fail = o.cholesky(M)
        ref = np.linalg.cholesky(M)
        err = np.abs(L - ref).max() / np.abs(ref).max()
        ok &= fail == -1 and err < 1e-12 and np.all(np.triu(L, 1) == 0)
        det.append("m=%d err=%.1e" % (m, err))
    Mbad = np.diag([4.0, 1.0, -2.0, 3.0])
    _, fail = o.cholesky(Mbad)
    ok &= fail == 2
    G = rng.standard_normal((5, 9))
    G[3] = 0.0  # rank deficient: row and pivot 3 are exactly zero
    _, fail2 = o.cholesky(G @ G.T)
    ok &= fail2 == 3
    det.append("planted fail=%d rank-deficient fail=%d" % (fail, fail2))
    return ok, "; ".join(det)


def pin_triangular(o):
    rng = np.random.default_rng(9)
    ok, det = True, []
    for m in (1, 6, 50):
        L = np.tril(rng.standard_normal((m, m))) + np.diag(rng.uniform(2, 3, m))
        v = rng.standard_normal(m)
        z = o.forward(L, v)
        y = o.backward(L, v)
        ez = np.abs(z - sl.solve_triangular(L, v, lower=True)).max()
        ey = np.abs(y - sl.solve_triangular(L, v, lower=True, trans="T")).max()
        ok &= ez < 1e-11 and ey < 1e-11
        det.append("m=%d %.1e %.1e" % (m, ez, ey))
    return ok, "; ".join(det)


def pin_gemv(o):
    rng = np.random.default_rng(10)
    A = rng.standard_normal((13, 29))
    v, u = rng.standard_normal(29), rng.standard_normal(13)
    e1 = np.abs(o.gemv(A, v) - A @ v).max()
    e2 = np.abs(o.gemv_t(A, u) - A.T @ u).max()
    return e1 < 1e-12 and e2 < 1e-12, "%.1e %.1e" % (e1, e2)


def pin_psi_theta_step(o):
    """psi is the largest of the ratios -dx_j/x_j, -ds_j/s_j; theta = alpha/psi
    unless psi <= 1; the step adds theta times the direction."""
    x = np.array([1.0, 2.0, 4.0])
    s = np.array([2.0, 1.0, 0.5])
    dx = np.array([-0.5, 1.0, -6.0])  # ratios 0.5, -0.5, 1.5
    ds = np.array([-1.0, -2.5, 0.1])  # ratios 0.5, 2.5, -0.2
    p = o.psi(x, s, dx, ds)
    ok = p == 2.5
    ok &= o.theta(2.5, ALPHA) == ALPHA / 2.5 and o.theta(1.0, ALPHA) == 1.0 and o.theta(0.7, ALPHA) == 1.0
    y, dy = np.array([1.0, -1.0]), np.array([0.5, 0.25])
    x1, y1, s1 = o.step(x, y, s, dx, dy, ds, 0.5)
    ok &= np.array_equal(x1, x + 0.5 * dx) and np.array_equal(y1, y + 0.5 * dy) and np.array_equal(s1, s + 0.5 * ds)
    D = o.scaling(x, s)
    ok &= np.array_equal(D, x / s)
    g = o.rel_gap(np.array([1.0, 2.0]), np.array([3.0, 1.0, 1.0]), np.array([1.0, 1.0, 1.0]), np.array([0.5, 0.5]))
    ok &= abs(g - (5.0 - 1.5) / 6.0) < 1e-15
    return ok, "psi=%r" % p


def pin_run_invariants(o, seeds=(0, 1)):
    """Along a run at 64 x 128: x, s > 0; psi >= 1/2; dual feasibility exact;
    primal drift bounded (it is the accumulated solve residual: A dx = M dy - r);
    the complementarity product obeys the step recurrence; the gap ends
    below tol."""
    ok, det = True, []
    for seed in seeds:
        lp = lpgen.workload("dense_64x128_f64", seed)
        res, pts = _iterates_of(o, lp)
        tr = res["trace"]
        psi_ok = bool(np.all(tr[:, 0] >= 0.5 - 1e-12))
        pos_ok = all(np.all(x > 0) and np.all(s > 0) for (x, y, s) in pts[:-1])
        dual = max(np.linalg.norm(lp.A64.T @ y + s - lp.c) / np.linalg.norm(lp.c) for (x, y, s) in pts)
        primal = max(np.linalg.norm(lp.A64 @ x - lp.b) / np.linalg.norm(lp.b) for (x, y, s) in pts)
        # x's after a step of length theta is (1 - theta) x's + theta^2 dx'ds
        # (third row of Eq. (3)); dx'ds = dy'(r - M dy) is the solve's
        # residual, so it is added back rather than assumed zero.
        rec = 0.0
        for k in range(len(pts) - 1):
            d = o.direction(lp.A64, pts[k][0], pts[k][2])
            xs0 = pts[k][0] @ pts[k][2]
            xs1 = pts[k + 1][0] @ pts[k + 1][2]
            th = tr[k, 1]
            rec = max(rec, abs(xs1 - (1 - th) * xs0 - th * th * (d["dx"] @ d["ds"])) / xs0)
        good = (res["status"] == oracle.OPTIMAL and psi_ok and pos_ok and dual < 1e-13 and primal < 1e-9
                and rec < 1e-13 and tr[-1, 2] < 1e-8)
        ok &= good
        det.append("seed=%d iters=%d dual=%.1e primal=%.1e rec=%.1e" % (seed, res["iters"], dual, primal, rec))
    return ok, "; ".join(det)


def pin_backward_error(o, seed=0):
    """Each Newton system is solved to a normwise backward error
    ||M dy - r|| / (||M|| ||dy|| + ||r||) below 1e-12."""
    lp = lpgen.workload("dense_64x128_f64", seed)
    res, pts = _iterates_of(o, lp)
    worst = 0.0
    for (x, y, s) in pts[:-1]:
        d = o.direction(lp.A64, x, s)
        M = (lp.A64 * d["D"]) @ lp.A64.T
        be = np.abs(M @ d["dy"] - d["r"]).max() / (np.abs(M).sum(1).max() * np.abs(d["dy"]).max()
                                                   + np.abs(d["r"]).max())
        worst = max(worst, be)
    return worst < 1e-12, "%.1e" % worst


def pin_not_spd(o):
    """A rank-deficient A (a zero row) makes M singular: reported, not trapped."""
    lp = lpgen.generate(4, 9, seed=3)
    A = lp.A64.copy()
    A[2] = 0.0
    b = A @ lp.x0
    c = A.T @ lp.y0 + lp.s0
    res = o.solve(A, b, c, lp.x0, lp.y0, lp.s0)
    return res["status"] == oracle.NOT_SPD and res["fail_index"] == 2, "status=%d idx=%d" % (res["status"],
                                                                                           res["fail_index"])


def infeasible_start(lp, seed):
    """A seeded interior point that satisfies neither A x = b nor A'y + s = c."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.5, 2.0, lp.n), rng.standard_normal(lp.m), rng.uniform(0.5, 2.0, lp.n)


def pin_infeasible_newton_system(o, m=4, n=9, seed=6):
    """Infeasible-start variant: the direction is the solution of the full
    (2n + m) x (2n + m) Newton system of Eq. (3) with the residuals
    b - A x and c - A'y - s on its right-hand side, solved here by LAPACK
    (numpy.linalg.solve), at an infeasible point and along a run."""
    lp = lpgen.generate(m, n, seed=seed)
    A = lp.A64
    x, y, s = infeasible_start(lp, seed)
    worst = 0.0
    for _ in range(4):
        K = np.zeros((2 * n + m, 2 * n + m))
        K[:m, :n] = A                                  # A dx            = b - A x
        K[m:m + n, n:n + m] = A.T                      # A' dy + ds      = c - A'y - s
        K[m:m + n, n + m:] = np.eye(n)
        K[m + n:, :n] = np.diag(s)                     # S dx + X ds     = -X s
        K[m + n:, n + m:] = np.diag(x)
        rhs = np.concatenate([lp.b - A @ x, lp.c - A.T @ y - s, -x * s])
        ref = np.linalg.solve(K, rhs)
        d = o.direction_infeasible(A, lp.b, lp.c, x, y, s)
        got = np.concatenate([d["dx"], d["dy"], d["ds"]])
        worst = max(worst, np.abs(got - ref).max() / np.abs(ref).max())
        th = 0.5 / max(np.max(-d["dx"] / x), np.max(-d["ds"] / s), 1.0)
        x, y, s = x + th * d["dx"], y + th * d["dy"], s + th * d["ds"]
    return worst < 1e-10, "%.1e" % worst


def pin_infeasible_feasible_start(o, seed=2):
    """From a feasible start the variant's system is the paper's: the same
    direction as ``direction`` to rounding."""
    lp = lpgen.generate(10, 25, seed=seed)
    d0 = o.direction(lp.A64, lp.x0, lp.s0)
    d1 = o.direction_infeasible(lp.A64, lp.b, lp.c, lp.x0, lp.y0, lp.s0)
    err = max(np.abs(d1[k] - d0[k]).max() / np.abs(d0[k]).max() for k in ("dx", "dy", "ds"))
    return err < 1e-11, "%.1e" % err


def pin_infeasible_runs(o, seeds=(0, 1, 2)):
    """Runs of the variant from infeasible points: the residuals shrink by
    (1 - theta_k) per step (the first two rows of Eq. (3); up to the solve's
    residual, which grows with max D / min D near the optimum), the
    iterate keeps at least the fraction 1 - alpha of each coordinate, and the
    run ends at the brute-force optimal vertex with both residuals (computed
    here) below tol."""
    ok, det = True, []
    # starts in [0.5, 2], and starts scaled by 0.1 (y = 0) that are still far
    # from feasible when the gap first falls below tol
    cases = [((m, n), seed, 1.0, 1e-9) for (m, n), seed in itertools.product(TINY, seeds)]
    cases += [((1, 3), 1, 0.1, 1e-6), ((4, 8), 0, 0.1, 1e-6), ((2, 8), 0, 0.1, 1e-6)]
    for (m, n), seed, scale, tol in cases:
        lp = lpgen.generate(m, n, seed=seed)
        x, y, s = infeasible_start(lp, 100 + seed)
        if scale != 1.0:
            x, y, s = scale * x, 0.0 * y, scale * s
        res = o.solve(lp.A64, lp.b, lp.c, x, y, s, alpha=ALPHA, tol=tol, keep_iterates=True, infeasible=True)
        pts = [(x, y, s)] + [(r[:n], r[n:n + m], r[n + m:]) for r in res["iterates"]]
        rp = [lp.b - lp.A64 @ p[0] for p in pts]
        rd = [lp.c - lp.A64.T @ p[1] - p[2] for p in pts]
        rec, frac = 0.0, True
        for k, th in enumerate(res["trace"][:, 1]):
            rec = max(rec, np.abs(rp[k + 1] - (1 - th) * rp[k]).max() / (1 + np.abs(rp[0]).max()),
                      np.abs(rd[k + 1] - (1 - th) * rd[k]).max() / (1 + np.abs(rd[0]).max()))
            frac &= bool(np.all(pts[k + 1][0] >= (1 - ALPHA) * pts[k][0] * (1 - 1e-12))
                         and np.all(pts[k + 1][2] >= (1 - ALPHA) * pts[k][2] * (1 - 1e-12)))
        opt, _ = brute_force_optimum(lp.A64, lp.b, lp.c)
        cx = float(lp.c @ res["x"])
        pres = np.abs(rp[-1]).max() / (1 + np.abs(lp.b).max())
        dres = np.abs(rd[-1]).max() / (1 + np.abs(lp.c).max())
        good = (res["status"] == oracle.OPTIMAL and rec < 1e-8 and frac and pres < tol and dres < tol
                and abs(cx - opt) <= 10 * tol * (1 + abs(opt)))
        ok &= bool(good)
        if not good:
            det.append("m=%d n=%d seed=%d status=%d rec=%.1e frac=%s pres=%.1e dres=%.1e cx=%.12g opt=%.12g"
                       % (m, n, seed, res["status"], rec, frac, pres, dres, cx, opt))
    return ok, "; ".join(det)


def pin_residuals(o, seed=3):
    """The relative residuals against numpy's products."""
    lp = lpgen.generate(7, 20, seed=seed)
    x, y, s = infeasible_start(lp, seed)
    got = o.residuals(lp.A64, lp.b, lp.c, x, y, s)
    want = (np.abs(lp.b - lp.A64 @ x).max() / (1 + np.abs(lp.b).max()),
            np.abs(lp.c - lp.A64.T @ y - s).max() / (1 + np.abs(lp.c).max()))
    err = max(abs(g - w) / w for g, w in zip(got, want))
    return err < 1e-13, "%.1e" % err


def pin_stop_rules(o, seed=5):
    """The loop's other stops (the cap of 500 and the stall rule of five steps
    shorter than 1e-12 are readings: the paper states neither).  A run capped
    at 3 iterations returns MAX_ITER after exactly 3 steps, on the uncapped
    run's third iterate bit for bit.  With alpha chosen so that every step has
    theta = alpha/psi = 0.5e-12 the run stops STALLED after exactly its fifth
    step; with theta = 2e-12 it does not stall within 8 steps (MAX_ITER).  The
    iterate barely moves at these step lengths, so psi stays within 1e-9 of
    its value at the start and theta within the factor 2 of the threshold.
    (The literal zero-direction stop cannot fire from an interior point:
    dx_j/x_j + ds_j/s_j = -1 for every j, pinned by the Newton identities.)"""
    lp = lpgen.generate(6, 15, seed=seed)
    full = o.solve(lp.A64, lp.b, lp.c, lp.x0, lp.y0, lp.s0, keep_iterates=True)
    cap = o.solve(lp.A64, lp.b, lp.c, lp.x0, lp.y0, lp.s0, max_iter=3)
    ok = full["iters"] > 3 and cap["status"] == oracle.MAX_ITER and cap["iters"] == 3
    n, m = lp.n, lp.m
    ok &= bool(np.array_equal(cap["x"], full["iterates"][2][:n]) and np.array_equal(cap["y"], full["iterates"][2][n:n + m]))
    d = o.direction(lp.A64, lp.x0, lp.s0)
    psi0 = o.psi(lp.x0, lp.s0, d["dx"], d["ds"])
    ok &= psi0 > 1.0
    lo = o.solve(lp.A64, lp.b, lp.c, lp.x0, lp.y0, lp.s0, alpha=0.5e-12 * psi0, max_iter=50)
    hi = o.solve(lp.A64, lp.b, lp.c, lp.x0, lp.y0, lp.s0, alpha=2e-12 * psi0, max_iter=8)
    ok &= lo["status"] == oracle.STALLED and lo["iters"] == 5
    ok &= hi["status"] == oracle.MAX_ITER and hi["iters"] == 8
    return ok, "cap=%d/%d lo=%d/%d hi=%d/%d psi0=%.3g" % (cap["status"], cap["iters"], lo["status"], lo["iters"],
                                                          hi["status"], hi["iters"], psi0)


PINS = [pin_textbook_lp, pin_full_step_branch, pin_brute_force, pin_m1_closed_form, pin_newton_identities, pin_sherman_morrison,
        pin_normal_matrix, pin_cholesky, pin_triangular, pin_gemv, pin_psi_theta_step, pin_run_invariants,
        pin_backward_error, pin_not_spd, pin_infeasible_newton_system, pin_infeasible_feasible_start,
        pin_infeasible_runs, pin_residuals, pin_stop_rules]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_oracle_pin(pin):
    ok, detail = pin(oracle.default)
    assert ok, detail


def test_thread_count_does_not_change_results():
    """OpenMP only splits independent outputs, so one thread and many give
    bit-identical runs."""
    code = ("import sys; sys.path.insert(0, %r); import lpgen, oracle, numpy as np;"
            "lp = lpgen.workload('dense_64x128_f64', 0);"
            "r = oracle.solve(lp.A64, lp.b, lp.c, lp.x0, lp.y0, lp.s0);"
            "sys.stdout.write(np.concatenate([r['x'], r['y'], r['s'], r['trace'].ravel()]).tobytes().hex())") % ROOT
    outs = []
    for threads in ("1", "3"):
        env = dict(os.environ, OMP_NUM_THREADS=threads)
        outs.append(subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                                   check=True).stdout)
    assert outs[0] == outs[1] and len(outs[0]) > 0


# Plausible mistakes, planted in a copy of the C source: each must fail a pin.
MUTANTS = [
    ("dx sign of x", "dx[j] = D[j] * (-ds[j]) - x[j];", "dx[j] = D[j] * (-ds[j]) + x[j];"),
    ("dx dropped term", "dx[j] = D[j] * (-ds[j]) - x[j];", "dx[j] = D[j] * (-ds[j]);"),
    ("ds sign", "ds[j] = -w[j];", "ds[j] = w[j];"),
    ("D inverted", "D[j] = x[j] / s[j];", "D[j] = s[j] / x[j];"),
    ("SYRK wrong row", "acc += (ap[j] * D[j]) * aq[j];", "acc += (ap[j] * D[j]) * ap[j];"),
    ("SYRK D dropped", "acc += (ap[j] * D[j]) * aq[j];", "acc += ap[j] * aq[j];"),
    ("rhs uses s", "or_gemv(m, n, A, x, r);", "or_gemv(m, n, A, s, r);"),
    ("cholesky wrong index", "acc -= li[k] * lj[k];", "acc -= li[k] * li[k];"),
    ("cholesky no sqrt", "const double ljj = sqrt(d);", "const double ljj = d;"),
    ("back-substitution transposed", "acc -= L[k * m + i] * y[k];", "acc -= L[i * m + k] * y[k];"),
    ("forward multiplies", "z[i] = acc / li[i];", "z[i] = acc * li[i];"),
    ("gemv_t transposed", "acc += A[p * n + j] * v[p];", "acc += A[j * m + p] * v[p];"),
    ("psi wrong scale", "double v = -ds[j] / s[j];", "double v = -ds[j] / x[j];"),
    ("psi sign", "double u = -dx[j] / x[j];", "double u = dx[j] / x[j];"),
    ("theta", "psi <= 1.0 ? 1.0 : alpha / psi", "psi <= 1.0 ? 1.0 : 1.0 / psi"),
    ("step y sign", "y[p] = y[p] + theta * dy[p];", "y[p] = y[p] - theta * dy[p];"),
    ("gap sign", "return (cx - by) / (1.0 + fabs(cx));", "return (cx + by) / (1.0 + fabs(cx));"),
    ("psi test strict", "if (psi <= 1.0) {", "if (psi < 0.0) {"),
    # the infeasible-start variant
    ("variant r_d sign of s", "rd[j] = (c[j] - w[j]) - s[j];", "rd[j] = (c[j] - w[j]) + s[j];"),
    ("variant rhs drops A D r_d", "r[p] = b[p] + z[p];", "r[p] = b[p];"),
    ("variant rhs uses A x", "r[p] = b[p] + z[p];", "r[p] = b[p] - z[p];"),
    ("variant ds drops r_d", "ds[j] = rd[j] - w[j];", "ds[j] = -w[j];"),
    ("variant u drops D", "u[j] = D[j] * rd[j];", "u[j] = rd[j];"),
    ("variant theta overshoots", "psi <= alpha ? 1.0 : alpha / psi", "psi <= 1.0 ? 1.0 : 1.0 / psi"),
    ("variant stop ignores residuals", "fabs(gap) < tol && res[0] < tol && res[1] < tol", "fabs(gap) < tol"),
    ("residual norm of b", "bn = fmax(bn, fabs(b[p]));", "bn = fmax(bn, fabs(t[p]));"),
    ("dual residual norm sign of s", "rdn = fmax(rdn, fabs((c[j] - w[j]) - s[j]));",
     "rdn = fmax(rdn, fabs((c[j] - w[j]) + s[j]));"),
    ("primal residual norm uses b only", "rp = fmax(rp, fabs(b[p] - t[p]));", "rp = fmax(rp, fabs(b[p]));"),
    ("variant theta full step at psi <= 1", "psi <= alpha ? 1.0 : alpha / psi", "psi <= 1.0 ? 1.0 : alpha / psi"),
    # the stop rules of the loop
    ("stall count", "if (small_steps >= 5) {", "if (small_steps >= 6) {"),
    ("stall threshold", "small_steps = theta < 1e-12 ? small_steps + 1 : 0;",
     "small_steps = theta < 1e-11 ? small_steps + 1 : 0;"),
    ("stall never counted", "small_steps = theta < 1e-12 ? small_steps + 1 : 0;", "small_steps = 0;"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistakes_fail_a_pin(name, old, new):
    src = open(oracle.SOURCE).read()
    assert src.count(old) == 1, "mutation anchor not found: " + old
    mutant = oracle.Oracle.from_source(src.replace(old, new))
    failed = []
    for pin in PINS:
        try:
            ok, _ = pin(mutant)
        except Exception:  # a crash (e.g. NaN into a library routine) also fails the pin
            ok = False
        if not ok:
            failed.append(pin.__name__)
            break
    assert failed, "planted mistake '%s' passed every pin" % name
