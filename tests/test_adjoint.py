"""The adjoint pdas_backward: sensitivities of L(x*) = w'x* at a final iterate
(x, y, s), from implicit differentiation of F = [Ax - b; A'y + s - c; Xs - sigma]
= 0 with sigma = x.*s held fixed.

The reference is independent of both the oracle and the GPU path: the
perturbed system F = 0 is re-solved by undamped Newton (dense numpy, FP64)
from the final iterate, and L is differenced centrally with one Richardson
step, (4 L'(h/2) - L'(h)) / 3 at h = 1e-6: near a vertex the curvature is
strong, and the plain central difference's O(h^2) term reached 3e-4 of the
derivative at 128 x 384.  A CPU
test first pins the adjoint itself: J' (la, lb, lc) = (g, 0, 0) with J the
Jacobian of F, whose reduced form is
    (A D A') la = A D g,  lb = D (A' la - g),
    dL/db = la, dL/dc = lb, dL/dA = -(la x' + y lb'),
against those finite differences.  The GPU test then checks pdas_backward,
which solves the reduced form and refines (la, lb, lc) on the full system
(lb = D (A' la - g) alone cancels where D is large).
"""
import numpy as np
import pytest
import torch

import lpgen
import oracle


def newton_fixed_sigma(A, b, c, x, y, s, sigma, iters=30):
    """Solve Ax = b, A'y + s = c, x.*s = sigma by Newton from (x, y, s)."""
    m, n = A.shape
    x, y, s = x.copy(), y.copy(), s.copy()
    N = 2 * n + m
    for _ in range(iters):
        F = np.concatenate([A @ x - b, A.T @ y + s - c, x * s - sigma])
        if np.abs(F).max() <= 1e-15 * (1 + np.abs(b).max() + np.abs(c).max()):
            break
        J = np.zeros((N, N))
        J[:m, :n] = A
        J[m:m + n, n:n + m] = A.T
        J[m:m + n, n + m:] = np.eye(n)
        J[m + n:, :n] = np.diag(s)
        J[m + n:, n + m:] = np.diag(x)
        dz = np.linalg.solve(J, -F)
        x += dz[:n]
        y += dz[n:n + m]
        s += dz[n + m:]
    return x, y, s


def fd_directional(A, b, c, x, y, s, w, dA, db, dc, h=1e-6):
    sigma = x * s

    def central(t):
        xp = newton_fixed_sigma(A + t * dA, b + t * db, c + t * dc, x, y, s, sigma)[0]
        xm = newton_fixed_sigma(A - t * dA, b - t * db, c - t * dc, x, y, s, sigma)[0]
        return (w @ xp - w @ xm) / (2 * t)

    return (4 * central(h / 2) - central(h)) / 3


def full_adjoint(A, x, y, s, g):
    """The adjoint solved densely on the full system J' (la, lb, lc) =
    (g, 0, 0), J the Jacobian of F (the matrix of the Newton system)."""
    m, n = A.shape
    N = 2 * n + m
    J = np.zeros((N, N))
    J[:m, :n] = A
    J[m:m + n, n:n + m] = A.T
    J[m:m + n, n + m:] = np.eye(n)
    J[m + n:, :n] = np.diag(s)
    J[m + n:, n + m:] = np.diag(x)
    lam = np.linalg.solve(J.T, np.concatenate([g, np.zeros(m + n)]))
    la, lb = lam[:m], lam[m:m + n]
    return -(np.outer(la, x) + np.outer(y, lb)), la, lb


def adjoint_formulas(A, x, y, s, g):
    """full_adjoint, after checking that the reduced normal equations
    (A D A') la = A D g give the same la."""
    dA, la, lb = full_adjoint(A, x, y, s, g)
    D = x / s
    la_reduced = np.linalg.solve((A * D) @ A.T, A @ (D * g))
    assert np.linalg.norm(la - la_reduced) <= 1e-8 * np.linalg.norm(la)
    return dA, la, lb


def early_stopped(m, n, seed, tol, storage="f64"):
    lp = lpgen.generate(m, n, seed=seed, storage=storage)
    r = oracle.solve(lp.A64, lp.b, lp.c, lp.x0, lp.y0, lp.s0, tol=tol)
    return lp, r["x"], r["y"], r["s"]


def test_adjoint_formulas_match_finite_differences():
    lp, x, y, s = early_stopped(12, 30, seed=5, tol=1e-6)
    rng = np.random.default_rng(0)
    w = rng.standard_normal(lp.n)
    dLdA, dLdb, dLdc = adjoint_formulas(lp.A64, x, y, s, w)
    for _ in range(3):
        dA, db, dc = rng.standard_normal(lp.A64.shape), rng.standard_normal(lp.m), rng.standard_normal(lp.n)
        fd_b = fd_directional(lp.A64, lp.b, lp.c, x, y, s, w, 0 * dA, db, 0 * dc)
        fd_c = fd_directional(lp.A64, lp.b, lp.c, x, y, s, w, 0 * dA, 0 * db, dc)
        fd_A = fd_directional(lp.A64, lp.b, lp.c, x, y, s, w, dA, 0 * db, 0 * dc)
        for an, fd in ((dLdb @ db, fd_b), (dLdc @ dc, fd_c), (np.sum(dLdA * dA), fd_A)):
            assert abs(an - fd) <= 2e-5 * abs(fd) + 1e-9, (an, fd)


@pytest.mark.gpu
@pytest.mark.parametrize("seed", [0, 1])
def test_backward_matches_finite_differences(seed):
    """128 x 384, FP32 storage, the FP32 mixed form with FP64 refinement,
    stopped at a relative gap of 1e-6; loss w'x with w ~ N(0,1)."""
    from paper_1502_03543_gb300 import build as B
    B.build()
    import paper_1502_03543_gb300 as P
    lp = lpgen.generate(128, 384, seed=seed, storage="f32")
    dv = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    A = torch.from_numpy(lp.A_store).cuda()
    x, y, s = dv(lp.x0), dv(lp.y0), dv(lp.s0)
    rng = np.random.default_rng(seed + 10)
    w = rng.standard_normal(lp.n)
    with P.Solver(lp.m, lp.n, "fp32_ir", torch.float32) as S:
        out = S.solve(A, dv(lp.b), dv(lp.c), x, y, s, alpha=0.95, tol=1e-6)
        assert out["status"] == 1
        dA, db, dc = S.backward(A, x, y, s, dv(w))
    xh, yh, sh = (t.cpu().numpy() for t in (x, y, s))
    dA, db, dc = dA.cpu().numpy(), db.cpu().numpy(), dc.cpu().numpy()
    # against the dense full-system adjoint at the same iterate: cond J ~ 4e4,
    # so the reference is good to ~1e-12; the reduced form alone (no
    # refinement on the full system) is off by ~2e-5 in dL/dc here.
    eA, eb, ec = full_adjoint(lp.A64, xh, yh, sh, w)
    for got, ref in ((db, eb), (dc, ec), (dA, eA)):
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= 1e-10, err
    for _ in range(3):
        pA, pb, pc = rng.standard_normal(lp.A64.shape), rng.standard_normal(lp.m), rng.standard_normal(lp.n)
        fd_b = fd_directional(lp.A64, lp.b, lp.c, xh, yh, sh, w, 0 * pA, pb, 0 * pc)
        fd_c = fd_directional(lp.A64, lp.b, lp.c, xh, yh, sh, w, 0 * pA, 0 * pb, pc)
        fd_A = fd_directional(lp.A64, lp.b, lp.c, xh, yh, sh, w, pA, 0 * pb, 0 * pc)
        for an, fd in ((db @ pb, fd_b), (dc @ pc, fd_c), (np.sum(dA * pA), fd_A)):
            assert abs(an - fd) <= 2e-5 * abs(fd) + 1e-9, (an, fd)


@pytest.mark.gpu
def test_backward_at_a_vertex_and_through_autograd():
    """Near a nondegenerate optimum x* -> x_B = B^{-1} b, so dL/db -> B^{-T} w_B;
    the same gradient comes out of torch.autograd through solve_lp."""
    from paper_1502_03543_gb300 import build as B
    B.build()
    import paper_1502_03543_gb300 as P
    lp = lpgen.generate(64, 160, seed=3)
    dv = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    A = dv(lp.A64)
    w = np.random.default_rng(4).standard_normal(lp.n)
    with P.Solver(lp.m, lp.n, "fp64") as S:
        b = dv(lp.b).requires_grad_(True)
        c = dv(lp.c).requires_grad_(True)
        xs = P.solve_lp(A, b, c, dv(lp.x0), dv(lp.y0), dv(lp.s0), S, alpha=0.95, tol=1e-10)
        loss = (xs * dv(w)).sum()
        loss.backward()
    basis = np.argsort(-xs.detach().cpu().numpy())[: lp.m]
    Bm = lp.A64[:, basis]
    vertex = np.linalg.solve(Bm.T, w[basis])
    got = b.grad.cpu().numpy()
    assert np.linalg.norm(got - vertex) <= 1e-4 * np.linalg.norm(vertex)
    assert c.grad is not None and torch.isfinite(c.grad).all()
