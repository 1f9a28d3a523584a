"""The batched adjoint (pdas_batch_backward): the sensitivities of
L = sum_i w_i' x*_i for a batch of LPs of 128 x 384 (FP32 storage, stopped at
a relative gap of 1e-6, w ~ N(0,1)), every LP differentiated in one launch
(one CTA per LP, its normal matrix formed and factored in the CTA).

Per LP, the batch's outputs at the batch's own final iterate are checked
against the dense full-system adjoint J'(la, lb, lc) = (g, 0, 0) (numpy,
FP64; independent of the oracle and of the GPU path) to 1e-10 normwise, as
pdas_backward is; on two LPs also against central finite differences of a
Newton re-solve of F = 0 with sigma held fixed (the reference of the
single-LP adjoint's tests), to the 1e-4 relative asked of the adjoint.  An
uneven batch covers the size buckets."""
import numpy as np
import pytest
import torch

import lpgen
from test_adjoint import fd_directional, full_adjoint

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pdas():
    from paper_1502_03543_gb300 import build as B
    B.build()
    import paper_1502_03543_gb300 as P
    assert torch.cuda.is_available()
    return P


def dv(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def solve_batch(P, sizes, tol, base_seed):
    lps = lpgen.batch(len(sizes[0]), storage="f32", base_seed=base_seed, sizes=sizes)
    pk = lpgen.pack(lps)
    A = torch.from_numpy(np.ascontiguousarray(pk["A"], dtype=np.float32)).cuda()
    b, c = dv(pk["b"]), dv(pk["c"])
    x, y, s = dv(pk["x0"]), dv(pk["y0"]), dv(pk["s0"])
    S = P.BatchSolver(pk["m"], pk["n"], A, b, c, x, y, s, tol=tol)
    out = S.solve()
    return lps, pk, S, (A, b, c, x, y, s), out


def offsets(pk):
    a_off = np.concatenate([[0], np.cumsum(pk["m"].astype(np.int64) * pk["n"])])
    m_off = np.concatenate([[0], np.cumsum(pk["m"])])
    n_off = np.concatenate([[0], np.cumsum(pk["n"])])
    return a_off, m_off, n_off


@pytest.mark.parametrize("sizes", [
    (np.full(12, 128), np.full(12, 384)),                                   # the differentiable batch's shape
    (np.array([20, 64, 65, 128, 130, 200, 256]), np.array([50, 190, 130, 384, 400, 600, 520])),  # every bucket
])
def test_batch_backward_matches_dense_adjoint(pdas, sizes):
    lps, pk, S, bufs, out = solve_batch(pdas, sizes, 1e-6, 2000)
    assert np.all(out["status"] == 1), out["status"]
    rng = np.random.default_rng(7)
    w = rng.standard_normal(int(pk["n"].sum()))
    dA, db, dc, status = S.backward(dv(w))
    assert np.all(status == 0), status
    x, y, s = (t.cpu().numpy() for t in bufs[3:])
    dA, db, dc = dA.cpu().numpy(), db.cpu().numpy(), dc.cpu().numpy()
    a_off, m_off, n_off = offsets(pk)
    for i, lp in enumerate(lps):
        xi, yi, si = x[n_off[i]:n_off[i + 1]], y[m_off[i]:m_off[i + 1]], s[n_off[i]:n_off[i + 1]]
        wi = w[n_off[i]:n_off[i + 1]]
        eA, eb, ec = full_adjoint(lp.A64, xi, yi, si, wi)
        got = (db[m_off[i]:m_off[i + 1]], dc[n_off[i]:n_off[i + 1]],
               dA[a_off[i]:a_off[i + 1]].reshape(lp.m, lp.n))
        for g, ref in zip(got, (eb, ec, eA)):
            err = np.linalg.norm(g - ref) / np.linalg.norm(ref)
            assert err <= 1e-10, (i, lp.m, lp.n, err)
    S.close()


def test_batch_backward_matches_finite_differences(pdas):
    sizes = (np.full(4, 128), np.full(4, 384))
    lps, pk, S, bufs, out = solve_batch(pdas, sizes, 1e-6, 3000)
    assert np.all(out["status"] == 1)
    rng = np.random.default_rng(8)
    w = rng.standard_normal(int(pk["n"].sum()))
    dA, db, dc, status = S.backward(dv(w), want_dA=True)
    assert np.all(status == 0)
    x, y, s = (t.cpu().numpy() for t in bufs[3:])
    dA, db, dc = dA.cpu().numpy(), db.cpu().numpy(), dc.cpu().numpy()
    a_off, m_off, n_off = offsets(pk)
    for i in (0, 3):
        lp = lps[i]
        xi, yi, si = x[n_off[i]:n_off[i + 1]], y[m_off[i]:m_off[i + 1]], s[n_off[i]:n_off[i + 1]]
        wi = w[n_off[i]:n_off[i + 1]]
        gA = dA[a_off[i]:a_off[i + 1]].reshape(lp.m, lp.n)
        gb, gc = db[m_off[i]:m_off[i + 1]], dc[n_off[i]:n_off[i + 1]]
        pA, pb, pc = rng.standard_normal(lp.A64.shape), rng.standard_normal(lp.m), rng.standard_normal(lp.n)
        eA, eb, ec = full_adjoint(lp.A64, xi, yi, si, wi)
        for g, ref in ((gb, eb), (gc, ec), (gA, eA)):
            assert np.linalg.norm(g - ref) <= 1e-10 * np.linalg.norm(ref)
        # h = 1e-7: at these iterates (max D / min D ~ 1e18) the curvature in A
        # is strong, and differences at h = 1e-6 still carried up to 2e-4 of
        # truncation error on the oracle's own iterate of one of these LPs
        # (1e-5: 9e-2, 1e-6: 6e-6, 1e-7: 3e-8 there)
        fd_b = fd_directional(lp.A64, lp.b, lp.c, xi, yi, si, wi, 0 * pA, pb, 0 * pc, h=1e-7)
        fd_c = fd_directional(lp.A64, lp.b, lp.c, xi, yi, si, wi, 0 * pA, 0 * pb, pc, h=1e-7)
        fd_A = fd_directional(lp.A64, lp.b, lp.c, xi, yi, si, wi, pA, 0 * pb, 0 * pc, h=1e-7)
        for an, fd in ((gb @ pb, fd_b), (gc @ pc, fd_c), (np.sum(gA * pA), fd_A)):
            # the agreement asked of the adjoint: 1e-4 relative
            assert abs(an - fd) <= 1e-4 * abs(fd) + 1e-9, (i, an, fd)
    S.close()
