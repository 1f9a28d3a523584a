"""Parity of the factor and the triangular solves at the benchmark's sizes.

The Cholesky of the normal matrix (Section V-A) runs at m = 8192 in the
benchmark: for the FP32 factor of the mixed forms that is one persistent
launch over nb = 64 tile rows (~43.8k tasks on 152 CTAs, a dedicated
diagonal CTA, ticket-ordered priorities), for the FP64 tier the same task
list in double-float, and for the plain form the FP64 panel factor.  These
tests factor the normal matrix the library itself forms at the seeded start
of the 4096 x 16384 and 8192 x 32768 workloads and check, through the C ABI:

  * sampled full rows of L L' against M, elementwise, within the backward
    error bound of a Cholesky whose multiply-adds carry relative error u:
    |L L' - M| <= g |L| |L'|, with g derived below for each arithmetic;
  * both triangular solves against the oracle's substitutions on the GPU's
    own L, normwise within 4 cond(L)^2 gamma_m(u) of the solve's precision
    (cond(L) estimated by power and inverse iteration, which can only
    underestimate it; the factor 4 covers that).
"""
import numpy as np
import pytest
import scipy.linalg
import torch

import lpgen
import oracle

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53
U32 = 2.0 ** -24

WORKLOADS = {4096: "dense_4096x16384_bf16_colscaled", 8192: "dense_8192x32768_bf16_colscaled"}


def gamma(n, u):
    return n * u / (1 - n * u)


@pytest.fixture(scope="module")
def pdas():
    from paper_1502_03543_gb300 import build as B
    B.build()
    import paper_1502_03543_gb300 as P
    assert torch.cuda.is_available()
    return P


@pytest.fixture(scope="module", params=sorted(WORKLOADS))
def case(request, pdas):
    lp = lpgen.workload(WORKLOADS[request.param], 0)
    A = torch.from_numpy(lp.A_store.view(np.int16).copy()).view(torch.bfloat16).cuda()
    yield lp, A
    del A
    torch.cuda.empty_cache()


def dv(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host64(t):
    return t.detach().cpu().numpy().astype(np.float64)


def sample_rows(m, seed=0):
    """First and last rows, rows on both sides of tile edges (128) and of the
    middle, and a few random ones."""
    rng = np.random.default_rng(seed)
    fixed = [0, 1, 127, 128, 129, m // 2 - 1, m // 2, m - 129, m - 128, m - 2, m - 1]
    return sorted(set(fixed) | set(int(p) for p in rng.integers(0, m, 6)))


def factor_rows_error(L, M, rows, g):
    """max over the sampled rows of |L L' - M|_pq / (g (|L| |L'|)_pq) (<= 1
    passes), and the largest |L L' - M|_pq / max|M| seen."""
    absL = np.abs(L)
    worst, normwise = 0.0, 0.0
    scale = np.abs(M).max()
    for p in rows:
        llt = L @ L[p]  # row p of L L' (L lower triangular: zeros above the diagonal)
        mrow = np.concatenate([M[p, : p + 1], M[p + 1:, p]])  # row p of the symmetric M from its lower triangle
        err = np.abs(llt - mrow)
        bound = g * (absL @ absL[p])
        worst = max(worst, float((err / bound).max()))
        normwise = max(normwise, float(err.max() / scale))
    return worst, normwise


def cond_estimate(L, iters=40, seed=1):
    """cond_2(L) = sqrt(cond_2(L L')) from power iteration on L L' and inverse
    iteration with LAPACK's triangular solves (both converge from the safe
    side: the estimate never exceeds the true condition number)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(L.shape[0])
    lam_max = 0.0
    for _ in range(iters):
        w = L @ (L.T @ v)
        lam_max = np.linalg.norm(w) / np.linalg.norm(v)
        v = w / np.linalg.norm(w)
    v = rng.standard_normal(L.shape[0])
    inv_max = 0.0
    for _ in range(iters):
        z = scipy.linalg.solve_triangular(L, v, lower=True)
        w = scipy.linalg.solve_triangular(L, z, lower=True, trans="T")
        inv_max = np.linalg.norm(w) / np.linalg.norm(v)
        v = w / np.linalg.norm(w)
    return float(np.sqrt(lam_max * inv_max))


def check_solves(S, L, m, u, seed, rhs0):
    """Two right-hand sides (A x0 of the seeded start and a random vector):
    the library's two triangular solves with its own factor against the
    oracle's FP64 substitutions on the same L."""
    kappa = cond_estimate(L)
    rng = np.random.default_rng(seed)
    worst = 0.0
    for rhs in (rhs0, rng.standard_normal(m)):
        x = S.factor_solve(dv(rhs)).cpu().numpy()
        xo = oracle.backward(L, oracle.forward(L, rhs))
        err = np.linalg.norm(x - xo) / np.linalg.norm(xo)
        bound = 4 * kappa ** 2 * gamma(m, u)
        assert err <= bound, (err, bound, kappa)
        worst = max(worst, err / bound)
    return kappa, worst


def test_tile_cholesky_fp32_full_size(pdas, case):
    """The FP32 tile factor of the mixed forms on the normal matrix that the
    BF16 tensor-core form builds at the seeded start (the benchmark's first
    factor).  Error bound: every trailing product L_ik L_jk' (K = 128) runs
    as BF16 plane products that are exact in FP32, drops terms below 2^-22
    of sum |L_ik||L_jk| and accumulates over 8 tensor-core steps that
    truncate (2^-23 each): 1.25 x 2^-20 per product, plus 2^-24 for the
    subtraction from C, over nb = m/128 steps; the factor and solve inside a
    tile add gamma_128 at u = 2^-23.  g = (nb + 1) 2^-19 + 256 x 2^-23 covers
    both with room; the normwise form 4 m u32 max|M| is checked too."""
    lp, A = case
    m, n = lp.m, lp.n
    nb = (m + 127) // 128
    with pdas.Solver(m, n, "bf16_ir", torch.bfloat16) as S:
        S.form_normal(A, dv(lp.x0), dv(lp.s0))
        M = host64(S.copy_matrix())
        S.factor()
        L = np.tril(host64(S.copy_matrix()))
        assert np.all(np.diag(L) > 0)
        g = (nb + 1) * 2.0 ** -19 + 256 * 2.0 ** -23
        worst, normwise = factor_rows_error(L, M, sample_rows(m), g)
        assert worst <= 1.0, worst
        assert normwise <= 4 * m * U32, normwise
        # the FP32 solves apply each diagonal tile's explicit inverse: the
        # forward error is FP32-grade times the conditioning
        kappa, sworst = check_solves(S, L, m, U32, seed=m, rhs0=lp.b)
    print("m=%d fp32 tile factor: |LL'-M| at %.2e of its bound, normwise %.1e; cond(L) ~ %.0f, solves at %.1e "
          "of their bound" % (m, worst, normwise, kappa, sworst))


def test_double_float_tile_factor_full_size(pdas, case):
    """The FP64 tier of a mixed form without its tensor-core parts
    (fp64_tier_tc = 0; the rule dspread_refactor = 1e-300 moves the handle
    to the tier at once): the normal matrix formed in double-float and
    factored by the FP32 factor's tile task list in double-float (hi + lo
    FP32 pairs: every multiply-add exact to a few units of 2^-46), then
    solved by FP64 substitution.  g = (m + 1) 2^-43 is the Cholesky bound
    gamma_{m+1} at a unit roundoff of 2^-43."""
    lp, A = case
    m, n = lp.m, lp.n
    x0, s0 = dv(lp.x0), dv(lp.s0)
    with pdas.Solver(m, n, "bf16_ir", torch.bfloat16, dspread_refactor=1e-300, fp64_tier_tc=0) as S:
        _, _, _, info = S.direction(A, x0, s0)
        assert info["used_fp64"] == 1 and info["normal_form"] == 2
        S.form_normal(A, x0, s0)
        M = host64(S.copy_matrix())
        S.factor()  # no step taken yet: the gap is unknown, so the double-float factor runs
        L = np.tril(host64(S.copy_matrix()))
        worst, normwise = factor_rows_error(L, M, sample_rows(m, seed=1), (m + 1) * 2.0 ** -43)
        assert worst <= 1.0, worst
        kappa, sworst = check_solves(S, L, m, U64, seed=m + 1, rhs0=lp.b)
    print("m=%d double-float tile factor: |LL'-M| at %.2e of its bound, normwise %.1e; cond(L) ~ %.0f, solves at "
          "%.1e of their bound" % (m, worst, normwise, kappa, sworst))


def test_fp64_factor_full_size(pdas, case):
    """The plain FP64 form: M formed in FP64, the FP64 panel factor, FP64
    substitution.  g = gamma_{m+1}(u64), the componentwise backward error
    bound of Cholesky in any summation order."""
    lp, A = case
    m, n = lp.m, lp.n
    with pdas.Solver(m, n, "fp64", torch.bfloat16) as S:
        S.form_normal(A, dv(lp.x0), dv(lp.s0))
        M = host64(S.copy_matrix())
        S.factor()
        L = np.tril(host64(S.copy_matrix()))
        worst, normwise = factor_rows_error(L, M, sample_rows(m, seed=2), gamma(m + 1, U64))
        assert worst <= 1.0, worst
        kappa, sworst = check_solves(S, L, m, U64, seed=m + 2, rhs0=lp.b)
    print("m=%d fp64 factor: |LL'-M| at %.2e of its bound, normwise %.1e; cond(L) ~ %.0f, solves at %.1e of "
          "their bound" % (m, worst, normwise, kappa, sworst))


def test_tensor_core_fp64_factor_full_size(pdas, case):
    """The FP64 tier's default factor: FP64 panels, trailing updates on the
    tensor cores from 7 fixed-point BF16 digits per panel row (exact digit
    products and sums).  Bound: gamma_{m+1}(u64) |L||L'| for the FP64
    arithmetic, plus the digits' rounding of entries below 1/8 of their
    panel row's largest (2^-56 of 2^e per entry) and the digit pairs left
    out, summed over the m / 64 panels: within 2^-40 sqrt(M_pp M_qq)."""
    lp, A = case
    m, n = lp.m, lp.n
    x0, s0 = dv(lp.x0), dv(lp.s0)
    with pdas.Solver(m, n, "bf16_ir", torch.bfloat16, dspread_refactor=1e-300) as S:
        _, _, _, info = S.direction(A, x0, s0)
        assert info["used_fp64"] == 1
        assert info["factor_form"] == 4, info  # the tensor-core factor, not a fallback after a failed pivot
        S.form_normal(A, x0, s0)
        M = host64(S.copy_matrix())
        S.factor()  # raises on a failed pivot (no fallback inside pdas_factor)
        L = np.tril(host64(S.copy_matrix()))
        d = np.sqrt(np.diag(M))
        absL = np.abs(L)
        worst, scaled = 0.0, 0.0
        for p in sample_rows(m, seed=3):
            err = np.abs(L @ L[p] - np.concatenate([M[p, : p + 1], M[p + 1:, p]]))
            bound = gamma(m + 1, U64) * (absL @ absL[p]) + 2.0 ** -40 * d[p] * d
            worst = max(worst, float((err / bound).max()))
            scaled = max(scaled, float((err / (d[p] * d)).max()))
        assert worst <= 1.0, worst
        assert scaled <= 1e-14, scaled
        kappa, sworst = check_solves(S, L, m, U64, seed=m + 3, rhs0=lp.b)
    print("m=%d tensor-core FP64 factor: |LL'-M| at %.2e of its bound, scaled %.1e; cond(L) ~ %.0f, solves at "
          "%.1e of their bound" % (m, worst, scaled, kappa, sworst))
