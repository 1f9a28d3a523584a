"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances come from the arithmetic:
  * a dot product of length n summed in two different orders in FP64 differs
    by at most 2 gamma_n sum|terms|, gamma_n = n u / (1 - n u), u = 2^-53
    (FP32: u = 2^-24) -- used elementwise for A v, A' u and M = A D A';
  * Cholesky factors and triangular solves of well-conditioned matrices agree
    to ~cond * u; 1e-11 relative leaves room on the test matrices;
  * whole iterates: the normwise 1e-9 relative agreement that the FP64 form
    must keep with the oracle at every iteration, and the optimal objective
    to 1e-8 relative for every form.
"""
import numpy as np
import pytest
import torch

import lpgen
import oracle

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53
U32 = 2.0 ** -24


def gamma(n, u):
    return n * u / (1 - n * u)


@pytest.fixture(scope="module")
def pdas():
    from paper_1502_03543_gb300 import build as B
    B.build()
    import paper_1502_03543_gb300 as P
    assert torch.cuda.is_available()
    return P


TORCH_DT = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}


def dev_A(lp):
    if lp.storage == "bf16":
        return torch.from_numpy(lp.A_store.view(np.int16).copy()).view(torch.bfloat16).cuda()
    return torch.from_numpy(np.ascontiguousarray(lp.A_store)).cuda()


def dv(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()


SHAPES = [(1, 2), (5, 37), (64, 128), (130, 520), (67, 301)]


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("m,n", SHAPES)
def test_gemv_and_gemv_t(pdas, storage, m, n):
    lp = lpgen.generate(m, n, seed=m + n, storage=storage, scaled=storage == "bf16")
    A = dev_A(lp)
    rng = np.random.default_rng(1)
    v, u = rng.standard_normal(n), rng.standard_normal(m)
    with pdas.Solver(m, n, "fp64", TORCH_DT[storage]) as S:
        r = host(S.gemv(A, dv(v)))
        w = host(S.gemv_t(A, dv(u)))
    ref_r, ref_w = oracle.gemv(lp.A64, v), oracle.gemv_t(lp.A64, u)
    bound_r = 2 * gamma(n, U64) * (np.abs(lp.A64) @ np.abs(v))
    bound_w = 2 * gamma(m, U64) * (np.abs(lp.A64).T @ np.abs(u))
    assert np.all(np.abs(r - ref_r) <= bound_r + 1e-300)
    assert np.all(np.abs(w - ref_w) <= bound_w + 1e-300)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("m,n", SHAPES + [(33, 4104), (130, 2048)])
def test_gemv_double_float_mixed_forms(pdas, storage, m, n):
    """The mixed forms run the passes over A in double-float on the FP32 pipes:
    each term a v carries <= 2^-47 relative error, the FP32 low part of a
    16- or 32-term partial sum adds <= 32 x 2^-48 of its terms, and the FP64
    accumulation of the partials gamma_n(u64): together well within 2^-41 of
    sum |a v|, some 10^5 times below FP32 accuracy.  exact_passes=1 restores
    the FP64 passes (FP64 bound)."""
    lp = lpgen.generate(m, n, seed=m + n + 7, storage=storage, scaled=storage == "bf16")
    A = dev_A(lp)
    rng = np.random.default_rng(2)
    v, u = rng.standard_normal(n), rng.standard_normal(m)
    ref_r, ref_w = oracle.gemv(lp.A64, v), oracle.gemv_t(lp.A64, u)
    mag_r, mag_w = np.abs(lp.A64) @ np.abs(v), np.abs(lp.A64).T @ np.abs(u)
    with pdas.Solver(m, n, "fp32_ir", TORCH_DT[storage]) as S:
        r, w = host(S.gemv(A, dv(v))), host(S.gemv_t(A, dv(u)))
    assert np.all(np.abs(r - ref_r) <= (2.0 ** -41 + 2 * gamma(n, U64)) * mag_r + 1e-300)
    assert np.all(np.abs(w - ref_w) <= (2.0 ** -41 + 2 * gamma(m, U64)) * mag_w + 1e-300)
    with pdas.Solver(m, n, "fp32_ir", TORCH_DT[storage], exact_passes=1) as S:
        r, w = host(S.gemv(A, dv(v))), host(S.gemv_t(A, dv(u)))
    assert np.all(np.abs(r - ref_r) <= 2 * gamma(n, U64) * mag_r + 1e-300)
    assert np.all(np.abs(w - ref_w) <= 2 * gamma(m, U64) * mag_w + 1e-300)


@pytest.mark.parametrize("storage", ["f64", "bf16"])
@pytest.mark.parametrize("m,n", SHAPES)
def test_normal_matrix_fp64(pdas, storage, m, n):
    lp = lpgen.generate(m, n, seed=7 * m + n, storage=storage, scaled=storage == "bf16")
    rng = np.random.default_rng(2)
    x, s = rng.uniform(0.01, 10, n), rng.uniform(0.01, 10, n)
    with pdas.Solver(m, n, "fp64", TORCH_DT[storage]) as S:
        S.form_normal(dev_A(lp), dv(x), dv(s))
        M = host(S.copy_matrix())
    D = oracle.scaling(x, s)
    ref = oracle.normal_matrix(lp.A64, D)
    bound = 2 * gamma(n + 2, U64) * ((np.abs(lp.A64) * D) @ np.abs(lp.A64).T)
    low = np.tril_indices(m)
    assert np.all(np.abs(M[low] - ref[low]) <= bound[low])


@pytest.mark.parametrize("m,n", SHAPES)
def test_normal_matrix_fp32_simt(pdas, m, n):
    lp = lpgen.generate(m, n, seed=3 * m + n, storage="f32")
    rng = np.random.default_rng(3)
    x, s = rng.uniform(0.1, 10, n), rng.uniform(0.1, 10, n)
    with pdas.Solver(m, n, "fp32_ir", torch.float32) as S:
        S.form_normal(dev_A(lp), dv(x), dv(s))
        M = host(S.copy_matrix()).astype(np.float64)
    D = oracle.scaling(x, s)
    ref = oracle.normal_matrix(lp.A64, D)
    # operands rounded to FP32 (A D and A exact), products and sums in FP32
    bound = 2 * gamma(n + 3, U32) * ((np.abs(lp.A64) * D) @ np.abs(lp.A64).T)
    low = np.tril_indices(m)
    assert np.all(np.abs(M[low] - ref[low]) <= bound[low])


def spd_matrix(m, seed):
    lp = lpgen.generate(m, 3 * m + 1, seed=seed)
    D = oracle.scaling(lp.x0, lp.s0)
    return oracle.normal_matrix(lp.A64, D)


@pytest.mark.parametrize("m", [1, 7, 64, 65, 200])
def test_cholesky_and_solves_fp64(pdas, m):
    M = spd_matrix(m, seed=m)
    Lo, fail = oracle.cholesky(M)
    assert fail == -1
    with pdas.Solver(m, m + 1, "fp64") as S:
        S.load_matrix(dv(M))
        S.factor()
        L = np.tril(host(S.copy_matrix()))
        rhs = np.random.default_rng(4).standard_normal(m)
        x = host(S.factor_solve(dv(rhs)))
    assert np.linalg.norm(L - Lo) <= 1e-11 * np.linalg.norm(Lo)
    # the triangular solves against the oracle's substitutions on the GPU's factor
    xo = oracle.backward(L, oracle.forward(L, rhs))
    assert np.linalg.norm(x - xo) <= 1e-11 * np.linalg.norm(xo)


@pytest.mark.parametrize("m", [7, 65, 200, 384, 700])  # the FP32 factor runs on 128 x 128 tiles
def test_cholesky_fp32(pdas, m):
    M = spd_matrix(m, seed=100 + m)
    Lo, _ = oracle.cholesky(M)
    with pdas.Solver(m, m + 1, "fp32_ir", torch.float32) as S:
        S.load_matrix(dv(M))
        S.factor()
        L = np.tril(host(S.copy_matrix()).astype(np.float64))
        rhs = np.random.default_rng(5).standard_normal(m)
        x = host(S.factor_solve(dv(rhs)))
    # FP32 factor of a well-conditioned matrix: backward error ~ m u32
    assert np.abs(L @ L.T - M).max() <= 4 * m * U32 * np.abs(M).max()
    # the FP32 factor's solves run in FP32 (a preconditioner, refined in FP64
    # by the mixed forms): forward error <= cond(L)^2 gamma_m(u32) per solve pair
    xo = oracle.backward(L, oracle.forward(L, rhs))
    assert np.linalg.norm(x - xo) <= 2 * np.linalg.cond(L) ** 2 * gamma(m, U32) * np.linalg.norm(xo)


@pytest.mark.parametrize("form,dt", [("fp64", torch.float64), ("fp32_ir", torch.float32)])
@pytest.mark.parametrize("m,bad", [(150, 97), (400, 300)])
def test_not_spd_reports_pivot(pdas, form, dt, m, bad):
    M = np.eye(m)
    M[bad, bad] = -1.0
    with pdas.Solver(m, m + 1, form, dt) as S:
        S.load_matrix(dv(M).to(dt))
        st = S.factor(raise_on_error=False)
        assert st == -3 and S.last_error_index() == bad


@pytest.mark.parametrize("bad", [10, 97, 290])
def test_not_spd_reports_pivot_tensor_core_factor(pdas, bad):
    """The FP64 tier's tensor-core factor at m = 300 (five 64-column panels,
    the last 44 wide) reports a pivot that is not positive with its index:
    in the first panel (the diagonal block's own launch), in a later panel
    (the block factored inside the previous panel's update) and in the last,
    narrower panel."""
    m = 300
    lp = lpgen.generate(m, 4 * m, seed=5, storage="bf16", scaled=True)
    M = np.eye(m)
    M[bad, bad] = -1.0
    with pdas.Solver(m, lp.n, "bf16_ir", torch.bfloat16, dspread_refactor=1e-300) as S:
        _, _, _, info = S.direction(dev_A(lp), dv(lp.x0), dv(lp.s0))
        assert info["factor_form"] == 4
        S.load_matrix(dv(M))
        st = S.factor(raise_on_error=False)
        assert st == -3 and S.last_error_index() == bad


def lapack_direction(A, x, s):
    D = x / s
    M = (A * D) @ A.T
    dy = np.linalg.solve(M, A @ x)
    w = A.T @ dy
    return D * w - x, dy, -w


def test_direction_matches_oracle(pdas):
    """Directions along the oracle's trajectory agree with the oracle's to
    1e-9, or -- once the normal matrix is ill-conditioned -- at least as well
    as an independent LAPACK solve of the same system does (4x margin)."""
    lp = lpgen.workload("dense_64x128_f64", 0)
    res = oracle.solve(lp.A64, lp.b, lp.c, lp.x0, lp.y0, lp.s0, keep_iterates=True)
    n, m = lp.n, lp.m
    pts = [(lp.x0, lp.s0)] + [(r[:n], r[n + m:]) for r in res["iterates"][:-1]]
    with pdas.Solver(m, n, "fp64") as S:
        A = dev_A(lp)
        for k in range(len(pts)):
            x, s = pts[k]
            d = oracle.direction(lp.A64, x, s)
            dx, dy, ds, _ = S.direction(A, dv(x), dv(s))
            lap = lapack_direction(lp.A64, x, s)
            # forward error of a backward-stable solve: ~u cond(M); dx = D w - x
            # cancels, which scales its relative error by ||D w|| / ||dx||
            kappa = np.linalg.cond((lp.A64 * d["D"]) @ lp.A64.T)
            amp = {0: np.linalg.norm(d["D"] * d["ds"]) / np.linalg.norm(d["dx"]), 1: 1.0, 2: 1.0}
            for i, (g, o, l) in enumerate(((host(dx), d["dx"], lap[0]), (host(dy), d["dy"], lap[1]),
                                           (host(ds), d["ds"], lap[2]))):
                err = np.linalg.norm(g - o) / np.linalg.norm(o)
                spread = np.linalg.norm(l - o) / np.linalg.norm(o)
                assert err <= max(1e-9, 4 * spread, 10 * U64 * kappa * amp[i]), (k, i, err, spread)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fp64_iterates_match_oracle_every_iteration(pdas, seed):
    """Iterates of the FP64 form against the oracle's at every iteration:
    normwise 1e-9 relative, or within 4x of the drift between the oracle and
    an independent LAPACK-based FP64 run (FP64 rounding amplified by the
    conditioning of A D A' sets that drift late in the solve).  Same number
    of iterations, same optimal objective to 1e-8."""
    from fp64_spread import iterate_spread, lapack_trajectory
    lp = lpgen.workload("dense_64x128_f64", seed)
    ref = oracle.solve(lp.A64, lp.b, lp.c, lp.x0, lp.y0, lp.s0, keep_iterates=True)
    n, m = lp.n, lp.m
    traj = lapack_trajectory(lp.A64, lp.b, lp.c, lp.x0, lp.y0, lp.s0, ref["iters"])
    spread = iterate_spread(ref["iterates"], traj, n, m)
    A, b, c = dev_A(lp), dv(lp.b), dv(lp.c)
    x, y, s = dv(lp.x0), dv(lp.y0), dv(lp.s0)
    first_above = None
    with pdas.Solver(m, n, "fp64") as S:
        for k in range(ref["iters"]):
            # the psi kernel itself is exact: the oracle's psi of the GPU's own
            # (deterministic) direction at the GPU's iterate, bit for bit
            gdx, _, gds, _ = S.direction(A, x, s)
            psi_exact = oracle.psi(host(x), host(s), host(gdx), host(gds))
            st, info = S.step(A, b, c, x, y, s, alpha=0.95)
            assert info["psi"] == psi_exact, (k, info["psi"], psi_exact)
            it = ref["iterates"][k]
            err = max(np.linalg.norm(host(g) - o) / np.linalg.norm(o)
                      for g, o in ((x, it[:n]), (y, it[n:n + m]), (s, it[n + m:])))
            bound = max(1e-9, 4 * spread[: k + 1].max())
            assert err <= bound, (k, err, spread[k])
            if err > 1e-9 and first_above is None:
                first_above = k

        assert info["rel_gap"] < 1e-8  # the oracle stops at this same iteration
    print("seed %d: first iteration above 1e-9: %s (LAPACK drift max %.1e)" % (seed, first_above, spread.max()))
    obj, obj_ref = float(lp.c @ host(x)), float(lp.c @ ref["x"])
    assert abs(obj - obj_ref) <= 1e-8 * abs(obj_ref)


def test_solve_entry_point_c1(pdas):
    lp = lpgen.workload("dense_64x128_f64", 0)
    ref = oracle.solve(lp.A64, lp.b, lp.c, lp.x0, lp.y0, lp.s0)
    x, y, s = dv(lp.x0), dv(lp.y0), dv(lp.s0)
    with pdas.Solver(lp.m, lp.n, "fp64") as S:
        out = S.solve(dev_A(lp), dv(lp.b), dv(lp.c), x, y, s, alpha=0.95, tol=1e-8)
    assert out["status"] == 1 and out["iters"] == ref["iters"]
    assert abs(float(lp.c @ host(x)) - float(lp.c @ ref["x"])) <= 1e-8 * abs(float(lp.c @ ref["x"]))


@pytest.mark.parametrize("seed", [0, 1])
def test_fp32_ir_objective_and_iterations(pdas, seed):
    lp = lpgen.generate(64, 128, seed=seed, storage="f32")
    ref = oracle.solve(lp.A64, lp.b, lp.c, lp.x0, lp.y0, lp.s0)
    x, y, s = dv(lp.x0), dv(lp.y0), dv(lp.s0)
    with pdas.Solver(lp.m, lp.n, "fp32_ir", torch.float32, dspread_refactor=0.0) as S:
        out = S.solve(dev_A(lp), dv(lp.b), dv(lp.c), x, y, s, alpha=0.95, tol=1e-8)
    assert out["status"] == 1
    obj_ref = float(lp.c @ ref["x"])
    assert abs(float(lp.c @ host(x)) - obj_ref) <= 1e-8 * abs(obj_ref)
    assert out["iters"] == ref["iters"]


def test_edge_cases(pdas):
    # m = 1 and n = m + 1
    for (m, n) in [(1, 2), (1, 9), (5, 6)]:
        lp = lpgen.generate(m, n, seed=11)
        ref = oracle.solve(lp.A64, lp.b, lp.c, lp.x0, lp.y0, lp.s0)
        x, y, s = dv(lp.x0), dv(lp.y0), dv(lp.s0)
        with pdas.Solver(m, n, "fp64") as S:
            out = S.solve(dev_A(lp), dv(lp.b), dv(lp.c), x, y, s)
        assert out["status"] == ref["status"] and out["iters"] == ref["iters"]
        assert abs(float(lp.c @ host(x)) - float(lp.c @ ref["x"])) <= 1e-8 * (1 + abs(float(lp.c @ ref["x"])))
    lp = lpgen.generate(6, 14, seed=12)
    with pdas.Solver(6, 14, "fp64") as S:
        A, b, c = dev_A(lp), dv(lp.b), dv(lp.c)
        # not interior: nothing modified
        x0 = lp.x0.copy()
        x0[3] = 0.0
        x, y, s = dv(x0), dv(lp.y0), dv(lp.s0)
        out = S.solve(A, b, c, x, y, s)
        assert out["status"] == -2 and np.array_equal(host(x), x0) and np.array_equal(host(y), lp.y0)
        # alpha outside (0, 1)
        x = dv(lp.x0)
        st, _ = S.step(A, b, c, x, y, s, alpha=1.0, raise_on_error=False)
        assert st == -1 and np.array_equal(host(x), lp.x0)
    # rank-deficient A: a zero row -> reported, iterate untouched
    A0 = lp.A64.copy()
    A0[2] = 0.0
    with pdas.Solver(6, 14, "fp64") as S:
        x, y, s = dv(lp.x0), dv(lp.y0), dv(lp.s0)
        out = S.solve(dv(A0), dv(A0 @ lp.x0), dv(A0.T @ lp.y0 + lp.s0), x, y, s)
        assert out["status"] == -3 and S.last_error_index() == 2
        assert np.array_equal(host(x), lp.x0)


def test_full_step_lp_is_exact(pdas):
    from conftest import load_fixture
    g = load_fixture("lp_2x4_one_step.txt")
    A = np.array(g["A"]).reshape(2, 4)
    x, y, s = dv(g["x0"]), dv(g["y0"]), dv(g["s0"])
    with pdas.Solver(2, 4, "fp64") as S:
        out = S.solve(dv(A), dv(g["b"]), dv(g["c"]), x, y, s)
    assert out["status"] == 2 and out["iters"] == 1
    assert np.array_equal(host(x), g["x_opt"]) and np.array_equal(host(y), g["y_opt"])
    assert np.array_equal(host(s), g["s_opt"])


def test_fp64_c2_first_iterations(pdas):
    """2048 x 8192 FP64: the first two iterates against the oracle."""
    lp = lpgen.workload("dense_2048x8192_f64", 0)
    n, m = lp.n, lp.m
    A, b, c = dev_A(lp), dv(lp.b), dv(lp.c)
    x, y, s = dv(lp.x0), dv(lp.y0), dv(lp.s0)
    xo, yo, so = lp.x0.copy(), lp.y0.copy(), lp.s0.copy()
    with pdas.Solver(m, n, "fp64") as S:
        for k in range(2):
            S.step(A, b, c, x, y, s, alpha=0.95)
            d = oracle.direction(lp.A64, xo, so)
            th = oracle.theta(oracle.psi(xo, so, d["dx"], d["ds"]), 0.95)
            xo, yo, so = oracle.step(xo, yo, so, d["dx"], d["dy"], d["ds"], th)
            for g, o in ((x, xo), (y, yo), (s, so)):
                assert np.linalg.norm(host(g) - o) <= 1e-9 * np.linalg.norm(o), k


def test_full_size_sampled_normal_matrix(pdas):
    """8192 x 32768 BF16-stored, column-scaled A: sampled entries of the FP64
    normal matrix and of A x against the oracle computed one by one."""
    lp = lpgen.workload("dense_8192x32768_bf16_colscaled", 0)
    m, n = lp.m, lp.n
    rng = np.random.default_rng(6)
    with pdas.Solver(m, n, "fp64", torch.bfloat16) as S:
        A = dev_A(lp)
        S.form_normal(A, dv(lp.x0), dv(lp.s0))
        M = S.copy_matrix()
        r = host(S.gemv(A, dv(lp.x0)))
        pairs = [(int(p), int(q)) for p, q in zip(rng.integers(0, m, 64), rng.integers(0, m, 64))]
        pairs = [(max(p, q), min(p, q)) for p, q in pairs] + [(m - 1, m - 1), (m - 1, 0), (0, 0)]
        got = {pq: float(M[pq[0], pq[1]]) for pq in pairs}
    D = lp.x0 / lp.s0
    for (p, q), g in got.items():
        o = oracle.normal_entry(lp.A64, D, p, q)
        bound = 2 * gamma(n + 2, U64) * float(np.abs(lp.A64[p]) * D @ np.abs(lp.A64[q]))
        assert abs(g - o) <= bound, (p, q)
    rows = rng.integers(0, m, 32)
    for p in rows:
        o = float(lp.A64[p] @ lp.x0)  # reference magnitude only
        bound = 2 * gamma(n, U64) * float(np.abs(lp.A64[p]) @ np.abs(lp.x0))
        assert abs(r[p] - oracle.gemv(lp.A64[p:p + 1], lp.x0)[0]) <= bound and np.isfinite(o)


# ---------------------------------------------------------------------------
# the BF16 tensor-core form

def tc_bound(A64, D, n, splits=2):
    """|M_tc - M| elementwise.  The split of A_q D into BF16 terms leaves
    2^-(8 splits) relative (plus FP32 rounding of D and of A_q D); products
    are exact; each 128-long chunk takes 8 splits accumulation steps on the
    tensor core (u = 2^-23, it truncates) and the chunk sums are added in
    round-to-nearest FP32 (u = 2^-24)."""
    rep = 2.0 ** (-8 * splits) + 2.0 ** -22
    acc = gamma(8 * splits + 1, 2.0 ** -23) + gamma(n // 128 + 2, 2.0 ** -24)
    return (rep + acc + rep * acc) * ((np.abs(A64) * D) @ np.abs(A64).T)


def scaled_error(Mt, Me):
    d = np.sqrt(np.diag(Me))
    low = np.tril_indices(Me.shape[0])
    return (np.abs(Mt - Me) / np.outer(d, d))[low].max()


TC_SHAPES = [(1, 2), (5, 37), (64, 128), (130, 520), (67, 301), (257, 1024), (300, 1000), (511, 640)]


@pytest.mark.parametrize("splits", [1, 2, 3])
@pytest.mark.parametrize("m,n", TC_SHAPES)
def test_normal_matrix_bf16_tensor_cores(pdas, m, n, splits):
    lp = lpgen.generate(m, n, seed=5 * m + n, storage="bf16", scaled=True)
    rng = np.random.default_rng(11)
    x, s = rng.uniform(0.01, 10, n), rng.uniform(0.01, 10, n)
    with pdas.Solver(m, n, "bf16_ir", torch.bfloat16, splits=splits) as S:
        S.form_normal(dev_A(lp), dv(x), dv(s))
        M = host(S.copy_matrix()).astype(np.float64)
    D = oracle.scaling(x, s)
    ref = oracle.normal_matrix(lp.A64, D)
    low = np.tril_indices(m)
    bound = tc_bound(lp.A64, D, n, splits)
    assert np.all(np.abs(M[low] - ref[low]) <= bound[low])
    # error relative to sqrt(M_pp M_qq): the split terms carry D.*A to 2^-16
    # (2 terms) and the chunked accumulation stays near FP32 rounding
    assert scaled_error(M, ref) <= {1: 1e-2, 2: 2e-5, 3: 1e-5}[splits]


@pytest.mark.parametrize("seed", [0, 1])
def test_bf16_ir_solve_matches_oracle(pdas, seed):
    lp = lpgen.generate(64, 128, seed=seed, storage="bf16", scaled=True)
    ref = oracle.solve(lp.A64, lp.b, lp.c, lp.x0, lp.y0, lp.s0)
    x, y, s = dv(lp.x0), dv(lp.y0), dv(lp.s0)
    with pdas.Solver(lp.m, lp.n, "bf16_ir", torch.bfloat16) as S:
        out = S.solve(dev_A(lp), dv(lp.b), dv(lp.c), x, y, s, alpha=0.95, tol=1e-8)
    assert out["status"] == 1
    obj_ref = float(lp.c @ ref["x"])
    assert abs(float(lp.c @ host(x)) - obj_ref) <= 1e-8 * abs(obj_ref)
    assert out["iters"] == ref["iters"]


@pytest.mark.parametrize("dspread", [1e8, 0.0])
def test_bf16_ir_solve_512x2048(pdas, dspread):  # with and without the max(D)/min(D) rule
    """A whole solve at 512 x 2048 (column-scaled BF16 A): the mixed form with
    FP64 refinement and the switch to FP64 reaches the oracle's optimal
    objective to 1e-8 in the same number of iterations, and keeps primal and
    dual feasibility."""
    lp = lpgen.generate(512, 2048, seed=0, storage="bf16", scaled=True)
    ref = oracle.solve(lp.A64, lp.b, lp.c, lp.x0, lp.y0, lp.s0)
    x, y, s = dv(lp.x0), dv(lp.y0), dv(lp.s0)
    A, b, c = dev_A(lp), dv(lp.b), dv(lp.c)
    sweeps, fp64 = [], []
    with pdas.Solver(lp.m, lp.n, "bf16_ir", torch.bfloat16, dspread_refactor=dspread) as S:
        for k in range(ref["iters"]):
            st, info = S.step(A, b, c, x, y, s, alpha=0.95)
            sweeps.append(info["refine_sweeps"])
            fp64.append(info["used_fp64"])
    print("dspread %g: refinement sweeps %s, FP64 iterations %d" % (dspread, sweeps, sum(fp64)))
    assert info["rel_gap"] < 1e-8
    obj_ref = float(lp.c @ ref["x"])
    assert abs(float(lp.c @ host(x)) - obj_ref) <= 1e-8 * abs(obj_ref)
    xh, yh, sh = host(x), host(y), host(s)
    assert np.linalg.norm(lp.A64 @ xh - lp.b) <= 1e-9 * np.linalg.norm(lp.b)
    assert np.linalg.norm(lp.A64.T @ yh + sh - lp.c) <= 1e-12 * np.linalg.norm(lp.c)


def tf32_bound(A64, D, n, splits=1):
    """|M_tf32 - M| elementwise.  One term: A and D.*A are each rounded to
    FP32 and then to TF32 (u = 2^-11, round to nearest even), so a product
    carries at most (1 + 2^-11 + 2^-24)^2 - 1 < 2^-10 + 2^-20 relative error.
    TF32 x 3: each operand is hi + lo with |v - hi - lo| <= 2^-24 |v| +
    2^-22 |v| and the dropped lo x lo product is below 2^-22 |a b|: < 2^-20
    together.  Each 64-long chunk takes 8 (24) tensor-core accumulation steps
    (u = 2^-23, truncating) and the chunk sums are added in round-to-nearest
    FP32 (u = 2^-24)."""
    rep = 2.0 ** -10 + 2.0 ** -20 if splits == 1 else 2.0 ** -20
    acc = gamma(8 * splits + 1, 2.0 ** -23) + gamma(n // 64 + 2, 2.0 ** -24)
    return (rep + acc + rep * acc) * ((np.abs(A64) * D) @ np.abs(A64).T)


@pytest.mark.parametrize("splits", [1, 3])
@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("m,n", TC_SHAPES)
def test_normal_matrix_tf32_tensor_cores(pdas, m, n, storage, splits):
    """TF32 form (tcgen05 kind::tf32, one product or TF32 x 3): the lower
    triangle of M = A D A' against the FP64 oracle within the rounding bound,
    and its scaled error near 2^-10 (one product) or FP32 level (three)."""
    lp = lpgen.generate(m, n, seed=7 * m + n, storage=storage)
    rng = np.random.default_rng(12)
    x, s = rng.uniform(0.01, 10, n), rng.uniform(0.01, 10, n)
    with pdas.Solver(m, n, "tf32_ir", TORCH_DT[storage], splits=splits) as S:
        S.form_normal(dev_A(lp), dv(x), dv(s))
        M = host(S.copy_matrix()).astype(np.float64)
    D = oracle.scaling(x, s)
    ref = oracle.normal_matrix(lp.A64, D)
    low = np.tril_indices(m)
    assert np.all(np.abs(M[low] - ref[low]) <= tf32_bound(lp.A64, D, n, splits)[low])
    assert scaled_error(M, ref) <= {1: 4e-3, 3: 1e-5}[splits]


def test_tf32_rounding_is_to_nearest_even(pdas):
    """Entries chosen so that A and D.*A are exact in TF32 or sit exactly on a
    tie: M = A D A' of a 1 x n problem must equal the sum of the TF32 values
    rounded to nearest even (ties: 1 + 2^-11 -> 1, 1 + 3 * 2^-11 -> 1 + 2^-9)."""
    n = 8
    a = np.array([1.0, 1 + 2.0 ** -11, 1 + 3 * 2.0 ** -11, 1 + 2.0 ** -10, 0.5, -0.25, 0.0, 1 + 2.0 ** -12])
    a_tf32 = np.array([1.0, 1.0, 1 + 2.0 ** -9, 1 + 2.0 ** -10, 0.5, -0.25, 0.0, 1.0])
    # every product and partial sum is a multiple of 2^-20 below 8: exact in FP32
    x, s = np.ones(n), np.ones(n)  # D = 1: D.*A = A
    with pdas.Solver(1, n, "tf32_ir", torch.float64, splits=1) as S:
        S.form_normal(dv(a.reshape(1, n)), dv(x), dv(s))
        M = host(S.copy_matrix()).astype(np.float64)
    assert M[0, 0] == float(np.sum(a_tf32 * a_tf32))


@pytest.mark.parametrize("splits", [1, 3])
@pytest.mark.parametrize("seed", [0, 1])
def test_tf32_ir_solve_matches_oracle(pdas, seed, splits):
    lp = lpgen.generate(64, 128, seed=seed, storage="f64")
    ref = oracle.solve(lp.A64, lp.b, lp.c, lp.x0, lp.y0, lp.s0)
    x, y, s = dv(lp.x0), dv(lp.y0), dv(lp.s0)
    with pdas.Solver(lp.m, lp.n, "tf32_ir", torch.float64, splits=splits) as S:
        out = S.solve(dev_A(lp), dv(lp.b), dv(lp.c), x, y, s, alpha=0.95, tol=1e-8)
    assert out["status"] == 1
    obj_ref = float(lp.c @ ref["x"])
    assert abs(float(lp.c @ host(x)) - obj_ref) <= 1e-8 * abs(obj_ref)
    assert out["iters"] == ref["iters"]


@pytest.mark.parametrize("splits", [1, 3])
def test_tf32_ir_c2_first_iterations(pdas, splits):
    """2048 x 8192 FP64-stored A in the TF32 form: the refined direction makes
    the first two iterates agree with the oracle's to 1e-9 normwise."""
    lp = lpgen.workload("dense_2048x8192_f64", 0)
    A, b, c = dev_A(lp), dv(lp.b), dv(lp.c)
    x, y, s = dv(lp.x0), dv(lp.y0), dv(lp.s0)
    xo, yo, so = lp.x0.copy(), lp.y0.copy(), lp.s0.copy()
    with pdas.Solver(lp.m, lp.n, "tf32_ir", torch.float64, splits=splits) as S:
        for k in range(2):
            st, info = S.step(A, b, c, x, y, s, alpha=0.95)
            assert not info["used_fp64"]
            d = oracle.direction(lp.A64, xo, so)
            th = oracle.theta(oracle.psi(xo, so, d["dx"], d["ds"]), 0.95)
            xo, yo, so = oracle.step(xo, yo, so, d["dx"], d["dy"], d["ds"], th)
            for g, o in ((x, xo), (y, yo), (s, so)):
                assert np.linalg.norm(host(g) - o) <= 1e-9 * np.linalg.norm(o), k


def infeasible_point(lp, seed):
    """A seeded interior point with A x != b and A'y + s != c."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.5, 2.0, lp.n), rng.standard_normal(lp.m), rng.uniform(0.5, 2.0, lp.n)


@pytest.mark.parametrize("form,storage", [("fp64", "f64"), ("fp32_ir", "f32"), ("bf16_ir", "bf16"),
                                          ("tf32_ir", "f64")])
def test_infeasible_direction_matches_oracle(pdas, form, storage):
    """Infeasible-start variant: the direction at an infeasible interior point
    against the oracle's, normwise to 1e-9 (the mixed forms refine dy to the
    FP64 backward-error level), and the residual rows of Eq. (3)."""
    lp = lpgen.generate(130, 520, seed=21, storage=storage)
    x, y, s = infeasible_point(lp, 5)
    ref = oracle.direction_infeasible(lp.A64, lp.b, lp.c, x, y, s)
    with pdas.Solver(lp.m, lp.n, form, TORCH_DT[storage], infeasible=1) as S:
        dx, dy, ds, info = S.direction_infeasible(dev_A(lp), dv(lp.b), dv(lp.c), dv(x), dv(y), dv(s))
    for got, want in ((dx, ref["dx"]), (dy, ref["dy"]), (ds, ref["ds"])):
        assert np.linalg.norm(host(got) - want) <= 1e-9 * np.linalg.norm(want)
    A = lp.A64
    assert np.abs(A @ host(dx) - (lp.b - A @ x)).max() <= 1e-9 * (1 + np.abs(lp.b).max())
    assert np.abs(A.T @ host(dy) + host(ds) - (lp.c - A.T @ y - s)).max() <= 1e-12 * (1 + np.abs(lp.c).max())


@pytest.mark.parametrize("seed", [0, 1])
def test_infeasible_fp64_iterates_match_oracle(pdas, seed):
    """FP64 form, infeasible start at 64 x 128: every iterate normwise to 1e-9
    of the oracle's, the same iteration count, and the reported residuals."""
    lp = lpgen.workload("dense_64x128_f64", seed)
    x0, y0, s0 = infeasible_point(lp, 50 + seed)
    ref = oracle.solve(lp.A64, lp.b, lp.c, x0, y0, s0, tol=1e-8, keep_iterates=True, infeasible=True)
    assert ref["status"] == oracle.OPTIMAL
    n, m = lp.n, lp.m
    A, b, c = dev_A(lp), dv(lp.b), dv(lp.c)
    x, y, s = dv(x0), dv(y0), dv(s0)
    with pdas.Solver(m, n, "fp64", infeasible=1) as S:
        for k in range(ref["iters"]):
            st, info = S.step(A, b, c, x, y, s, alpha=0.95)
            assert st == 0
            it = ref["iterates"][k]
            for g, o in ((x, it[:n]), (y, it[n:n + m]), (s, it[n + m:])):
                assert np.linalg.norm(host(g) - o) <= 1e-9 * np.linalg.norm(o), k
            # the reported residuals are those of the GPU's iterate (sums
            # that cancel: rounding ~ n u |A| |x| / (1 + |b|)), and track the
            # oracle's run until they reach the floor that the solves'
            # forward error sets (~1e-10 here), where the two runs' rounding
            # decides them
            pres, dres = oracle.residuals(lp.A64, lp.b, lp.c, host(x), host(y), host(s))
            assert abs(info["pres"] - pres) <= 1e-9 * pres + 1e-13, k
            assert abs(info["dres"] - dres) <= 1e-9 * dres + 1e-13, k
            pres_o, dres_o = ref["res_trace"][k]
            assert abs(info["pres"] - pres_o) <= 1e-3 * pres_o + 1e-10, k
            assert abs(info["dres"] - dres_o) <= 1e-3 * dres_o + 1e-10, k
        x, y, s = dv(x0), dv(y0), dv(s0)
        out = S.solve(A, b, c, x, y, s, alpha=0.95, tol=1e-8)
    assert out["status"] == 1 and out["iters"] == ref["iters"]


@pytest.mark.parametrize("form,storage", [("bf16_ir", "bf16"), ("fp32_ir", "f32"), ("tf32_ir", "f64")])
def test_infeasible_mixed_solve(pdas, form, storage):
    """Mixed forms from an infeasible start at 512 x 2048: the oracle's optimal
    objective to 1e-8 and both residuals below the tolerance."""
    lp = lpgen.generate(512, 2048, seed=3, storage=storage, scaled=storage == "bf16")
    x0, y0, s0 = infeasible_point(lp, 8)
    ref = oracle.solve(lp.A64, lp.b, lp.c, x0, y0, s0, tol=1e-8, infeasible=True)
    assert ref["status"] == oracle.OPTIMAL
    x, y, s = dv(x0), dv(y0), dv(s0)
    with pdas.Solver(lp.m, lp.n, form, TORCH_DT[storage], infeasible=1) as S:
        out = S.solve(dev_A(lp), dv(lp.b), dv(lp.c), x, y, s, alpha=0.95, tol=1e-8)
    assert out["status"] == 1
    obj_ref = float(lp.c @ ref["x"])
    assert abs(float(lp.c @ host(x)) - obj_ref) <= 1e-8 * abs(obj_ref)
    pres, dres = oracle.residuals(lp.A64, lp.b, lp.c, host(x), host(y), host(s))
    assert pres < 1e-8 and dres < 1e-8
    assert abs(out["iters"] - ref["iters"]) <= 1


def test_infeasible_entry_needs_the_option(pdas):
    lp = lpgen.generate(5, 12, seed=1)
    x, y, s = infeasible_point(lp, 1)
    with pdas.Solver(lp.m, lp.n, "fp64") as S:
        with pytest.raises(pdas.PdasError):
            S.direction_infeasible(dev_A(lp), dv(lp.b), dv(lp.c), dv(x), dv(y), dv(s))


def test_full_size_bf16_tensor_core_sampled(pdas):
    """8192 x 32768, the benchmark's configuration (BF16 tensor-core form,
    the default 3 split terms of D.*A): sampled entries of M against the
    oracle one by one within the 3-term bound of tc_bound, and the
    direction's defining identities at full size."""
    lp = lpgen.workload("dense_8192x32768_bf16_colscaled", 0)
    m, n = lp.m, lp.n
    rng = np.random.default_rng(12)
    with pdas.Solver(m, n, "bf16_ir", torch.bfloat16) as S:
        assert S.options.splits in (0, 3)  # 0 selects the default, 3
        A = dev_A(lp)
        x, s = dv(lp.x0), dv(lp.s0)
        S.form_normal(A, x, s)
        M = S.copy_matrix()
        pairs = [(int(p), int(q)) for p, q in zip(rng.integers(0, m, 48), rng.integers(0, m, 48))]
        pairs = [(max(p, q), min(p, q)) for p, q in pairs] + [(m - 1, m - 1), (m - 1, 0), (0, 0), (4095, 4095)]
        got = {pq: float(M[pq[0], pq[1]]) for pq in pairs}
        del M
        dx, dy, ds, info = S.direction(A, x, s)
    # the identities through the FP64 passes (the ones the direction uses; the
    # component entry points of a default mixed handle run the double-float pass)
    with pdas.Solver(m, n, "bf16_ir", torch.bfloat16, exact_passes=1) as E:
        adx = host(E.gemv(A, dx))
        w = host(E.gemv_t(A, dy))
    D = lp.x0 / lp.s0
    diag = {p: oracle.normal_entry(lp.A64, D, p, p) for pq in got for p in pq}
    for (p, q), g in got.items():
        o = oracle.normal_entry(lp.A64, D, p, q)
        t = float((np.abs(lp.A64[p]) * D) @ np.abs(lp.A64[q]))
        # the handle runs the default 3 split terms (as the benchmark does)
        rep, acc = 2.0 ** -24 + 2.0 ** -22, gamma(8 * 3 + 1, 2.0 ** -23) + gamma(n // 128 + 2, 2.0 ** -24)
        assert abs(g - o) <= (rep + acc + rep * acc) * t, (p, q, g, o)
        assert abs(g - o) <= 1e-5 * np.sqrt(diag[p] * diag[q]), (p, q)
    # A dx = M dy - A x is the refinement residual: at most refine accept x ||A x||
    r = lp.A64 @ lp.x0
    assert np.abs(adx).max() <= 1e-11 * np.abs(r).max(), np.abs(adx).max() / np.abs(r).max()
    assert np.array_equal(host(ds), -w)
    xh, sh = lp.x0, lp.s0
    assert np.abs(host(dx) / xh + host(ds) / sh + 1).max() <= 1e-10
    print("full-size direction: refinement sweeps %d, residual %.2e" % (info["refine_sweeps"], info["refine_resid"]))


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_gemv_widening_special_values(pdas, storage):
    """The passes over A widen FP32 / BF16 to FP64 bit by bit on the integer
    pipes: signed zeros, FP32 subnormals and values near the FP32 range
    limits must widen exactly (checked through A v with one-hot v)."""
    m, n = 4, 64
    vals = np.array([0.0, -0.0, 1.0, -1.5, 3.0e38, -2.5e-38, 1.0e-40, -7.0e-45, 65504.0, 1.17549435e-38,
                     np.float32(np.pi), -np.float32(1e-3)], dtype=np.float64)
    A64 = np.zeros((m, n))
    A64.flat[: vals.size] = vals
    A64.flat[vals.size: 2 * vals.size] = -vals
    if storage == "f32":
        At = torch.from_numpy(A64.astype(np.float32)).cuda()
        ref = A64.astype(np.float32).astype(np.float64)
    else:
        bits = lpgen.round_bf16_bits(A64)
        At = torch.from_numpy(bits.view(np.int16).copy()).view(torch.bfloat16).cuda()
        ref = lpgen.bf16_bits_to_f64(bits)
    with pdas.Solver(m, n, "fp64", TORCH_DT[storage]) as S:
        for j in range(n):
            e = np.zeros(n)
            e[j] = 1.0
            col = host(S.gemv(At, dv(e)))
            # bit for bit what the oracle's A v gives (a sum started at +0 turns -0 into +0)
            want = oracle.gemv(ref, e)
            assert np.array_equal(col.view(np.int64), want.view(np.int64)), (j, col, want)


# ---------------------------------------------------------------------------
# the FP64 tier of a mixed form: double-float normal matrix, dropped columns

@pytest.mark.parametrize("storage", ["bf16", "f32"])
@pytest.mark.parametrize("m,n", [(5, 37), (130, 520), (257, 1024)])
def test_double_float_normal_matrix(pdas, storage, m, n):
    """Once a mixed form runs an FP64 factor, M is formed in double-float on
    the FP32 pipes (A exact in FP32): D.*A to ~2^-48 and TwoSum accumulation,
    so |M_df - M| <= 2 n 2^-46 (|A| D |A|') elementwise."""
    lp = lpgen.generate(m, n, seed=m + 3, storage=storage, scaled=True)
    rng = np.random.default_rng(13)
    x, s = rng.uniform(0.01, 10, n), rng.uniform(0.01, 10, n)
    form = "bf16_ir" if storage == "bf16" else "fp32_ir"
    with pdas.Solver(m, n, form, TORCH_DT[storage], dspread_refactor=1e-300, fp64_tier_tc=0) as S:
        A = dev_A(lp)
        _, _, _, info = S.direction(A, dv(x), dv(s))  # the rule switches to the FP64 tier at once
        assert info["used_fp64"] == 1 and info["fp64_reason"] == 1 and info["normal_form"] == 2
        S.form_normal(A, dv(x), dv(s))
        M = host(S.copy_matrix())
    D = oracle.scaling(x, s)
    ref = oracle.normal_matrix(lp.A64, D)
    low = np.tril_indices(m)
    bound = 2 * n * 2.0 ** -46 * ((np.abs(lp.A64) * D) @ np.abs(lp.A64).T)
    assert np.all(np.abs(M[low] - ref[low]) <= bound[low])
    assert scaled_error(M, ref) <= 1e-12


@pytest.mark.parametrize("storage", ["bf16", "f32"])
def test_fp64_tier_whole_solve(pdas, storage):
    """A mixed form forced into its FP64 tier from the first iteration
    (double-float M of the significant columns, FP64 factor, PCG on the whole
    M) reaches the oracle's objective in the oracle's number of iterations."""
    lp = lpgen.generate(256, 1024, seed=21, storage=storage, scaled=True)
    ref = oracle.solve(lp.A64, lp.b, lp.c, lp.x0, lp.y0, lp.s0)
    x, y, s = dv(lp.x0), dv(lp.y0), dv(lp.s0)
    A, b, c = dev_A(lp), dv(lp.b), dv(lp.c)
    form = "bf16_ir" if storage == "bf16" else "fp32_ir"
    cols = []
    forms = []
    with pdas.Solver(lp.m, lp.n, form, TORCH_DT[storage], dspread_refactor=1e-300) as S:
        for k in range(ref["iters"]):
            st, info = S.step(A, b, c, x, y, s, alpha=0.95)
            assert info["used_fp64"] == 1
            cols.append(info["factor_columns"])
            forms.append(info["normal_form"])
    # BF16 A: the tensor-core digit planes (4), unless a factor failed and the
    # iteration re-formed M in FP64 (3); FP32 A: double-float (2)
    assert set(forms) <= ({4, 3} if storage == "bf16" else {2, 3}) and forms[0] == (4 if storage == "bf16" else 2)
    assert info["rel_gap"] < 1e-8
    obj_ref = float(lp.c @ ref["x"])
    assert abs(float(lp.c @ host(x)) - obj_ref) <= 1e-8 * abs(obj_ref)
    assert min(cols) < lp.n  # columns were dropped late in the solve
    xh, yh, sh = host(x), host(y), host(s)
    assert np.linalg.norm(lp.A64 @ xh - lp.b) <= 1e-9 * np.linalg.norm(lp.b)
    assert np.linalg.norm(lp.A64.T @ yh + sh - lp.c) <= 1e-12 * np.linalg.norm(lp.c)


@pytest.mark.parametrize("m", [320, 300])
def test_tensor_core_factor_whole_solve(pdas, m):
    """BF16 A forced into the FP64 tier from the first iteration at m = 320
    and 300 (above the size where the tier's factor moves to the tensor
    cores: five 64-column panels, ragged trailing tiles; at 300 the last
    panel is 44 columns wide, so the diagonal block factored inside the last
    update is narrower than a panel): every iteration's direction comes from
    the digit-plane normal matrix and the tensor-core factor (no fallback
    after a failed pivot), and the solve reaches the oracle's objective in
    the oracle's number of iterations."""
    lp = lpgen.generate(m, 4 * m, seed=23, storage="bf16", scaled=True)
    ref = oracle.solve(lp.A64, lp.b, lp.c, lp.x0, lp.y0, lp.s0)
    x, y, s = dv(lp.x0), dv(lp.y0), dv(lp.s0)
    A, b, c = dev_A(lp), dv(lp.b), dv(lp.c)
    with pdas.Solver(lp.m, lp.n, "bf16_ir", torch.bfloat16, dspread_refactor=1e-300) as S:
        for k in range(ref["iters"]):
            st, info = S.step(A, b, c, x, y, s, alpha=0.95)
            assert info["used_fp64"] == 1 and info["normal_form"] == 4 and info["factor_form"] == 4, (k, info)
    assert info["rel_gap"] < 1e-8
    obj_ref = float(lp.c @ ref["x"])
    assert abs(float(lp.c @ host(x)) - obj_ref) <= 1e-8 * abs(obj_ref)


@pytest.mark.parametrize("m", [300, 700, 1000])
def test_tensor_core_factor_ragged(pdas, m):
    """The FP64 tier's tensor-core factor (FP64 diagonal blocks, the next
    panel's block factored inside the update, FP64 panel rows, trailing
    updates from exact digit planes) at sizes that are not multiples of the
    64-column panel or the 128-row tile.  Every row of |LL' - M| within
    gamma_{m+1}(u64) |L||L'| plus the digits' truncation (2^-40 of
    sqrt(M_pp M_qq), as at full size)."""
    lp = lpgen.generate(m, 4 * m, seed=m, storage="bf16", scaled=True)
    A = dev_A(lp)
    x0, s0 = dv(lp.x0), dv(lp.s0)
    with pdas.Solver(m, lp.n, "bf16_ir", torch.bfloat16, dspread_refactor=1e-300) as S:
        _, _, _, info = S.direction(A, x0, s0)
        assert info["used_fp64"] == 1 and info["factor_form"] == 4, info
        S.form_normal(A, x0, s0)
        M = host(S.copy_matrix()).astype(np.float64)
        S.factor()
        L = np.tril(host(S.copy_matrix()).astype(np.float64))
    Ml = np.tril(M) + np.tril(M, -1).T
    d = np.sqrt(np.diag(Ml))
    err = np.abs(L @ L.T - Ml)
    bound = gamma(m + 1, U64) * (np.abs(L) @ np.abs(L).T) + 2.0 ** -40 * np.outer(d, d)
    assert np.all(err <= bound), float((err / bound).max())
    assert float((err / np.outer(d, d)).max()) <= 1e-14


def test_stop_rules_match_oracle(pdas):
    """The cap and the stall rule of pdas_solve against the oracle's (both are
    readings: the paper states neither).  A run capped at 3 iterations
    returns MAX_ITER on the oracle's third iterate (normwise 1e-9); with
    alpha chosen so that every step has theta = alpha/psi = 0.5e-12 the run
    stops STALLED after exactly 5 steps, with theta = 2e-12 it does not stall
    within 8 steps."""
    lp = lpgen.generate(6, 15, seed=5)
    n, m = lp.n, lp.m
    ref = oracle.solve(lp.A64, lp.b, lp.c, lp.x0, lp.y0, lp.s0, max_iter=3)
    d = oracle.direction(lp.A64, lp.x0, lp.s0)
    psi0 = oracle.psi(lp.x0, lp.s0, d["dx"], d["ds"])
    A, b, c = dev_A(lp), dv(lp.b), dv(lp.c)
    with pdas.Solver(m, n, "fp64", max_iter=3) as S:
        x, y, s = dv(lp.x0), dv(lp.y0), dv(lp.s0)
        out = S.solve(A, b, c, x, y, s)
        assert out["status"] == 3 and out["iters"] == 3 and ref["status"] == oracle.MAX_ITER
        for g, o in ((x, ref["x"]), (y, ref["y"]), (s, ref["s"])):
            assert np.linalg.norm(host(g) - o) <= 1e-9 * np.linalg.norm(o)
    with pdas.Solver(m, n, "fp64", max_iter=8) as S:
        for theta, status, iters in ((0.5e-12, 4, 5), (2e-12, 3, 8)):
            x, y, s = dv(lp.x0), dv(lp.y0), dv(lp.s0)
            out = S.solve(A, b, c, x, y, s, alpha=theta * psi0)
            assert (out["status"], out["iters"]) == (status, iters), (theta, out)


def test_bounded_wait_times_out_and_recovers(pdas):
    """Failure detection without a fault: the blocked triangular solves hand
    results from block to block through bounded waits.  With a 1 us limit the
    wait of block 1 for block 0 (a few us of work) gives up, the call returns
    PDAS_ERR_TIMEOUT instead of hanging, and every block leaves the launch.
    With the default limit restored, the same handle solves again, bit for
    bit as before, and against the oracle's substitutions on its factor."""
    m = 4096
    rng = np.random.default_rng(31)
    G = rng.standard_normal((m, m + 64))
    M = G @ G.T / (m + 64) + np.eye(m)
    rhs = rng.standard_normal(m)
    with pdas.Solver(m, m + 1, "fp32_ir", torch.float32) as S:
        S.load_matrix(dv(M).float())
        S.factor()
        first = host(S.factor_solve(dv(rhs)))
        S.set_wait_limit(1)
        with pytest.raises(pdas.PdasError) as err:
            S.factor_solve(dv(rhs))
        assert err.value.code == -5  # PDAS_ERR_TIMEOUT
        S.set_wait_limit(0)
        again = host(S.factor_solve(dv(rhs)))
        L = np.tril(host(S.copy_matrix()).astype(np.float64))
    assert np.array_equal(first, again)
    xo = oracle.backward(L, oracle.forward(L, rhs))
    assert np.linalg.norm(again - xo) <= 1e-4 * np.linalg.norm(xo)


def digit_bound(A64, D, kept):
    """|M_dig - M| elementwise for the tensor-core digit planes of the FP64
    tier (kept columns only): the FP64 rounding of D_j A_qj and the final
    FP64 combination (within 2 gamma_{k+2}(u64) sum |A_pj| D_j |A_qj|, which
    also covers the oracle's own rounding), the rounding of A entries below
    2^-32 of their row's largest to the last digit (<= 2^-40 2^ea_p each,
    times sum_j |B_qj|), and the digit pairs of weight 8 and more that are
    not formed (<= 2^-62 2^(ea_p + eb_q) per column)."""
    Ak, Dk = A64[:, kept], D[kept]
    k = Ak.shape[1]
    B = np.abs(Ak) * Dk
    ea = np.array([np.frexp(v)[1] if v > 0 else 0 for v in np.abs(Ak).max(1)], dtype=np.float64)
    eb = np.array([np.frexp(v)[1] if v > 0 else 0 for v in B.max(1)], dtype=np.float64)
    S = np.abs(Ak) @ B.T
    return (2 * gamma(k + 2, U64) * S + np.outer(2.0 ** (ea - 40), B.sum(1))
            + k * 2.0 ** -62 * np.exp2(ea[:, None] + eb[None, :]))


def kept_columns(D, m, drop_tol=1e-10, drop_keep=1.25):
    """The columns the FP64 tier factors (the rule of pdas_options.drop_tol /
    drop_keep): D_j >= drop_tol max D, at least ceil(drop_keep m) of the largest."""
    n = D.size
    t = drop_tol * D.max()
    kmin = min(max(int(np.ceil(drop_keep * m)), m), n)
    if np.count_nonzero(D >= t) < kmin:
        t = np.sort(D)[::-1][kmin - 1]
    return np.nonzero(D >= t)[0]


@pytest.mark.parametrize("m,n,spread", [(5, 37, 1e2), (130, 520, 1e6), (257, 1024, 1e2), (300, 1000, 1e20),
                                        (200, 3000, 1e30), (1024, 4096, 1e4)])
def test_digit_normal_matrix(pdas, m, n, spread):
    """The FP64 tier's normal matrix of a BF16-stored A on the tensor cores
    (fixed-point BF16 digit planes, exact products and exact sums): against
    the oracle's FP64 normal matrix of the kept columns, elementwise within
    digit_bound, and FP64-grade relative to sqrt(M_pp M_qq).  D = x/s spans
    about spread^2; beyond 1e10 the tier drops columns (the gather path of
    the planes)."""
    lp = lpgen.generate(m, n, seed=m + 11, storage="bf16", scaled=True)
    rng = np.random.default_rng(17)
    x = np.exp(rng.uniform(-0.5, 0.5, n) * np.log(spread))
    s = 1.0 / np.exp(rng.uniform(-0.5, 0.5, n) * np.log(spread))
    with pdas.Solver(m, n, "bf16_ir", torch.bfloat16, dspread_refactor=1e-300) as S:
        A = dev_A(lp)
        # a direction at a benign point: the rule moves the handle to its FP64 tier for good
        _, _, _, info = S.direction(A, dv(np.ones(n)), dv(np.ones(n)))
        assert info["used_fp64"] == 1 and info["fp64_reason"] == 1 and info["normal_form"] == 4
        S.form_normal(A, dv(x), dv(s))
        M = host(S.copy_matrix())
    D = oracle.scaling(x, s)
    kept = kept_columns(D, m)
    if spread >= 1e20:
        assert kept.size < n  # the gather path of the planes runs
    ref = oracle.normal_matrix(lp.A64[:, kept], D[kept])
    low = np.tril_indices(m)
    assert np.all(np.abs(M[low] - ref[low]) <= digit_bound(lp.A64, D, kept)[low])
    assert scaled_error(M, ref) <= 1e-13


def test_digit_tier_option_off(pdas):
    """fp64_tier_tc = 0 keeps the double-float formation of the FP64 tier."""
    lp = lpgen.generate(130, 520, seed=3, storage="bf16", scaled=True)
    x, s = np.ones(lp.n), np.ones(lp.n)
    with pdas.Solver(lp.m, lp.n, "bf16_ir", torch.bfloat16, dspread_refactor=1e-300, fp64_tier_tc=0) as S:
        _, _, _, info = S.direction(dev_A(lp), dv(x), dv(s))
    assert info["normal_form"] == 2
