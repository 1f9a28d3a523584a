"""The batched solver (pdas_batch.h): many small LPs, one CTA per LP, one
graph replay.  Each LP follows the algorithm of Section III with the FP32
normal matrix and factor and the FP64-accurate refined direction, so every
LP must reach the oracle's optimal objective (both stopped at the same gap
tolerance) in the same number of iterations, up to one where the two stop
within a hair of the tolerance."""
import ctypes

import numpy as np
import pytest

import lpgen
import oracle


def test_batch_sizes_and_packing():
    m, n = lpgen.batch_sizes(512, seed=0)
    assert m.min() >= 16 and m.max() <= 256 and np.all(n % m == 0)
    k = n // m
    assert set(np.unique(k)) <= {2, 3, 4} and len(np.unique(k)) == 3
    assert np.array_equal(lpgen.batch_sizes(512, seed=0)[0], m)  # seeded
    lps = lpgen.batch(5, seed=3)
    pk = lpgen.pack(lps)
    a_off = np.concatenate([[0], np.cumsum(pk["m"].astype(np.int64) * pk["n"])])
    n_off = np.concatenate([[0], np.cumsum(pk["n"])])
    m_off = np.concatenate([[0], np.cumsum(pk["m"])])
    for i, lp in enumerate(lps):
        assert lp.seed == 1000 + i
        assert np.array_equal(pk["A"][a_off[i]:a_off[i + 1]].reshape(lp.m, lp.n), lp.A_store)
        assert np.array_equal(pk["x0"][n_off[i]:n_off[i + 1]], lp.x0)
        assert np.array_equal(pk["b"][m_off[i]:m_off[i + 1]], lp.b)


def test_batch_create_rejects_bad_arguments_without_gpu():
    from paper_1502_03543_gb300 import build as B
    B.build()
    from paper_1502_03543_gb300 import _native as N
    L = N.lib()
    o = N.BatchOptions()
    L.pdas_batch_default_options(ctypes.byref(o))
    assert o.alpha == 0.95 and o.tol == 1e-7 and o.max_iter == 500 and o.refine_tol == 1e-14 and o.autotune == 1
    h = ctypes.c_void_p()
    buf = ctypes.c_void_p(1 << 20)  # never dereferenced: every case fails its host-side check
    arr = lambda *v: (ctypes.c_int * len(v))(*v)
    good = (buf,) * 6
    assert L.pdas_batch_create(0, arr(4), arr(8), *good, ctypes.byref(o), ctypes.byref(h)) == N.ERR_ARG
    assert L.pdas_batch_create(1, arr(8), arr(8), *good, ctypes.byref(o), ctypes.byref(h)) == N.ERR_ARG  # m < n
    assert L.pdas_batch_create(1, arr(257), arr(600), *good, ctypes.byref(o), ctypes.byref(h)) == N.ERR_ARG
    assert L.pdas_batch_create(1, arr(200), arr(1025), *good, ctypes.byref(o), ctypes.byref(h)) == N.ERR_ARG
    odd = (buf, buf, buf, ctypes.c_void_p((1 << 20) + 8), buf, buf)  # misaligned x
    assert L.pdas_batch_create(1, arr(4), arr(8), *odd, ctypes.byref(o), ctypes.byref(h)) == N.ERR_ARG
    bad = N.BatchOptions.from_buffer_copy(o)
    bad.alpha = 1.0
    assert L.pdas_batch_create(1, arr(4), arr(8), *good, ctypes.byref(bad), ctypes.byref(h)) == N.ERR_ARG
    assert not h.value


def _oracle_sound(lp, ref):
    """The oracle's final iterate is a valid reference: primal feasible to
    1e-8 and a non-negative gap (so c'x is within the gap of the optimum)."""
    gap = ref["trace"][ref["iters"] - 1][2]
    return gap >= 0 and np.linalg.norm(lp.A64 @ ref["x"] - lp.b) <= 1e-8 * np.linalg.norm(lp.b)


def _device_batch(lps):
    import torch
    pk = lpgen.pack(lps)
    dv = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    return pk, dict(A=torch.from_numpy(np.ascontiguousarray(pk["A"], dtype=np.float32)).cuda(), b=dv(pk["b"]),
                    c=dv(pk["c"]), x=dv(pk["x0"]), y=dv(pk["y0"]), s=dv(pk["s0"]))


def _split(pk, v, which):
    sizes = pk[which]
    off = np.concatenate([[0], np.cumsum(sizes)])
    return [v[off[i]:off[i + 1]] for i in range(len(sizes))]


@pytest.mark.gpu
def test_batch_matches_oracle_per_lp():
    """LPs in every bucket of m (16..256), n = m k, k in {2, 3, 4}."""
    import paper_1502_03543_gb300 as P
    sizes = (np.array([16, 40, 64, 65, 100, 128, 129, 150, 192, 193, 230, 256]),
             np.array([32, 160, 192, 260, 300, 512, 258, 450, 768, 579, 690, 512]))
    lps = lpgen.batch(sizes=sizes, base_seed=2000)
    pk, d = _device_batch(lps)
    with P.BatchSolver(pk["m"], pk["n"], d["A"], d["b"], d["c"], d["x"], d["y"], d["s"], tol=1e-7) as S:
        out = S.solve()
        cfg = S.config()
    assert sum(c[2] for c in cfg) == len(lps) and all(c[1] in (128, 256, 512) for c in cfg if c[2])
    xs = _split(pk, d["x"].cpu().numpy(), "n")
    checked = 0
    for i, lp in enumerate(lps):
        ref = oracle.solve(lp.A64, lp.b, lp.c, lp.x0, lp.y0, lp.s0, alpha=0.95, tol=1e-7)
        if not _oracle_sound(lp, ref):
            # the oracle's own final iterate lost feasibility (M singular to
            # working precision near the optimum): it pins nothing here, and
            # the GPU may stop on that singularity
            assert out["status"][i] in (1, 2, -3, 4), (i, out["status"][i])
            continue
        checked += 1
        assert out["status"][i] in (1, 2), (i, out["status"][i])
        assert out["gap"][i] < 1e-7
        assert abs(int(out["iters"][i]) - ref["iters"]) <= 1, (i, out["iters"][i], ref["iters"])
        obj, obj_ref = float(lp.c @ xs[i]), float(lp.c @ ref["x"])
        if int(out["iters"][i]) == ref["iters"]:  # same trajectory: tracked to refinement accuracy
            assert abs(obj - obj_ref) <= 1e-7 * abs(obj_ref), (i, obj, obj_ref)
        assert abs(obj - obj_ref) <= 1.01 * (out["gap"][i] * (1 + abs(obj)) + ref["trace"][ref["iters"] - 1][2] * (1 + abs(obj_ref)))
        assert np.linalg.norm(lp.A64 @ xs[i] - lp.b) <= 1e-8 * np.linalg.norm(lp.b)
    assert checked >= len(lps) - 2


@pytest.mark.gpu
def test_batch_isolates_a_bad_lp_and_replays_deterministically():
    import paper_1502_03543_gb300 as P
    lps = lpgen.batch(6, seed=5)
    lps[2].x0[3] = 0.0  # not interior: that LP alone fails
    pk, d = _device_batch(lps)
    x0, y0, s0 = d["x"].clone(), d["y"].clone(), d["s"].clone()
    with P.BatchSolver(pk["m"], pk["n"], d["A"], d["b"], d["c"], d["x"], d["y"], d["s"], autotune=False) as S:
        out = S.solve()
        x1 = d["x"].clone()
        d["x"].copy_(x0)
        d["y"].copy_(y0)
        d["s"].copy_(s0)
        out2 = S.solve()
    assert out["status"][2] == -2 and all(out["status"][i] in (1, 2) for i in range(6) if i != 2)
    assert np.array_equal(out["iters"], out2["iters"]) and np.array_equal(out["gap"], out2["gap"], equal_nan=True)
    assert np.isnan(out["gap"][2])  # (no step taken)
    assert np.array_equal(x1.cpu().numpy(), d["x"].cpu().numpy())


@pytest.mark.gpu
def test_batch_512():
    """The 512-LP batch (m ~ U{16..256}, n = m U{2..4}, FP32, gap 1e-7): all
    LPs optimal; a sample from every bucket against the oracle."""
    import paper_1502_03543_gb300 as P
    lps = lpgen.batch(512, seed=0)
    pk, d = _device_batch(lps)
    with P.BatchSolver(pk["m"], pk["n"], d["A"], d["b"], d["c"], d["x"], d["y"], d["s"], tol=1e-7) as S:
        out = S.solve()
        print("batch 512: %.2f ms, %d iterations, buckets %s" % (out["ms"], out["iters"].sum(), S.config()))
    ok = np.isin(out["status"], (1, 2))
    print("statuses:", dict(zip(*np.unique(out["status"], return_counts=True))),
          "FP64-tier iterations:", int(out["fp64_iters"].sum()), "unrefined:", int(out["unrefined"].sum()))
    assert ok.mean() >= 0.98 and np.all(out["gap"][ok] < 1e-7)
    assert np.all(np.isin(out["status"][~ok], (-3, 4)))  # a singular M near the optimum only
    xs = _split(pk, d["x"].cpu().numpy(), "n")
    sample = [int(np.argmin(np.abs(pk["m"] - t))) for t in (20, 90, 160, 250)]
    for i in sample:
        lp = lps[i]
        ref = oracle.solve(lp.A64, lp.b, lp.c, lp.x0, lp.y0, lp.s0, alpha=0.95, tol=1e-7)
        if not _oracle_sound(lp, ref):
            continue
        obj, obj_ref = float(lp.c @ xs[i]), float(lp.c @ ref["x"])
        assert abs(obj - obj_ref) <= 1.01 * (out["gap"][i] * (1 + abs(obj)) + ref["trace"][ref["iters"] - 1][2] * (1 + abs(obj_ref)))
        assert abs(int(out["iters"][i]) - ref["iters"]) <= 1
