"""The paper's own solver of the normal equations on the GPU (Section V-A:
the Woodbury identity as n rank-one updates of A A', the Egidi-Maponi
recurrence; include/pdas_woodbury.h), through the C ABI.

It is compared with the oracle's direction dy (Cholesky of A D A' in FP64)
and with an independent numpy run of the same recurrence (the CPU test
solver of the oracle pins), at early iterates of the oracle's own runs,
where every intermediate matrix is well conditioned (smallest |den_l| at
least 1e-3; below that the recurrence itself loses accuracy, which is why
the library's direction uses the Cholesky path)."""
import numpy as np
import pytest
import torch

import lpgen
import oracle
from test_oracle_pins import sherman_morrison_dy

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


@pytest.mark.parametrize("m,n,seed,storage", [(4, 10, 0, "f64"), (6, 15, 1, "f64"), (8, 20, 2, "f64"),
                                              (64, 128, 0, "f64"), (37, 161, 3, "f32"), (130, 520, 4, "bf16")])
def test_woodbury_matches_oracle_and_cpu_recurrence(pdas, m, n, seed, storage):
    lp = lpgen.generate(m, n, seed=seed, storage=storage, scaled=storage == "bf16")
    res = oracle.solve(lp.A64, lp.b, lp.c, lp.x0, lp.y0, lp.s0, max_iter=3, keep_iterates=True)
    pts = [(lp.x0, lp.s0)] + [(r[:n], r[n + m:]) for r in res["iterates"]]
    if storage == "bf16":
        A = torch.from_numpy(lp.A_store.view(np.int16).copy()).view(torch.bfloat16).cuda()
    else:
        A = torch.from_numpy(np.ascontiguousarray(lp.A_store)).cuda()
    checked = 0
    with pdas.WoodburySolver(m, n, A.dtype) as W:
        W.prepare(A)
        for x, s in pts:
            D = x / s
            r = oracle.gemv(lp.A64, x)
            dy, min_den = W.solve(A, dv(D), dv(r))
            dy = dy.cpu().numpy()
            dy_cpu, min_den_cpu = sherman_morrison_dy(lp.A64, D, r)
            assert abs(min_den - min_den_cpu) <= 1e-8 * max(1.0, min_den_cpu)
            if min_den_cpu < 1e-3:
                continue
            want = oracle.direction(lp.A64, x, s)["dy"]
            assert np.abs(dy - want).max() <= 1e-9 * np.abs(want).max(), (np.abs(dy - want).max(), min_den)
            assert np.abs(dy - dy_cpu).max() <= 1e-9 * np.abs(dy_cpu).max()
            checked += 1
    assert checked >= 2


def test_woodbury_argument_checks(pdas):
    from paper_1502_03543_gb300 import _native as N
    import ctypes
    h = ctypes.c_void_p()
    assert N.lib().pdas_woodbury_create(5, 5, N.A_F64, None, ctypes.byref(h)) == N.ERR_ARG  # m < n required
    assert N.lib().pdas_woodbury_create(20000, 40000, N.A_F64, None, ctypes.byref(h)) == N.ERR_ARG
    lp = lpgen.generate(4, 9, seed=1)
    with pdas.WoodburySolver(4, 9) as W:
        with pytest.raises(pdas.PdasError):  # solve before prepare
            W.solve(dv(lp.A64), dv(np.ones(9)), dv(np.ones(4)))
