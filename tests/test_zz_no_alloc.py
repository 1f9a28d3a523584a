"""pdas_gemv_t_noalloc: A' u for callers that cannot allocate device memory
(code running under someone else's stream capture, memory owned by another
framework's pool, real-time loops).  It keeps its scratch in a fixed
file-scope device array instead of a handle's workspace; these checks call it
through the C ABI and compare it with the handle-based pdas_gemv_t and with
the oracle's A' u.

This file is collected last on purpose, so that a failure here cannot stop
a run of the other tests early."""
import ctypes

import numpy as np
import pytest
import torch

import lpgen
import oracle

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53
DT = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}


def dev_A(lp):
    if lp.storage == "bf16":
        return torch.from_numpy(lp.A_store.view(np.int16).copy()).view(torch.bfloat16).cuda()
    return torch.from_numpy(np.ascontiguousarray(lp.A_store)).cuda()


@pytest.mark.parametrize("m,n,storage", [(5, 37, "f64"), (130, 520, "bf16"), (300, 1001, "f32"),
                                         (2048, 8192, "f64"), (1024, 40000, "bf16")])
def test_noalloc_matches_handle_entry_point_twice(m, n, storage):
    from paper_1502_03543_gb300 import build as B
    B.build()
    import paper_1502_03543_gb300 as P
    from paper_1502_03543_gb300 import _native as N

    lp = lpgen.generate(m, n, seed=m, storage=storage, scaled=storage == "bf16")
    A = dev_A(lp)
    rng = np.random.default_rng(9)
    us = [torch.from_numpy(rng.standard_normal(m)).cuda() for _ in range(2)]
    stream = torch.cuda.current_stream()
    with P.Solver(m, n, "fp64", DT[storage]) as S:
        refs = [S.gemv_t(A, u).cpu().numpy() for u in us]
    absA = np.abs(lp.A64)
    for u, ref in zip(us, refs):  # two calls in a row share the scratch
        out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        st = N.lib().pdas_gemv_t_noalloc(m, n, {"f64": N.A_F64, "f32": N.A_F32, "bf16": N.A_BF16}[storage],
                                         ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert st == N.OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        # two FP64 summation orders of the same m-term column sums
        bound = 2 * (m * U64 / (1 - m * U64)) * (absA.T @ np.abs(u.cpu().numpy()))
        assert np.all(np.abs(got - ref) <= bound)
        assert np.all(np.abs(got - oracle.gemv_t(lp.A64, u.cpu().numpy())) <= bound)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1502_03543_gb300 import _native as N
    limit = (8 << 20) // 8 - 32  # (PDAS_NOALLOC_SCRATCH_BYTES - 256) / 8
    one = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(one.data_ptr())
    assert N.lib().pdas_gemv_t_noalloc(1, limit + 1, N.A_F64, p, p, p, None) == N.ERR_ARG
    assert N.lib().pdas_gemv_t_noalloc(0, 5, N.A_F64, p, p, p, None) == N.ERR_ARG
