"""The task order of the single-launch tile Cholesky (host logic, no GPU).

The kernel hands tasks out in list order and a CTA waits only for the tile
counters its task needs.  It cannot deadlock if every task's waits are met
once all EARLIER tasks have finished; executing the list in order on the CPU
checks exactly that, and checks that the list is complete.  Replaying the
tile operations of the list in numpy (FP64) must give the Cholesky factor.
Task kinds: 0 = last update of diagonal tile (l, l), then its factor; 1 =
last update of tile (i, l), i >= l + 2, then its solve against L_ll; 2 =
update of tile (i, l) by step k <= l - 2, or k = l - 1 when i = l + 1; 3 =
inverse of the diagonal factor L_ll (for the blocked triangular solves); 4 =
solve of the sub-diagonal tile (l + 1, l) against L_ll, all its updates
applied (run with kind 0 by one CTA, in the order 0(0), 4(1,0), 0(1), ...)."""
import ctypes

import numpy as np
import pytest

FINAL_DIAG, FINAL_OFF, UPDATE, INV, CHAIN_SOLVE = 0, 1, 2, 3, 4
TILE = 128


def tasks(m, nproc=304):
    from paper_1502_03543_gb300 import build as B
    B.build()
    from paper_1502_03543_gb300 import _native as N
    L = N.lib()
    n = L.pdas_chol_tile_tasks(m, nproc, None, 0)
    out = (ctypes.c_int32 * max(1, 4 * n))()
    assert L.pdas_chol_tile_tasks(m, nproc, out, n) == n
    return [tuple(int(v) for v in row) for row in np.frombuffer(out, dtype=np.int32)[: 4 * n].reshape(n, 4)]


@pytest.mark.parametrize("m,nproc", [(1, 304), (128, 304), (129, 1), (300, 2), (1000, 304), (4096, 304),
                                     (4096, 7), (8192, 304)])
def test_every_task_once_and_waits_met_by_earlier_tasks(m, nproc):
    got = tasks(m, nproc)
    nb = -(-m // TILE)
    want = {(FINAL_DIAG, l, l, l - 1) for l in range(nb)}
    want |= {(FINAL_OFF, i, l, l - 1) for l in range(nb) for i in range(l + 2, nb)}
    want |= {(CHAIN_SOLVE, l + 1, l, l) for l in range(nb - 1)}
    want |= {(UPDATE, i, l, k) for l in range(nb) for k in range(l - 1) for i in range(l, nb)}
    want |= {(UPDATE, l + 1, l, l - 1) for l in range(1, nb - 1)}
    want |= {(INV, l, l, 0) for l in range(nb)}
    assert len(got) == len(set(got)) and set(got) == want
    state = np.zeros((nb, nb), dtype=np.int64)  # updates applied; l + 1 once final
    for kind, i, l, k in got:
        if kind == INV:
            assert state[l, l] == l + 1
            continue
        if kind == UPDATE:
            assert state[i, k] >= k + 1 and state[l, k] >= k + 1 and state[i, l] == k
            state[i, l] = k + 1
            continue
        if kind == CHAIN_SOLVE:
            assert i == l + 1 and state[l, l] == l + 1 and state[i, l] == l
            state[i, l] = l + 1
            continue
        if l > 0:  # the last update, by tile column l - 1
            assert state[i, l - 1] >= l and state[l, l - 1] >= l and state[i, l] == l - 1
        if kind == FINAL_OFF:
            assert state[l, l] == l + 1  # the diagonal factor it solves against
        state[i, l] = l + 1
    assert all(state[i, l] == l + 1 for l in range(nb) for i in range(l, nb))


@pytest.mark.parametrize("m", [300, 513])
def test_replaying_the_tasks_gives_the_factor(m):
    rng = np.random.default_rng(m)
    G = rng.standard_normal((m, m + 7))
    M = G @ G.T + m * np.eye(m)
    W = np.tril(M).copy()
    s = lambda t: slice(t * TILE, min(m, (t + 1) * TILE))
    for kind, i, l, k in tasks(m, 3):
        if kind == INV:
            continue
        if kind == CHAIN_SOLVE:
            W[s(i), s(l)] = np.linalg.solve(W[s(l), s(l)], W[s(i), s(l)].T).T
            continue
        if kind == UPDATE or l > 0:
            kk = k if kind == UPDATE else l - 1
            W[s(i), s(l)] -= W[s(i), s(kk)] @ W[s(l), s(kk)].T
        if kind == FINAL_DIAG:
            B = np.tril(W[s(l), s(l)])
            W[s(l), s(l)] = np.linalg.cholesky(B + np.tril(B, -1).T)
        elif kind == FINAL_OFF:
            W[s(i), s(l)] = np.linalg.solve(W[s(l), s(l)], W[s(i), s(l)].T).T
    W = np.tril(W)
    assert np.abs(W - np.linalg.cholesky(M)).max() <= 1e-12 * np.abs(W).max()


def test_the_chain_order_is_consistent_with_the_list():
    """One CTA runs kinds 0 and 4 in the order 0(0), 4(1,0), 0(1), 4(2,1), ...,
    the others the remaining tasks in list order.  The list must place every
    chain task after everything it waits for and before everything that
    waits for it, so that order is a topological one too."""
    for m in (300, 1000, 4096):
        got = tasks(m, 5)
        pos = {t: n for n, t in enumerate(got)}
        nb = -(-m // TILE)
        chain = []
        for l in range(nb):
            chain.append((FINAL_DIAG, l, l, l - 1))
            if l + 1 < nb:
                chain.append((CHAIN_SOLVE, l + 1, l, l))
        assert [pos[t] for t in chain] == sorted(pos[t] for t in chain)
