"""Seeded synthetic LP generator shared by the tests, the benchmark and the
smoke check.

It holds none of the method's arithmetic: it only draws the random data and
builds a strictly feasible primal-dual start, so that the GPU library and the
CPU oracle can be fed the very same arrays.  The paper (arXiv:1502.03543)
measures on dense LPs whose sizes and data are not given; these inputs stand
in for them.

Recipe (numpy ``default_rng(seed)``, PCG64), draws in this order:
  1. Z ~ N(0,1), shape (m, n), row-major;
  2. optionally sigma ~ U(0.1, 10) per column and A = Z * sigma (columns scaled);
  3. A rounded to its storage dtype with round-to-nearest-even: "f64", "f32"
     or "bf16".  The rounded A defines the LP for every consumer;
  4. x0 ~ U(0.5, 1.5)^n;  5. s0 ~ U(0.5, 1.5)^n;  6. y0 ~ N(0,1)^m;
  7. b = A x0 and c = A' y0 + s0 in FP64, each sum taken left to right in
     increasing index order with separate multiply and add, so the arrays are
     bit-identical on every machine.
x0 > 0 is then primal feasible and (y0, s0 > 0) dual feasible: an interior
start as the algorithm of Section III requires.
"""
from __future__ import annotations

import dataclasses

import numpy as np

STORAGE = ("f64", "f32", "bf16")


def round_bf16_bits(a: np.ndarray) -> np.ndarray:
    """Round float values to bfloat16 (round to nearest, ties to even) and
    return the raw 16-bit patterns as uint16.  Inputs are first rounded to
    float32 (exact for every value produced here that is then rounded again
    to bf16 only when the float32 value is not a tie; the two-step rounding
    is the definition used by the storage format, stated here explicitly)."""
    a32 = np.ascontiguousarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return r.astype(np.uint16)


def bf16_bits_to_f64(bits: np.ndarray) -> np.ndarray:
    """Exact widening of bfloat16 bit patterns to float64."""
    u32 = bits.astype(np.uint32) << 16
    return u32.view(np.float32).astype(np.float64)


@dataclasses.dataclass
class LP:
    m: int
    n: int
    storage: str
    A_store: np.ndarray  # float64 / float32 / uint16 (bf16 bits), shape (m, n)
    A64: np.ndarray  # exact float64 widening of A_store
    b: np.ndarray
    c: np.ndarray
    x0: np.ndarray
    y0: np.ndarray
    s0: np.ndarray
    seed: int
    scaled: bool


def _ltr_matvec(A64: np.ndarray, v: np.ndarray) -> np.ndarray:
    """A v with each row sum taken left to right (column by column)."""
    AT = np.asfortranarray(A64).T  # C-contiguous view of columns
    out = np.zeros(A64.shape[0])
    for j in range(A64.shape[1]):
        out += AT[j] * v[j]
    return out


def _ltr_rmatvec(A64: np.ndarray, v: np.ndarray) -> np.ndarray:
    """A' v with each column sum taken top to bottom (row by row)."""
    out = np.zeros(A64.shape[1])
    for p in range(A64.shape[0]):
        out += A64[p] * v[p]
    return out


def generate(m: int, n: int, seed: int = 0, storage: str = "f64", scaled: bool = False) -> LP:
    """Draw one LP by the recipe in the module docstring."""
    if storage not in STORAGE:
        raise ValueError("storage must be one of %s" % (STORAGE,))
    rng = np.random.default_rng(seed)
    Z = rng.standard_normal((m, n))
    if scaled:
        sigma = rng.uniform(0.1, 10.0, n)
        Z *= sigma
    if storage == "f64":
        A_store = Z
        A64 = Z
    elif storage == "f32":
        A_store = Z.astype(np.float32)
        A64 = A_store.astype(np.float64)
    else:
        A_store = round_bf16_bits(Z)
        A64 = bf16_bits_to_f64(A_store)
    del Z
    x0 = rng.uniform(0.5, 1.5, n)
    s0 = rng.uniform(0.5, 1.5, n)
    y0 = rng.standard_normal(m)
    b = _ltr_matvec(A64, x0)
    c = _ltr_rmatvec(A64, y0) + s0
    return LP(m, n, storage, A_store, A64, b, c, x0, y0, s0, seed, scaled)


# The dense LP workloads, by shape and storage.
WORKLOADS = {
    "dense_64x128_f64": dict(m=64, n=128, storage="f64", scaled=False, tol=1e-8),
    "dense_2048x8192_f64": dict(m=2048, n=8192, storage="f64", scaled=False, tol=1e-8),
    "dense_8192x32768_bf16_colscaled": dict(m=8192, n=32768, storage="bf16", scaled=True, tol=1e-8),
    # a mid-size case of the same family, for kernel profiles (A is 134 MB, larger than L2)
    "dense_4096x16384_bf16_colscaled": dict(m=4096, n=16384, storage="bf16", scaled=True, tol=1e-8),
}


def workload(name: str, seed: int = 0) -> LP:
    w = WORKLOADS[name]
    return generate(w["m"], w["n"], seed=seed, storage=w["storage"], scaled=w["scaled"])


# ---- batches of small LPs ---------------------------------------------------
def batch_sizes(count: int = 512, seed: int = 0, m_lo: int = 16, m_hi: int = 256, k_lo: int = 2, k_hi: int = 4):
    """Sizes of a batch of uneven LPs: numpy default_rng(seed) draws
    m ~ U{m_lo..m_hi} for every instance, then k ~ U{k_lo..k_hi}; n = m k."""
    rng = np.random.default_rng(seed)
    m = rng.integers(m_lo, m_hi + 1, count)
    k = rng.integers(k_lo, k_hi + 1, count)
    return m.astype(np.int64), (m * k).astype(np.int64)


def batch(count: int = 512, seed: int = 0, storage: str = "f32", base_seed: int = 1000, sizes=None):
    """The LPs of a batch: instance i is generate(m_i, n_i, seed=base_seed + i)
    with the sizes of batch_sizes(count, seed) (or the given (m, n) arrays)."""
    m, n = sizes if sizes is not None else batch_sizes(count, seed)
    return [generate(int(m[i]), int(n[i]), seed=base_seed + i, storage=storage) for i in range(len(m))]


def pack(lps):
    """Concatenate a batch in LP order: A (each A_i row-major, in its storage
    dtype), b, c, x0, y0, s0 (float64), and the m, n arrays; the offsets of
    LP i are the prefix sums of m_k n_k, m_k and n_k over k < i."""
    A = np.concatenate([lp.A_store.ravel() for lp in lps])
    cat = lambda f: np.concatenate([getattr(lp, f) for lp in lps]).astype(np.float64)
    return dict(A=A, b=cat("b"), c=cat("c"), x0=cat("x0"), y0=cat("y0"), s0=cat("s0"),
                m=np.array([lp.m for lp in lps], dtype=np.int32), n=np.array([lp.n for lp in lps], dtype=np.int32))


BATCHES = {
    # 512 LPs, m ~ U{16..256}, n = m U{2..4}, FP32 storage, instance seeds 1000 + i
    "batch_512_f32": dict(count=512, seed=0, storage="f32", tol=1e-7),
    # the differentiable batch: 256 LPs of 128 x 384, FP32 storage, instance
    # seeds 1000 + i, stopped at a gap of 1e-6; loss sum_i w_i' x*_i
    "adjoint_256_f32": dict(count=256, m=128, n=384, storage="f32", tol=1e-6),
}
