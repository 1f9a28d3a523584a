"""The seeded LP generator: bf16 storage rounding agrees with torch's
round-to-nearest-even conversion, the start is strictly interior and
feasible, and the draws are reproducible."""
import numpy as np
import torch

import lpgen


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    v = np.concatenate([rng.standard_normal(100000) * 10.0 ** rng.integers(-20, 20, 100000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.005859375, 3.0e38]])
    ours = lpgen.round_bf16_bits(v)
    ref = torch.from_numpy(v.astype(np.float32)).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(ours, ref)
    back = lpgen.bf16_bits_to_f64(ours)
    assert np.array_equal(back, torch.from_numpy(ours.view(np.int16)).view(torch.bfloat16).double().numpy())


def test_start_is_interior_and_feasible():
    for storage, scaled in [("f64", False), ("f32", False), ("bf16", True)]:
        lp = lpgen.generate(17, 45, seed=3, storage=storage, scaled=scaled)
        assert lp.A_store.shape == (17, 45)
        assert np.all(lp.x0 >= 0.5) and np.all(lp.x0 <= 1.5) and np.all(lp.s0 >= 0.5) and np.all(lp.s0 <= 1.5)
        assert np.abs(lp.A64 @ lp.x0 - lp.b).max() <= 1e-12 * np.abs(lp.A64).sum(1).max()
        assert np.abs(lp.A64.T @ lp.y0 + lp.s0 - lp.c).max() <= 1e-12 * (1 + np.abs(lp.A64).sum(0).max())
        if storage == "f32":
            assert np.array_equal(lp.A64, lp.A_store.astype(np.float64))


def test_reproducible():
    a = lpgen.generate(8, 20, seed=11, storage="bf16", scaled=True)
    b = lpgen.generate(8, 20, seed=11, storage="bf16", scaled=True)
    assert np.array_equal(a.A_store, b.A_store) and np.array_equal(a.b, b.b) and np.array_equal(a.c, b.c)
    c = lpgen.generate(8, 20, seed=12, storage="bf16", scaled=True)
    assert not np.array_equal(a.A_store, c.A_store)
