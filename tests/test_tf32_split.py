"""The TF32 operand arithmetic behind the tensor-core normal matrix, on the
CPU: rounding an FP32 value to TF32 (10 stored mantissa bits) by the bit
manipulation the fold kernel uses matches round-to-nearest-even by its
definition, and the hi + lo split of TF32 x 3 leaves the relative errors that
the parity bound of the GPU test assumes (2^-22 per operand, 2^-20 per
product)."""
import numpy as np


def round_tf32_bits(f32):
    """Add one less than half the TF32 spacing plus the lowest kept bit, then
    clear the 13 dropped bits (finite inputs)."""
    u = f32.view(np.uint32).astype(np.uint64)
    u = (u + 0xFFF + ((u >> 13) & 1)) & 0xFFFFE000
    return u.astype(np.uint32).view(np.float32)


def round_tf32_definition(f32):
    """The nearest value with 13 trailing zero mantissa bits; ties to the one
    whose last kept bit is 0."""
    u = f32.view(np.uint32).astype(np.int64)
    lo = u & ~0x1FFF                      # same sign: towards zero
    hi = lo + 0x2000                      # away from zero
    flo = lo.astype(np.uint32).view(np.float32).astype(np.float64)
    fhi = hi.astype(np.uint32).view(np.float32).astype(np.float64)
    x = f32.astype(np.float64)
    dlo, dhi = np.abs(x - flo), np.abs(fhi - x)
    even_lo = ((lo >> 13) & 1) == 0
    pick_lo = (dlo < dhi) | ((dlo == dhi) & even_lo)
    return np.where(pick_lo, lo, hi).astype(np.uint32).view(np.float32)


def test_bit_trick_is_round_to_nearest_even():
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(200000) * np.exp(rng.uniform(-30, 30, 200000))).astype(np.float32)
    # exact ties and neighbours of ties
    base = rng.integers(0x3F800000, 0x40000000, 20000, dtype=np.uint32) & ~np.uint32(0x1FFF)
    ties = np.concatenate([base | 0x1000, base | 0x0FFF, base | 0x1001, base | 0x3000]).view(np.float32)
    x = np.concatenate([x, ties, -ties, np.float32([0.0, -0.0, 1.0, 2.0 ** -126, 3.0e38])])
    assert np.array_equal(round_tf32_bits(x).view(np.uint32), round_tf32_definition(x).view(np.uint32))
    # the tie cases of the GPU test: 1 + 2^-11 -> 1, 1 + 3 2^-11 -> 1 + 2^-9
    t = np.float32([1 + 2.0 ** -11, 1 + 3 * 2.0 ** -11])
    assert list(round_tf32_bits(t)) == [1.0, 1 + 2.0 ** -9]


def split(v64):
    a32 = v64.astype(np.float32)
    hi = round_tf32_bits(a32)
    lo = round_tf32_bits((a32 - hi).astype(np.float32))  # a32 - hi is exact in FP32
    return hi.astype(np.float64), lo.astype(np.float64)


def test_split_and_product_errors():
    rng = np.random.default_rng(1)
    a = rng.standard_normal(400000) * np.exp(rng.uniform(-5, 5, 400000))
    b = rng.standard_normal(400000) * np.exp(rng.uniform(-5, 5, 400000))
    a0, a1 = split(a)
    b0, b1 = split(b)
    ea = np.abs(a - a0 - a1) / np.abs(a)
    assert ea.max() <= 2.0 ** -24 + 2.0 ** -22 * (1 + 2.0 ** -24)
    prod = a0 * b0 + a0 * b1 + a1 * b0   # each product exact in FP32 (11 x 11 bits)
    assert (np.abs(prod - a * b) / np.abs(a * b)).max() <= 2.0 ** -20
    # one TF32 product: 2^-10 + 2^-20
    one = round_tf32_bits(a.astype(np.float32)).astype(np.float64) * round_tf32_bits(b.astype(np.float32))
    assert (np.abs(one - a * b) / np.abs(a * b)).max() <= 2.0 ** -10 + 2.0 ** -20
    # every product of planes is exact in FP32
    for p, q in ((a0, b0), (a0, b1), (a1, b0)):
        pq = p * q
        assert np.array_equal(pq.astype(np.float32).astype(np.float64), pq)
