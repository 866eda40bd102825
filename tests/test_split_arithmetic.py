"""Host-side checks of the arithmetic the tensor-core forms rest on (no GPU):

* the three-part BF16 split used by the split precision: hi = bf16(x),
  mid = bf16(x - hi), lo = bf16(x - hi - mid), each residual computed in
  FP32, reconstructs every FP32 value x with |x| >= 2^-100 exactly
  (hi + mid + lo == x, summed in FP64), and both residuals are exact in
  FP32; below that the last residual can fall under BF16's normal range and
  lose bits (a value that small adds nothing to a squared distance at FP32
  precision);
* the three part products the split form leaves out (mid*lo, lo*mid, lo*lo)
  are below 2^-23 |x||y| together, the bound the stated error uses;
* the 8-bit form: 255 x for x = k/255 rounds to the integer k, and every
  integer 0..255 is exact in BF16, so its products are exact.

BF16 rounding is emulated bit by bit (round to nearest, ties to even, on the
upper 16 bits of the FP32 pattern)."""
import numpy as np

rng = np.random.Generator(np.random.PCG64(2310))


def bf16_round(x32):
    """Round FP32 values to BF16 (nearest, ties to even), returned as FP32."""
    u = np.asarray(x32, np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32)


def split3(x32):
    hi = bf16_round(x32)
    r1 = (x32 - hi).astype(np.float32)
    mid = bf16_round(r1)
    r2 = (r1 - mid).astype(np.float32)
    lo = bf16_round(r2)
    return hi, mid, lo, r1, r2


def sample_fp32(m):
    # wide exponent range, both signs, plus edge patterns
    e = rng.uniform(-100, 120, m)
    x = (rng.choice([-1.0, 1.0], m) * rng.uniform(1.0, 2.0, m) * 2.0 ** e).astype(np.float32)
    edges = np.array([0.0, 1.0, -1.0, 1.0 / 255.0, 2.0 ** -100, np.float32(1.0 - 2.0 ** -24), 65504.0,
                      np.float32(1.0 + 2.0 ** -23), 123456.789, 3.0e38], np.float32)
    return np.concatenate([x, edges])


def test_three_part_split_is_exact():
    x = sample_fp32(200_000)
    x = x[(x == 0) | (np.abs(x) >= 2.0 ** -100)]
    hi, mid, lo, r1, r2 = split3(x)
    # residuals exact in FP32 (the FP64 differences equal the FP32 ones)
    np.testing.assert_array_equal(r1.astype(np.float64), x.astype(np.float64) - hi.astype(np.float64))
    np.testing.assert_array_equal(r2.astype(np.float64), r1.astype(np.float64) - mid.astype(np.float64))
    # the last part holds the remaining bits exactly
    np.testing.assert_array_equal(lo, r2)
    np.testing.assert_array_equal(hi.astype(np.float64) + mid.astype(np.float64) + lo.astype(np.float64),
                                  x.astype(np.float64))


def test_dropped_products_bound():
    x, y = sample_fp32(50_000), sample_fp32(50_000)
    x, y = x[np.abs(x) > 1e-30], y[: (np.abs(x) > 1e-30).sum()]
    keep = np.abs(y) > 1e-30
    x, y = x[keep], y[keep]
    hx, mx, lx, _, _ = split3(x)
    hy, my, ly, _, _ = split3(y)
    f = lambda v: v.astype(np.float64)
    dropped = np.abs(f(mx) * f(ly)) + np.abs(f(lx) * f(my)) + np.abs(f(lx) * f(ly))
    assert (dropped <= 2.0 ** -23 * np.abs(f(x) * f(y))).all()
    # the six kept products recover the product to that bound
    kept = (f(lx) * f(hy) + f(hx) * f(ly) + f(mx) * f(my) + f(mx) * f(hy) + f(hx) * f(my) + f(hx) * f(hy))
    assert (np.abs(kept - f(x) * f(y)) <= 2.0 ** -23 * np.abs(f(x) * f(y))).all()


def test_eight_bit_values_are_exact_integers_in_bf16():
    k = np.arange(256)
    x = (k / 255.0).astype(np.float32)          # the data: exact multiples of 1/255 as FP32
    scaled = np.rint(x * np.float32(255.0)).astype(np.float32)
    np.testing.assert_array_equal(scaled, k.astype(np.float32))
    np.testing.assert_array_equal(bf16_round(scaled), scaled)  # 0..255 need at most 8 significant bits
    # a product of two such integers is exact in FP32, and a sum of d <= 784
    # of them stays an integer below 2^24 while the data norms stay below 258
    assert 255 * 255 * 784 > 2 ** 24 and 258 * 255 * 255 < 2 ** 24
