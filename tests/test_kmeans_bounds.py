"""CPU checks of the error bounds behind the tensor-core k-means margins,
with TF32 rounding emulated bit for bit in numpy (10 explicit mantissa bits):

* one product per pair (operands truncated to TF32): |f.c - t(f).t(c)| is
  below (2^-9 + 2^-20) sum |f_j c_j|;
* split operands (x = hi + lo + r, hi and lo rounded to nearest, ties away
  from zero): |r| <= 2^-22 |x| and |f.c - (hi.hi + hi.lo + lo.hi)| <= 3.01
  2^-22 sum |f_j c_j|;
* the margins the kernel uses cover twice these terms plus the FP32
  accumulation of the products (one ulp per addition);
* the centroid update's fixed point: the integer recipe gives floor(x 2^sh)
  exactly across binades and for subnormals, and the scale keeps n partial
  sums below 2^62."""
import numpy as np

TF32_DROP = 13  # mantissa bits FP32 has beyond TF32


def tf32_trunc(x):
    u = np.asarray(x, np.float32).view(np.uint32)
    return (u & np.uint32(~((1 << TF32_DROP) - 1) & 0xFFFFFFFF)).view(np.float32)


def tf32_rna(x):
    """Round to nearest, ties away from zero: add half of the dropped part to the magnitude bits."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = (u + (1 << (TF32_DROP - 1))) & ~np.uint64((1 << TF32_DROP) - 1)
    return r.astype(np.uint32).view(np.float32)


def split(x):
    x = np.asarray(x, np.float32)
    hi = tf32_rna(x)
    lo = tf32_rna((x - hi).astype(np.float32))  # x - hi is exact in FP32
    return hi, lo


def rows(seed, n=4000, d=128):
    rng = np.random.default_rng(seed)
    scale = np.exp(rng.uniform(-8, 8, (n, 1)))  # rows over many binades
    return (rng.standard_normal((n, d)) * scale).astype(np.float32)


def test_tf32_rounding_emulation():
    x = np.array([1.0, 1.0 + 2.0 ** -10, 1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11, -(1.0 + 2.0 ** -11)], np.float32)
    assert tf32_trunc(x).tolist() == [1.0, 1.0 + 2.0 ** -10, 1.0, 1.0 + 2.0 ** -10, -1.0]
    # ties (exactly half an ulp of TF32) go away from zero
    assert tf32_rna(x).tolist() == [1.0, 1.0 + 2.0 ** -10, 1.0 + 2.0 ** -10, 1.0 + 2.0 ** -9, -(1.0 + 2.0 ** -10)]


def test_split_residual_bound():
    x = rows(1).ravel()
    hi, lo = split(x)
    r = x.astype(np.float64) - hi.astype(np.float64) - lo.astype(np.float64)
    assert np.all(np.abs(r) <= 2.0 ** -22 * np.abs(x.astype(np.float64)))
    assert np.all(tf32_trunc(hi) == hi) and np.all(tf32_trunc(lo) == lo)  # both parts are TF32 values


def test_product_error_bounds():
    F, C = rows(2), rows(3, n=100)
    f64, c64 = F.astype(np.float64), C.astype(np.float64)
    exact = f64 @ c64.T
    mag = np.abs(f64) @ np.abs(c64).T
    single = tf32_trunc(F).astype(np.float64) @ tf32_trunc(C).astype(np.float64).T
    assert np.all(np.abs(exact - single) <= (2.0 ** -9 + 2.0 ** -20) * mag)
    fh, fl = (a.astype(np.float64) for a in split(F))
    ch, cl = (a.astype(np.float64) for a in split(C))
    three = fh @ ch.T + fh @ cl.T + fl @ ch.T
    err = np.abs(exact - three)
    assert np.all(err <= 3.01 * 2.0 ** -22 * mag)
    # the split products are far more accurate than the single ones on the same data
    assert err.max() / mag.max() < 2.0 ** -20 < np.abs(exact - single).max() / mag.max()


def test_margins_cover_the_bounds():
    d = 128
    acc_single = d * 2.0 ** -23       # FP32 accumulation of d products, one ulp per addition
    acc_split = 3 * d * 2.0 ** -23    # three products per K step
    assert 2.0 * (2.0 ** -9 + 2.0 ** -20 + acc_single) <= 2.0 ** -7
    assert 2.0 * (3.01 * 2.0 ** -22 + acc_split) <= 2.0 ** -12


def fix_shift(bmax, n):
    """The centroid sums' scale: n < 2^nb, max |F_ij| < 2^e (frexp), sh = 62 - nb - e, at most 187."""
    if not bmax > 0:
        return 0
    e = int(np.frexp(np.float32(bmax))[1])
    return min(62 - int(n).bit_length() - e, 187)


def fix_value(x, sh):
    """floor(x 2^sh) by the integer recipe of the update: the signed significand placed at bit 39 and shifted
    right arithmetically by 189 - sh - e (e = 1 and no implicit bit for subnormals), shifts clamped to 63."""
    u = int(np.array([x], np.float32).view(np.uint32)[0])
    e = (u >> 23) & 255
    hi = ((u << 7) & 0x3FFFFF80) | (0x40000000 if e else 0)
    amt = min(189 - sh - max(e, 1), 63)
    assert amt >= 1
    v = -hi if u >> 31 else hi
    return (v << 32) >> amt


def test_fixed_point_centroid_sums():
    from fractions import Fraction

    rng = np.random.default_rng(5)
    for n, lo, hi_exp in ((1000, -30, 0), (3, -140, -125), (1 << 20, -10, 10)):
        x = (rng.standard_normal(min(n, 3000)) * np.exp2(rng.uniform(lo, hi_exp, min(n, 3000)))).astype(np.float32)
        sh = fix_shift(np.abs(x).max(), n)
        q = [fix_value(v, sh) for v in x]
        exact = [Fraction(float(v)) * Fraction(2) ** sh for v in x]
        assert all(e - 1 < qi <= e for qi, e in zip(q, exact))  # floor: error below one unit of 2^-sh
        # n values of magnitude up to max|x| keep every partial sum below 2^62
        assert int(n) * max(abs(qi) for qi in q) < 2 ** 62
    # subnormal data: the cap keeps the shift at or below 187, where every subnormal is a whole number of units
    assert fix_shift(np.float32(1e-44), 10) == 187
    assert fix_value(np.float32(1e-44), 187) == int(Fraction(float(np.float32(1e-44))) * Fraction(2) ** 187)
