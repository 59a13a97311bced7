"""CPU checks of the error bounds behind the tensor-core k-means margins,
with TF32 rounding emulated bit for bit in numpy (10 explicit mantissa bits):

* one product per pair (operands truncated to TF32): |f.c - t(f).t(c)| is
  below (2^-9 + 2^-20) sum |f_j c_j|;
* split operands (x = hi + lo + r, hi and lo rounded to nearest, ties away
  from zero): |r| <= 2^-22 |x| and |f.c - (hi.hi + hi.lo + lo.hi)| <= 3.01
  2^-22 sum |f_j c_j|;
* the margins the kernel uses cover twice these terms plus the FP32
  accumulation of the products (one ulp per addition)."""
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
