"""The (hi, lo) FP32 arithmetic of the GMRES basis, emulated on the CPU.

The Gram-Schmidt kernels hold the Krylov vectors as FP32 (hi, lo) pairs and
form every product with its rounding error (an FMA) and every sum with
Knuth's two-sum, in round-to-nearest FP32 operations the compiler may not
contract.  The same sequence of operations is written here in numpy float32
(an FMA is emulated exactly: a float32 product is exact in float64) and
compared with exact rational arithmetic:
- the error-free transformations are exact;
- a dot product keeps about 48 bits (error below 1e-13 of the sum of
  |terms|, where FP32 alone would give about 1e-7);
- a Gram-Schmidt update that cancels down to 1e-9 of its terms keeps its
  absolute error below 1e-13 of the terms;
- dropping a product's rounding error (a planted mistake) breaks the bound.
"""

from fractions import Fraction

import numpy as np

f32 = np.float32


def add(a, b):
    return f32(f32(a) + f32(b))


def sub(a, b):
    return f32(f32(a) - f32(b))


def mul(a, b):
    return f32(f32(a) * f32(b))


def fma(a, b, c):
    return f32(np.float64(f32(a)) * np.float64(f32(b)) + np.float64(f32(c)))


def two_sum(a, b):
    s = add(a, b)
    bb = sub(s, a)
    return s, add(sub(a, sub(s, bb)), sub(b, bb))


def df_mac(acc, a, b, keep_error=True):
    """acc += a b: the product with its rounding error, the sum compensated."""
    p = mul(a, b)
    e = fma(a, b, -p) if keep_error else f32(0)
    s, t = two_sum(acc[0], p)
    return (s, add(acc[1], add(t, e)))


def df_small(acc, a, b):
    return (acc[0], fma(a, b, acc[1]))


def renorm(acc):
    return two_sum(acc[0], acc[1])


def split(x):
    h = f32(x)
    return h, f32(np.float64(x) - np.float64(h))


def exact(x):
    return Fraction(float(x))


def test_error_free_transformations_are_exact():
    rng = np.random.default_rng(1)
    for _ in range(2000):
        a, b = (f32(v) for v in rng.standard_normal(2) * 10.0 ** rng.integers(-6, 6, 2))
        s, e = two_sum(a, b)
        assert exact(s) + exact(e) == exact(a) + exact(b)
        p = mul(a, b)
        assert exact(p) + exact(fma(a, b, -p)) == exact(a) * exact(b)


def _dot(vh, vl, w, keep_error=True):
    acc = (f32(0), f32(0))
    for i in range(len(w)):
        acc = df_mac(acc, vh[i], w[i], keep_error)
        acc = df_small(acc, vl[i], w[i])
    return renorm(acc)


def test_dot_product_keeps_about_48_bits():
    """A basis vector in (hi, lo) pairs against an FP32 operator output (exact as a hi part)."""
    rng = np.random.default_rng(2)
    n = 3000
    v = rng.standard_normal(n)
    w = rng.standard_normal(n).astype(np.float32)
    vh, vl = zip(*(split(x) for x in v))
    got = _dot(vh, vl, w)
    ref = sum((exact(vh[i]) + exact(vl[i])) * exact(w[i]) for i in range(n))
    scale = sum(abs(exact(vh[i]) * exact(w[i])) for i in range(n))
    err = float(abs(exact(got[0]) + exact(got[1]) - ref) / scale)
    assert err < 1e-13, err
    # the planted mistake: the products' rounding errors dropped (an FP32 dot product)
    bad = _dot(vh, vl, w, keep_error=False)
    err_bad = float(abs(exact(bad[0]) + exact(bad[1]) - ref) / scale)
    assert err_bad > 1e-10, err_bad


def test_cancelling_gram_schmidt_update():
    """x - sum_k v_k h_k with x equal to the sum up to 1e-9: the update of a vector that the
    basis almost spans, in the kernel's order (renormalised every eighth term)."""
    rng = np.random.default_rng(3)
    K = 60
    vs = rng.standard_normal(K)
    hs = rng.standard_normal(K)
    vsp = [split(x) for x in vs]
    hsp = [split(x) for x in hs]
    x = float(sum(np.float64(vh) * np.float64(hh) for (vh, _), (hh, _) in zip(vsp, hsp))) + 1e-9
    acc = split(x)
    for k in range(K):
        (vh, vl), (hh, hl) = vsp[k], hsp[k]
        acc = df_mac(acc, -vh, hh)
        acc = df_small(acc, -vh, hl)
        acc = df_small(acc, -vl, hh)
        if k % 8 == 7:
            acc = renorm(acc)
    acc = renorm(acc)
    xs = split(x)
    ref = exact(xs[0]) + exact(xs[1]) - sum(
        (exact(vh) + exact(vl)) * (exact(hh) + exact(hl)) for (vh, vl), (hh, hl) in zip(vsp, hsp))
    scale = sum(abs(exact(vh) * exact(hh)) for (vh, _), (hh, _) in zip(vsp, hsp))
    err = float(abs(exact(acc[0]) + exact(acc[1]) - ref) / scale)
    assert float(abs(ref) / scale) < 1e-8  # the update did cancel
    assert err < 1e-13, err
