"""The split arithmetic behind the mixed-precision cell products, emulated
bit by bit in numpy (no GPU, no library code).

The tensor-core filter keeps binary32 accuracy by splitting operands into
lower-precision terms:

* BF16x3: v = b1 + b2 + b3 with b1 = bf16(v), b2 = bf16(v - b1),
  b3 = bf16(v - b1 - b2) (round to nearest even); six of the nine cross
  products are accumulated, dropping a2 y3 + a3 y2 + a3 y3.
* 3xTF32: x = hi + lo with hi = tf32(x) (round half away) and lo = x - hi;
  hi hi + hi lo + lo hi, dropping lo lo.

These tests pin the facts the kernels rely on: the bf16 split of a binary32
value is exact (24 = 3 x 8 significant bits, every remainder exact in
binary32), and the dropped products bound the error of one product by about
2^-23 (BF16x3) and 2^-21 (3xTF32) relative, below or at binary32 rounding.
"""
import numpy as np


def bf16(x):
    """Round binary32 to bfloat16 (8 significant bits), nearest even; finite inputs."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def tf32(x):
    """Round binary32 to TF32 (11 significant bits), half away from zero; finite inputs."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x1000) & 0xFFFFE000
    return b.astype(np.uint32).view(np.float32)


def split3(v):
    v = np.asarray(v, np.float32)
    b1 = bf16(v)
    r1 = (v - b1).astype(np.float32)
    b2 = bf16(r1)
    r2 = (r1 - b2).astype(np.float32)
    return b1, b2, bf16(r2), r1, r2


def _values(seed, n=200000, span=60):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(n) * np.exp2(rng.integers(-span, span, n))).astype(np.float32)


def test_bf16_rounding_special_values():
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: nearest even keeps 1
    assert bf16(np.float32(1 + 2 ** -8)) == 1.0
    assert bf16(np.float32(1 + 3 * 2 ** -8)) == np.float32(1 + 2 ** -6)
    assert bf16(np.float32(-1.5)) == -1.5
    # 8 significant bits survive unchanged
    assert bf16(np.float32(255.0)) == 255.0 and bf16(np.float32(257.0)) == 256.0


def test_bf16x3_split_of_binary32_is_exact():
    v = _values(1)
    b1, b2, b3, r1, r2 = split3(v)
    v64 = v.astype(np.float64)
    assert np.array_equal(v64 - b1, r1.astype(np.float64))          # remainders exact in binary32
    assert np.array_equal(r1.astype(np.float64) - b2, r2.astype(np.float64))
    assert np.array_equal(b1.astype(np.float64) + b2 + b3, v64)      # the three terms sum to v
    # each term carries at most 8 significant bits: bf16 of it is itself
    for t in (b1, b2, b3):
        assert np.array_equal(bf16(t), t)


def test_bf16x3_six_products_error_bound():
    a, y = _values(2, span=20), _values(3, span=20)
    a1, a2, a3, _, _ = [t.astype(np.float64) for t in split3(a)]
    y1, y2, y3, _, _ = [t.astype(np.float64) for t in split3(y)]
    six = a3 * y1 + a2 * y2 + a1 * y3 + a2 * y1 + a1 * y2 + a1 * y1
    exact = a.astype(np.float64) * y.astype(np.float64)
    rel = np.abs(six - exact) / np.abs(exact)
    assert rel.max() <= 2.0 ** -23 * 1.01
    # the bound is attained to within a small factor: the dropped terms matter
    assert rel.max() > 2.0 ** -26
    # dropping one of the six kept terms would break binary32 accuracy
    five = six - a2 * y2
    assert (np.abs(five - exact) / np.abs(exact)).max() > 2.0 ** -20


def test_3xtf32_error_bound():
    x, z = _values(4, span=20), _values(5, span=20)
    xh, zh = tf32(x), tf32(z)
    xl = tf32((x - xh).astype(np.float32))       # the MMA reads lo as TF32 too
    zl = tf32((z - zh).astype(np.float32))
    xh, zh, xl, zl = [t.astype(np.float64) for t in (xh, zh, xl, zl)]
    three = xh * zh + xh * zl + xl * zh
    exact = x.astype(np.float64) * z.astype(np.float64)
    rel = np.abs(three - exact) / np.abs(exact)
    assert rel.max() <= 2.0 ** -20
    # one TF32 product alone keeps about 11 bits
    one = (xh * zh - exact) / exact
    assert np.abs(one).max() > 2.0 ** -12


def test_bf16x3_dot_product_against_binary32():
    """A cell-row dot product of n_e = 343 terms: the BF16x3 six-product sum
    accumulated in binary32 stays within a small multiple of the binary32
    dot product's own rounding error."""
    rng = np.random.default_rng(6)
    ne = 343
    A = rng.standard_normal((64, ne)).astype(np.float32)
    Y = rng.standard_normal((ne, 16)).astype(np.float32)
    exact = A.astype(np.float64) @ Y.astype(np.float64)
    a = [t for t in split3(A)[:3]]
    y = [t for t in split3(Y)[:3]]
    acc = np.zeros((64, 16), np.float32)
    for (i, j) in [(2, 0), (1, 1), (0, 2), (1, 0), (0, 1), (0, 0)]:
        acc = (acc + (a[i].astype(np.float64) @ y[j].astype(np.float64)).astype(np.float32)).astype(np.float32)
    f32 = (A @ Y).astype(np.float32)
    scale = np.abs(A).astype(np.float64) @ np.abs(Y).astype(np.float64)
    err_split = np.abs(acc - exact) / scale
    err_f32 = np.abs(f32 - exact) / scale
    assert err_split.max() < 8 * max(err_f32.max(), 2.0 ** -24)
