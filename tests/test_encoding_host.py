"""The integer encoding of the back-substitution and the grouped query, on the CPU.

For int32 tables whose finite entries are below 2^24 the kernels read the int32 bit
patterns as float32 values (m -> m x 2^-149: subnormal below 2^23, the lowest normal
binade up to 2^24) and add and compare them as floats.  The claims they rely on, checked
here with IEEE float32 arithmetic (numpy keeps subnormals):
  - the float sum of two encoded values is the encoding of the integer sum while that
    sum stays below 2^24, and at or above 2^24 it never decodes to a value below 2^24;
  - float order is integer order;
  - SPQ_INF_I32 (2^29) encodes a float far above every such sum, and +inf stays above it.
"""

import numpy as np

INF_I32 = 1 << 29


def enc(m):
    return np.asarray(m, dtype=np.int32).view(np.float32)


def dec(f):
    return np.asarray(f, dtype=np.float32).view(np.int32).astype(np.int64)


def test_sums_below_2_24_are_exact_integer_sums():
    rng = np.random.default_rng(11)
    a = rng.integers(0, 1 << 24, size=200_000)
    b = rng.integers(0, 1 << 24, size=200_000)
    keep = a + b < (1 << 24)
    a, b = a[keep], b[keep]
    s = enc(a) + enc(b)
    assert s.dtype == np.float32
    assert np.array_equal(dec(s), a + b)
    # the edges: 0, the subnormal / normal boundary 2^23, the largest exact sum
    edges = np.array([[0, 0], [1, 0], [(1 << 23) - 1, 1], [1 << 23, 0], [(1 << 23) - 5, 7],
                      [(1 << 24) - 1, 0], [(1 << 23), (1 << 23) - 1]], dtype=np.int64)
    assert np.array_equal(dec(enc(edges[:, 0]) + enc(edges[:, 1])), edges.sum(axis=1))


def test_sums_at_or_above_2_24_never_decode_below_it():
    rng = np.random.default_rng(12)
    a = rng.integers(0, 1 << 24, size=200_000)
    b = rng.integers(0, 1 << 24, size=200_000)
    keep = a + b >= (1 << 24)
    s = dec(enc(a[keep]) + enc(b[keep]))
    assert (s >= (1 << 24)).all()


def test_float_order_is_integer_order_and_inf_is_above():
    rng = np.random.default_rng(13)
    x = rng.integers(0, 1 << 25, size=100_000)
    y = rng.integers(0, 1 << 25, size=100_000)
    assert np.array_equal(enc(x) < enc(y), x < y)
    assert np.array_equal(np.minimum(enc(x), enc(y)).view(np.int32), np.minimum(x, y))
    inf = enc(INF_I32)
    biggest = enc((1 << 24) - 1) + enc((1 << 24) - 1)
    assert inf > biggest and inf > enc(x).max()
    assert np.float32(np.inf) > inf
    # three-term query sums of finite entries stay below the encoded infinity
    assert enc((1 << 24) - 1) + enc((1 << 24) - 1) + enc((1 << 24) - 1) < inf
