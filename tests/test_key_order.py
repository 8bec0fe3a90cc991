"""The k-nearest-neighbour kernels order candidates by (d^2, index) comparing the 64-bit patterns
of the non-negative FP64 squared distances as unsigned integers.  This pins the fact that makes
that exact: for non-negative doubles (zero, subnormals, normals, infinity) the unsigned order of
the bit patterns is the order of the values, and equal patterns are equal values."""
import numpy as np


def _bits(x):
    return np.asarray(x, np.float64).view(np.uint64)


def test_bit_pattern_order_is_value_order_for_non_negative_doubles():
    rng = np.random.default_rng(7)
    parts = [
        np.abs(rng.standard_normal(20000)) * 10.0 ** rng.integers(-300, 300, 20000),
        rng.random(5000) * 2.0 ** -1060,                     # subnormals
        np.array([0.0, 5e-324, 2.2250738585072014e-308, 1.0, np.nextafter(1.0, 2.0), 1.7976931348623157e308,
                  np.inf]),
    ]
    x = np.concatenate(parts)
    order_by_value = np.argsort(x, kind="stable")
    order_by_bits = np.argsort(_bits(x), kind="stable")
    assert np.array_equal(x[order_by_value], x[order_by_bits])
    a, b = x[: len(x) // 2], x[len(x) // 2 : 2 * (len(x) // 2)]
    assert np.array_equal(a < b, _bits(a) < _bits(b))
    assert np.array_equal(a == b, _bits(a) == _bits(b))


def test_squared_distances_are_never_negative_zero():
    """dx*dx + dy*dy with round-to-nearest is +0 when it is zero, so no -0.0 (whose pattern sorts
    last) reaches the comparison."""
    rng = np.random.default_rng(3)
    dx = np.concatenate([rng.standard_normal(1000), [0.0, -0.0, 1e-200, -1e-200]])
    dy = np.concatenate([rng.standard_normal(1000), [-0.0, 0.0, -1e-200, 1e-200]])
    d2 = dx * dx + dy * dy
    assert not np.any(np.signbit(d2))
