"""The leaf host pass (normalise + round) of the mixed-precision forms, on CPU.

A mixed-precision DAG stores each leaf as complex64 values x * 2^-e, where e
is the exponent that brings the largest |component| of the leaf into
[0.5, 1) (frexp), and the product x * 2^-e (exact in FP64) is rounded once to
the nearest float.  New data of the same leaf keeps e while its largest
component stays in (2^(e-32), 2^e]; otherwise e is chosen again.  The FP64
form stores the values as they are.  These tests restate that definition
with numpy and compare the library's host store with it bit for bit; they
need no GPU (the store is then pageable host memory).
"""
import math

import numpy as np
import pytest

L = pytest.importorskip("paper_2511_02257_b300")

LT, SHAPE = 3, (4, 5)


def _expected(x, e):
    return (np.asarray(x, np.complex128) * math.ldexp(1.0, -e)).astype(np.complex64)


def _frexp_exp(x):
    m = float(np.max(np.abs(np.concatenate([x.real.ravel(), x.imag.ravel()]))))
    return 0 if m == 0.0 or not math.isfinite(m) else math.frexp(m)[1]


def _data(rng, scale):
    return scale * (rng.standard_normal((LT,) + SHAPE) + 1j * rng.standard_normal((LT,) + SHAPE))


def _same(a, b):
    return np.array_equal(a.view(np.uint32), b.view(np.uint32))


@pytest.mark.parametrize("precision", ["tf32x3", "bf16x3"])
@pytest.mark.parametrize("scale", [1.0, 3e5, 2.0 ** -40, 7.5e-300])
def test_first_data_sets_the_exponent(precision, scale):
    rng = np.random.default_rng(int(abs(math.log2(scale))) + 1)
    x = _data(rng, scale)
    d = L.Dag(LT, precision)
    u = d.add_leaf(SHAPE, x)
    got, e = d.leaf_store(u)
    assert e == _frexp_exp(x)
    assert _same(got, _expected(x, e).reshape(LT, -1))
    # the largest component lands in [0.5, 1)
    m = np.max(np.abs(np.concatenate([got.real.ravel(), got.imag.ravel()])))
    assert 0.5 <= m <= 1.0  # rounding may carry the largest to 1.0
    d.close()


def test_new_data_keeps_the_exponent_inside_its_range():
    rng = np.random.default_rng(3)
    x = _data(rng, 1.0)
    d = L.Dag(LT, "tf32x3")
    u = d.add_leaf(SHAPE, x)
    _, e0 = d.leaf_store(u)
    top = math.ldexp(1.0, e0)
    # largest component exactly 2^e: kept (the upper bound is inclusive)
    y = _data(rng, 1.0)
    y = y / np.max(np.abs(np.concatenate([y.real.ravel(), y.imag.ravel()]))) * top
    d.set_leaf_data(u, y)
    got, e = d.leaf_store(u)
    assert e == e0 and _same(got, _expected(y, e0).reshape(LT, -1))
    # much smaller, still above 2^(e-32): kept, values scaled by the old exponent
    z = y * 2.0 ** -30
    d.set_leaf_data(u, z)
    got, e = d.leaf_store(u)
    assert e == e0 and _same(got, _expected(z, e0).reshape(LT, -1))
    # at 2^(e-32) or below: a new exponent
    w = y * 2.0 ** -33
    d.set_leaf_data(u, w)
    got, e = d.leaf_store(u)
    assert e == _frexp_exp(w) and e < e0 - 30
    assert _same(got, _expected(w, e).reshape(LT, -1))
    # above 2^e: a new exponent
    v = y * 3.0
    d.set_leaf_data(u, v)
    got, e = d.leaf_store(u)
    assert e == _frexp_exp(v)
    assert _same(got, _expected(v, e).reshape(LT, -1))
    d.close()


def test_zero_infinite_and_nan_components():
    d = L.Dag(LT, "tf32x3")
    x = np.zeros((LT,) + SHAPE, np.complex128)
    u = d.add_leaf(SHAPE, x)
    got, e = d.leaf_store(u)
    assert e == 0 and not np.any(got)
    # an infinite component: no finite scale, the exponent is 0
    y = np.full((LT,) + SHAPE, 0.25 + 0.5j)
    y[1, 2, 3] = complex(np.inf, 1.0)
    d.set_leaf_data(u, y)
    got, e = d.leaf_store(u)
    assert e == 0 and np.isinf(got[1].reshape(SHAPE)[2, 3].real)
    # a NaN component never sets the scale and is stored as NaN
    z = np.full((LT,) + SHAPE, 3.0 - 1.0j)
    z[0, 0, 0] = complex(np.nan, 0.0)
    d.set_leaf_data(u, z)
    got, e = d.leaf_store(u)
    assert e == math.frexp(3.0)[1]
    assert np.isnan(got[0, 0].real)
    rest = np.delete(got.ravel(), 0)
    assert _same(rest, np.delete(_expected(z, e).ravel(), 0))
    d.close()


def test_fp64_store_is_the_data():
    rng = np.random.default_rng(5)
    x = _data(rng, 1e7)
    d = L.Dag(LT, "fp64")
    u = d.add_leaf(SHAPE, x)
    got, e = d.leaf_store(u)
    assert e == 0 and np.array_equal(got.view(np.float64), x.reshape(LT, -1).view(np.float64))
    d.close()


def test_large_leaf_split_over_host_threads():
    """A leaf of 2^22 complex values is normalised by several host threads:
    the same store as the single-pass definition, including the exponent
    found as the maximum over the threads' partial maxima."""
    rng = np.random.default_rng(9)
    lt, shape = 4, (1024, 1024)
    x = rng.standard_normal((lt,) + shape) + 1j * rng.standard_normal((lt,) + shape)
    x[3, 1000, 7] = 40.0 + 0.0j   # the largest component, in the last thread's range
    d = L.Dag(lt, "tf32x3")
    u = d.add_leaf(shape, x)
    got, e = d.leaf_store(u)
    assert e == math.frexp(40.0)[1]
    assert _same(got, _expected(x, e).reshape(lt, -1))
    d.close()


def test_read_leaf_store_errors():
    d = L.Dag(LT, "tf32x3")
    a = d.add_leaf(SHAPE)                     # no data yet
    b = d.add_leaf(SHAPE, np.ones((LT,) + SHAPE))
    c = d.add_contraction(a, b, [0, 1], [0, 1])
    with pytest.raises(L.LqcError):
        d.leaf_store(a)                       # LQC_ERR_STATE
    with pytest.raises(L.LqcError):
        d.leaf_store(c)                       # not a leaf
    d.close()
