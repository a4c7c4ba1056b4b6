"""Pins of the oracle's float32 path: a float32 volume is filtered on 65536
grey levels spanning its range (level = floor((v - lo) * 65535 / d + 1/2), back
as lo + level * d / 65535, float32 rounding at every step).  Pinned by the
span of the levels, the round-trip bound through the identity filter, the
exact reduction to the 16-bit filters when the volume already holds the
levels 0..65535, constant volumes and monotonicity."""
import numpy as np
import pytest

import oracle
import phantoms

NONE = oracle.Config(threshold_mode="none")


def _ct_like(shape, seed):
    rng = np.random.default_rng(seed)
    # attenuation-like values with negative air, soft tissue and a dense insert
    v = rng.normal(0.0, 40.0, shape).astype(np.float32) - np.float32(1000.0)
    v[shape[0] // 4:, shape[1] // 4:, :] += np.float32(1040.0)
    v[shape[0] // 2:, :, shape[2] // 3:] += np.float32(2200.5)
    return v.astype(np.float32)


def test_levels_span_the_range():
    v = _ct_like((6, 7, 9), 501)
    q, lo, hi = oracle.quantize_f32(v)
    assert q.dtype == np.uint16 and lo == v.min() and hi == v.max()
    assert q.min() == 0 and q.max() == 65535
    assert q[np.unravel_index(np.argmin(v), v.shape)] == 0
    assert q[np.unravel_index(np.argmax(v), v.shape)] == 65535


def test_round_trip_through_the_identity_filter():
    # mean at r = 0 with the gate off is the identity on levels: the output is
    # the value's level mapped back, within half a step (plus float32 rounding)
    v = _ct_like((7, 8, 9), 502)
    out = oracle.filter_volume_f32(v, oracle.MEAN, 0, cfg=NONE)
    step = (float(v.max()) - float(v.min())) / 65535
    ulp = np.spacing(np.float32(np.abs(v).max()))
    assert np.abs(out.astype(np.float64) - v).max() <= 0.52 * step + 2 * float(ulp)


@pytest.mark.parametrize("f", range(8))
def test_levels_already_on_the_grid_reduce_to_the_16bit_filter(f):
    # a float32 volume holding the integers 0..65535 (both ends present): the
    # scale is exactly 1, the levels are the values, and the result is the
    # 16-bit filter's, as floats
    u = phantoms.random_volume((7, 6, 5), 503 + f, "u16")
    u.reshape(-1)[0], u.reshape(-1)[1] = 0, 65535
    got = oracle.filter_volume_f32(u.astype(np.float32), f, 1)
    want = oracle.filter_volume(u, f, 1).astype(np.float32)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("f", range(8))
def test_constant_volume_unchanged(f):
    v = np.full((5, 6, 7), -123.25, np.float32)
    out = oracle.filter_volume_f32(v, f, 2)
    assert (out == np.float32(-123.25)).all()


def test_levels_are_monotone():
    rng = np.random.default_rng(504)
    v = np.sort(rng.normal(0, 1e3, 4096).astype(np.float32)).reshape(4, 32, 32)
    q, _, _ = oracle.quantize_f32(v)
    assert (np.diff(q.reshape(-1).astype(np.int64)) >= 0).all()


def test_non_finite_values_are_rejected():
    v = np.zeros((3, 3, 3), np.float32)
    for bad in (np.nan, np.inf, -np.inf):
        v[1, 1, 1] = bad
        with pytest.raises(ValueError):
            oracle.quantize_f32(v)
