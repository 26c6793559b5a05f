"""The shifted geometric mean against its closed form and special cases."""

import math

import pytest

from paper_2311_12180_gb300.metrics import shifted_geometric_mean as sgm


def test_constant_values_give_that_value():
    assert sgm([3.0] * 7) == pytest.approx(3.0, rel=1e-12)


def test_two_values_closed_form():
    # sqrt((1 + 10)(100 + 10)) - 10
    assert sgm([1.0, 100.0]) == pytest.approx(math.sqrt(11.0 * 110.0) - 10.0, rel=1e-12)


def test_shift_zero_is_the_geometric_mean_and_order_does_not_matter():
    assert sgm([2.0, 8.0], shift=0.0) == pytest.approx(4.0, rel=1e-12)
    assert sgm([5.0, 0.5, 40.0]) == pytest.approx(sgm([40.0, 5.0, 0.5]), rel=1e-12)


def test_between_min_and_max_and_below_arithmetic_mean():
    v = [0.1, 2.0, 30.0, 400.0]
    s = sgm(v)
    assert min(v) < s < max(v) and s < sum(v) / len(v)


def test_empty_and_invalid():
    assert sgm([]) == 0.0
    with pytest.raises(ValueError):
        sgm([-20.0])
