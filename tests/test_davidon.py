"""CPU checks of Davidon's cubic-interpolation search (the spin-rate study's
optimiser, Sec. 6.1) on functions with known maxima."""
import math

import pytest

from paper_2407_16032_b300.davidon import davidon_maximize


def test_quadratic_maximum_is_found_in_one_step():
    # the cubic through a quadratic's values and slopes is the quadratic
    calls = []

    def fg(x):
        calls.append(x)
        return -(x - 6.26) ** 2 + 3.0, -2.0 * (x - 6.26)

    x, f, g, hist = davidon_maximize(fg, 3.0, 8.0, maxit=1)
    assert abs(x - 6.26) < 1e-12 and abs(f - 3.0) < 1e-12
    assert len(calls) == 3


@pytest.mark.parametrize("a,b", [(0.2, 3.0), (0.5, 2.5)])
def test_smooth_maximum_within_tolerance(a, b):
    # sin(x) + x / 10 on [a, b]: maximum where cos x = -1/10, x = acos(-0.1)
    fg = lambda x: (math.sin(x) + 0.1 * x, math.cos(x) + 0.1)
    x, f, g, hist = davidon_maximize(fg, a, b, xtol=1e-8, gtol=1e-10, maxit=20)
    assert abs(x - math.acos(-0.1)) < 1e-6
    assert len(hist) < 12          # superlinear: a handful of evaluations


def test_an_interval_without_a_bracketed_maximum_is_rejected():
    with pytest.raises(ValueError):
        davidon_maximize(lambda x: (x, 1.0), 0.0, 1.0)
