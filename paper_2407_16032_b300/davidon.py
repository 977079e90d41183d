"""Davidon's cubic-interpolation search on an interval (the optimiser of the
spin-rate study, Sec. 6.1): from the values and derivatives of a smooth function
at the two ends of an interval that brackets an extremum, the extremum of the
cubic that matches all four numbers is evaluated next, and the end whose
derivative has the same sign is moved there.

For a minimum with f'(a) < 0 < f'(b) the cubic's minimiser is
    z = 3 (f(a) - f(b)) / (b - a) + f'(a) + f'(b),
    w = sqrt(z^2 - f'(a) f'(b)),
    x = b - (b - a) (f'(b) + w - z) / (f'(b) - f'(a) + 2 w)
(Davidon's interpolation formula as given in Fletcher's Practical Methods of
Optimization, Sec. 2.6); a maximum of f is the minimum of -f. A quadratic is
interpolated exactly, so it is found in one step.
"""
from __future__ import annotations

import math


def _cubic_min(a, fa, ga, b, fb, gb):
    z = 3.0 * (fa - fb) / (b - a) + ga + gb
    w = math.sqrt(max(z * z - ga * gb, 0.0))
    den = gb - ga + 2.0 * w
    if den == 0.0:
        return 0.5 * (a + b)
    return b - (b - a) * (gb + w - z) / den


def davidon_maximize(fg, a, b, xtol=1e-2, gtol=0.0, maxit=12, guard=0.05):
    """Maximise f on [a, b] given fg(x) -> (f(x), f'(x)) with f'(a) > 0 >
    f'(b). Each step evaluates the interpolating cubic's maximiser, kept at
    least guard (b - a) inside the interval, and replaces the end whose
    derivative sign it shares. Stops when the interval is shorter than xtol,
    |f'| <= gtol at the new point, or after maxit steps. Returns (x, f(x),
    f'(x), history of (x, f, f') in evaluation order)."""
    fa, ga = fg(a)
    fb, gb = fg(b)
    hist = [(a, fa, ga), (b, fb, gb)]
    if not (ga > 0.0 > gb):
        raise ValueError(f"davidon_maximize: [{a}, {b}] does not bracket a maximum (f' = {ga}, {gb})")
    best = max(hist, key=lambda h: h[1])
    for _ in range(maxit):
        if b - a <= xtol:
            break
        x = _cubic_min(a, -fa, -ga, b, -fb, -gb)
        x = min(max(x, a + guard * (b - a)), b - guard * (b - a))
        fx, gx = fg(x)
        hist.append((x, fx, gx))
        if fx > best[1]:
            best = (x, fx, gx)
        if abs(gx) <= gtol:
            break
        if gx > 0.0:
            a, fa, ga = x, fx, gx
        else:
            b, fb, gb = x, fx, gx
    return best[0], best[1], best[2], hist
