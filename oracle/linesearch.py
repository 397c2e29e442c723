"""Strong-Wolfe line search for the Gauss-Newton step (test infrastructure).

The paper's experiments take the GN step length from a Moré-Thuente line
search (Sec. 5, third-party toolbox). This module restates a published
strong-Wolfe method from its description: the bracketing phase and the zoom
phase of Nocedal & Wright, Numerical Optimization (2nd ed.), Algorithms 3.5 and
3.6, with the trial point of the zoom phase at the minimiser of the cubic
Hermite interpolant of the bracket ends (their Eq. 3.59), kept at least 10 % of
the bracket away from either end (else bisection). Where the two values
compared in the zoom phase agree to within a few units of rounding, the
derivative decides instead (a reading: the published algorithm
assumes exact function values).

phi(alpha) = J(v + alpha p) and phi'(alpha) = g(v + alpha p)^T p. A returned
step satisfies the strong Wolfe conditions
    phi(alpha) <= phi(0) + c1 alpha phi'(0),   |phi'(alpha)| <= c2 |phi'(0)|.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

OK, NOT_DESCENT, MAX_EVALS = 0, 1, 2
EPS = 2.0 ** -52


@dataclass
class LineSearchResult:
    alpha: float
    phi: float
    dphi: float
    evals: int
    status: int
    last: bool          # the accepted step is the last point evaluated


def cubic_min(a, fa, da, b, fb, db):
    """Minimiser of the cubic through (a, fa, da), (b, fb, db), or None."""
    if a == b:
        return None
    d1 = da + db - 3.0 * (fa - fb) / (a - b)
    disc = d1 * d1 - da * db
    if disc < 0.0:
        return None
    d2 = math.copysign(math.sqrt(disc), b - a)
    den = db - da + 2.0 * d2
    if den == 0.0:
        return None
    return b - (b - a) * (db + d2 - d1) / den


def strong_wolfe(phi, phi0, dphi0, alpha1=1.0, c1=1e-4, c2=0.9, alpha_max=10.0, max_evals=30):
    """Step length satisfying the strong Wolfe conditions (N&W Algs. 3.5 / 3.6)."""
    if not dphi0 < 0.0:
        return LineSearchResult(alpha1, math.nan, math.nan, 0, NOT_DESCENT, False)
    evals = 0

    def ev(a):
        nonlocal evals
        evals += 1
        f, d = phi(a)
        return f, d

    def zoom(lo, flo, dlo, hi, fhi, dhi):
        while evals < max_evals:
            width = hi - lo
            a = cubic_min(lo, flo, dlo, hi, fhi, dhi)
            lo_b, hi_b = min(lo, hi), max(lo, hi)
            pad = 0.1 * abs(width)
            if a is None or not (lo_b + pad <= a <= hi_b - pad):
                a = 0.5 * (lo + hi)
            f, d = ev(a)
            # values equal to within rounding carry no information: let the
            # derivative decide (the flat region near a minimiser)
            flat = abs(f - flo) <= 16.0 * EPS * max(abs(f), abs(flo))
            if f > phi0 + c1 * a * dphi0 or (f >= flo and not flat):
                hi, fhi, dhi = a, f, d
            else:
                if abs(d) <= -c2 * dphi0:
                    return LineSearchResult(a, f, d, evals, OK, True)
                if d * (hi - lo) >= 0.0:
                    hi, fhi, dhi = lo, flo, dlo
                lo, flo, dlo = a, f, d
        return LineSearchResult(lo, flo, dlo, evals, MAX_EVALS, False)

    a_prev, f_prev, d_prev = 0.0, phi0, dphi0
    a = alpha1
    first = True
    while evals < max_evals:
        f, d = ev(a)
        if f > phi0 + c1 * a * dphi0 or (not first and f >= f_prev):
            return zoom(a_prev, f_prev, d_prev, a, f, d)
        if abs(d) <= -c2 * dphi0:
            return LineSearchResult(a, f, d, evals, OK, True)
        if d >= 0.0:
            return zoom(a, f, d, a_prev, f_prev, d_prev)
        a_prev, f_prev, d_prev = a, f, d
        a = min(2.0 * a, alpha_max)
        if a == a_prev:  # at alpha_max and still descending
            return LineSearchResult(a, f, d, evals, MAX_EVALS, True)
        first = False
    return LineSearchResult(a_prev, f_prev, d_prev, evals, MAX_EVALS, False)
