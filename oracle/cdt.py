"""Cumulative table of the oracle's discrete Gaussian (TEST INFRASTRUCTURE ONLY).

The error distribution G(sigma) of the paper's encryption (Section 2.4) is
read as the discrete Gaussian on the integers |x| <= 19 (six standard
deviations of sigma = 3.2) with probability proportional to
exp(-x^2 / (2 sigma^2)).  A sample inverts the cumulative distribution on a
63-bit uniform integer u: the value is -19 plus the number of thresholds
C_i <= u, where C_i = floor(2^63 * P(X <= -19 + i)) for i = 0..37.

The thresholds are computed here with mpmath at 60 significant digits.
"""
import functools

import mpmath

SIGMA = mpmath.mpf("3.2")
SUPPORT = 19


@functools.lru_cache(maxsize=None)
def cdt_table():
    with mpmath.workdps(60):
        sigma = mpmath.mpf("3.2")
        xs = list(range(-SUPPORT, SUPPORT + 1))
        rho = [mpmath.exp(-mpmath.mpf(x) ** 2 / (2 * sigma ** 2)) for x in xs]
        z = mpmath.fsum(rho)
        out = []
        run = mpmath.mpf(0)
        scale = mpmath.mpf(2) ** 63
        for i in range(2 * SUPPORT):
            run += rho[i]
            out.append(int(mpmath.floor(scale * run / z)))
    return tuple(out)


def probabilities():
    """Exact-at-60-digits probabilities of -19..19, for distribution checks."""
    with mpmath.workdps(60):
        sigma = mpmath.mpf("3.2")
        xs = list(range(-SUPPORT, SUPPORT + 1))
        rho = [mpmath.exp(-mpmath.mpf(x) ** 2 / (2 * sigma ** 2)) for x in xs]
        z = mpmath.fsum(rho)
        return [float(v / z) for v in rho]
