"""Brenner's series for two equal spheres squeezing along their line of centres (Sec. 3, eq. Brenner).

|F| = 8 pi mu a |v| sinh(alpha) sum_{n>=1} n(n+1)/((2n-1)(2n+3)) [ ratio_n - 1 ],
ratio_n = (4 cosh^2((n+1/2) alpha) + (2n+1)^2 sinh^2 alpha) / (2 sinh((2n+1) alpha) - (2n+1) sinh(2 alpha)),
cosh(alpha) = 1 + delta/2 (delta = gap / a).

The bracket is evaluated after dividing numerator and denominator by exp((2n+1) alpha),
which is algebraically identical and avoids overflow for large n alpha.
"""
import math

import numpy as np


def bracket_direct(n, alpha):
    """ratio_n - 1 exactly as printed (overflows for (2n+1) alpha > ~700)."""
    num = 4.0 * np.cosh((n + 0.5) * alpha) ** 2 + (2 * n + 1) ** 2 * np.sinh(alpha) ** 2
    den = 2.0 * np.sinh((2 * n + 1) * alpha) - (2 * n + 1) * np.sinh(2 * alpha)
    return num / den - 1.0


def bracket_scaled(n, alpha):
    """ratio_n - 1 with numerator and denominator divided by exp((2n+1) alpha)."""
    x = (2 * n + 1) * alpha
    e1 = np.exp(-x)
    e2 = np.exp(-2.0 * x)
    m = 2 * n + 1
    num = 2.0 * e1 + 2.0 * e2 + m * m * math.sinh(alpha) ** 2 * e1 + m * math.sinh(2 * alpha) * e1
    den = 1.0 - e2 - m * math.sinh(2 * alpha) * e1
    return num / den


def squeeze_force(delta, speed=1.0, visc=1.0, radius=1.0):
    """|F^(k)| for each sphere of a pair approaching each other, each at |v| = speed."""
    alpha = math.acosh(1.0 + delta / 2.0)
    n_max = int(80.0 / alpha) + 200
    n = np.arange(1, n_max + 1, dtype=np.float64)
    terms = n * (n + 1) / ((2 * n - 1) * (2 * n + 3)) * bracket_scaled(n, alpha)
    return 8.0 * math.pi * visc * radius * speed * math.sinh(alpha) * float(np.sum(terms))
