"""Pins for the Brenner series (Sec. 3 eq. Brenner) against its two classical limits."""
import math

import numpy as np

from oracle import brenner


def test_scaled_bracket_matches_printed_form():
    n = np.arange(1, 60, dtype=float)
    for delta in (1e-2, 0.3, 1.0):
        a = math.acosh(1 + delta / 2)
        assert np.allclose(brenner.bracket_scaled(n, a), brenner.bracket_direct(n, a), rtol=1e-9, atol=1e-13)


def test_far_field_limit():
    # well-separated spheres approaching each other: each moves against the other's
    # Stokeslet field 3a/(2d) U, so F/(6 pi mu a U) = 1 + 3a/(2d) + O((a/d)^2)
    for d in (200.0, 1000.0):
        f = brenner.squeeze_force(d - 2.0) / (6 * math.pi)
        assert abs(f - (1 + 1.5 / d)) < 5.0 / d ** 2


def test_lubrication_limit():
    # near contact: F/(6 pi mu a U) = 1/(2 delta) + (9/20) ln(1/delta) + O(1)
    c = [brenner.squeeze_force(d) / (6 * math.pi) - (1 / (2 * d) + 0.45 * math.log(1 / d)) for d in (1e-3, 1e-4, 1e-5)]
    assert abs(c[1] - c[2]) < 2e-3 and abs(c[0] - c[1]) < 5e-3
    assert 1.0 < c[2] < 2.0


def test_scaling_with_speed_viscosity_radius():
    f = brenner.squeeze_force(0.1)
    assert math.isclose(brenner.squeeze_force(0.1, speed=2.0, visc=3.0, radius=1.5), f * 9.0, rel_tol=1e-13)
