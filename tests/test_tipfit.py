"""Pins of the tip-radius estimator used by the solutal checks: exact on a
parabolic interface, and close to the radius of a circle."""
from __future__ import annotations

import math

import numpy as np
import pytest

from tipfit import contour_x, tip_radius


def _field(nx, ny, xi_of_y, width=2.5):
    """phi = tanh((x_i(y) - x)/(sqrt2 W)): solid (phi > 0) left of x_i(y)."""
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    return np.tanh((xi_of_y(y) - x) / (math.sqrt(2.0) * width))


def test_contour_is_linear_interpolation():
    row = np.array([1.0, 0.5, 0.25, -0.75, -1.0])
    assert contour_x(row, 0) == pytest.approx(2.25)
    assert math.isnan(contour_x(-np.ones(5), 0))
    assert math.isnan(contour_x(np.ones(5), 0))


@pytest.mark.parametrize("r", [6.0, 15.0, 40.0])
@pytest.mark.parametrize("arm", ["px", "mx", "py"])
def test_parabola_radius_is_recovered(r, arm):
    n, c = 201, 100
    xt = 160.3
    phi = _field(n, n, lambda y: xt - (y - c) ** 2 / (2 * r))
    if arm == "mx":
        phi = phi[:, ::-1]
    if arm == "py":
        phi = phi.T
    # the tanh profile is symmetric about phi = 0, so the contour is exact
    # to the linear interpolation of a smooth profile
    assert tip_radius(phi, c, c, arm, w=min(8, int(r))) == pytest.approx(r, rel=0.01)


def test_circle_radius_is_close():
    n, c, R = 201, 100, 30.0
    y, x = np.mgrid[0:n, 0:n].astype(float)
    phi = np.tanh((R - np.hypot(x - c, y - c)) / (math.sqrt(2.0) * 2.5))
    # over |y| <= R/4 the circle differs from its osculating parabola by
    # y^4/(8 R^3): the fitted radius is within 2 %
    assert tip_radius(phi, c, c, "px", w=int(R / 4)) == pytest.approx(R, rel=0.02)
