"""Tip radius of a dendrite arm from a phase field, for the checks of the
solutal case (Sec. 4.3).  The paper reports tip radii without saying how they
were measured; here (reading R23) the phi = 0 contour is located row by row
near the tip by linear interpolation and the parabola x = x_tip - y^2/(2 r)
is fitted to it by least squares over rows |y - y_axis| <= w.  Test
infrastructure only: it reads fields the solver has already returned."""
from __future__ import annotations

import numpy as np


def contour_x(row: np.ndarray, x0: int) -> float:
    """Outermost phi > 0 -> phi <= 0 crossing at x >= x0 along one row, by
    linear interpolation; NaN if the row has no solid beyond x0 or the solid
    reaches the row's end."""
    pos = np.nonzero(row[x0:] > 0)[0]
    if len(pos) == 0:
        return float("nan")
    i = x0 + int(pos[-1])
    if i + 1 >= len(row):
        return float("nan")
    a, b = row[i], row[i + 1]
    return i + a / (a - b)


def orient(phi: np.ndarray, cx: float, cy: float, arm: str):
    """View of phi (rows y, columns x) in which the arm grows along +x from
    (cx, cy): 'px' as is, 'mx' mirrored in x, 'py' transposed."""
    if arm == "px":
        return phi, cx, cy
    if arm == "mx":
        return phi[:, ::-1], phi.shape[1] - 1 - cx, cy
    if arm == "py":
        return phi.T, cy, cx
    raise ValueError(arm)


def tip_radius(phi: np.ndarray, cx: float, cy: float, arm: str = "px", w: int = 8) -> float:
    """Radius (lattice units) of the parabola fitted to the phi = 0 contour
    of the arm within w rows of its axis."""
    f, cx, cy = orient(phi, cx, cy, arm)
    x0, yc = int(round(cx)), int(round(cy))
    js = np.arange(-w, w + 1)
    xs = np.array([contour_x(f[yc + j], x0) for j in js])
    ok = np.isfinite(xs)
    if ok.sum() < 5:
        return float("nan")
    A = np.stack([np.ones(ok.sum()), -(js[ok].astype(float) ** 2)], 1)
    _, b = np.linalg.lstsq(A, xs[ok], rcond=None)[0]
    return 1.0 / (2.0 * b) if b > 0 else float("nan")
