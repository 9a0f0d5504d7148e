"""The sub-cube argument used to check the 10^9-cell heat cube on sampled cells.

RK4 applies the 7-point operator four times a step, so after N steps a cell
depends only on cells within 4 N steps of it along the grid.  A sub-cube that
extends 4 N + 1 cells beyond the sampled cell (where the grid allows), with
the full grid's spacing, must therefore give that cell exactly the full grid's
result, whatever its own faces do.  Checked here with the oracle alone.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W


def _window(c, r, l):
    w = min(l, 2 * r + 1)
    s = min(max(c - r, 0), l - w)
    return s, w


@pytest.mark.parametrize("method", ["mm", "cgb"])
def test_sub_cube_reproduces_full_grid(method):
    l, N, dt = 24, 2, 0.02
    alpha = 0.4 / (6 * dt * l * l)
    T = N * dt
    lo, hi = W.random_box(l ** 3, seed=5, centre=(0.0, 1.0), width=(0.0, 0.1))
    flo, fhi = O.reach(method, "heat", lo, hi, t_final=T, dt=dt, params=(alpha, l, 1))
    flo, fhi = flo.reshape(l, l, l), fhi.reshape(l, l, l)
    Lo, Hi = lo.reshape(l, l, l), hi.reshape(l, l, l)
    r = 4 * N + 1
    for (z, y, x) in [(0, 0, 0), (23, 23, 23), (0, 12, 5), (12, 12, 12), (9, 14, 10)]:
        (sz, w), (sy, _), (sx, _) = _window(z, r, l), _window(y, r, l), _window(x, r, l)
        sub = np.s_[sz:sz + w, sy:sy + w, sx:sx + w]
        wlo, whi = O.reach(method, "heat", Lo[sub].ravel(), Hi[sub].ravel(), t_final=T, dt=dt,
                           params=(alpha * (l / w) ** 2, w, 1 if sz == 0 else 0))
        k = ((z - sz) * w + (y - sy)) * w + (x - sx)
        assert abs(wlo[k] - flo[z, y, x]) <= 1e-13 * max(1.0, abs(flo[z, y, x]))
        assert abs(whi[k] - fhi[z, y, x]) <= 1e-13 * max(1.0, abs(fhi[z, y, x]))


def test_too_small_sub_cube_differs():
    """The converse: a sub-cube only 4 N - 1 cells wide around an interior
    cell lets its insulated faces reach the cell (so the margin is needed)."""
    l, N, dt = 24, 2, 0.02
    alpha = 0.4 / (6 * dt * l * l)
    T = N * dt
    lo, hi = W.random_box(l ** 3, seed=5, centre=(0.0, 1.0), width=(0.0, 0.1))
    flo, _ = O.reach("mm", "heat", lo, hi, t_final=T, dt=dt, params=(alpha, l, 1))
    r = 4 * N - 1
    z = y = x = 12
    (s, w) = _window(z, r, l)
    sub = np.s_[s:s + w, s:s + w, s:s + w]
    wlo, _ = O.reach("mm", "heat", lo.reshape(l, l, l)[sub].ravel(), hi.reshape(l, l, l)[sub].ravel(),
                     t_final=T, dt=dt, params=(alpha * (l / w) ** 2, w, 0))
    k = ((z - s) * w + (y - s)) * w + (x - s)
    assert wlo[k] != flo.reshape(l, l, l)[z, y, x]
