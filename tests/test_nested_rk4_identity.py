"""The nested form of classic RK4 for a linear system with a constant input.

For dy/dt = C y + p (C, p constant) one classic RK4 step (Sec. 3.1, Algorithm 1
as read in the oracle) and the nested form

    y1 = y + h/4 f(y),  y2 = y + h/3 f(y1),  y3 = y + h/2 f(y2),  y+ = y + h f(y3)

are the same polynomial in h C applied to f(y) = C y + p.  The CUDA path takes
the nested form for the linear halves (the traffic CGB radius with its constant
contraction matrix, the heat cube), the oracle the classic stages; these tests
check the identity in exact rational arithmetic, so that only rounding can
separate the two.
"""
from fractions import Fraction as F
import random

import pytest


def matvec(C, y):
    return [sum(c * v for c, v in zip(row, y)) for row in C]


def f(C, p, y):
    return [a + b for a, b in zip(matvec(C, y), p)]


def axpy(a, x, y):
    return [a * xi + yi for xi, yi in zip(x, y)]


def classic(C, p, y, h):
    k1 = f(C, p, y)
    k2 = f(C, p, axpy(h / 2, k1, y))
    k3 = f(C, p, axpy(h / 2, k2, y))
    k4 = f(C, p, axpy(h, k3, y))
    acc = [a + 2 * b + 2 * c + d for a, b, c, d in zip(k1, k2, k3, k4)]
    return axpy(h / 6, acc, y)


def nested(C, p, y, h):
    y1 = axpy(h / 4, f(C, p, y), y)
    y2 = axpy(h / 3, f(C, p, y1), y)
    y3 = axpy(h / 2, f(C, p, y2), y)
    return axpy(h, f(C, p, y3), y)


def traffic_radius_matrix(n, v, w):
    # r' = C r + [p]: v from the left neighbour, w from the right one (reading R3)
    C = [[F(0)] * n for _ in range(n)]
    for i in range(n):
        if i > 0:
            C[i][i - 1] = v
        if i < n - 1:
            C[i][i + 1] = w
    return C


@pytest.mark.parametrize("n,steps", [(1, 3), (5, 4), (9, 3)])
def test_nested_equals_classic_on_the_traffic_radius(n, steps):
    rng = random.Random(n)
    v, w, h = F(1, 2), F(1, 6), F(1, 100)
    C = traffic_radius_matrix(n, v, w)
    p = [F(rng.randint(1, 9), 2)] + [F(0)] * (n - 1)   # the input half-width enters cell 0
    y = [F(rng.randint(1, 50), 7) for _ in range(n)]
    a, b = list(y), list(y)
    for _ in range(steps):
        a, b = classic(C, p, a, h), nested(C, p, b, h)
        assert a == b


def test_nested_equals_classic_on_a_dense_linear_system():
    rng = random.Random(7)
    n = 6
    C = [[F(rng.randint(-9, 9), rng.randint(1, 9)) for _ in range(n)] for _ in range(n)]
    p = [F(rng.randint(-9, 9), 5) for _ in range(n)]
    y = [F(rng.randint(-20, 20), 3) for _ in range(n)]
    h = F(3, 40)
    assert classic(C, p, y, h) == nested(C, p, y, h)


def test_the_identity_fails_for_a_nonlinear_right_hand_side():
    # the nested form is not RK4 in general: with f(y) = y^2 the two differ,
    # which is why the kernels keep the stage form for the nonlinear halves
    def fq(y):
        return [yi * yi for yi in y]

    y, h = [F(1, 2)], F(1, 10)
    k1 = fq(y)
    k2 = fq(axpy(h / 2, k1, y))
    k3 = fq(axpy(h / 2, k2, y))
    k4 = fq(axpy(h, k3, y))
    rk4 = axpy(h / 6, [a + 2 * b + 2 * c + d for a, b, c, d in zip(k1, k2, k3, k4)], y)
    y1 = axpy(h / 4, fq(y), y)
    y2 = axpy(h / 3, fq(y1), y)
    y3 = axpy(h / 2, fq(y2), y)
    nest = axpy(h, fq(y3), y)
    assert rk4 != nest
