"""Pins of the FP64 oracle against facts other than itself.

Each test checks the oracle against a closed form, an invariant, a published
known-answer table, the defining inequalities of the paper's methods (Sec. 2.1)
evaluated by brute force, or exhaustive sampling on tiny systems.  A dropped
term, a wrong sign or index, a transposed operand or a wrong RK4 weight in
``oracle/oracle.c`` makes at least one of them fail.
"""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.linalg

import oracle as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rk4_poly(Z):
    """RK4 applied to y' = Z y / h gives y <- p(Z) y with p the degree-4 Taylor
    polynomial of exp (Butcher, Numerical Methods for ODEs, Sec. 23)."""
    Z = np.atleast_2d(Z)
    I = np.eye(Z.shape[0])
    return I + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24


def rk4_input_poly(Z):
    """For y' = A y + p with constant p, one RK4 step adds h * phi(hA) p with
    phi(Z) = I + Z/2 + Z^2/6 + Z^3/24."""
    Z = np.atleast_2d(Z)
    I = np.eye(Z.shape[0])
    return I + Z / 2 + Z @ Z / 6 + Z @ Z @ Z / 24


# ------------------------------------------------------------------ Philox
def test_philox_known_answers():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(v, 16) for v in line.split()])
    assert len(rows) == 3
    for r in rows:
        assert O.philox4x32_10(r[0:4], r[4:6]) == tuple(r[6:10])


def test_uniform_stream_properties():
    u = np.array([O.uniform(7, j, i, 0) for j in range(200) for i in range(50)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert np.all(u * 2.0**53 == np.floor(u * 2.0**53))  # 53-bit grid
    assert abs(u.mean() - 0.5) < 0.01
    assert abs(u.var() - 1.0 / 12.0) < 0.005
    # the tag, the sample index, the component index and the seed all change the draw
    assert O.uniform(7, 3, 4, 0) != O.uniform(7, 3, 4, 1)
    assert O.uniform(7, 3, 4, 0) != O.uniform(7, 4, 3, 0)
    assert O.uniform(7, 3, 4, 0) != O.uniform(8, 3, 4, 0)
    assert O.uniform(1 << 32, 0, 0, 0) != O.uniform(0, 0, 0, 0)
    # all 53 bits are used: the lowest one is set about half the time
    assert 0.45 < np.mean((u * 2.0**53).astype(np.int64) & 1) < 0.55


def test_uniform_is_the_stated_conversion_of_philox():
    # counter (i, j, tag, 0), key (seed mod 2^32, seed div 2^32), U = top 53 bits of w0:w1
    seed, j, i, tag = (5 << 32) + 77, 12, 345, 1
    w = O.philox4x32_10([i, j, tag, 0], [seed & 0xFFFFFFFF, seed >> 32])
    assert O.uniform(seed, j, i, tag) == (((w[0] << 32) | w[1]) >> 11) * 2.0**-53


def test_mc_sample_bound_values():
    # Sec. 2.1 / Algorithm 4, m = ceil((2n/eps) ln(2n/delta)), evaluated by hand:
    # 20 ln 20 = 59.91; 640 ln 3200 = 5165.38 (a base-10 log would give 2244)
    assert O.mc_samples(1, 0.1, 0.1) == 60
    assert O.mc_samples(16, 0.05, 0.01) == 5166


def test_nsteps_reading():
    assert O.nsteps(10.0, 0.01) == 1000
    assert O.nsteps(0.05, 1e-4) == 500
    assert O.nsteps(2.0, 0.01) == 200
    assert O.nsteps(0.0, 0.1) == 0
    for bad in [(1.0, 0.3), (1.0, 0.0), (1.0, -0.1), (float("nan"), 0.1), (-1.0, 0.1)]:
        with pytest.raises(O.OracleError):
            O.nsteps(*bad)


# ------------------------------------------------------------------ RK4 (Algorithm 1, reading R1)
@pytest.mark.parametrize("lam", [-1.3, 0.7, -20.0])
def test_rk4_scalar_stability_polynomial(lam):
    h, T = 0.05, 2.0
    N = O.nsteps(T, h)
    y = O.flow("linear", [1.0], [0.0], t_final=T, dt=h, A=[[lam]])
    expect = rk4_poly(h * lam)[0, 0] ** N
    assert y[0] == pytest.approx(expect, rel=1e-13)


def test_rk4_exact_on_nilpotent_system():
    # A^5 = 0 -> exp(hA) equals its degree-4 Taylor polynomial, so RK4 is exact
    A = W.linear_nilpotent(5, seed=3)
    x0 = np.array([0.3, -1.0, 2.0, 0.5, 1.5])
    T = 1.7
    y = O.flow("linear", x0, np.zeros(5), t_final=T, dt=0.1, A=A)
    np.testing.assert_allclose(y, scipy.linalg.expm(A * T) @ x0, rtol=0, atol=1e-12)


def test_rk4_fourth_order_convergence():
    m = 3
    x0 = np.array([0.4, -0.7, 0.9, 0.1, 0.0, -0.2])
    w = np.array([0.01, -0.005, 0.0])
    T = 2.0
    ref = O.flow("osc", x0, w, t_final=T, dt=0.00125)
    errs = [np.abs(O.flow("osc", x0, w, t_final=T, dt=h) - ref).max() for h in (0.04, 0.02, 0.01)]
    assert 13.0 < errs[0] / errs[1] < 19.0
    assert 13.0 < errs[1] / errs[2] < 19.0


# ------------------------------------------------------------------ linear test system (C5)
def _exact_linear_hull(A, lo, hi, plo, phi, T):
    n = A.shape[0]
    aug = np.zeros((2 * n, 2 * n))
    aug[:n, :n] = A
    aug[:n, n:] = np.eye(n)
    E2 = scipy.linalg.expm(aug * T)
    E, G = E2[:n, :n], E2[:n, n:]
    Ep, Em = np.maximum(E, 0), np.minimum(E, 0)
    Gp, Gm = np.maximum(G, 0), np.minimum(G, 0)
    return Ep @ lo + Em @ hi + Gp @ plo + Gm @ phi, Ep @ hi + Em @ lo + Gp @ phi + Gm @ plo


def _discrete_linear_hull(A, lo, hi, plo, phi, h, N):
    """Exact reachable set of the RK4 map itself: x_N = P^N x0 + S p."""
    n = A.shape[0]
    P = rk4_poly(h * A)
    Q = h * rk4_input_poly(h * A)
    PN = np.linalg.matrix_power(P, N)
    S = np.zeros((n, n))
    Pk = np.eye(n)
    for _ in range(N):
        S += Pk @ Q
        Pk = Pk @ P
    Pp, Pm = np.maximum(PN, 0), np.minimum(PN, 0)
    Sp, Sm = np.maximum(S, 0), np.minimum(S, 0)
    return Pp @ lo + Pm @ hi + Sp @ plo + Sm @ phi, Pp @ hi + Pm @ lo + Sp @ phi + Sm @ plo


@pytest.mark.parametrize("method", ["mm", "cgb"])
def test_linear_metzler_matches_expm_hull(method):
    n, T, h = 4, 1.0, 0.01
    A = W.linear_metzler(n, seed=11)
    lo, hi = W.random_box(n, seed=12)
    plo, phi = W.random_box(n, seed=13, centre=(-0.2, 0.2), width=(0.0, 0.1))
    glo, ghi = O.reach(method, "linear", lo, hi, plo, phi, t_final=T, dt=h, A=A)
    elo, ehi = _exact_linear_hull(A, lo, hi, plo, phi, T)
    np.testing.assert_allclose(glo, elo, rtol=0, atol=1e-8)
    np.testing.assert_allclose(ghi, ehi, rtol=0, atol=1e-8)


@pytest.mark.parametrize("method", ["mm", "cgb"])
def test_linear_metzler_equals_discrete_rk4_hull(method):
    # P = p(hA) >= 0 elementwise when h max|a_ii| <= 1, so both bounds are the
    # exact reachable set of the RK4 map
    n, h, N = 4, 0.01, 150
    A = W.linear_metzler(n, seed=21)
    lo, hi = W.random_box(n, seed=22)
    plo, phi = W.random_box(n, seed=23, centre=(-0.2, 0.2), width=(0.0, 0.1))
    assert (rk4_poly(h * A) >= 0).all()
    glo, ghi = O.reach(method, "linear", lo, hi, plo, phi, t_final=N * h, dt=h, A=A)
    dlo, dhi = _discrete_linear_hull(A, lo, hi, plo, phi, h, N)
    np.testing.assert_allclose(glo, dlo, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(ghi, dhi, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("method", ["mm", "cgb"])
def test_linear_general_contains_discrete_hull(method):
    n, h, N = 4, 0.02, 100
    A = W.linear_general(n, seed=31)
    assert (A - np.diag(np.diag(A)) < 0).any()  # not Metzler
    lo, hi = W.random_box(n, seed=32)
    plo, phi = W.random_box(n, seed=33, centre=(-0.2, 0.2), width=(0.0, 0.1))
    glo, ghi = O.reach(method, "linear", lo, hi, plo, phi, t_final=N * h, dt=h, A=A)
    dlo, dhi = _discrete_linear_hull(A, lo, hi, plo, phi, h, N)
    assert (glo <= dlo + 1e-12).all() and (ghi >= dhi - 1e-12).all()


# ------------------------------------------------------------------ traffic (Sec. 5.1, reading R6)
def test_traffic_free_flow_fixed_point():
    # x_i = 70, d = 35: every flux equals 35 (= v x < c, < w (xbar - x)), so x stays put
    n = 9
    x = np.full(n, 70.0)
    assert np.all(O.rhs("traffic", x, [35.0]) == 0.0)
    lo, hi = O.reach("mm", "traffic", x, x, [35.0], [35.0], t_final=3.0, dt=0.01)
    assert np.all(lo == 70.0) and np.all(hi == 70.0)


def test_traffic_mass_balance():
    # Interior fluxes telescope: sum_i dx_i/dt = d - f_{n-1}.  While the last cell
    # stays above c/v = 80 its outflow is the capacity 40, so the total density
    # changes by exactly (d - 40) T; RK4 preserves this linear invariant.
    n, T, h, d = 8, 2.0, 0.01, 35.0
    x0 = np.full(n, 150.0)
    plo, phi = O.reach_pipe("mm", "traffic", x0, x0, [d], [d], t_final=T, dt=h, every=1)
    assert plo[:, -1].min() > 85.0
    xT = O.flow("traffic", x0, [d], t_final=T, dt=h)
    assert xT.sum() == pytest.approx(x0.sum() + (d - 40.0) * T, abs=1e-9)
    assert np.all(plo[-1] == xT)


def test_traffic_mm_is_corner_trajectories():
    wl = W.traffic_small(16)
    lo, hi = O.reach("mm", "traffic", wl["x_lo"], wl["x_hi"], wl["w_lo"], wl["w_hi"],
                     t_final=wl["t_final"], dt=wl["dt"])
    flo = O.flow("traffic", wl["x_lo"], wl["w_lo"], t_final=wl["t_final"], dt=wl["dt"])
    fhi = O.flow("traffic", wl["x_hi"], wl["w_hi"], t_final=wl["t_final"], dt=wl["dt"])
    assert np.array_equal(lo, flo) and np.array_equal(hi, fhi)
    assert lo[0] == pytest.approx(83.333, abs=1e-3) and hi[0] == pytest.approx(236.667, abs=1e-3)


def test_traffic_cgb_radius_closed_form():
    # the traffic contraction matrix is constant, so the radius obeys the linear
    # ODE r' = C r + [p]; with C read off g by unit probes the radius must match
    # expm of that ODE (RK4 error O(h^4))
    n, T, h = 6, 2.0, 0.01
    c0 = np.linspace(60, 200, n)
    C = np.column_stack([O.growth("traffic", c0, np.eye(n)[j], [0.0]) for j in range(n)])
    hp = O.growth("traffic", c0, np.zeros(n), [1.0])
    lo, hi = c0 - 3.0, c0 + 3.0
    glo, ghi = O.reach("cgb", "traffic", lo, hi, [35.0], [45.0], t_final=T, dt=h)
    aug = np.zeros((n + 1, n + 1))
    aug[:n, :n] = C
    aug[:n, n] = hp * 5.0
    E = scipy.linalg.expm(aug * T)
    r = E[:n, :n] @ np.full(n, 3.0) + E[:n, n]
    np.testing.assert_allclose((ghi - glo) / 2, r, rtol=1e-9)


# ------------------------------------------------------------------ KS grid (C8, C9)
@pytest.mark.parametrize("k", [1, 3, 7])
def test_ks_linear_part_fourier_symbol(k):
    # -u_xx - u_xxxx by central differences has the symbol
    # 4 sin^2(th/2)/dx^2 - 16 sin^4(th/2)/dx^4 on the mode cos(th i)
    n, dx = 32, math.pi / 4
    th = 2 * math.pi * k / n
    u = np.cos(th * np.arange(n))
    f = O.rhs("ks", u, params=(dx, 0.0, 1.0, 1.0))
    lam = 4 * math.sin(th / 2) ** 2 / dx**2 - 16 * math.sin(th / 2) ** 4 / dx**4
    np.testing.assert_allclose(f, lam * u, rtol=0, atol=1e-12)


def test_ks_nonlinear_term_closed_form():
    # -u u_x with u = sin(th i): -sin(th i) cos(th i) sin(th)/dx
    n, dx, k = 24, 0.3, 2
    th = 2 * math.pi * k / n
    i = np.arange(n)
    u = np.sin(th * i)
    f = O.rhs("ks", u, params=(dx, 1.0, 0.0, 0.0))
    np.testing.assert_allclose(f, -np.sin(th * i) * np.cos(th * i) * math.sin(th) / dx, atol=1e-13)


def test_ks_mean_is_conserved():
    n = 128
    wl = W.ks_grid(n)
    u0 = 0.5 * (wl["x_lo"] + wl["x_hi"])
    uT = O.flow("ks", u0, t_final=0.05, dt=1e-4, params=wl["params"])
    assert abs(uT.sum() - u0.sum()) < 1e-12 * n
    assert np.abs(uT - u0).max() > 1e-5  # it did move


@pytest.mark.parametrize("method", ["mm", "cgb"])
def test_ks_shift_invariance(method):
    n, k = 40, 7
    wl = W.ks_grid(n, t_final=0.01)
    a = O.reach(method, "ks", wl["x_lo"], wl["x_hi"], t_final=0.01, dt=1e-4, params=wl["params"])
    b = O.reach(method, "ks", np.roll(wl["x_lo"], k), np.roll(wl["x_hi"], k), t_final=0.01,
                dt=1e-4, params=wl["params"])
    assert np.array_equal(np.roll(a[0], k), b[0]) and np.array_equal(np.roll(a[1], k), b[1])


# ------------------------------------------------------------------ oscillator chain (C10)
def _osc_as_linear(m, ka, kc):
    n = 2 * m
    A = np.zeros((n, n))
    for i in range(m):
        A[i, m + i] = 1.0
        A[m + i, i] = -ka - 2 * kc
        if i > 0:
            A[m + i, i - 1] = kc
        if i < m - 1:
            A[m + i, i + 1] = kc
    return A


@pytest.mark.parametrize("method", ["mm", "cgb"])
def test_osc_without_cubic_term_is_the_linear_chain(method):
    m = 4
    q = W.osc_query(m, seed=5, half_width=1e-2, t_final=2.0)
    prm = (1.0, 0.0, 0.5)
    wlo = np.concatenate([np.zeros(m), q["w_lo"]])
    whi = np.concatenate([np.zeros(m), q["w_hi"]])
    a = O.reach(method, "osc", q["x_lo"], q["x_hi"], q["w_lo"], q["w_hi"], t_final=2.0,
                dt=q["dt"], params=prm)
    b = O.reach(method, "linear", q["x_lo"], q["x_hi"], wlo, whi, t_final=2.0, dt=q["dt"],
                A=_osc_as_linear(m, 1.0, 0.5))
    np.testing.assert_allclose(a[0], b[0], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(a[1], b[1], rtol=1e-12, atol=1e-14)


# ------------------------------------------------------------------ defining properties (Sec. 2.1)
def _systems():
    g = np.random.default_rng(99)
    A = W.linear_general(5, seed=41)
    return [
        ("traffic", 6, None, None, lambda n: (g.uniform(0, 320, n), g.uniform(0, 30, n)), 1),
        ("ks", 8, (math.pi / 4, 1.0, 1.0, 1.0), None,
         lambda n: (g.uniform(-1, 1, n), g.uniform(0, 0.5, n)), 0),
        ("osc", 6, None, None, lambda n: (g.uniform(-1.5, 1.5, n), g.uniform(0, 0.5, n)), 3),
        ("linear", 5, None, A, lambda n: (g.uniform(-1, 1, n), g.uniform(0, 0.5, n)), 5),
    ]


@pytest.mark.parametrize("sysdef", _systems(), ids=lambda s: s[0])
def test_decomposition_properties(sysdef):
    kind, n, prm, A, draw, nw = sysdef
    g = np.random.default_rng(7)
    for trial in range(20):
        c, hw = draw(n)
        x, xh = c - hw, c + hw
        p = g.uniform(30, 40, nw) if kind == "traffic" else g.uniform(-0.1, 0.0, nw)
        ph = p + g.uniform(0, 0.05, nw)
        kw = dict(params=prm, A=A)
        # d(x, p, x, p) = f(x, p)
        np.testing.assert_allclose(O.decomp(kind, x, p, x, p, **kw), O.rhs(kind, x, p, **kw),
                                   rtol=1e-13, atol=1e-12)
        d0 = O.decomp(kind, x, p, xh, ph, **kw)
        u0 = O.decomp(kind, xh, ph, x, p, **kw)
        # monotone in the off-diagonal arguments (finite increases, box kept ordered)
        for j in range(n):
            e = np.zeros(n)
            e[j] = 0.5 * hw[j] + 1e-3
            d1 = O.decomp(kind, x + e, p, xh + e, ph, **kw)
            for i in range(n):
                if i == j:
                    continue
                # raising x_j (lower argument) may not lower d_i(x, ., xh, .)
                dx_only = O.decomp(kind, x + np.where(np.arange(n) == j, min(e[j], xh[j] - x[j]), 0),
                                   p, xh, ph, **kw)
                assert dx_only[i] >= d0[i] - 1e-12 * (1 + abs(d0[i]))
                dxh_only = O.decomp(kind, x, p, xh + e, ph, **kw)
                assert dxh_only[i] <= d0[i] + 1e-12 * (1 + abs(d0[i]))
            del d1
        # the decomposition bounds f over the box with the diagonal argument held
        for _ in range(30):
            y = x + g.random(n) * (xh - x)
            q = p + g.random(nw) * (ph - p)
            fy_lo = O.rhs(kind, np.where(np.eye(n, dtype=bool), x[:, None], y[None, :]).diagonal()
                          if False else y, q, **kw)
            for i in range(n):
                yl = y.copy()
                yl[i] = x[i]
                yu = y.copy()
                yu[i] = xh[i]
                assert d0[i] <= O.rhs(kind, yl, q, **kw)[i] + 1e-12 * (1 + abs(d0[i]))
                assert u0[i] >= O.rhs(kind, yu, q, **kw)[i] - 1e-12 * (1 + abs(u0[i]))
            del fy_lo


def _num_jacobian(kind, y, p, kw, eps=1e-6):
    n = y.size
    J = np.empty((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = eps
        J[:, j] = (O.rhs(kind, y + e, p, **kw) - O.rhs(kind, y - e, p, **kw)) / (2 * eps)
    return J


@pytest.mark.parametrize("sysdef", _systems(), ids=lambda s: s[0])
def test_contraction_matrix_is_the_box_supremum(sysdef):
    # Sec. 2.1: C_ii >= J_ii, C_ij >= |J_ij|.  Every Jacobian entry of these
    # systems is affine or monotone in |x| on each coordinate, so its supremum
    # over the box is attained at a corner: g(c, r) - [p] must equal
    # sum_j sup_corners(J_ij) r_j, not merely exceed it.
    kind, n, prm, A, draw, nw = sysdef
    kw = dict(params=prm, A=A)
    g = np.random.default_rng(5)
    for trial in range(4):
        c, r = draw(n)
        if kind == "traffic":
            c = g.uniform(20, 300, n)
            r = g.uniform(0, 2, n)
            p = np.array([40.0])
        else:
            p = np.zeros(nw)
        corners = np.array(list(itertools.product([-1.0, 1.0], repeat=n)))
        Csup = np.full((n, n), -np.inf)
        for s in corners:
            J = _num_jacobian(kind, c + s * r, p, kw)
            Jb = np.abs(J)
            Jb[np.diag_indices(n)] = J.diagonal()
            Csup = np.maximum(Csup, Jb)
        gr = O.growth(kind, c, r, np.zeros(max(nw, 0)), **kw)
        expect = Csup @ r
        if kind == "traffic":
            # piecewise-linear fluxes: corners need not hit every regime; the
            # constant C must dominate the sampled supremum
            assert (gr >= expect - 1e-8).all()
        else:
            np.testing.assert_allclose(gr, expect, rtol=1e-7, atol=1e-7)


def test_traffic_contraction_matrix_is_tight_over_all_states():
    # random states in [0, 320] visit every regime of the min; the sampled
    # supremum of the Jacobian then equals the constant bound exactly
    n = 5
    g = np.random.default_rng(3)
    C = np.column_stack([O.growth("traffic", np.zeros(n), np.eye(n)[j], [0.0]) for j in range(n)])
    Csup = np.full((n, n), -np.inf)
    for _ in range(3000):
        J = _num_jacobian("traffic", g.uniform(1, 319, n), np.array([40.0]), {}, eps=1e-7)
        Jb = np.abs(J)
        Jb[np.diag_indices(n)] = J.diagonal()
        Csup = np.maximum(Csup, Jb)
    np.testing.assert_allclose(C, Csup, atol=1e-6)


# ------------------------------------------------------------------ brute force (C11)
BRUTE = [
    ("traffic", np.array([100.0, 110.0, 95.0]), np.array([110.0, 120.0, 100.0]),
     np.array([35.0]), np.array([45.0]), 3.0, 0.01, None, None),
    ("ks", np.array([0.1, -0.2, 0.3, 0.0]), np.array([0.15, -0.1, 0.35, 0.1]),
     np.zeros(0), np.zeros(0), 0.1, 1e-3, (math.pi / 4, 1.0, 1.0, 1.0), None),
    ("osc", np.array([0.5, -0.3, 0.0, 0.1]), np.array([0.52, -0.28, 0.02, 0.12]),
     np.array([-0.01, -0.01]), np.array([0.01, 0.01]), 2.0, 0.005, None, None),
    ("linear", np.array([-0.1, 0.2, 0.5]), np.array([0.1, 0.3, 0.6]),
     np.array([-0.1, 0.0, 0.1]), np.array([0.1, 0.05, 0.1]), 1.5, 0.01, None,
     W.linear_general(3, seed=51)),
]


@pytest.mark.parametrize("case", BRUTE, ids=lambda c: c[0])
def test_brute_force_samples_inside_mm_and_cgb(case):
    kind, lo, hi, wlo, whi, T, h, prm, A = case
    kw = dict(params=prm, A=A)
    n, nw = lo.size, wlo.size
    mm = O.reach("mm", kind, lo, hi, wlo, whi, t_final=T, dt=h, **kw)
    cg = O.reach("cgb", kind, lo, hi, wlo, whi, t_final=T, dt=h, **kw)
    g = np.random.default_rng(17)
    pts = [np.array(c) for c in itertools.product(*[np.linspace(0, 1, 4)] * n)]
    pts += [g.random(n) for _ in range(300)]
    worst = np.inf
    for k, u in enumerate(pts):
        x0 = lo + u * (hi - lo)
        w = wlo + (g.random(nw) if k % 2 else (k // 2) % 2 * np.ones(nw)) * (whi - wlo)
        xT = O.flow(kind, x0, w, t_final=T, dt=h, **kw)
        for blo, bhi in (mm, cg):
            worst = min(worst, (xT - blo).min(), (bhi - xT).min())
    assert worst >= 0.0, f"a trajectory left the box by {-worst}"


# ------------------------------------------------------------------ Monte Carlo (Algorithm 4)
def test_mc_box_is_elementwise_min_max_of_samples():
    wl = W.traffic_small(16)
    lo, hi, fin = O.reach("mc", "traffic", wl["x_lo"], wl["x_hi"], wl["w_lo"], wl["w_hi"],
                          t_final=1.0, dt=0.01, m=64, seed=3, return_finals=True)
    assert np.array_equal(lo, fin.min(axis=0)) and np.array_equal(hi, fin.max(axis=0))


@pytest.mark.parametrize("prec", [64, 32])
def test_mc_samples_are_uniform_in_the_initial_box(prec):
    n, m = 5, 4000
    lo, hi = W.random_box(n, seed=61, width=(0.1, 1.0))
    _, _, fin = O.reach("mc", "linear", lo, hi, np.zeros(n), np.zeros(n), t_final=0.0, dt=0.1,
                        A=np.zeros((n, n)), m=m, seed=9, prec=prec, return_finals=True)
    u = (fin - lo) / (hi - lo)
    assert (u >= -1e-7).all() and (u < 1 + 1e-7).all()
    assert np.abs(u.mean(axis=0) - 0.5).max() < 0.02
    if prec == 32:
        assert np.array_equal(fin, fin.astype(np.float32).astype(np.float64))
    else:
        j, i = 17, 3
        assert fin[j, i] == lo[i] + (hi[i] - lo[i]) * O.uniform(9, j, i, 0)


def test_mc_samples_the_inputs_too():
    # reading R4: with A = 0 the final state is x0 + T p, which recovers every
    # sampled input; they must follow the input stream (tag 1)
    n, m, T = 3, 500, 2.0
    lo, hi = np.zeros(n), np.zeros(n)
    plo, phi = np.array([-1.0, 0.0, 2.0]), np.array([1.0, 0.5, 2.0])
    _, _, fin = O.reach("mc", "linear", lo, hi, plo, phi, t_final=T, dt=0.5, A=np.zeros((n, n)),
                        m=m, seed=4, return_finals=True)
    p = fin / T
    assert p[:, 0].min() < -0.9 and p[:, 0].max() > 0.9 and np.all(p[:, 2] == 2.0)
    assert p[7, 1] == pytest.approx(0.5 * O.uniform(4, 7, 1, 1), rel=1e-14)


def test_mc_inside_mm_traffic_config():
    wl = W.traffic_small(16)
    args = (wl["x_lo"], wl["x_hi"], wl["w_lo"], wl["w_hi"])
    kw = dict(t_final=wl["t_final"], dt=wl["dt"])
    mlo, mhi = O.reach("mm", "traffic", *args, **kw)
    clo, chi = O.reach("mc", "traffic", *args, **kw, m=1000, seed=0)
    assert (clo >= mlo).all() and (chi <= mhi).all()


# ------------------------------------------------------------------ degenerate boxes (C13)
@pytest.mark.parametrize("kind", ["traffic", "ks", "osc", "linear"])
def test_zero_width_box_is_one_trajectory(kind):
    g = np.random.default_rng(2)
    n = 6
    prm = None
    A = W.linear_general(n, seed=71) if kind == "linear" else None
    if kind == "traffic":
        x = g.uniform(50, 200, n)
        w = np.array([40.0])
    elif kind == "ks":
        x = g.uniform(-0.5, 0.5, n)
        w = np.zeros(0)
    else:
        x = g.uniform(-1, 1, n)
        w = g.uniform(-0.01, 0.01, O.input_dim(kind, n))
    kw = dict(t_final=0.5, dt=0.005, params=prm, A=A)
    traj = O.flow(kind, x, w, **kw)
    mlo, mhi = O.reach("mm", kind, x, x, w, w, **kw)
    np.testing.assert_allclose(mlo, traj, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(mhi, traj, rtol=1e-12, atol=1e-12)
    clo, chi = O.reach("cgb", kind, x, x, w, w, **kw)
    assert np.array_equal(clo, traj) and np.array_equal(chi, traj)  # r stays exactly 0
    slo, shi = O.reach("mc", kind, x, x, w, w, **kw, m=8, seed=1)
    assert np.array_equal(slo, traj) and np.array_equal(shi, traj)


# ------------------------------------------------------------------ reach pipe (Sec. 5.5)
@pytest.mark.parametrize("method", ["mm", "cgb"])
def test_pipe_rows_are_intermediate_boxes(method):
    wl = W.traffic_small(8)
    args = (wl["x_lo"], wl["x_hi"], wl["w_lo"], wl["w_hi"])
    plo, phi = O.reach_pipe(method, "traffic", *args, t_final=1.0, dt=0.01, every=25)
    assert plo.shape == (4, 8)
    for q in range(4):
        lo, hi = O.reach(method, "traffic", *args, t_final=0.25 * (q + 1), dt=0.01)
        np.testing.assert_allclose(plo[q], lo, rtol=1e-14)
        np.testing.assert_allclose(phi[q], hi, rtol=1e-14)


# ------------------------------------------------------------------ 3-D heat diffusion (Sec. 5.4, reading R12)
def _heat_matrix(l, kh, open_face):
    """Graph Laplacian of the l^3 grid assembled from the PDE's stencil: each
    present neighbour contributes kh (u_nb - u_i); below z = 0 an open face
    contributes kh (0 - u_i)."""
    n = l ** 3
    A = np.zeros((n, n))
    idx = lambda x, y, z: x + l * (y + l * z)
    for z in range(l):
        for y in range(l):
            for x in range(l):
                i = idx(x, y, z)
                for dxx, dyy, dzz in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    X, Y, Z = x + dxx, y + dyy, z + dzz
                    if 0 <= X < l and 0 <= Y < l and 0 <= Z < l:
                        A[i, idx(X, Y, Z)] += kh
                        A[i, i] -= kh
                    elif Z < 0 and open_face:
                        A[i, i] -= kh
    return A


@pytest.mark.parametrize("method", ["mm", "cgb"])
@pytest.mark.parametrize("open_face", [0.0, 1.0])
def test_heat_equals_the_assembled_linear_system(method, open_face):
    l, alpha = 3, 0.02
    kh = alpha * l * l
    lo, hi = W.random_box(l ** 3, seed=81, centre=(0.0, 1.0), width=(0.0, 0.1))
    a = O.reach(method, "heat", lo, hi, t_final=1.0, dt=0.01, params=(alpha, l, open_face))
    A = _heat_matrix(l, kh, open_face)
    z = np.zeros(l ** 3)
    b = O.reach(method, "linear", lo, hi, z, z, t_final=1.0, dt=0.01, A=A)
    np.testing.assert_allclose(a[0], b[0], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(a[1], b[1], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("k", [(1, 0, 0), (0, 2, 1), (3, 1, 2)])
def test_heat_neumann_cosine_modes(k):
    # with every face insulated, cos(pi k (x + 1/2) / l) in each direction is an
    # eigenvector of the discrete operator with eigenvalue -2 kh sum(1 - cos(pi k / l))
    l, alpha = 6, 0.01
    kh = alpha * l * l
    c = [np.cos(np.pi * kk * (np.arange(l) + 0.5) / l) for kk in k]
    u = np.einsum("z,y,x->zyx", c[2], c[1], c[0]).reshape(-1)
    lam = -2.0 * kh * sum(1.0 - np.cos(np.pi * kk / l) for kk in k)
    np.testing.assert_allclose(O.rhs("heat", u, params=(alpha, l, 0.0)), lam * u, atol=1e-12)


def test_heat_is_conserved_in_a_closed_box_and_leaks_through_the_open_face():
    l, alpha = 5, 0.01
    kh = alpha * l * l
    u0 = np.random.default_rng(8).random(l ** 3)
    closed = O.flow("heat", u0, t_final=2.0, dt=0.01, params=(alpha, l, 0.0))
    assert abs(closed.sum() - u0.sum()) < 1e-12 * u0.sum()
    # open face: the total changes at -kh times the heat of the bottom layer
    du = O.rhs("heat", u0, params=(alpha, l, 1.0))
    assert du.sum() == pytest.approx(-kh * u0[: l * l].sum(), rel=1e-12)


# ------------------------------------------------------------------ quadrotor swarm (Sec. 5.2, reading R13)
QM, QG = 1.4, 9.81
QPRM = (QM, QG, QM * QG, 0.054, 0.061, 0.104)   # Jx != Jy so that a swapped inertia shows


def _agent(pos=(0, 0, 0), vel=(0, 0, 0), ang=(0, 0, 0), rate=(0, 0, 0)):
    return np.array([*pos, *vel, *ang, *rate], dtype=float)


def test_quad_hover_is_an_equilibrium():
    x = _agent(pos=(1.0, -2.0, 3.0))
    d = O.rhs("quad", x, np.zeros(3), params=QPRM)
    np.testing.assert_allclose(d, 0.0, atol=1e-14)


@pytest.mark.parametrize("ang,unit", [
    # (phi, theta, psi) -> (ddp_n / a, ddp_e / a, (ddh - g) / a) with a = F/m,
    # worked out by hand from the paper's equations
    ((math.pi / 2, 0.0, 0.0), (0.0, 1.0, 0.0)),
    ((0.0, math.pi / 2, 0.0), (-1.0, 0.0, 0.0)),
    ((0.0, math.pi / 2, math.pi / 2), (0.0, -1.0, 0.0)),
    ((math.pi / 2, 0.0, math.pi / 2), (-1.0, 0.0, 0.0)),
    ((math.pi, 0.0, 0.0), (0.0, 0.0, 1.0)),
    ((0.0, 0.0, 1.0), (0.0, 0.0, -1.0)),
])
def test_quad_accelerations_at_right_angles(ang, unit):
    a = QPRM[2] / QM
    d = O.rhs("quad", _agent(ang=ang), np.zeros(3), params=QPRM)
    np.testing.assert_allclose(d[3:6], (a * unit[0], a * unit[1], QG + a * unit[2]), atol=1e-12)


def test_quad_thrust_direction_has_unit_length():
    # (ddp_n, ddp_e, g - ddh) / a is the third column of a rotation matrix
    g = np.random.default_rng(11)
    a = QPRM[2] / QM
    for _ in range(200):
        x = _agent(ang=g.uniform(-4, 4, 3))
        d = O.rhs("quad", x, np.zeros(3), params=QPRM)
        v = np.array([d[3], d[4], QG - d[5]]) / a
        assert abs(np.linalg.norm(v) - 1.0) < 1e-13


def test_quad_passive_rows_and_inputs():
    g = np.random.default_rng(12)
    x = g.uniform(-1, 1, 24)
    tau = g.uniform(-1, 1, 6)
    d = O.rhs("quad", x, tau, params=QPRM)
    for k in range(2):
        y, dy, t = x[12 * k:12 * k + 12], d[12 * k:12 * k + 12], tau[3 * k:3 * k + 3]
        np.testing.assert_array_equal(dy[0:3], y[3:6])
        np.testing.assert_array_equal(dy[6:9], y[9:12])
        np.testing.assert_allclose(dy[9:12], t / np.array(QPRM[3:6]), rtol=1e-15)


def test_quad_flow_at_constant_attitude_is_a_parabola():
    # no torque and no angular rate: the acceleration is constant, so RK4 is exact
    ang = (0.3, -0.2, 1.1)
    x0 = _agent(pos=(1.0, 2.0, -3.0), vel=(0.5, -0.25, 0.1), ang=ang)
    acc = O.rhs("quad", x0, np.zeros(3), params=QPRM)[3:6]
    T = 1.5
    x = O.flow("quad", x0, np.zeros(3), t_final=T, dt=0.05, params=QPRM)
    np.testing.assert_allclose(x[0:3], x0[0:3] + x0[3:6] * T + 0.5 * acc * T * T, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(x[3:6], x0[3:6] + acc * T, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(x[6:9], ang, rtol=0, atol=0)


def test_quad_flow_of_the_angles_under_constant_torque():
    tau = np.array([0.01, -0.02, 0.03])
    x0 = _agent(ang=(0.0, 0.0, 0.2), rate=(0.0, 0.0, 0.0))
    T = 1.0
    x = O.flow("quad", x0, tau, t_final=T, dt=0.01, params=QPRM)
    J = np.array(QPRM[3:6])
    np.testing.assert_allclose(x[9:12], tau / J * T, rtol=1e-13)
    np.testing.assert_allclose(x[6:9], x0[6:9] + 0.5 * tau / J * T * T, rtol=1e-12)


def test_quad_agents_are_independent():
    g = np.random.default_rng(13)
    K = 4
    c = g.uniform(-0.5, 0.5, 12 * K)
    lo, hi = c - 0.01, c + 0.01
    wl = g.uniform(-0.02, 0.0, 3 * K)
    wh = wl + 0.02
    for method in ("mm", "cgb"):
        a = O.reach(method, "quad", lo, hi, wl, wh, t_final=0.5, dt=0.01, params=QPRM)
        for k in range(K):
            s, t = slice(12 * k, 12 * k + 12), slice(3 * k, 3 * k + 3)
            b = O.reach(method, "quad", lo[s], hi[s], wl[t], wh[t], t_final=0.5, dt=0.01, params=QPRM)
            np.testing.assert_array_equal(a[0][s], b[0])
            np.testing.assert_array_equal(a[1][s], b[1])


def test_quad_decomposition_at_a_point_is_f():
    g = np.random.default_rng(14)
    for _ in range(50):
        x = g.uniform(-4, 4, 12)
        p = g.uniform(-1, 1, 3)
        np.testing.assert_array_equal(O.decomp("quad", x, p, x, p, params=QPRM),
                                      O.rhs("quad", x, p, params=QPRM))


def _single_angle_range(j, lo, hi, fixed):
    """Exact range of the acceleration rows over an interval of angle j (the
    other angles fixed): sampling with the endpoints and every multiple of
    pi/2 inside (where sine and cosine have their extrema)."""
    crit = [k * math.pi / 2 for k in range(math.ceil(lo / (math.pi / 2)), math.floor(hi / (math.pi / 2)) + 1)]
    t = np.concatenate([np.linspace(lo, hi, 401), [lo, hi], crit])
    vals = []
    for v in t:
        ang = list(fixed)
        ang[j] = v
        vals.append(O.rhs("quad", _agent(ang=ang), np.zeros(3), params=QPRM)[3:6])
    vals = np.array(vals)
    return vals.min(axis=0), vals.max(axis=0)


@pytest.mark.parametrize("j,fixed", [(0, (0.0, 0.0, 0.0)), (1, (0.0, 0.0, 0.0)), (2, (0.0, 0.7, 0.0)),
                                     (0, (0.0, 0.0, 0.9))])
def test_quad_decomposition_is_tight_when_one_angle_varies(j, fixed):
    # with one angle varying, each acceleration has that angle in one factor (or
    # none), so the interval extension is the exact range: this pins the
    # extremum logic of the interval sine and cosine, including wide intervals
    g = np.random.default_rng(15 + j)
    intervals = [(-0.3, 0.2), (1.2, 1.9), (-1.9, -1.2), (2.9, 3.4), (-7.0, 0.5), (0.1, 6.5), (-3.5, -2.9)]
    intervals += [tuple(sorted(g.uniform(-7, 7, 2))) for _ in range(6)]
    for lo_a, hi_a in intervals:
        x = _agent(ang=fixed)
        xh = x.copy()
        x[6 + j], xh[6 + j] = lo_a, hi_a
        dlo = O.decomp("quad", x, np.zeros(3), xh, np.zeros(3), params=QPRM)
        dhi = O.decomp("quad", xh, np.zeros(3), x, np.zeros(3), params=QPRM)
        rmin, rmax = _single_angle_range(j, lo_a, hi_a, fixed)
        np.testing.assert_allclose(dlo[3:6], rmin, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(dhi[3:6], rmax, rtol=1e-12, atol=1e-12)


def test_quad_decomposition_bounds_f_on_the_box_and_is_monotone():
    g = np.random.default_rng(16)
    for _ in range(20):
        c = g.uniform(-3, 3, 12)
        h = g.uniform(0, 0.6, 12)
        lo, hi = c - h, c + h
        p = np.zeros(3)
        dlo = O.decomp("quad", lo, p, hi, p, params=QPRM)
        dhi = O.decomp("quad", hi, p, lo, p, params=QPRM)
        for _ in range(100):
            f = O.rhs("quad", g.uniform(lo, hi), p, params=QPRM)
            assert np.all(dlo[3:6] <= f[3:6] + 1e-12) and np.all(f[3:6] <= dhi[3:6] + 1e-12)
        # shrinking the box (raising x, lowering xh) can only raise d(x, xh)
        lo2 = lo + g.uniform(0, 1, 12) * h
        hi2 = hi - g.uniform(0, 1, 12) * h
        d2 = O.decomp("quad", lo2, p, hi2, p, params=QPRM)
        assert np.all(d2[3:6] >= dlo[3:6] - 1e-12)


def _fd_jacobian(x, eps=1e-6):
    J = np.empty((12, 12))
    for j in range(12):
        e = np.zeros(12)
        e[j] = eps
        J[:, j] = (O.rhs("quad", x + e, np.zeros(3), params=QPRM) -
                   O.rhs("quad", x - e, np.zeros(3), params=QPRM)) / (2 * eps)
    return J


def test_quad_growth_bounds_the_jacobian():
    # a box with one angle of nonzero radius isolates one column of C in the
    # acceleration rows: C_ij r_j >= |J_ij(y)| r_j at every y in the box
    g = np.random.default_rng(17)
    for _ in range(12):
        c = _agent(ang=g.uniform(-3, 3, 3))
        for j in range(3):
            r = np.zeros(12)
            r[6 + j] = g.uniform(0.01, 0.5)
            dr = O.growth("quad", c, r, np.zeros(3), params=QPRM)
            Cj = dr[3:6] / r[6 + j]
            best = np.zeros(3)
            for t in np.linspace(-1, 1, 41):
                y = c.copy()
                y[6 + j] += t * r[6 + j]
                Jy = np.abs(_fd_jacobian(y)[3:6, 6 + j])
                assert np.all(Jy <= Cj + 1e-6)
                best = np.maximum(best, Jy)
            # the natural extension overestimates where the angle occurs twice
            # (dependency), by at most the enclosure widths: O(a r_j)
            assert np.all(Cj <= best + 2.0 * QPRM[2] / QM * r[6 + j] + 1e-6)


def test_quad_growth_structure():
    g = np.random.default_rng(18)
    c = g.uniform(-1, 1, 12)
    r = g.uniform(0, 0.1, 12)
    hp = g.uniform(0, 0.01, 3)
    dr = O.growth("quad", c, r, hp, params=QPRM)
    np.testing.assert_array_equal(dr[0:3], r[3:6])
    np.testing.assert_array_equal(dr[6:9], r[9:12])
    np.testing.assert_allclose(dr[9:12], hp / np.array(QPRM[3:6]), rtol=1e-15)
    np.testing.assert_array_equal(O.growth("quad", c, np.zeros(12), np.zeros(3), params=QPRM), 0.0)
    # at a point the angular entries equal |J| exactly (the interval extension of
    # a point is the point)
    J = _fd_jacobian(c)
    r1 = np.zeros(12)
    r1[6:9] = 1e-9
    dr1 = O.growth("quad", c, r1, np.zeros(3), params=QPRM)
    np.testing.assert_allclose(dr1[3:6] / 1e-9, np.abs(J[3:6, 6:9]).sum(axis=1), rtol=1e-5)


@pytest.mark.parametrize("method", ["mm", "cgb"])
def test_quad_boxes_contain_sampled_trajectories(method):
    g = np.random.default_rng(19)
    K = 3
    c = np.concatenate([_agent(pos=g.uniform(-5, 5, 3), vel=g.uniform(-1, 1, 3),
                               ang=(*g.uniform(-0.3, 0.3, 2), g.uniform(-3, 3)), rate=g.uniform(-0.1, 0.1, 3))
                        for _ in range(K)])
    h = np.tile(np.array([0.05] * 3 + [0.01] * 3 + [0.02] * 3 + [0.01] * 3), K)
    wl = np.tile([-0.005, -0.005, -0.002], K)
    wh = -wl
    lo, hi = O.reach(method, "quad", c - h, c + h, wl, wh, t_final=1.0, dt=0.01, params=QPRM)
    _, _, finals = O.reach("mc", "quad", c - h, c + h, wl, wh, t_final=1.0, dt=0.01, params=QPRM,
                           m=64, seed=5, return_finals=True)
    assert np.all(finals >= lo - 1e-9) and np.all(finals <= hi + 1e-9)


def test_quad_point_box_is_the_trajectory():
    x0 = _agent(pos=(1, 2, 3), vel=(0.1, 0.2, 0.3), ang=(0.2, -0.1, 2.0), rate=(0.05, -0.02, 0.1))
    tau = np.array([0.003, -0.001, 0.002])
    traj = O.flow("quad", x0, tau, t_final=1.0, dt=0.01, params=QPRM)
    for method in ("mm", "cgb"):
        lo, hi = O.reach(method, "quad", x0, x0, tau, tau, t_final=1.0, dt=0.01, params=QPRM)
        np.testing.assert_allclose(lo, traj, rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(hi, traj, rtol=1e-13, atol=1e-13)


# ------------------------------------------------------------------ box-evaluated traffic C (reading R14)
TLP = O.TRAFFIC_LOCAL_PRM


def _traffic_fd_jacobian(x, eps=1e-5):
    n = x.size
    J = np.empty((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = eps
        J[:, j] = (O.rhs("traffic", x + e, [40.0], params=TLP) - O.rhs("traffic", x - e, [40.0], params=TLP)) / (2 * eps)
    return J


@pytest.mark.parametrize("regime", [(1.0, 60.0), (60.0, 250.0), (240.0, 320.0), (0.0, 320.0)])
def test_traffic_local_growth_bounds_the_jacobian(regime):
    # C r >= J_ii r_i + sum_{j != i} |J_ij| r_j at every point of the box
    g = np.random.default_rng(int(regime[0]) + 5)
    n = 10
    for _ in range(8):
        a = g.uniform(*regime, n)
        b = g.uniform(*regime, n)
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        c, r = (lo + hi) / 2, (hi - lo) / 2
        dr = O.growth("traffic", c, r, [0.0], params=TLP)
        for _ in range(60):
            y = g.uniform(lo, hi)
            J = _traffic_fd_jacobian(y)
            need = np.abs(J) @ r - np.abs(np.diag(J)) * r + np.diag(J) * r
            # (a difference quotient across a kink lies between the one-sided slopes)
            assert np.all(dr >= need - 1e-7 * (1.0 + r.sum()))


def test_traffic_local_is_tighter_than_the_global_bound():
    g = np.random.default_rng(6)
    for _ in range(20):
        c = g.uniform(0, 320, 12)
        r = g.uniform(0, 30, 12)
        loc = O.growth("traffic", c, r, [2.0], params=TLP)
        glob = O.growth("traffic", c, r, [2.0], params=O.TRAFFIC_PRM)
        assert np.all(loc <= glob + 1e-12)


def test_traffic_local_free_flow_and_congested_boxes():
    v, w = 0.5, 1.0 / 6.0
    g = np.random.default_rng(7)
    n = 8
    # free flow everywhere in the box: C = v on the subdiagonal, -v on the diagonal
    c = g.uniform(3, 8, n)
    r = g.uniform(0.5, 2, n)
    dr = O.growth("traffic", c, r, [1.5], params=TLP)
    want = -v * r
    want[1:] += v * r[:-1]
    want[0] += 1.5
    np.testing.assert_allclose(dr, want, rtol=1e-14, atol=1e-14)
    # congested everywhere (the last cell flows at capacity): w on the
    # superdiagonal, -w on the diagonal of every cell with a congested inflow
    c = g.uniform(302, 308, n)
    r = g.uniform(0.5, 2, n)
    dr = O.growth("traffic", c, r, [1.5], params=TLP)
    want = np.zeros(n)
    want[:-1] += w * r[1:]
    want[1:] -= w * r[1:]
    want[0] += 1.5
    np.testing.assert_allclose(dr, want, rtol=1e-14, atol=1e-14)


def test_traffic_local_cgb_contains_sampled_trajectories():
    wl = W.traffic_small(16)
    lo, hi = O.reach("cgb", "traffic", wl["x_lo"], wl["x_hi"], wl["w_lo"], wl["w_hi"], t_final=2.0, dt=0.01,
                     params=TLP)
    glo, ghi = O.reach("cgb", "traffic", wl["x_lo"], wl["x_hi"], wl["w_lo"], wl["w_hi"], t_final=2.0, dt=0.01)
    _, _, finals = O.reach("mc", "traffic", wl["x_lo"], wl["x_hi"], wl["w_lo"], wl["w_hi"], t_final=2.0,
                           dt=0.01, m=200, seed=1, return_finals=True)
    assert np.all(finals >= lo - 1e-9) and np.all(finals <= hi + 1e-9)
    # and it is tighter than the global bound on this workload
    assert np.all(hi - lo <= ghi - glo + 1e-9) and np.sum(hi - lo) < 0.9 * np.sum(ghi - glo)


def test_traffic_local_capacity_box():
    # with capacity 20, densities in [105, 145] flow at capacity everywhere
    # (v x > 20 and w (xbar - x) > 20): every entry of C vanishes
    prm = (20.0, 0.5, 1.0 / 6.0, 320.0, 1.0)
    g = np.random.default_rng(8)
    c = g.uniform(110, 140, 9)
    r = g.uniform(0.5, 5, 9)
    dr = O.growth("traffic", c, r, [0.75], params=prm)
    want = np.zeros(9)
    want[0] = 0.75
    np.testing.assert_array_equal(dr, want)


# ------------------------------------------------------------------ outward rounding (reading R15)
from fractions import Fraction as Fr  # noqa: E402

TSP = O.TRAFFIC_SOUND_PRM


def _exact_traffic_rk4(x, d, h, N, prm, radius=False, hp=None):
    """Classic RK4 (R1) of the traffic chain (R6), or of its CGB radius
    dynamics C r + [p], in exact rational arithmetic."""
    cap, v, w, xbar = (Fr(p) for p in prm[:4])
    n = len(x)

    def f(y):
        if radius:
            return [(v * y[i - 1] if i > 0 else 0) + (w * y[i + 1] if i < n - 1 else 0) + (hp if i == 0 else 0)
                    for i in range(n)]
        flux = [min(cap, v * y[i], w * (xbar - y[i + 1])) if i < n - 1 else min(cap, v * y[i]) for i in range(n)]
        return [(d if i == 0 else flux[i - 1]) - flux[i] for i in range(n)]

    z = list(x)
    for _ in range(N):
        k1 = f(z)
        k2 = f([z[i] + h / 2 * k1[i] for i in range(n)])
        k3 = f([z[i] + h / 2 * k2[i] for i in range(n)])
        k4 = f([z[i] + h * k3[i] for i in range(n)])
        z = [z[i] + h / 6 * (k1[i] + 2 * k2[i] + 2 * k3[i] + k4[i]) for i in range(n)]
    return z


@pytest.mark.parametrize("seed", range(6))
def test_sound_boxes_contain_the_exact_arithmetic_result(seed):
    g = np.random.default_rng(40 + seed)
    n, N, dt = int(g.integers(3, 6)), int(g.integers(3, 7)), 0.05
    c = g.uniform(5, 315, n)
    hw = g.uniform(0, 8, n)
    lo, hi = c - hw, c + hw
    dl = float(g.uniform(20, 40))
    dh = dl + float(g.uniform(0, 10))
    T = N * dt
    h = Fr(dt)
    X0, X1 = [Fr(a) for a in lo], [Fr(a) for a in hi]
    # MM: two corner trajectories
    mlo, mhi = O.reach("mm", "traffic", lo, hi, [dl], [dh], t_final=T, dt=dt, params=TSP)
    elo = _exact_traffic_rk4(X0, Fr(dl), h, N, TSP)
    ehi = _exact_traffic_rk4(X1, Fr(dh), h, N, TSP)
    assert all(Fr(mlo[i]) <= elo[i] for i in range(n))
    assert all(Fr(mhi[i]) >= ehi[i] for i in range(n))
    # CGB: center and radius in exact arithmetic
    clo, chi = O.reach("cgb", "traffic", lo, hi, [dl], [dh], t_final=T, dt=dt, params=TSP)
    cc = _exact_traffic_rk4([(a + b) / 2 for a, b in zip(X0, X1)], (Fr(dl) + Fr(dh)) / 2, h, N, TSP)
    rr = _exact_traffic_rk4([(b - a) / 2 for a, b in zip(X0, X1)], None, h, N, TSP, radius=True,
                            hp=(Fr(dh) - Fr(dl)) / 2)
    assert all(Fr(clo[i]) <= cc[i] - rr[i] for i in range(n))
    assert all(Fr(chi[i]) >= cc[i] + rr[i] for i in range(n))


@pytest.mark.parametrize("method", ["mm", "cgb"])
def test_sound_boxes_contain_the_nearest_rounded_boxes(method):
    wl = W.traffic_small(16)
    args = (wl["x_lo"], wl["x_hi"], wl["w_lo"], wl["w_hi"])
    a = O.reach(method, "traffic", *args, t_final=10.0, dt=0.01)
    b = O.reach(method, "traffic", *args, t_final=10.0, dt=0.01, params=TSP)
    assert np.all(b[0] <= a[0]) and np.all(b[1] >= a[1])
    # the outward rounding costs a few ulps per step, nothing more
    scale = np.abs(a[1]).max()
    assert np.max(a[0] - b[0]) < 1e-11 * scale and np.max(b[1] - a[1]) < 1e-11 * scale
    assert np.max(a[0] - b[0]) > 0 and np.max(b[1] - a[1]) > 0


def _is_down(x, exact):
    return Fr(x) <= exact < Fr(np.nextafter(x, np.inf))


def _is_up(x, exact):
    return Fr(np.nextafter(x, -np.inf)) < exact <= Fr(x)


def test_sound_primitives_are_the_directed_roundings():
    g = np.random.default_rng(50)
    vals = np.concatenate([g.uniform(-1, 1, 60) * 10.0 ** g.integers(-8, 9, 60), [0.1, 1.0 / 3, 320.0, -40.0]])
    for a in vals[:32]:
        for b in vals[32:]:
            A, B = Fr(a), Fr(b)
            assert _is_down(O.sound_op("add_dn", a, b), A + B)
            assert _is_up(O.sound_op("add_up", a, b), A + B)
            assert _is_down(O.sound_op("mul_dn", a, b), A * B)
            assert _is_up(O.sound_op("mul_up", a, b), A * B)
            if b > 0:
                assert _is_down(O.sound_op("div_dn", a, b), A / B)
                assert _is_up(O.sound_op("div_up", a, b), A / B)


def test_sound_constant_interval_product():
    c = 0.01 / 6
    cl, cu = O.sound_op("div_dn", 0.01, 6.0), O.sound_op("div_up", 0.01, 6.0)
    assert Fr(cl) <= Fr(0.01) / 6 <= Fr(cu)
    for ql, qu in [(-3.7, 2.9), (0.3, 5.1), (-8.2, -1.3)]:
        rl, ru = O.sound_mul_pos(cl, cu, ql, qu)
        lo_exact = min(Fr(cl) * Fr(ql), Fr(cu) * Fr(ql))
        hi_exact = max(Fr(cl) * Fr(qu), Fr(cu) * Fr(qu))
        assert _is_down(rl, lo_exact) and _is_up(ru, hi_exact)
    del c


@pytest.mark.parametrize("regime", [(1.0, 60.0), (90.0, 200.0), (250.0, 319.0), (0.0, 320.0)])
def test_traffic_sound_rhs_encloses_the_exact_range(regime):
    g = np.random.default_rng(int(regime[0]) + 51)
    cap, v, w, xbar = (Fr(p) for p in TSP[:4])
    n = 7
    for _ in range(20):
        a, b = g.uniform(*regime, n), g.uniform(*regime, n)
        yl, yu = np.minimum(a, b), np.maximum(a, b)
        if _ == 0:
            yu = yl.copy()   # a point: the enclosure of one value
        dl = float(g.uniform(20, 40))
        du = dl + float(g.uniform(0, 5))
        kl, ku = O.traffic_sound_rhs(yl, yu, dl, du, params=TSP)
        L, U = [Fr(x) for x in yl], [Fr(x) for x in yu]
        fmin = [min(cap, v * L[i], w * (xbar - U[i + 1])) if i < n - 1 else min(cap, v * L[i]) for i in range(n)]
        fmax = [min(cap, v * U[i], w * (xbar - L[i + 1])) if i < n - 1 else min(cap, v * U[i]) for i in range(n)]
        for i in range(n):
            inl, inu = (Fr(dl), Fr(du)) if i == 0 else (fmin[i - 1], fmax[i - 1])
            emin, emax = inl - fmax[i], inu - fmin[i]
            assert Fr(kl[i]) <= emin and Fr(ku[i]) >= emax
            # and no looser than a few roundings of the operands (fluxes up to
            # cap, congestion terms up to w xbar)
            tol = Fr(8 * np.spacing(64.0))
            assert emin - Fr(kl[i]) <= tol and Fr(ku[i]) - emax <= tol


@pytest.mark.parametrize("v", [0.5, 0.45])
def test_traffic_sound_radius_rhs_is_an_upper_bound(v):
    g = np.random.default_rng(52)
    prm = (40.0, v, 1.0 / 6.0, 320.0, 0.0, 1.0)
    v, w = Fr(prm[1]), Fr(prm[2])
    for _ in range(30):
        n = 6
        r = g.uniform(0, 10, n) * 10.0 ** g.integers(-3, 3)
        hp = float(g.uniform(0, 5))
        dr = O.traffic_sound_radius_rhs(r, hp, params=prm)
        R_ = [Fr(x) for x in r]
        for i in range(n):
            e = (Fr(hp) if i == 0 else 0) + (v * R_[i - 1] if i > 0 else 0) + (w * R_[i + 1] if i < n - 1 else 0)
            assert Fr(dr[i]) >= e
            assert Fr(dr[i]) - e <= Fr(4 * np.spacing(float(e) if e > 0 else 1.0))


@pytest.mark.parametrize("method", ["mm", "cgb"])
def test_sound_zero_horizon_contains_the_box(method):
    # with no step the exact method returns the initial box itself: the
    # outward-rounded center and radius must reproduce it or contain it
    g = np.random.default_rng(53)
    for k in range(40):
        if k % 2:
            # hi - lo exact (Sterbenz) and lo + hi inexact half of the time: the
            # center's rounding alone decides the containment
            a, b = g.uniform(100, 120, 9), g.uniform(100, 120, 9)
            lo, hi = np.minimum(a, b), np.maximum(a, b)
        else:
            c = g.uniform(0, 320, 9)
            h = g.uniform(0, 10, 9) * 10.0 ** g.integers(-6, 1)
            lo, hi = c - h, c + h
        blo, bhi = O.reach(method, "traffic", lo, hi, [30.0], [40.0], t_final=0.0, dt=0.01, params=TSP)
        assert np.all(blo <= lo) and np.all(bhi >= hi)
