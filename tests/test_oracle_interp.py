"""Pins of the oracle's interpolants (Sec. 3.4, Eqs. 15-22).

Independent routes: polynomial reproduction, the cubic-Hermite definition of
Catmull-Rom (central-difference tangents), the Cox-de Boor recursion for the
uniform cubic B-spline, the prefilter's defining three-point relation, and
convergence orders on a smooth field.
"""
import numpy as np
import pytest

import oracle

TWO_PI = 2 * np.pi


def interior_points(n, count, margin, seed):
    # Points whose whole stencil stays inside [0, n-1] without wrapping (grid units).
    rng = np.random.default_rng(seed)
    return rng.uniform(margin, n - 1 - margin, size=(count, 2))


def at(n, f, scheme, pts_grid):
    dx = TWO_PI / n
    return oracle.interp(f, scheme, pts_grid[:, 0] * dx, pts_grid[:, 1] * dx)


def node_values(n, fun):
    g = np.arange(n, dtype=float)
    X, Y = np.meshgrid(g, g, indexing="xy")
    return fun(X, Y)


def test_bilinear_reproduces_bilinear_polynomials():
    n = 16
    fun = lambda x, y: 1.0 + 2.0 * x - 3.0 * y + 0.5 * x * y
    pts = interior_points(n, 500, 0.0, 1)
    pts[:5] = [[3, 4], [3.5, 4], [3, 4.25], [0, 0], [7.75, 2.5]]
    np.testing.assert_allclose(at(n, node_values(n, fun), oracle.BILINEAR, pts),
                               fun(pts[:, 0], pts[:, 1]), atol=1e-12)


def test_catmull_rom_reproduces_quadratics_not_cubics():
    n = 16
    quad = lambda x, y: (1 + 0.3 * x - 0.2 * x * x) * (2 - 0.5 * y + 0.1 * y * y)
    pts = interior_points(n, 500, 1.0, 2)
    np.testing.assert_allclose(at(n, node_values(n, quad), oracle.CATMULL_ROM, pts),
                               quad(pts[:, 0], pts[:, 1]), atol=1e-11)
    cubic = lambda x, y: x ** 3
    err = np.abs(at(n, node_values(n, cubic), oracle.CATMULL_ROM, pts) - pts[:, 0] ** 3)
    assert err.max() > 1e-2


def hermite_central(pm1, p0, p1, p2, s):
    # Cubic Hermite segment with central-difference tangents (Catmull-Rom).
    m0, m1 = 0.5 * (p1 - pm1), 0.5 * (p2 - p0)
    h00, h10 = 2 * s ** 3 - 3 * s ** 2 + 1, s ** 3 - 2 * s ** 2 + s
    h01, h11 = -2 * s ** 3 + 3 * s ** 2, s ** 3 - s ** 2
    return h00 * p0 + h10 * m0 + h01 * p1 + h11 * m1


def test_catmull_rom_equals_tensor_cubic_hermite_with_wrap():
    n = 8
    rng = np.random.default_rng(3)
    f = rng.standard_normal((n, n))
    pts = rng.uniform(-3 * n, 4 * n, size=(300, 2))   # includes wrapped and negative points
    got = at(n, f, oracle.CATMULL_ROM, pts)
    for (x, y), g in zip(pts, got):
        i, j = int(np.floor(x)), int(np.floor(y))
        s, t = x - i, y - j
        rows = []
        for b in range(-1, 3):
            r = [f[(j + b) % n, (i + a) % n] for a in range(-1, 3)]
            rows.append(hermite_central(*r, s))
        assert abs(hermite_central(*rows, t) - g) < 1e-12


def cox_de_boor(k, p, x):
    # B-spline basis N_{k,p}(x) on the integer knots k, k+1, ..., k+p+1.
    if p == 0:
        return 1.0 if k <= x < k + 1 else 0.0
    return ((x - k) / p) * cox_de_boor(k, p - 1, x) + ((k + p + 1 - x) / p) * cox_de_boor(k + 1, p - 1, x)


def test_raw_bspline_equals_cox_de_boor_cubic():
    # Raw samples as B-spline coefficients: f(x) = sum_k c_k beta3(x - k),
    # beta3(x) = N_{-2,3}(x) is the centred cubic B-spline.
    n = 8
    rng = np.random.default_rng(4)
    c = rng.standard_normal((n, n))
    pts = rng.uniform(0, n, size=(200, 2))
    got = at(n, c, oracle.BSPLINE, pts)
    for (x, y), g in zip(pts, got):
        i, j = int(np.floor(x)), int(np.floor(y))
        ref = 0.0
        for b in range(-1, 3):
            for a in range(-1, 3):
                wx = cox_de_boor(-2, 3, x - (i + a))
                wy = cox_de_boor(-2, 3, y - (j + b))
                ref += wx * wy * c[(j + b) % n, (i + a) % n]
        assert abs(ref - g) < 1e-12


def test_raw_bspline_smooths_cubics_by_second_derivative():
    # Approximating spline: for a cubic p, sum_k p(k) beta3(x - k) = p(x) + p''(x)/6.
    n = 16
    p = lambda x, y: 0.01 * x ** 3 - 0.1 * x * x + x + 0.02 * y ** 3
    pxx_plus_pyy = lambda x, y: 0.06 * x - 0.2 + 0.12 * y
    pts = interior_points(n, 300, 1.0, 5)
    got = at(n, node_values(n, p), oracle.BSPLINE, pts)
    np.testing.assert_allclose(got, p(pts[:, 0], pts[:, 1]) + pxx_plus_pyy(pts[:, 0], pts[:, 1]) / 6,
                               atol=1e-11)


def test_prefilter_solves_three_point_relation_and_interpolates():
    n = 32
    rng = np.random.default_rng(6)
    f = rng.standard_normal((n, n))
    c = oracle.bspline_prefilter(f)
    sx = (np.roll(c, 1, axis=1) + 4 * c + np.roll(c, -1, axis=1)) / 6
    sxy = (np.roll(sx, 1, axis=0) + 4 * sx + np.roll(sx, -1, axis=0)) / 6
    np.testing.assert_allclose(sxy, f, atol=1e-12)
    g = np.arange(n, dtype=float)
    X, Y = np.meshgrid(g, g, indexing="xy")
    pts = np.stack([X.ravel(), Y.ravel()], axis=1)
    np.testing.assert_allclose(at(n, c, oracle.BSPLINE, pts), f.ravel(), atol=1e-12)


@pytest.mark.parametrize("scheme", [oracle.BILINEAR, oracle.CATMULL_ROM, oracle.BSPLINE])
def test_interpolants_return_node_values(scheme):
    n = 16
    rng = np.random.default_rng(7)
    f = rng.standard_normal((n, n))
    stencil = oracle.bspline_prefilter(f) if scheme == oracle.BSPLINE else f
    g = np.arange(n, dtype=float)
    X, Y = np.meshgrid(g, g, indexing="xy")
    pts = np.stack([X.ravel(), Y.ravel()], axis=1)
    np.testing.assert_allclose(at(n, stencil, scheme, pts), f.ravel(), atol=1e-12)


@pytest.mark.parametrize("scheme,order", [(oracle.BILINEAR, 2), (oracle.CATMULL_ROM, 3),
                                          (oracle.BSPLINE, 4)])
def test_convergence_order_on_smooth_field(scheme, order):
    fun = lambda x, y: np.sin(x) * np.sin(2 * y) + np.cos(3 * x + y)
    rng = np.random.default_rng(8)
    xy = rng.uniform(0, TWO_PI, size=(4000, 2))
    errs = []
    for n in (32, 64, 128):
        X, Y = np.meshgrid(np.arange(n) * TWO_PI / n, np.arange(n) * TWO_PI / n, indexing="xy")
        f = fun(X, Y)
        if scheme == oracle.BSPLINE:
            f = oracle.bspline_prefilter(f)
        got = oracle.interp(f, scheme, xy[:, 0], xy[:, 1])
        errs.append(np.max(np.abs(got - fun(xy[:, 0], xy[:, 1]))))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - order) < 0.35), rates


def test_periodic_images_give_the_same_value():
    n = 16
    rng = np.random.default_rng(9)
    f = rng.standard_normal((n, n))
    xy = rng.uniform(0, TWO_PI, size=(50, 2))
    for scheme in (0, 1, 2):
        a = oracle.interp(f, scheme, xy[:, 0], xy[:, 1])
        b = oracle.interp(f, scheme, xy[:, 0] - 3 * TWO_PI, xy[:, 1] + 5 * TWO_PI)
        np.testing.assert_allclose(a, b, atol=1e-11)
