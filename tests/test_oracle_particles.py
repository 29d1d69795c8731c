"""Pins of the oracle's particle integrators (Secs. 3.2, 3.3, 5.3).

Closed forms of Eq. 3 in uniform flows (steady and linearly varying in
time), the printed transit-time table (Table 1), fourth-order convergence,
and conservation of the streamfunction along tracer paths in Taylor-Green.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2607_17836_b300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "uniform_transit_times.txt")


def uniform_fields(n, ux, uy):
    return np.full((n, n), float(ux)), np.full((n, n), float(uy))


def run_uniform(st, dt, t_end, x0=0.25, scheme=oracle.BILINEAR):
    n = 16
    u, v = uniform_fields(n, 1.0, 0.0)
    x, y = np.array([x0]), np.array([0.25])
    vx, vy = np.zeros(1), np.zeros(1)
    for _ in range(int(round(t_end / dt))):
        oracle.particles_rk4(scheme, dt, st, u, v, u, v, x, y, vx, vy)
    return x[0], y[0], vx[0], vy[0]


@pytest.mark.parametrize("st", [0.1, 1.0, 10.0])
@pytest.mark.parametrize("scheme", [0, 1, 2])
def test_uniform_flow_closed_form(st, scheme):
    # Eq. 28: v = 1 - exp(-t/St), x = x0 + t - St (1 - exp(-t/St)).
    t = 1.0
    x, y, vx, vy = run_uniform(st, 1e-3, t, scheme=scheme)
    assert abs(vx - (1 - math.exp(-t / st))) < 1e-10
    assert abs(x - (0.25 + t - st * (1 - math.exp(-t / st)))) < 1e-10
    assert y == 0.25 and vy == 0.0


def test_transit_time_table():
    # Time to go from x = 0.25 to x = 0.5 from rest (Table 1), dt = 1e-3 as in
    # the paper, crossing located by linear interpolation between steps.
    rows = np.loadtxt(GOLDEN)
    n, dt = 16, 1e-3
    u, v = uniform_fields(n, 1.0, 0.0)
    for st, t_ref in rows:
        x, y, vx, vy = np.array([0.25]), np.array([0.25]), np.zeros(1), np.zeros(1)
        t, xprev = 0.0, 0.25
        while x[0] < 0.5:
            xprev = x[0]
            oracle.particles_rk4(0, dt, st, u, v, u, v, x, y, vx, vy)
            t += dt
        t_cross = t - dt * (x[0] - 0.5) / (x[0] - xprev)
        assert abs(t_cross - t_ref) <= 5e-4 + 1e-6, (st, t_cross, t_ref)


def test_linearly_varying_flow_uses_theta_in_the_right_direction():
    # u(t) = a + c t between snapshots (exact under linear time blending):
    # v = a + c t - c St + (v0 - a + c St) e^{-t/St},
    # x = x0 + a t + c t^2/2 - c St t + (v0 - a + c St) St (1 - e^{-t/St}).
    n, dt, st, a, c = 16, 1e-2, 0.3, 0.5, 2.0
    x, y, vx, vy = np.array([1.0]), np.array([2.0]), np.zeros(1), np.zeros(1)
    steps = 100
    for k in range(steps):
        un, vn = uniform_fields(n, a + c * k * dt, 0.0)
        un1, vn1 = uniform_fields(n, a + c * (k + 1) * dt, 0.0)
        oracle.particles_rk4(0, dt, st, un, vn, un1, vn1, x, y, vx, vy)
    t = steps * dt
    A = -a + c * st
    v_ex = a + c * t - c * st + A * math.exp(-t / st)
    x_ex = 1.0 + a * t + 0.5 * c * t * t - c * st * t + A * st * (1 - math.exp(-t / st))
    assert abs(vx[0] - v_ex) < 1e-8 and abs(x[0] - x_ex) < 1e-8
    # tracers in the same flow move by the exact integral of u(t)
    xt, yt = np.array([1.0]), np.array([2.0])
    for k in range(steps):
        un, vn = uniform_fields(n, a + c * k * dt, 0.0)
        un1, vn1 = uniform_fields(n, a + c * (k + 1) * dt, 0.0)
        oracle.particles_rk4(0, dt, 0.0, un, vn, un1, vn1, xt, yt)
    assert abs(xt[0] - (1.0 + a * t + 0.5 * c * t * t)) < 1e-12


def test_rk4_is_fourth_order():
    st, t = 0.5, 1.0
    exact = 0.25 + t - st * (1 - math.exp(-t / st))
    errs = [abs(run_uniform(st, dt, t)[0] - exact) for dt in (0.1, 0.05, 0.025)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - 4) < 0.3), rates


@pytest.mark.parametrize("scheme,tol", [(oracle.CATMULL_ROM, 2e-4), (oracle.BSPLINE, 2e-5)])
def test_tracers_conserve_streamfunction_in_taylor_green(scheme, tol):
    # Steady TG u = sin x cos y, v = -cos x sin y has psi = sin x sin y
    # constant along paths; the residual drift is interpolation error.
    n = 64
    X, Y = inputs.grid(n)
    u, v = np.sin(X) * np.cos(Y), -np.cos(X) * np.sin(Y)
    if scheme == oracle.BSPLINE:
        u, v = oracle.bspline_prefilter(u), oracle.bspline_prefilter(v)
    xy = inputs.uniform_positions(256, seed=21)
    x, y = xy[:, 0].copy(), xy[:, 1].copy()
    psi0 = np.sin(x) * np.sin(y)
    for _ in range(200):
        oracle.particles_rk4(scheme, 1e-2, 0.0, u, v, u, v, x, y)
    assert np.max(np.abs(np.sin(x) * np.sin(y) - psi0)) < tol


def test_coupled_taylor_green_tracers_conserve_streamfunction():
    # Decaying TG keeps its shape, so tracers stay on their streamlines.
    wl = inputs.taylor_green_64()
    c = oracle.Coupled(wl.n, wl.nu, wl.dt, wl.omega0(), scheme=oracle.BILINEAR)
    xy = inputs.uniform_positions(4096, seed=1)
    c.add_species(xy, 0.0)
    psi0 = np.sin(xy[:, 0]) * np.sin(xy[:, 1])
    c.step(wl.steps)
    s = c.species[0]
    assert np.max(np.abs(np.sin(s.x) * np.sin(s.y) - psi0)) < 2e-4
    st = c.stats()
    assert abs(st["energy"] - 0.25 * math.exp(-4 * wl.nu * wl.dt * wl.steps)) < 1e-12
    assert st["msd"][0][0] > 0 and st["step"] == wl.steps


def test_zero_slip_start_and_small_stokes_limit():
    # A species with vxy=None starts at the interpolated fluid velocity; as
    # St -> 0 inertial paths approach tracer paths (Sec. 3.3).
    wl = inputs.taylor_green_64()
    c = oracle.Coupled(wl.n, wl.nu, wl.dt, wl.omega0(), scheme=oracle.CATMULL_ROM)
    xy = inputs.uniform_positions(64, seed=2)
    c.add_species(xy, 0.0)
    c.add_species(xy, 1e-3)
    u = c._level[0]
    np.testing.assert_allclose(c.species[1].vx, oracle.interp(u, 1, xy[:, 0], xy[:, 1]), atol=0)
    c.step(100)
    d = np.hypot(c.species[0].x - c.species[1].x, c.species[0].y - c.species[1].y)
    assert d.max() < 1e-4


def test_cluster_index_of_uniform_points_is_near_zero():
    xy = inputs.uniform_positions(400_000, seed=3)
    assert abs(oracle.cluster_index(xy[:, 0], xy[:, 1])) < 0.1
    # all P particles in one of B boxes: mean P/B, Var = P^2 (B-1)/B^2,
    # so Var/mean - 1 = P (B-1)/B - 1
    x = np.full(1000, 0.01)
    assert abs(oracle.cluster_index(x, x) - (1000 * 4095 / 4096 - 1)) < 1e-9
    # exactly k particles at every box centre: Var = 0, so the index is -1;
    # shifting some by whole periods (2 pi m) must not move them between boxes
    B, k = 64, 3
    c = (np.arange(B) + 0.5) * (2 * np.pi / B)
    X, Y = np.meshgrid(c, c)
    xs = np.tile(X.ravel(), k) + 2 * np.pi * np.repeat([0, -3, 5], B * B)
    ys = np.tile(Y.ravel(), k) + 2 * np.pi * np.repeat([2, 0, -1], B * B)
    assert oracle.cluster_index(xs, ys) == pytest.approx(-1.0, abs=1e-12)


@pytest.mark.parametrize("scheme,tol", [(oracle.CATMULL_ROM, 5e-5), (oracle.BSPLINE, 2e-6)])
def test_streamfunction_velocity_is_the_centred_difference(scheme, tol):
    # Eq. 11 on psi = sin x sin y: centred differences of width 2 dx give
    # u = sin x cos y * sin(dx)/dx and v = -cos x sin y * sin(dx)/dx exactly,
    # so the oracle must reproduce the sinc factor (1 - dx^2/6), not the
    # analytic velocity: this pins the formula's axes, sign and width.
    n = 64
    X, Y = inputs.grid(n)
    psi = np.sin(X) * np.sin(Y)
    if scheme == oracle.BSPLINE:
        psi = oracle.bspline_prefilter(psi)
    xy = inputs.uniform_positions(500, seed=31)
    u, v = oracle.psi_velocity(psi, scheme, xy[:, 0], xy[:, 1])
    d = 2 * np.pi / n
    sinc = np.sin(d) / d
    np.testing.assert_allclose(u, np.sin(xy[:, 0]) * np.cos(xy[:, 1]) * sinc, atol=tol)
    np.testing.assert_allclose(v, -np.cos(xy[:, 0]) * np.sin(xy[:, 1]) * sinc, atol=tol)
    # ... and the sinc factor is resolved: the plain analytic velocity is off
    assert np.max(np.abs(u - np.sin(xy[:, 0]) * np.cos(xy[:, 1]))) > 10 * tol


def test_streamfunction_and_velocity_tracers_agree_short_time():
    # Both tracer paths follow the same flow; they differ by O(dx^2).
    wl = inputs.taylor_green_64()
    a = oracle.Coupled(wl.n, wl.nu, wl.dt, wl.omega0(), scheme=oracle.BSPLINE)
    b = oracle.Coupled(wl.n, wl.nu, wl.dt, wl.omega0(), scheme=oracle.BSPLINE, tracer_velocity=1)
    xy = inputs.uniform_positions(256, seed=32)
    a.add_species(xy, 0.0)
    b.add_species(xy, 0.0)
    a.step(100)
    b.step(100)
    d = np.hypot(a.species[0].x - b.species[0].x, a.species[0].y - b.species[0].y)
    assert 1e-6 < d.max() < 1e-3   # paths differ, by O(dx^2) of the distance travelled


def test_msd_standard_error_against_the_statistics_module_and_closed_forms():
    import statistics
    rng = np.random.default_rng(11)
    x0, y0 = rng.uniform(0, 6, 257), rng.uniform(0, 6, 257)
    x, y = x0 + rng.normal(0, 0.7, 257), y0 + rng.normal(0, 1.3, 257)
    sx, sy = oracle.msd_sem(x, y, x0, y0)
    for got, d in ((sx, x - x0), (sy, y - y0)):
        q = [float(v) * float(v) for v in d]
        assert got == pytest.approx(statistics.stdev(q) / np.sqrt(len(q)), rel=1e-12)
    # every particle displaced alike: no spread (up to the rounding of x0 + d - x0)
    assert oracle.msd_sem(x0 + 0.4, y0 - 2.0, x0, y0) == pytest.approx((0.0, 0.0), abs=1e-15)
    # half displaced by a, half not: squared displacements a^2 and 0,
    # sample variance n a^4 / (4 (n - 1)), standard error a^2 / (2 sqrt(n - 1))
    n, a = 100, 0.3
    xs = np.zeros(n)
    xs[: n // 2] = a
    sx, sy = oracle.msd_sem(xs, np.zeros(n), np.zeros(n), np.zeros(n))
    assert sx == pytest.approx(a * a / (2.0 * np.sqrt(n - 1)), rel=1e-12) and sy == 0.0
    assert oracle.msd_sem([1.0], [2.0], [0.0], [0.0]) == (0.0, 0.0)


def test_diffusivity_of_ballistic_motion():
    # x = x0 + U t: msd = U^2 t^2, so D = U^2 t / 2
    t, ux, uy = 3.5, 0.2, -1.1
    x0 = np.linspace(0, 1, 50)
    m = oracle.msd(x0 + ux * t, x0 + uy * t, x0, x0)
    dxy = oracle.diffusivity(m, t)
    assert dxy[0] == pytest.approx(ux * ux * t / 2, rel=1e-12)
    assert dxy[1] == pytest.approx(uy * uy * t / 2, rel=1e-12)
    assert oracle.diffusivity(m, 0.0) == (0.0, 0.0)
