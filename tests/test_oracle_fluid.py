"""Pins of the oracle's pseudospectral AB2 vorticity solver (Sec. 3.1).

Each check comes from outside the oracle: closed-form solutions, analytic
derivatives of chosen fields, exact invariants of the Galerkin-truncated
system, and the input generator's own energy normalisation.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2607_17836_b300 import inputs


def grid(n):
    return inputs.grid(n)


def test_taylor_green_closed_form_integrating_factor():
    # omega = 2 sin x sin y has a zero nonlinear term, so the viscous
    # integrating factor makes every step exact: omega(t) = 2 exp(-2 nu t) sin x sin y.
    n, nu, dt, steps = 32, 0.01, 1e-3, 200
    X, Y = grid(n)
    f = oracle.Flow(n, nu, dt, inputs.taylor_green(n), ab2_mode=0)
    assert np.max(np.abs(f.nonlinear())) < 1e-12
    f.step(steps)
    w = f.fields(("w",))["w"]
    exact = 2 * math.exp(-2 * nu * dt * steps) * np.sin(X) * np.sin(Y)
    assert np.max(np.abs(w - exact)) < 1e-12


def test_taylor_green_explicit_ab2_is_second_order():
    # Paper's Eq. 10 with the viscous term inside R: O(dt^2) against the closed form.
    n, nu, T = 16, 0.5, 1.0
    X, Y = grid(n)
    errs = []
    for dt in (0.02, 0.01, 0.005):
        f = oracle.Flow(n, nu, dt, inputs.taylor_green(n), ab2_mode=1)
        f.step(int(round(T / dt)))
        w = f.fields(("w",))["w"]
        errs.append(np.max(np.abs(w - 2 * math.exp(-2 * nu * T) * np.sin(X) * np.sin(Y))))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.5 < r2 < 4.5, errs


def test_taylor_green_diagnostics_closed_form():
    # u = sin x cos y, v = -cos x sin y: E = 1/4, Z = 1/2, P = 1.
    f = oracle.Flow(32, 0.0, 1e-3, inputs.taylor_green(32))
    e, z, p = f.diagnostics()
    assert abs(e - 0.25) < 1e-13 and abs(z - 0.5) < 1e-13 and abs(p - 1.0) < 1e-13


def test_velocity_and_bracket_against_analytic_field():
    # omega = sin x + cos 2y  ->  psi = sin x + cos(2y)/4 (omega = -lap psi),
    # u = psi_y, v = -psi_x (Eq. 2); Eq. 1 bracket [psi, omega] = psi_x w_y - psi_y w_x.
    n = 32
    X, Y = grid(n)
    w0 = np.sin(X) + np.cos(2 * Y)
    f = oracle.Flow(n, 0.0, 1e-3, w0)
    fl = f.fields(("u", "v", "w"))
    psi_x, psi_y = np.cos(X), -0.5 * np.sin(2 * Y)
    w_x, w_y = np.cos(X), -2 * np.sin(2 * Y)
    np.testing.assert_allclose(fl["u"], psi_y, atol=1e-13)
    np.testing.assert_allclose(fl["v"], -psi_x, atol=1e-13)
    np.testing.assert_allclose(fl["w"], w0, atol=1e-13)
    bracket = psi_x * w_y - psi_y * w_x
    # the oracle's nonlinear term N = u w_x + v w_y enters as d omega/dt = -N
    np.testing.assert_allclose(-f.nonlinear(), bracket, atol=1e-12)


@pytest.mark.parametrize("mode", [0, 1])
def test_first_step_follows_vorticity_equation(mode):
    # Forward difference of one tiny step against the right-hand side of Eq. 1.
    n, nu, dt = 32, 0.05, 1e-7
    X, Y = grid(n)
    w0 = np.sin(X) + np.cos(2 * Y)
    f = oracle.Flow(n, nu, dt, w0, ab2_mode=mode)
    f.step(1)
    w1 = f.fields(("w",))["w"]
    psi_x, psi_y = np.cos(X), -0.5 * np.sin(2 * Y)
    w_x, w_y = np.cos(X), -2 * np.sin(2 * Y)
    lap_w = -np.sin(X) - 4 * np.cos(2 * Y)
    rhs = psi_x * w_y - psi_y * w_x + nu * lap_w
    np.testing.assert_allclose((w1 - w0) / dt, rhs, atol=2e-6)


def test_two_thirds_mask_and_mean_removal():
    # n = 64: modes with |k| <= 21 survive the initial projection, |k| = 22 does not.
    n = 64
    X, Y = grid(n)
    keep = np.cos(21 * X) + np.sin(21 * Y) + np.cos(5 * X + 21 * Y)
    drop = np.cos(22 * X) + np.sin(22 * Y) + np.cos(3 * X + 22 * Y) + 0.7
    f = oracle.Flow(n, 0.0, 1e-3, keep + drop)
    np.testing.assert_allclose(f.fields(("w",))["w"], keep, atol=1e-12)


def test_generator_energy_is_unit():
    # The input generator normalises its field with its own numpy FFT to unit
    # kinetic energy over the (2 pi)^2 domain; the oracle reports the mean.
    w0 = inputs.decaying_turbulence(64, seed=11, k0=4.0)
    e, _, _ = oracle.Flow(64, 0.0, 1e-3, w0).diagnostics()
    assert abs(e * (2 * np.pi) ** 2 - 1.0) < 1e-12


def test_inviscid_invariants_conserved():
    # The 2/3-truncated system conserves E and Z exactly in continuous time,
    # so with nu = 0 the only drift is AB2's own O(dt^2) error: halving dt
    # over the same time must cut it fourfold.  (A non-conservative nonlinear
    # term would leave an O(1) drift that does not shrink with dt.)
    w0 = inputs.decaying_turbulence(64, seed=12, k0=4.0)
    drift = []
    for dt in (2e-3, 1e-3, 5e-4):
        f = oracle.Flow(64, 0.0, dt, w0)
        e0, z0, _ = f.diagnostics()
        f.step(int(round(0.1 / dt)))
        e1, z1, _ = f.diagnostics()
        drift.append((abs(e1 - e0) / e0, abs(z1 - z0) / z0))
    d = np.array(drift)
    assert np.all(d[0] < 1e-4)
    ratios = d[:-1] / d[1:]
    assert np.all((ratios > 3.6) & (ratios < 4.4)), ratios


@pytest.mark.parametrize("mode", [0, 1])
def test_energy_and_enstrophy_budgets(mode):
    # dE/dt = -2 nu Z and dZ/dt = -2 nu P, integrated by the trapezoid rule;
    # the residual is the time discretisation's, so it is O(dt^2): a dropped
    # or misweighted viscous term would leave an O(1) residual instead.
    nu, T = 0.02, 0.06
    w0 = inputs.decaying_turbulence(64, seed=13, k0=4.0)
    res = []
    for dt in (2e-3, 1e-3, 5e-4):
        f = oracle.Flow(64, nu, dt, w0, ab2_mode=mode)
        hist = [f.diagnostics()]
        for _ in range(int(round(T / dt))):
            f.step(1)
            hist.append(f.diagnostics())
        h = np.array(hist)
        dE, dZ = h[-1, 0] - h[0, 0], h[-1, 1] - h[0, 1]
        intZ = dt * (h[1:-1, 1].sum() + 0.5 * (h[0, 1] + h[-1, 1]))
        intP = dt * (h[1:-1, 2].sum() + 0.5 * (h[0, 2] + h[-1, 2]))
        res.append((abs(dE + 2 * nu * intZ) / abs(dE), abs(dZ + 2 * nu * intP) / abs(dZ)))
    r = np.array(res)
    assert np.all(r[0] < 1e-3)
    ratios = r[:-1] / r[1:]
    assert np.all((ratios > 3.6) & (ratios < 4.4)), ratios
