"""Pins of the oracle's kinematic flow (Sec. 5.2) against what the
mathematics fixes: the velocity is the curl of the streamfunction
(checked by spectral differentiation of the grid field), the steady cellular
limit conserves the streamfunction along tracer paths, the analytic RK4 is
fourth order, and the early mean-square displacement is ballistic with
<|u|^2> = alpha^2 / 2."""
import numpy as np
import pytest

import oracle
from paper_2607_17836_b300 import inputs

PAPER = dict(alpha=3.6 * np.pi, k=1.0, eps=0.6 * np.pi, omega=1.8, phi=0.0)


def spectral_d(f, axis):
    n = f.shape[0]
    k = np.fft.fftfreq(n, d=1.0 / n)
    fh = np.fft.fft(f, axis=axis)
    shape = [1, 1]
    shape[axis] = n
    return np.real(np.fft.ifft(1j * k.reshape(shape) * fh, axis=axis))


@pytest.mark.parametrize("params", [PAPER, dict(alpha=1.3, k=3.0, eps=0.4, omega=2.5, phi=0.7)])
def test_velocity_is_the_curl_of_the_streamfunction(params):
    n, t = 64, 0.37
    f = oracle.kinematic_fields(n, t, **params)
    # arrays are [j][i]: axis 1 is x, axis 0 is y
    scale = np.max(np.abs(f["u"]))
    np.testing.assert_allclose(spectral_d(f["psi"], 0), f["u"], atol=1e-12 * scale)
    np.testing.assert_allclose(-spectral_d(f["psi"], 1), f["v"], atol=1e-12 * scale)
    div = spectral_d(f["u"], 1) + spectral_d(f["v"], 0)
    assert np.max(np.abs(div)) < 1e-11 * scale
    lap = spectral_d(spectral_d(f["psi"], 1), 1) + spectral_d(spectral_d(f["psi"], 0), 0)
    np.testing.assert_allclose(-lap, f["omega"], atol=1e-11 * np.max(np.abs(f["omega"])))
    # the point evaluation agrees with the grid field at the nodes
    xs = np.arange(n) * (2 * np.pi / n)
    x, y = np.meshgrid(xs, xs)
    u, v = oracle.kinematic_velocity(x, y, t, **params)
    np.testing.assert_array_equal(u, f["u"])
    np.testing.assert_array_equal(v, f["v"])


def test_steady_cells_conserve_the_streamfunction_along_paths():
    p = dict(PAPER, eps=0.0)
    xy = inputs.uniform_positions(500, 3)
    x, y = xy[:, 0].copy(), xy[:, 1].copy()
    psi = lambda a, b: (p["alpha"] / p["k"]) * np.sin(p["k"] * a) * np.sin(p["k"] * b)
    p0 = psi(x, y)
    for s in range(2000):
        x, y = oracle.tracers_rk4_analytic(1e-3, s * 1e-3, x, y, **p)
    assert np.max(np.abs(psi(x, y) - p0)) < 1e-9 * p["alpha"]


def test_analytic_rk4_is_fourth_order():
    xy = inputs.uniform_positions(64, 4)
    t_end = 0.5

    def run(dt):
        x, y = xy[:, 0].copy(), xy[:, 1].copy()
        for s in range(int(round(t_end / dt))):
            x, y = oracle.tracers_rk4_analytic(dt, s * dt, x, y, **PAPER)
        return x, y

    ref = run(0.0003125)
    errs = []
    for dt in (0.01, 0.005, 0.0025):
        x, y = run(dt)
        errs.append(np.max(np.hypot(x - ref[0], y - ref[1])))
    for a, b in zip(errs, errs[1:]):
        assert 12.0 < a / b < 20.0, errs


def test_early_mean_square_displacement_is_ballistic():
    # MSD(t) / t^2 -> <|u|^2> = alpha^2 / 2 over uniformly placed tracers
    xy = inputs.uniform_positions(40000, 5)
    dt = 1e-4
    x, y = oracle.tracers_rk4_analytic(dt, 0.0, xy[:, 0].copy(), xy[:, 1].copy(), **PAPER)
    m = oracle.msd(x, y, xy[:, 0], xy[:, 1])
    assert (m[0] + m[1]) / dt ** 2 == pytest.approx(PAPER["alpha"] ** 2 / 2, rel=0.03)


def test_the_three_routes_agree_for_a_short_time():
    xy = inputs.uniform_positions(200, 6)
    runs = [oracle.KinematicRun(128, 1e-3, PAPER, xy, ap) for ap in ("analytic", "velocity", "psi")]
    for r in runs:
        r.step(200)
    for r in runs[1:]:
        # interpolation error of order dx^2 per unit time over t = 0.2
        assert np.max(np.hypot(r.x - runs[0].x, r.y - runs[0].y)) < 5e-3
