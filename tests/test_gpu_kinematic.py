"""The kinematic tracer benchmark of Sec. 5.2 through the C ABI
(el_create_kinematic): the prescribed oscillating Taylor-Green field on the
grid and in the statistics, tracer parity with the FP64 oracle for the three
routes (the field at the particle, the interpolated velocity, the
interpolated streamfunction) and every interpolant, and the paper's finding
that the three routes give the same mean-square displacement (here: within
three combined standard errors)."""
import numpy as np
import pytest

import oracle
from paper_2607_17836_b300 import elpath, inputs
from parity import POS_ATOL

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# the paper's configuration with its 2 km domain mapped onto [0, 2 pi):
# lengths and speeds scale by pi (k = 1, alpha = 3.6 pi, eps = 0.3 L = 0.6 pi)
PAPER = dict(alpha=3.6 * np.pi, k=1.0, eps=0.6 * np.pi, omega=1.8, phi=0.0)
N, DT = 128, 1e-3


def kin_flow(interp, tracer_velocity=0, params=PAPER, np_=1000, n=N, prefilter=True):
    g = elpath.Flow(n, 0.0, DT, None, interp=interp, max_species=1, max_particles=np_,
                    tracer_velocity=tracer_velocity, kinematic=params, sort_every=25,
                    bspline_prefilter=prefilter)
    return g


ROUTES = [("analytic", elpath.ANALYTIC, 0, 0), ("velocity", 0, 0, 0), ("velocity", 1, 0, 1),
          ("velocity", 2, 0, 2), ("psi", 0, 1, 0), ("psi", 1, 1, 1), ("psi", 2, 1, 2)]


@pytest.mark.parametrize("route", ROUTES, ids=[f"{r[0]}-{r[3]}" for r in ROUTES])
def test_tracers_match_the_oracle(route):
    approach, interp, tv, scheme = route
    xy = inputs.uniform_positions(1000, 17)
    g = kin_flow(interp, tv)
    g.set_particles(0, xy, 0.0)
    g.step(300)
    ref = oracle.KinematicRun(N, DT, PAPER, xy, approach, scheme=scheme)
    ref.step(300)
    got, _ = g.particles(0, 1000)
    err = np.max(np.hypot(got[:, 0] - ref.x, got[:, 1] - ref.y))
    assert err <= POS_ATOL, err
    g.close()


@pytest.mark.parametrize("interp", [0, 2])
def test_fields_and_exact_statistics(interp):
    g = kin_flow(interp, np_=1)
    g.step(37)
    t = 37 * DT
    f = oracle.kinematic_fields(N, t, **PAPER)
    for which, key in ((0, "omega"), (1, "u"), (2, "v")):
        np.testing.assert_allclose(g.field(which), f[key], rtol=0,
                                   atol=1e-12 * np.max(np.abs(f[key])))
    # the particle stencil's node values: the field itself, or for the
    # prefiltered B-spline its interpolating spline coefficients (the oracle
    # solves the cyclic system in physical space)
    for which, key in ((3, "u"), (4, "v")):
        ref = oracle.bspline_prefilter(f[key]) if interp == 2 else f[key]
        np.testing.assert_allclose(g.field(which), ref, rtol=0, atol=3e-6 * np.max(np.abs(ref)))
    s = g.stats()
    k = np.fft.fftfreq(N, d=1.0 / N)
    wh = np.fft.fft2(f["omega"])
    gx = np.real(np.fft.ifft2(1j * k[None, :] * wh))
    gy = np.real(np.fft.ifft2(1j * k[:, None] * wh))
    assert s["energy"] == pytest.approx(0.5 * np.mean(f["u"] ** 2 + f["v"] ** 2), rel=1e-12)
    assert s["enstrophy"] == pytest.approx(0.5 * np.mean(f["omega"] ** 2), rel=1e-12)
    assert s["palinstrophy"] == pytest.approx(0.5 * np.mean(gx ** 2 + gy ** 2), rel=1e-10)
    g.close()


def test_three_routes_give_the_same_dispersion():
    xy = inputs.uniform_positions(1000, 7)
    flows = {"analytic": kin_flow(elpath.ANALYTIC), "velocity": kin_flow(0),
             "psi": kin_flow(0, tracer_velocity=1)}
    for g in flows.values():
        g.set_particles(0, xy, 0.0)
    worst = 0.0
    for _ in range(4):
        st = {}
        for name, g in flows.items():
            g.step(5000)
            st[name] = g.stats()
        a = st["analytic"]
        for name in ("velocity", "psi"):
            b = st[name]
            for ax in range(2):
                gap = abs(a["msd"][0][ax] - b["msd"][0][ax])
                worst = max(worst, gap / np.hypot(a["msd_sem"][0][ax], b["msd_sem"][0][ax]))
        assert a["t"] == pytest.approx(b["t"])
    assert worst < 3.0, worst
    for g in flows.values():
        g.close()


def test_checkpoint_and_argument_errors():
    xy = inputs.uniform_positions(500, 8)
    g = kin_flow(1)
    g.set_particles(0, xy, 0.0)
    g.step(40)
    image = g.save_state()
    g.step(60)
    a, _ = g.particles(0, 500)
    h = kin_flow(1)
    h.load_state(image)
    h.step(60)
    b, _ = h.particles(0, 500)
    np.testing.assert_array_equal(a, b)
    other = kin_flow(1, params=dict(PAPER, eps=0.5))
    with pytest.raises(elpath.ElpathError) as e:
        other.load_state(image)                    # another field
    assert e.value.status == 1
    with pytest.raises(elpath.ElpathError) as e:
        kin_flow(elpath.ANALYTIC).set_particles(0, xy, 1.0)   # the analytic route is for tracers
    assert e.value.status == 1
    for bad in (dict(PAPER, k=1.5), dict(PAPER, k=0.0), dict(PAPER, k=60.0)):
        with pytest.raises(elpath.ElpathError):
            kin_flow(0, params=bad)
    with pytest.raises(elpath.ElpathError):
        kin_flow(elpath.ANALYTIC, tracer_velocity=1)
    with pytest.raises(elpath.ElpathError):       # a solved flow has no analytic field
        elpath.Flow(N, 1e-3, DT, inputs.taylor_green(N), interp=elpath.ANALYTIC)
    batch = elpath.Batch(2)
    with pytest.raises(elpath.ElpathError):
        batch.add(g)
    batch.close()
    for f in (g, h, other):
        f.close()
