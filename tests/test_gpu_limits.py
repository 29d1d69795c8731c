"""The ends of the grid-size range (n = 16 and n = 4096 points per side) on
the C-ABI path, every interpolation scheme, tracers and inertial particles.

  * n = 16: decaying turbulence against the full FP64 oracle (fluid and
    particles), with the 4 x 4 cubic stencils wrapping around a grid only
    four stencils wide and the coarsest re-binning tiles re-sorting every
    5 steps.
  * n = 4096: the inviscid Taylor-Green vortex omega = 2 sin x sin y, a
    steady solution (its nonlinear term vanishes identically), so the
    vorticity must stay omega_0 and the velocity must stay
    (sin x cos y, -cos x sin y); particles are compared with the oracle's
    RK4 driven by those exact levels (a 4096^2 FP64 oracle fluid solve takes
    minutes per step).  Particles cross about 20 cells in 300 steps.  With no
    viscosity nothing damps the highest kept modes, where AB2 amplifies
    advection by 1 + (k u dt)^4 / 4 per step: at dt = 5e-4 (k dt ~ 0.7) the
    FP32 rounding noise grew to 3e-3 of omega in 100 steps; dt = 1e-4 keeps the
    growth below 3 % over the run.
"""
import numpy as np
import pytest

import oracle
from paper_2607_17836_b300 import elpath, inputs
from parity import OMEGA_RTOL, POS_ATOL, OracleRun, oracle_stencil, rel_linf

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SCHEMES = (oracle.BILINEAR, oracle.CATMULL_ROM, oracle.BSPLINE)


def test_smallest_grid_16_matches_the_oracle():
    n, nu, dt = 16, 1e-2, 5e-2
    w0 = inputs.decaying_turbulence(n, 5, k0=3.0)
    sets = [(0.0, inputs.uniform_positions(500, 6)), (0.5, inputs.uniform_positions(500, 7))]
    o = OracleRun(n, nu, dt, w0)
    for scheme in SCHEMES:
        for st, xy in sets:
            o.add(scheme, st, xy)
    flows = []
    for scheme in SCHEMES:
        g = elpath.Flow(n, nu, dt, w0, interp=scheme, max_species=2, max_particles=1000,
                        sort_every=5)
        g.set_tuning(128, 5, 2)              # 4 x 4-cell tiles: the largest shift n = 16 allows
        for k, (st, xy) in enumerate(sets):
            g.set_particles(k, xy, st)
        flows.append(g)
    for g in flows:
        g.step(100)
    o.step(100)
    w_ref = o.flow.fields(("w",))["w"]
    for g in flows:
        assert rel_linf(g.field(0), w_ref) < OMEGA_RTOL
    for g in flows:
        g.step(100)
    o.step(100)
    for scheme, g in enumerate(flows):
        for k, (st, _) in enumerate(sets):
            pos, vel = g.particles(k, 500)
            err = np.max(np.abs(pos - o.positions(2 * scheme + k)))
            assert err < POS_ATOL, (scheme, k, err)
            if st > 0:
                assert np.max(np.abs(vel - o.velocities(2 * scheme + k))) < 1e-4
        assert g.stats()["finite"]
        g.close()


def test_largest_grid_4096_steady_taylor_green():
    n, dt, steps = 4096, 1e-4, 300
    x = np.arange(n) * (2.0 * np.pi / n)
    sx, cx = np.sin(x), np.cos(x)
    u0 = np.multiply.outer(cx, sx)           # [j][i]: sin(x_i) cos(y_j)
    v0 = -np.multiply.outer(sx, cx)          # -cos(x_i) sin(y_j)
    w0 = 2.0 * np.multiply.outer(sx, sx)     # 2 sin(x_i) sin(y_j)
    sets = [(0.0, inputs.uniform_positions(2000, 11)), (1.0, inputs.uniform_positions(2000, 12))]
    for scheme in SCHEMES:
        g = elpath.Flow(n, 0.0, dt, w0, interp=scheme, max_species=2, max_particles=4000,
                        sort_every=20)
        for k, (st, xy) in enumerate(sets):
            g.set_particles(k, xy, st)
        g.step(steps)
        if scheme == oracle.BILINEAR:        # the fluid does not depend on the scheme
            assert rel_linf(g.field(0), w0) < OMEGA_RTOL
            assert rel_linf(g.field(1), u0) < OMEGA_RTOL
            assert rel_linf(g.field(2), v0) < OMEGA_RTOL
        su, sv = oracle_stencil(u0, v0, scheme)
        for k, (st, xy) in enumerate(sets):
            X, Y = xy[:, 0].copy(), xy[:, 1].copy()
            if st > 0:                       # zero slip: the fluid velocity at the start
                VX, VY = oracle.interp(su, scheme, X, Y), oracle.interp(sv, scheme, X, Y)
            else:
                VX = VY = None
            for _ in range(steps):           # steady levels: n and n+1 are the same field
                oracle.particles_rk4(scheme, dt, st, su, sv, su, sv, X, Y, VX, VY)
            pos, vel = g.particles(k, len(xy))
            err = np.max(np.abs(pos - np.stack([X, Y], axis=1)))
            assert err < POS_ATOL, (scheme, k, err)
            travelled = np.max(np.hypot(X - xy[:, 0], Y - xy[:, 1])) / (2.0 * np.pi / n)
            assert travelled > 15.0          # the test crosses many cells
            if st > 0:
                assert np.max(np.abs(vel - np.stack([VX, VY], axis=1))) < 1e-4
        assert g.stats()["finite"]
        g.close()
