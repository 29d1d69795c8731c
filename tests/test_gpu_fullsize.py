"""Full-size workloads in the benchmark's launch configuration, compared with
the FP64 oracle on sampled particles (particles are independent, so the
oracle integrates just the sampled ones in the same fluid).

  * 1024^2 decaying turbulence, 1M tracers + 1M inertial particles at each
    of St = 0.1, 1, 10, each of the three schemes: vorticity after 100 steps,
    sampled positions and velocities after 200 steps;
  * 2048^2 double shear layer, 16M inertial particles at St = 1, Catmull-Rom:
    vorticity after 100 steps, every 64th particle (250,000 of them) after
    200 steps (about 0.8 s of oracle work per step on the host).
"""
import numpy as np
import pytest

from paper_2607_17836_b300 import elpath, inputs
from parity import OMEGA_RTOL, POS_ATOL, OracleRun, record, rel_linf

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SORT_EVERY = 20  # as in the benchmark


def test_decaying_turbulence_1024_all_schemes():
    wl = inputs.decaying_turbulence_1024()
    w0 = wl.omega0()
    stride = 244                                  # ~4100 sampled particles per species
    xys = [inputs.uniform_positions(s.count, s.seed) for s in wl.species]
    o = OracleRun(wl.n, wl.nu, wl.dt, w0)
    for scheme in (0, 1, 2):
        for s, xy in zip(wl.species, xys):
            o.add(scheme, s.st, xy[::stride])
    flows = []
    for scheme in (0, 1, 2):
        g = elpath.Flow(wl.n, wl.nu, wl.dt, w0, interp=scheme, max_species=4,
                        max_particles=wl.particles, sort_every=SORT_EVERY)
        for k, (s, xy) in enumerate(zip(wl.species, xys)):
            g.set_particles(k, xy, s.st)
        flows.append(g)
    for g in flows:
        g.step(100)
    o.step(100)
    w_ref = o.flow.fields(("w",))["w"]
    name = "decaying turbulence 1024^2, 4 x 1M"
    for scheme, g in enumerate(flows):
        werr = rel_linf(g.field(0), w_ref)
        record(name, scheme, "omega L-inf rel., 100 steps", werr, OMEGA_RTOL)
        assert werr < OMEGA_RTOL
    for g in flows:
        g.step(100)
    o.step(100)
    for scheme, g in enumerate(flows):
        for k, s in enumerate(wl.species):
            pos, vel = g.particles(k, s.count)
            ref = o.positions(4 * scheme + k)
            err = np.max(np.abs(pos[::stride] - ref))
            record(name, scheme, "max position error, 200 steps (every 244th)", err, POS_ATOL)
            assert err < POS_ATOL, (scheme, k, err)
            if s.st > 0:
                verr = np.max(np.abs(vel[::stride] - o.velocities(4 * scheme + k)))
                record(name, scheme, "max velocity error, 200 steps (every 244th)", verr, 1e-4)
                assert verr < 1e-4
        st = g.stats()
        assert st["finite"]
        g.close()


def test_kelvin_helmholtz_2048_16M():
    wl = inputs.kelvin_helmholtz_2048()
    w0 = wl.omega0()
    sp = wl.species[0]
    xy = inputs.uniform_positions(sp.count, sp.seed)
    g = elpath.Flow(wl.n, wl.nu, wl.dt, w0, interp=1, max_species=1, max_particles=sp.count,
                    sort_every=SORT_EVERY)
    g.set_particles(0, xy, sp.st)
    o = OracleRun(wl.n, wl.nu, wl.dt, w0)
    o.add(1, sp.st, xy[::64])
    name = "shear layer 2048^2, 16M at St = 1"
    g.step(100)
    o.step(100)
    werr = rel_linf(g.field(0), o.flow.fields(("w",))["w"])
    record(name, 1, "omega L-inf rel., 100 steps", werr, OMEGA_RTOL)
    assert werr < OMEGA_RTOL
    g.step(100)
    o.step(100)
    pos, vel = g.particles(0, sp.count)
    perr = np.max(np.abs(pos[::64] - o.positions(0)))
    verr = np.max(np.abs(vel[::64] - o.velocities(0)))
    record(name, 1, "max position error, 200 steps (every 64th)", perr, POS_ATOL)
    record(name, 1, "max velocity error, 200 steps (every 64th)", verr, 1e-4)
    assert perr < POS_ATOL
    assert verr < 1e-4
    g.close()
