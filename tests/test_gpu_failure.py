"""Failure detection without any GPU fault, and determinism.

A simulation made unstable on the host (a time step far beyond the AB2
stability limit) blows up; el_get_stats reports it as EL_ENONFINITE with the
flow still usable (readback works, it can be destroyed cleanly).  Identical
runs give identical bits (the reductions are in a fixed order and no kernel
depends on scheduling), whatever the block size of the particle step:
a cheap race detector.
"""
import numpy as np
import pytest

from paper_2607_17836_b300 import elpath, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_blow_up_is_reported_as_non_finite():
    n = 64
    g = elpath.Flow(n, 1e-4, 2.0, inputs.decaying_turbulence(n, 3, k0=6.0), interp=1,
                    max_species=1, max_particles=500)
    g.set_particles(0, inputs.uniform_positions(500, 4), 1.0)
    status = None
    for _ in range(40):
        g.step(5)
        s = g.stats(allow_nonfinite=True)
        if not s["finite"]:
            with pytest.raises(elpath.ElpathError) as e:
                g.stats()
            status = e.value.status
            break
    assert status == 6                                 # EL_ENONFINITE
    # the flow is still usable: readback and destruction work
    w = g.field(0)
    assert w.shape == (n, n)
    xy, _ = g.particles(0, 500)
    assert xy.shape == (500, 2)
    g.close()


def test_stable_runs_report_finite_statistics():
    n = 64
    g = elpath.Flow(n, 1e-3, 1e-3, inputs.decaying_turbulence(n, 3, k0=6.0), interp=0,
                    max_species=1, max_particles=500)
    g.set_particles(0, inputs.uniform_positions(500, 4), 0.0)
    g.step(200)
    assert g.stats()["finite"]
    g.close()


def run(case_threads, interp, sort_every, gather=elpath.GATHER_AUTO):
    n = 128
    g = elpath.Flow(n, 1e-4, 5e-4, inputs.decaying_turbulence(n, 12), interp=interp,
                    max_species=2, max_particles=6000, sort_every=sort_every)
    g.set_particles(0, inputs.uniform_positions(3000, 1), 0.0)
    g.set_particles(1, inputs.uniform_positions(3000, 2), 1.0)
    g.set_tuning(case_threads, sort_every, 0, gather)
    g.step(150)
    s = g.stats()
    out = [g.field(0)] + list(g.particles(0, 3000)) + list(g.particles(1, 3000))
    out.append(np.array([s["energy"], s["enstrophy"], s["palinstrophy"]]
                        + [m for p in s["msd"] for m in p] + s["cluster"]
                        + [m for p in s["msd_sem"] for m in p]))
    g.close()
    return out


@pytest.mark.parametrize("interp", [0, 1, 2])
def test_reruns_are_bitwise_identical(interp):
    a = run(256, interp, 10)
    b = run(256, interp, 10)
    c = run(128, interp, 17)          # another block size and re-binning cadence
    # the two stencil gathers of the cubic schemes (register copy, warp-shared
    # patch in shared memory): the same arithmetic on the same values
    d = run(512, interp, 10, elpath.GATHER_REGISTERS)
    e = run(128, interp, 0, elpath.GATHER_SHARED)
    for x, y, z, u, v in zip(a, b, c, d, e):
        np.testing.assert_array_equal(x, y)
        np.testing.assert_array_equal(x, z)
        np.testing.assert_array_equal(x, u)
        np.testing.assert_array_equal(x, v)


def test_non_finite_host_inputs_are_refused_and_leave_the_flow_unchanged():
    # NaN / Inf injected through every host input: the initial vorticity,
    # particle positions (and positions too far out for the image count),
    # particle velocities and the Stokes number.  Each call fails with
    # EL_EINVAL and a flow keeps its state.  Positions and velocities are
    # checked on the device, on the staged copy; capacity carved for a refused
    # call is handed back (species 1 below has none before the bad calls, and
    # takes a good set afterwards).
    n = 32
    w0 = inputs.decaying_turbulence(n, 3, k0=4.0)
    for bad in (np.nan, np.inf, -np.inf):
        w = w0.copy()
        w[5, 7] = bad
        with pytest.raises(elpath.ElpathError) as e:
            elpath.Flow(n, 1e-3, 1e-3, w, interp=0, max_species=1, max_particles=10)
        assert e.value.status == 1 and "non-finite" in str(e.value)
    g = elpath.Flow(n, 1e-3, 1e-3, w0, interp=1, max_species=2, max_particles=200)
    xy = inputs.uniform_positions(100, 5)
    g.set_particles(0, xy, 1.0)
    g.step(3)
    before = [g.field(0)] + list(g.particles(0, 100))
    # (position value at xy[17, 1] = element 35, velocity at vxy[3, 0] =
    # element 6, Stokes number, expected message)
    cases = ((np.nan, 0.0, 1.0, "xy[35]"), (np.inf, 0.0, 0.0, "xy[35]"), (2e9, 0.0, 0.0, "xy[35]"),
             (None, np.nan, 1.0, "vxy[6]"), (None, 0.0, np.nan, "st must"),
             (None, 0.0, np.inf, "st must"))
    for bad_xy, bad_v, st, msg in cases:
        p = xy.copy()
        if bad_xy is not None:
            p[17, 1] = bad_xy
        v = np.zeros_like(p)
        v[3, 0] = bad_v
        with pytest.raises(elpath.ElpathError) as e:
            g.set_particles(0, p, st, v)
        assert e.value.status == 1 and msg in str(e.value), str(e.value)
    for _ in range(3):                               # species 1 has no capacity yet
        for bad in (np.nan, np.inf):
            p = xy.copy()
            p[40, 0] = bad
            with pytest.raises(elpath.ElpathError) as e:
                g.set_particles(1, p, 0.0)
            assert e.value.status == 1 and "xy[80]" in str(e.value)
    after = [g.field(0)] + list(g.particles(0, 100))
    for a, b in zip(before, after):
        np.testing.assert_array_equal(a, b)
    assert g.stats()["np"][1] == 0
    g.set_particles(1, xy, 0.0)                      # the refused carves were handed back:
    g.step(2)                                        # 200 = max_particles still fits
    s = g.stats()
    assert s["finite"] and s["np"][:2] == [100, 100]
    g.close()
