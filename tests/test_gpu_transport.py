"""Transport statistics (Sec. 5.5, Sec. 6) through the C ABI: the standard
error of the mean-square displacement and the diffusivity D = msd / (2 t)
in el_get_stats, against the FP64 oracle on the same particle positions, and
the paper's particle-number convergence check (msd curves of 100 to 2000
tracers agree within their standard errors)."""
import numpy as np
import pytest

import oracle
from paper_2607_17836_b300 import elpath, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_standard_error_and_diffusivity_match_the_oracle():
    n, nu, dt = 128, 1e-4, 5e-4
    species = [(3001, 0.0, 5), (1500, 1.0, 6), (1, 0.0, 7)]  # a one-particle slot: no spread
    g = elpath.Flow(n, nu, dt, inputs.decaying_turbulence(n, 9), interp=1,
                    max_species=len(species), max_particles=sum(c for c, _, _ in species),
                    sort_every=11)
    starts = []
    for k, (c, st, seed) in enumerate(species):
        xy = inputs.uniform_positions(c, seed)
        starts.append(xy)
        g.set_particles(k, xy, st)
    s0 = g.stats()
    # at t = 0: D is defined as 0; the split-precision positions reproduce x0
    # up to rounding, so the spread of the squared displacements is ~0
    assert s0["diffusivity"][0] == (0.0, 0.0)
    assert s0["msd_sem"][0] == pytest.approx((0.0, 0.0), abs=1e-12)
    g.step(400)
    s = g.stats()
    t = s["t"]
    assert t == pytest.approx(400 * dt)
    for k, (c, _, _) in enumerate(species):
        xy, _ = g.particles(k, c)
        x0, y0 = starts[k][:, 0], starts[k][:, 1]
        ref_m = oracle.msd(xy[:, 0], xy[:, 1], x0, y0)
        ref_e = oracle.msd_sem(xy[:, 0], xy[:, 1], x0, y0)
        ref_d = oracle.diffusivity(ref_m, t)
        np.testing.assert_allclose(s["msd"][k], ref_m, rtol=1e-9)
        np.testing.assert_allclose(s["msd_sem"][k], ref_e, rtol=1e-7, atol=1e-15)
        np.testing.assert_allclose(s["diffusivity"][k], ref_d, rtol=1e-9)
    assert s["msd_sem"][2] == (0.0, 0.0)
    g.close()


def test_particle_number_convergence_within_standard_errors():
    # Sec. 5.5: 100, 500, 1000 and 2000 tracers in one decaying flow give msd
    # curves whose differences stay within the combined standard errors
    n, nu, dt = 128, 1e-4, 5e-4
    sets = [(100, 31), (500, 32), (1000, 33), (2000, 34)]
    g = elpath.Flow(n, nu, dt, inputs.decaying_turbulence(n, 21), interp=0, max_species=4,
                    max_particles=sum(c for c, _ in sets), sort_every=20)
    for k, (c, seed) in enumerate(sets):
        g.set_particles(k, inputs.uniform_positions(c, seed), 0.0)
    worst = 0.0
    for _ in range(4):
        g.step(2000)
        s = g.stats()
        for i in range(len(sets)):
            for j in range(i + 1, len(sets)):
                for a in range(2):
                    gap = abs(s["msd"][i][a] - s["msd"][j][a])
                    bound = np.hypot(s["msd_sem"][i][a], s["msd_sem"][j][a])
                    assert bound > 0
                    worst = max(worst, gap / bound)
        # D(t) is msd / (2 t) for every species
        for k in range(len(sets)):
            for a in range(2):
                assert s["diffusivity"][k][a] == pytest.approx(s["msd"][k][a] / (2 * s["t"]))
    assert worst < 3.0, worst
    g.close()
