"""Batched engine and autotuner (through the C ABI).

A member of a batch does the same arithmetic as the same simulation stepped
alone, whatever else is in the batch and whenever it joined; the tuning
knobs change no result.
"""
import numpy as np
import pytest

from paper_2607_17836_b300 import elpath, inputs
from parity import OMEGA_RTOL, POS_ATOL, rel_linf

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SPECS = [  # (n, scheme, [(count, St)], nu, dt)
    (32, 0, [(777, 0.0), (300, 1.0)], 1e-3, 2e-3),
    (64, 1, [(5000, 0.1)], 5e-4, 1e-3),
    (128, 2, [(2049, 0.0), (1000, 10.0), (257, 1.0)], 1e-4, 5e-4),
    (256, 0, [(20000, 1.0)], 1e-4, 5e-4),
]


def make(spec, seed, sort_every=7):
    n, scheme, species, nu, dt = spec
    g = elpath.Flow(n, nu, dt, inputs.decaying_turbulence(n, seed), interp=scheme,
                    max_species=len(species), max_particles=sum(c for c, _ in species),
                    sort_every=sort_every)
    for k, (c, st) in enumerate(species):
        g.set_particles(k, inputs.uniform_positions(c, seed * 10 + k), st)
    return g


def state(g, spec):
    out = [g.field(0)]
    for k, (c, _) in enumerate(spec[2]):
        out.extend(g.particles(k, c))
    return out


def assert_same(a, b):
    assert rel_linf(a[0], b[0]) < OMEGA_RTOL
    for x, y in zip(a[1:], b[1:]):
        assert np.max(np.abs(x - y)) <= POS_ATOL


def test_members_match_their_solo_runs():
    steps = 40
    solo = []
    for m, spec in enumerate(SPECS):
        g = make(spec, 100 + m)
        g.step(steps)
        solo.append(state(g, spec))
        g.close()
    batch = elpath.Batch(8)
    flows = [make(spec, 100 + m) for m, spec in enumerate(SPECS)]
    for g in flows:
        batch.add(g)
    batch.step(steps)
    for g, spec, ref in zip(flows, SPECS, solo):
        assert g.stats()["step"] == steps
        assert_same(state(g, spec), ref)
    # one launch per stage for the whole batch: the fused step's four for the
    # 256^2 member, the spectral and nonlinear stages for the others, the
    # particle stage once per scheme present (three here), the step counters:
    # 10 of our kernels per step
    l0 = batch.kernel_launches()
    batch.step(3)
    assert batch.kernel_launches() - l0 == 3 * 10
    batch.close()


def test_members_joining_and_leaving_at_different_steps():
    # member A runs 15 steps alone, then joins B (fresh) for 25; then A leaves
    # and B continues 10 more in the batch.
    a_spec, b_spec = SPECS[1], SPECS[2]
    ref_a = make(a_spec, 7)
    ref_a.step(40)
    ref_b = make(b_spec, 8)
    ref_b.step(35)
    a = make(a_spec, 7)
    a.step(15)
    b = make(b_spec, 8)
    batch = elpath.Batch(4)
    batch.add(a)
    batch.add(b)
    batch.step(25)
    batch.remove(a)
    a.step(0)
    batch.step(10)
    assert a.stats()["step"] == 40 and b.stats()["step"] == 35
    assert_same(state(a, a_spec), state(ref_a, a_spec))
    assert_same(state(b, b_spec), state(ref_b, b_spec))
    with pytest.raises(elpath.ElpathError) as e:
        b.step(1)                                  # members step only with their batch
    assert e.value.status == 5
    batch.close()


def test_autotune_changes_no_result():
    spec = (128, 1, [(30000, 1.0), (10000, 0.0)], 1e-4, 5e-4)
    ref = make(spec, 3, sort_every=20)
    tuned = make(spec, 3, sort_every=20)
    best = tuned.autotune(trial_steps=6)
    assert best["rk4_threads"] in (128, 256, 512) and best["ms_per_step"] > 0
    steps_done = tuned.stats()["step"]
    ref.step(steps_done)
    a, b = state(tuned, spec), state(ref, spec)
    np.testing.assert_array_equal(a[1], b[1])      # bitwise: block size and sort order
    np.testing.assert_array_equal(a[3], b[3])      # do not enter the arithmetic
    batch = elpath.Batch(4)
    flows = [make(s, 50 + m) for m, s in enumerate(SPECS[:3])]
    for g in flows:
        batch.add(g)
    bbest = batch.autotune(trial_steps=4)
    assert bbest["ms_per_step"] > 0
    batch.close()


FUSED_CASES = [  # (interp, bspline_prefilter, tracer_velocity, ab2_mode): planes 4, 4, 6, 5, 7
    (0, 1, 0, 0),
    (1, 1, 0, 1),
    (2, 1, 0, 0),
    (0, 1, 1, 0),
    (2, 1, 1, 1),
]


def make_fused(case, seed, n=1024):
    interp, pre, tv, mode = case
    g = elpath.Flow(n, 1e-4, 5e-4 * 1024 / n, inputs.decaying_turbulence(n, seed), interp=interp,
                    bspline_prefilter=pre, tracer_velocity=tv, ab2_mode=mode, max_species=2,
                    max_particles=6000, sort_every=7)
    g.set_particles(0, inputs.uniform_positions(3000, seed + 1), 0.0)
    g.set_particles(1, inputs.uniform_positions(3000, seed + 2), 1.0)
    return g


# (grid, case): the 1024^2 cases, a 2048^2 member on the fused step (4 planes)
# and one on the cuFFT path (the streamfunction plane: 5 planes), a 512^2 and a
# 256^2 member on the fused step
FUSED_MEMBERS = [(1024, c) for c in FUSED_CASES] + [(2048, (1, 1, 0, 1)), (2048, (0, 1, 1, 0)),
                                                     (512, (0, 1, 0, 0)), (256, (2, 1, 0, 1))]


def test_fused_members_equal_their_solo_runs_bit_for_bit():
    # members on the fused grids take the fused fluid step in the batch too
    # (one launch of each fused kernel per grid and plane count, every member
    # in it): the same kernels' arithmetic as alone, so the same bits,
    # whatever the plane count, the AB2 form or the step each member joined
    # at (members at odd and even steps share a launch).  A 256^2 member steps
    # beside them.
    head = [0, 3, 1, 4, 2, 1, 0, 2, 5]  # steps alone before joining
    steps = 12
    refs = []
    for m, (n, case) in enumerate(FUSED_MEMBERS):
        g = make_fused(case, 40 + 5 * m, n)
        g.step(head[m] + steps)
        refs.append((g.field(0), g.particles(0, 3000)[0], g.particles(1, 3000)))
        g.close()
    small = make(SPECS[3], 9)
    small_ref = make(SPECS[3], 9)
    small_ref.step(steps)
    batch = elpath.Batch(12)
    flows = []
    for m, (n, case) in enumerate(FUSED_MEMBERS):
        g = make_fused(case, 40 + 5 * m, n)
        g.step(head[m])
        flows.append(g)
        batch.add(g)
    batch.add(small)
    batch.step(steps)
    for g, (w, p0, (p1, v1)) in zip(flows, refs):
        np.testing.assert_array_equal(g.field(0), w)
        np.testing.assert_array_equal(g.particles(0, 3000)[0], p0)
        q1, u1 = g.particles(1, 3000)
        np.testing.assert_array_equal(q1, p1)
        np.testing.assert_array_equal(u1, v1)
    assert_same(state(small, SPECS[3]), state(small_ref, SPECS[3]))
    for g in flows + [small]:
        batch.remove(g)
        g.close()
    small_ref.close()
    batch.close()


# (n, scheme, tracer_velocity, [(count, St)]): per species, at least 2
# particles per cell takes the warp-shared stencil patch (automatic gather),
# fewer the per-thread register stencils
CLASS_SPECS = [
    (64, 1, 0, [(20000, 1.0), (800, 0.0)]),    # Catmull-Rom: patch and registers in one member
    (64, 2, 1, [(12000, 0.0), (9000, 10.0)]),  # B-spline, streamfunction tracers: patch
    (32, 0, 0, [(3000, 0.1)]),                 # bilinear (persistent class)
    (128, 2, 0, [(1500, 1.0)]),                # B-spline: registers
]


def make_class(spec, seed):
    n, scheme, tv, species = spec
    g = elpath.Flow(n, 1e-3, 1e-3 * 64 / n, inputs.decaying_turbulence(n, seed), interp=scheme,
                    tracer_velocity=tv, max_species=len(species),
                    max_particles=sum(c for c, _ in species), sort_every=5)
    for k, (c, st) in enumerate(species):
        g.set_particles(k, inputs.uniform_positions(c, seed * 10 + k), st)
    return g


def test_gather_classes_equal_their_solo_runs_bit_for_bit():
    # The batched particle step launches once per (scheme, stencil gather)
    # class present, each entry (a member's species) taking the gather its
    # own density picks; a flow alone picks one gather for all its species by
    # the densest.  Both gathers do the same arithmetic on the same values,
    # so every member ends bit for bit as alone.
    steps = 15
    refs = []
    for m, spec in enumerate(CLASS_SPECS):
        g = make_class(spec, 70 + m)
        g.step(steps)
        refs.append([g.field(0)] + [a for k, (c, _) in enumerate(spec[3]) for a in g.particles(k, c)])
        g.close()
    batch = elpath.Batch(8)
    flows = [make_class(spec, 70 + m) for m, spec in enumerate(CLASS_SPECS)]
    for g in flows:
        batch.add(g)
    batch.step(steps)
    for g, spec, ref in zip(flows, CLASS_SPECS, refs):
        got = [g.field(0)] + [a for k, (c, _) in enumerate(spec[3]) for a in g.particles(k, c)]
        for x, y in zip(got, ref):
            np.testing.assert_array_equal(x, y)
    # classes present: bilinear, Catmull-Rom registers and patch, B-spline
    # registers and patch (5 particle launches); the fluid step: the 64^2 and
    # 32^2 and 128^2 members on the batched spectral / cuFFT / nonlinear
    # stages (not fused grids); the step counters
    l0 = batch.kernel_launches()
    batch.step(2)
    per_step = (batch.kernel_launches() - l0) / 2
    assert per_step == 5 + 2 + 1
    for g in flows:
        batch.remove(g)
        g.close()
    batch.close()
