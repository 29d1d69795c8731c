"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Small grids span several thread blocks and ragged tails; the full-size
workloads (1024^2 decaying turbulence with 4 x 1M particles, 2048^2 shear
layer with 16M particles) run in the same launch configuration as the
benchmark and are compared on sampled particles the oracle integrates one
by one.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2607_17836_b300 import elpath, inputs
from parity import (GATHER_RTOL, OMEGA_RTOL, POS_ATOL, STATS_RTOL, TWO_PI, OracleRun, decaying,
                    gpu_flow, oracle_stencil, record, rel_linf)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_taylor_green_64_tracers_config():
    # 64^2 Taylor-Green, nu = 0.01, dt = 1e-3, 200 steps, 4096 tracers, bilinear.
    wl = inputs.taylor_green_64()
    xy = inputs.uniform_positions(4096, seed=1)
    g = gpu_flow(wl.n, wl.nu, wl.dt, wl.omega0(), interp=0, max_particles=4096)
    g.set_particles(0, xy, 0.0)
    o = OracleRun(wl.n, wl.nu, wl.dt, wl.omega0())
    o.add(0, 0.0, xy)
    g.step(wl.steps)
    o.step(wl.steps)
    X, Y = inputs.grid(wl.n)
    exact = 2 * math.exp(-2 * wl.nu * wl.dt * wl.steps) * np.sin(X) * np.sin(Y)
    w = g.field(0)
    wl_name = "Taylor-Green 64^2, 4096 tracers"
    record(wl_name, 0, "omega L-inf rel. vs closed form, 200 steps", rel_linf(w, exact), 2e-6)
    assert rel_linf(w, exact) < 2e-6   # FP32 storage: ~steps^0.5 * 2^-24 unbiased
    werr = rel_linf(w, o.flow.fields(("w",))["w"])
    record(wl_name, 0, "omega L-inf rel., 200 steps", werr, OMEGA_RTOL)
    assert werr < OMEGA_RTOL
    pos, _ = g.particles(0, 4096)
    perr = np.max(np.abs(pos - o.positions(0)))
    record(wl_name, 0, "max position error, 200 steps", perr, POS_ATOL)
    assert perr < POS_ATOL
    st = g.stats()
    assert abs(st["energy"] - 0.25 * math.exp(-4 * wl.nu * wl.dt * wl.steps)) < 1e-6
    psi0 = np.sin(xy[:, 0]) * np.sin(xy[:, 1])
    assert np.max(np.abs(np.sin(pos[:, 0]) * np.sin(pos[:, 1]) - psi0)) < 2e-4


@pytest.mark.parametrize("mode", [0, 1])
def test_vorticity_parity_128(mode):
    n, nu, dt = 128, 1e-4, 5e-4
    w0 = decaying(n, seed=5)
    g = gpu_flow(n, nu, dt, w0, ab2_mode=mode, max_species=0)
    o = oracle.Flow(n, nu, dt, w0, ab2_mode=mode)
    for steps in (1, 9, 90):
        g.step(steps)
        o.step(steps)
        of = o.fields(("u", "v", "w"))
        if steps == 90:
            record(f"decaying 128^2, AB2 mode {mode}", None, "omega L-inf rel., 100 steps",
                   rel_linf(g.field(0), of["w"]), OMEGA_RTOL)
        assert rel_linf(g.field(0), of["w"]) < OMEGA_RTOL
        assert rel_linf(g.field(1), of["u"]) < OMEGA_RTOL
        assert rel_linf(g.field(2), of["v"]) < OMEGA_RTOL
    e, z, p = o.diagnostics()
    st = g.stats()
    assert abs(st["energy"] - e) < 1e-5 * e
    assert abs(st["enstrophy"] - z) < 1e-5 * z
    assert abs(st["palinstrophy"] - p) < 1e-5 * p


@pytest.mark.parametrize("scheme,prefilter", [(0, True), (1, True), (2, True), (2, False)])
def test_gather_parity(scheme, prefilter):
    # The gather on the GPU's own stencil fields vs the oracle's interpolant
    # on the same values: isolates the interpolation arithmetic.
    n = 64
    g = gpu_flow(n, 1e-3, 1e-3, decaying(n, seed=6, k0=6.0), interp=scheme, prefilter=prefilter)
    g.step(3)
    prev = (g.field(3), g.field(4))
    g.step(1)
    cur = (g.field(3), g.field(4))
    rng = np.random.default_rng(7)
    pts = rng.uniform(-2 * TWO_PI, 3 * TWO_PI, size=(20011, 2))
    pts[:8] = [[0, 0], [TWO_PI, 0], [-1e-12, 3.0], [TWO_PI - 1e-12, 1.0],
               [TWO_PI / n * 5, TWO_PI / n * 7], [1e-7, TWO_PI - 1e-7], [100.0, -100.0], [3, 3]]
    d = torch.from_numpy(pts).cuda()
    for theta in (0.0, 0.5, 1.0):
        uv = g.sample_velocity(d, theta).cpu().numpy()
        ref = []
        for comp in (0, 1):
            a = oracle.interp(prev[comp], scheme, pts[:, 0], pts[:, 1])
            b = oracle.interp(cur[comp], scheme, pts[:, 0], pts[:, 1])
            ref.append((1 - theta) * a + theta * b)
        ref = np.stack(ref, axis=1)
        gerr = np.max(np.abs(uv - ref)) / np.max(np.abs(ref))
        record("gather, 64^2 field, 20011 points" + ("" if prefilter else " (raw B-spline)"), scheme,
               "interpolated velocity rel. error", gerr, GATHER_RTOL)
        assert gerr < GATHER_RTOL, theta
    if scheme == 2 and prefilter:
        # the GPU's spectral prefilter vs the oracle's cyclic tridiagonal solve
        u = g.field(1)
        assert rel_linf(cur[0], oracle.bspline_prefilter(u)) < GATHER_RTOL


@pytest.mark.parametrize("scheme", [0, 1, 2])
def test_coupled_particles_parity_128(scheme):
    # Tracers and three Stokes numbers, ragged counts, 200 coupled steps.
    n, nu, dt = 128, 1e-4, 5e-4
    w0 = decaying(n, seed=8)
    counts = [1, 257, 3001, 12345]
    sts = [0.0, 0.1, 1.0, 10.0]
    g = gpu_flow(n, nu, dt, w0, interp=scheme, max_species=4, max_particles=sum(counts),
                 sort_every=7)
    o = OracleRun(n, nu, dt, w0)
    xys = []
    for s, (c, st) in enumerate(zip(counts, sts)):
        xy = inputs.uniform_positions(c, seed=100 + s)
        xys.append(xy)
        g.set_particles(s, xy, st)
        o.add(scheme, st, xy)
    # zero-slip start: velocities equal the interpolated fluid velocity
    for s in (1, 2, 3):
        _, v = g.particles(s, counts[s])
        assert np.max(np.abs(v - o.velocities(s))) < GATHER_RTOL * 10
    g.step(200)
    o.step(200)
    for s in range(4):
        pos, vel = g.particles(s, counts[s])
        perr = np.max(np.abs(pos - o.positions(s)))
        record("decaying 128^2, 4 species (1-12345 particles)", scheme,
               "max position error, 200 steps", perr, POS_ATOL)
        assert perr < POS_ATOL, s
        if sts[s] > 0:
            assert np.max(np.abs(vel - o.velocities(s))) < 1e-4, s


def test_periodic_crossing_and_unwrapping():
    # Steady shear omega = cos y: u = -sin y, v = 0 exactly, so particles
    # stream along x across the periodic boundary many times.
    n = 32
    X, Y = inputs.grid(n)
    g = gpu_flow(n, 0.0, 0.01, np.cos(Y), interp=1, max_species=2, max_particles=2 * 500)
    o = OracleRun(n, 0.0, 0.01, np.cos(Y))
    rng = np.random.default_rng(9)
    xy = np.stack([rng.uniform(-TWO_PI, TWO_PI, 500), rng.uniform(0, TWO_PI, 500)], axis=1)
    xy[:4] = [[0.0, 3 * np.pi / 2], [-1e-9, np.pi / 2], [TWO_PI, 1.0], [TWO_PI * 7, 4.0]]
    for s, st in enumerate((0.0, 0.5)):
        g.set_particles(s, xy, st)
        o.add(1, st, xy)
    g.step(1500)
    o.step(1500)
    for s in range(2):
        pos, _ = g.particles(s, 500)
        assert np.max(np.abs(pos - o.positions(s))) < POS_ATOL
        assert np.max(np.abs(pos[:, 0] - xy[:, 0])) > 2 * TWO_PI   # wrapped at least twice


def test_new_particles_mid_run_keep_or_rebuild_the_step_graphs():
    # Particles set again in the same numbers keep the flow's captured step
    # graphs (they read the particle state through the device species table);
    # other numbers rebuild them.  Either way the new particles then follow
    # the oracle's trajectories from the level they were set at.
    n, nu, dt = 64, 1e-3, 1e-3
    w0 = decaying(n, seed=21, k0=6.0)
    g = gpu_flow(n, nu, dt, w0, interp=1, max_species=2, max_particles=6000, sort_every=7)
    o = OracleRun(n, nu, dt, w0)
    first = inputs.uniform_positions(3000, seed=22)
    g.set_particles(0, first, 0.0)
    g.set_particles(1, first, 1.0)
    g.step(30)
    o.step(30)
    for count, seed in ((3000, 23), (1234, 24)):     # the same numbers, then others
        xy = inputs.uniform_positions(count, seed)
        g.set_particles(0, xy, 0.0)
        g.set_particles(1, xy, 1.0)
        k0 = len(o.sets)
        o.add(1, 0.0, xy)
        o.add(1, 1.0, xy)
        g.step(25)
        o.step(25)
        for s in range(2):
            pos, _ = g.particles(s, count)
            perr = np.max(np.abs(pos - o.positions(k0 + s)))
            record("particles set again mid-run, 64^2", 1, "max position error, 25 steps", perr,
                   POS_ATOL)
            assert perr < POS_ATOL, (count, s, perr)
    g.close()


def test_empty_and_single_species_and_sort_invariance():
    n, nu, dt = 64, 1e-3, 1e-3
    w0 = decaying(n, seed=10, k0=6.0)
    xy = inputs.uniform_positions(5000, seed=11)
    res = []
    for sort_every in (0, 1, 5):
        g = gpu_flow(n, nu, dt, w0, interp=1, max_species=3, max_particles=5001,
                     sort_every=sort_every)
        g.set_particles(0, xy, 1.0)
        g.set_particles(1, xy[:0], 0.0)    # empty species
        g.set_particles(2, xy[:1], 0.0)    # single particle
        g.step(50)
        res.append((g.particles(0, 5000), g.particles(2, 1), g.stats()))
    for r in res[1:]:
        # results do not depend on the order the sort leaves particles in
        np.testing.assert_array_equal(r[0][0], res[0][0][0])
        np.testing.assert_array_equal(r[0][1], res[0][0][1])
        np.testing.assert_array_equal(r[1][0], res[0][1][0])
        assert r[2]["msd"][0] == res[0][2]["msd"][0]
        assert r[2]["cluster"][0] == res[0][2]["cluster"][0]
    assert res[0][2]["np"][:3] == [5000, 0, 1]


def test_stats_parity_and_determinism():
    n, nu, dt = 128, 1e-4, 5e-4
    w0 = decaying(n, seed=12)
    xy = inputs.uniform_positions(20000, seed=13)
    runs = []
    for _ in range(2):
        g = gpu_flow(n, nu, dt, w0, interp=0, max_species=2, max_particles=40000, sort_every=10)
        g.set_particles(0, xy, 0.0)
        g.set_particles(1, xy, 1.0)
        g.step(100)
        runs.append(g.stats())
    assert runs[0] == runs[1]       # bitwise identical
    o = OracleRun(n, nu, dt, w0)
    o.add(0, 0.0, xy)
    o.add(0, 1.0, xy)
    o.step(100)
    e, z, p = o.flow.diagnostics()
    st = runs[0]
    assert abs(st["energy"] - e) < 1e-5 * e
    for k in range(2):
        s = o.sets[k]
        mx, my = oracle.msd(s["x"], s["y"], s["x0"], s["y0"])
        assert abs(st["msd"][k][0] - mx) < 1e-4 * mx
        assert abs(st["msd"][k][1] - my) < 1e-4 * my
        c = oracle.cluster_index(s["x"], s["y"])
        assert abs(st["cluster"][k] - c) < 1e-3 * max(1.0, abs(c))


def test_long_run_statistics_256():
    # Chaotic run: compare dispersion and clustering, not trajectories.
    n, nu, dt, steps = 256, 1e-4, 5e-4, 2000
    w0 = decaying(n, seed=14)
    sts = [0.0, 0.1, 1.0, 10.0]
    cnt = 8192
    g = gpu_flow(n, nu, dt, w0, interp=0, max_species=4, max_particles=4 * cnt, sort_every=20)
    o = OracleRun(n, nu, dt, w0)
    for s, st in enumerate(sts):
        xy = inputs.uniform_positions(cnt, seed=200 + s)
        g.set_particles(s, xy, st)
        o.add(0, st, xy)
    g.step(steps)
    o.step(steps)
    gs = g.stats()
    for k in range(4):
        s = o.sets[k]
        mx, my = oracle.msd(s["x"], s["y"], s["x0"], s["y0"])
        assert abs(gs["msd"][k][0] - mx) < STATS_RTOL * mx
        assert abs(gs["msd"][k][1] - my) < STATS_RTOL * my
        c = oracle.cluster_index(s["x"], s["y"])
        assert abs(gs["cluster"][k] - c) < STATS_RTOL * max(1.0, abs(c))


def test_argument_errors():
    n = 32
    w0 = decaying(n, seed=15, k0=4.0)
    with pytest.raises(elpath.ElpathError) as e:
        elpath.Flow(n, -1.0, 1e-3, w0)
    assert e.value.status == 1
    g = gpu_flow(n, 1e-3, 1e-3, w0, max_species=1, max_particles=10)
    xy = inputs.uniform_positions(11, seed=1)
    with pytest.raises(elpath.ElpathError):
        g.set_particles(0, xy, 0.0)          # beyond capacity
    with pytest.raises(elpath.ElpathError):
        g.set_particles(1, xy[:5], 0.0)      # no such species slot
    bad = xy[:5].copy()
    bad[2, 0] = np.nan
    with pytest.raises(elpath.ElpathError):
        g.set_particles(0, bad, 0.0)
    with pytest.raises(elpath.ElpathError):
        g.set_particles(0, xy[:5], -1.0)
    with pytest.raises(elpath.ElpathError) as e:
        g.set_tuning(128, 20, 0, 3)          # no such stencil gather
    assert e.value.status == 1
    assert g.tuning()["gather"] == elpath.GATHER_AUTO
    # a failed call leaves the flow usable
    g.set_particles(0, xy[:5], 0.0)
    g.step(2)
    assert g.stats()["np"][0] == 5
    # workspace too small
    desc = elpath.make_desc(n, 1e-3, 1e-3)
    need = elpath.workspace_bytes(desc)
    small = torch.empty(need - 4096, dtype=torch.uint8, device="cuda")
    with pytest.raises(elpath.ElpathError) as e:
        elpath.Flow(n, 1e-3, 1e-3, w0, workspace=small)
    assert e.value.status == 2


@pytest.mark.parametrize("scheme", [0, 1, 2])
def test_no_uninitialised_reads(scheme):
    # A workspace full of NaN bytes (0xFF) must give the same bits as a zeroed
    # one: every value the path reads is written first.
    n = 64
    w0 = decaying(n, seed=16, k0=6.0)
    xy = inputs.uniform_positions(3000, seed=17)
    outs = []
    for fill in (0, 255):
        desc = elpath.make_desc(n, 1e-3, 1e-3, interp=scheme, max_species=2, max_particles=6000,
                                sort_every=4)
        ws = torch.full((elpath.workspace_bytes(desc),), fill, dtype=torch.uint8, device="cuda")
        g = elpath.Flow(n, 1e-3, 1e-3, w0, interp=scheme, max_species=2, max_particles=6000,
                        sort_every=4, workspace=ws)
        g.set_particles(0, xy, 1.0)
        g.set_particles(1, xy, 0.0)
        g.step(9)
        st = g.stats()
        outs.append((g.particles(0, 3000), g.particles(1, 3000)[0], g.field(0), st["msd"][:2]))
        g.close()
    a, b = outs
    np.testing.assert_array_equal(a[0][0], b[0][0])
    np.testing.assert_array_equal(a[0][1], b[0][1])
    np.testing.assert_array_equal(a[1], b[1])
    np.testing.assert_array_equal(a[2], b[2])
    assert a[3] == b[3]


@pytest.mark.parametrize("scheme", [0, 1, 2])
def test_streamfunction_tracers_parity(scheme):
    # tracer_velocity = 1: tracers use Eq. 11 (streamfunction + centred
    # differences), inertial particles the interpolated velocity.
    n, nu, dt = 128, 1e-4, 5e-4
    w0 = decaying(n, seed=18)
    g = gpu_flow(n, nu, dt, w0, interp=scheme, max_species=2, max_particles=8000, sort_every=9,
                 tracer_velocity=1)
    o = OracleRun(n, nu, dt, w0)
    xy = inputs.uniform_positions(4000, seed=19)
    g.set_particles(0, xy, 0.0)
    g.set_particles(1, xy, 1.0)
    o.add(scheme, 0.0, xy, psi=True)
    o.add(scheme, 1.0, xy)
    g.step(200)
    o.step(200)
    for s in range(2):
        pos, _ = g.particles(s, 4000)
        perr = np.max(np.abs(pos - o.positions(s)))
        record("streamfunction tracers (Eq. 11) + inertial, 128^2", scheme,
               "max position error, 200 steps", perr, POS_ATOL)
        assert perr < POS_ATOL, s
