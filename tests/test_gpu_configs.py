"""The large workloads at their configured sizes, against the FP64 oracle.

  * decaying turbulence, 1024^2, 1M tracers + 1M particles at each of
    St = 0.1, 1, 10, each interpolation scheme, 2000 steps;
  * the double shear layer, 2048^2, 16M particles at St = 1, Catmull-Rom,
    4000 steps;
  * the 64-member ensemble (256^2-1024^2, 1e4-1e6 particles each), batched
    (their fluid steps fused; FFT pools for any on cuFFT) against each member stepped alone;
  * the served stream's first 16 requests at their drawn sizes (grids up to
    2048^2, up to 8.5M particles, up to ~2000 steps, both served schemes),
    served together against each run alone.

The long runs are chaotic, so they are compared on statistics: the
mean-square displacement per axis and the clustering index of the same
particles the oracle integrated (every 16th / 64th of each species), within
1 % of the oracle's.  The oracle's values come from
tests/golden/make_config_statistics.py, which runs only the FP64 oracle
(about 15 and 45 minutes of host time); the GPU side runs here in seconds.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2607_17836_b300 import elpath, inputs, serve
from parity import OMEGA_RTOL, POS_ATOL, STATS_RTOL, record, rel_linf

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
SORT_EVERY = 20  # as in the benchmark


def golden(name):
    with open(os.path.join(GOLDEN, f"{name}_statistics.json")) as fh:
        return json.load(fh)


def compare_statistics(name, wl, gold, flow, xys, scheme, label):
    """Step `flow` through the golden checkpoints; at each compare the
    sampled particles' statistics with the oracle's."""
    stride = gold["stride"]
    done = 0
    marks = sorted(gold["checkpoints"], key=int)
    span = f"steps {', '.join(marks)}"
    for mark in marks:
        flow.step(int(mark) - done)
        done = int(mark)
        cp = gold["checkpoints"][mark]
        st = flow.stats()
        assert st["finite"] and st["step"] == done
        e_rel = abs(st["energy"] - cp["energy"]) / cp["energy"]
        record(label, scheme, f"energy rel. difference ({span})", e_rel, STATS_RTOL)
        assert e_rel < STATS_RTOL
        for row in cp["sets"]:
            if row["scheme"] != scheme:
                continue
            k = row["species"]
            pos, _ = flow.particles(k, wl.species[k].count)
            sub, x0 = pos[::stride], xys[k][::stride]
            assert sub.shape[0] == row["sampled"]
            mx, my = oracle.msd(sub[:, 0], sub[:, 1], x0[:, 0], x0[:, 1])
            c = oracle.cluster_index(sub[:, 0], sub[:, 1])
            msd_rel = max(abs(mx - row["msd"][0]) / row["msd"][0],
                          abs(my - row["msd"][1]) / row["msd"][1])
            c_rel = abs(c - row["cluster"]) / max(1.0, abs(row["cluster"]))
            what = f"every species, {span}"
            record(label, scheme, f"MSD rel. difference, per axis ({what})", msd_rel, STATS_RTOL)
            record(label, scheme, f"clustering index difference / max(1, |C|) ({what})", c_rel,
                   STATS_RTOL)
            assert msd_rel < STATS_RTOL, (mark, k, msd_rel)
            assert c_rel < STATS_RTOL, (mark, k, c, row["cluster"])
            if "positions" in row:
                ref = np.asarray(row["positions"])
                pstride = gold["position_stride"]
                perr = float(np.max(np.abs(pos[::pstride] - ref)))
                record(label, scheme, f"max position error after {mark} steps (every species, "
                       f"every {pstride}th particle)", perr, None)


@pytest.mark.parametrize("scheme", [0, 1, 2])
def test_decaying_turbulence_1024_statistics_2000_steps(scheme):
    gold = golden("decaying_turbulence_1024")
    wl = inputs.decaying_turbulence_1024()
    assert gold["n"] == wl.n and [s["seed"] for s in gold["species"]] == [s.seed for s in wl.species]
    xys = [inputs.uniform_positions(s.count, s.seed) for s in wl.species]
    g = elpath.Flow(wl.n, wl.nu, wl.dt, wl.omega0(), interp=scheme, max_species=4,
                    max_particles=wl.particles, sort_every=SORT_EVERY)
    for k, s in enumerate(wl.species):
        g.set_particles(k, xys[k], s.st)
    compare_statistics("decaying_turbulence_1024", wl, gold, g, xys, scheme,
                       "decaying turbulence 1024^2, 4 x 1M (oracle: every 16th)")
    g.close()


def test_kelvin_helmholtz_2048_statistics_4000_steps():
    gold = golden("kelvin_helmholtz_2048")
    wl = inputs.kelvin_helmholtz_2048()
    sp = wl.species[0]
    xys = [inputs.uniform_positions(sp.count, sp.seed)]
    g = elpath.Flow(wl.n, wl.nu, wl.dt, wl.omega0(), interp=1, max_species=1,
                    max_particles=sp.count, sort_every=SORT_EVERY)
    g.set_particles(0, xys[0], sp.st)
    compare_statistics("kelvin_helmholtz_2048", wl, gold, g, xys, 1,
                       "shear layer 2048^2, 16M at St = 1 (oracle: every 64th)")
    g.close()


def test_ensemble_64_members_batched_equal_alone():
    wls = inputs.ensemble_members(64)
    steps = 30
    w0s = [wl.omega0() for wl in wls]
    xys = [inputs.uniform_positions(wl.species[0].count, wl.species[0].seed) for wl in wls]

    def member(m):
        wl, sp = wls[m], wls[m].species[0]
        g = elpath.Flow(wl.n, wl.nu, wl.dt, w0s[m], interp=0, max_species=1,
                        max_particles=sp.count, sort_every=SORT_EVERY)
        g.set_particles(0, xys[m], sp.st)
        return g

    batch = elpath.Batch(64)
    flows = [member(m) for m in range(64)]
    for n in (256, 512, 1024):          # one FFT pool per grid size of cuFFT members, as the benchmark
        k = sum(1 for wl, g in zip(wls, flows) if wl.n == n and not g.fused)
        if k:
            batch.add_fft_pool(n, k)
    for g in flows:
        batch.add(g)
    batch.step(steps)
    mixed = []
    for m, g in enumerate(flows):
        assert g.stats()["step"] == steps
        mixed.append((g.field(0), g.particles(0, wls[m].species[0].count)[0]))
    batch.close()
    for g in flows:
        g.close()
    torch.cuda.empty_cache()
    worst_w = worst_p = 0.0
    for m in range(64):
        g = member(m)
        g.step(steps)
        w, pos = g.field(0), g.particles(0, wls[m].species[0].count)[0]
        g.close()
        worst_w = max(worst_w, rel_linf(mixed[m][0], w))
        worst_p = max(worst_p, float(np.max(np.abs(mixed[m][1] - pos))))
    record("ensemble, 64 members, batched vs alone", 0, "omega L-inf rel., 30 steps", worst_w, OMEGA_RTOL)
    record("ensemble, 64 members, batched vs alone", 0, "max position difference, 30 steps",
           worst_p, POS_ATOL)
    assert worst_w < OMEGA_RTOL
    assert worst_p < POS_ATOL


def test_served_stream_first_16_requests_equal_alone():
    reqs = inputs.served_requests(count=16)
    pools = {128: 4}
    srv = serve.Server(hbm_budget=100 << 30, max_members=64, tick_steps=50, keep_positions=True,
                       fft_pool_slots=pools)
    results = srv.run(inputs.served_requests(count=16), time_scale=0.05, timeout=600)
    srv.close()
    torch.cuda.empty_cache()
    assert len(results) == 16
    overlapped = sum(1 for r in results if any(o.admitted < r.finished and r.admitted < o.finished
                                               for o in results if o.rid != r.rid))
    assert overlapped >= 8, "requests should have shared the GPU"
    by_id = {r.rid: r for r in results}
    worst_p = worst_e = 0.0
    for req in reqs:
        res = by_id[req.rid]
        g = serve.build_flow(req, None, "cuda")
        g.step(req.workload.steps)
        pos, _ = g.particles(0, req.workload.particles)
        st = g.stats()
        g.close()
        assert res.stats["step"] == req.workload.steps
        worst_p = max(worst_p, float(np.max(np.abs(res.positions - pos))))
        worst_e = max(worst_e, abs(res.stats["energy"] - st["energy"]) / st["energy"])
    name = "served stream, first 16 requests (128^2-2048^2, to 8.5M particles)"
    record(name, None, "max position difference, served vs alone", worst_p, POS_ATOL)
    record(name, None, "energy rel. difference, served vs alone", worst_e, 1e-6)
    assert worst_p <= POS_ATOL
    assert worst_e <= 1e-6
