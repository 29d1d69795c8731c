"""Continuous-batching server: every request finishes with the result it has
when run alone, requests arriving while others run are admitted as memory
frees up, and the HBM budget is never exceeded."""
import numpy as np
import pytest

from paper_2607_17836_b300 import elpath, inputs, serve
from parity import POS_ATOL

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def small_stream(count=12):
    return inputs.served_requests(count=count, rate=200.0, seed=77, grids=(32, 64, 128),
                                  max_particles=2e4, steps=(10, 60))


@pytest.mark.parametrize("pools", [None, {32: 2, 64: 2, 128: 2}], ids=["own_ffts", "fft_pools"])
def test_served_results_equal_solo_runs_and_budget_holds(pools):
    # with FFT pools, members of a grid size that find a free slot transform
    # together (the pools' memory counts against the budget)
    reqs = small_stream()
    need = [elpath.workspace_bytes(serve.request_desc(r)) for r in reqs]
    pool_bytes = 0
    if pools:
        probe = elpath.Batch(1)
        pool_bytes = sum(probe.add_fft_pool(n, k) for n, k in pools.items())
        probe.close()
    budget = int(2.5 * max(need)) + pool_bytes     # forces queueing: only a few fit at once
    srv = serve.Server(hbm_budget=budget, max_members=8, tick_steps=7, keep_positions=True,
                       fft_pool_slots=pools)
    results = srv.run(small_stream(), time_scale=1.0, timeout=300)
    srv.close()
    assert len(results) == len(reqs)
    assert srv.peak_used <= budget
    admitted_late = [r for r in results if r.admitted > r.arrival + 1e-3]
    assert admitted_late, "the budget should have made some requests wait"
    by_id = {r.rid: r for r in results}
    for req in reqs:
        res = by_id[req.rid]
        g = serve.build_flow(req, None, "cuda")
        g.step(req.workload.steps)
        pos, _ = g.particles(0, req.workload.particles)
        st = g.stats()
        g.close()
        assert res.stats["step"] == req.workload.steps
        assert np.max(np.abs(res.positions - pos)) <= POS_ATOL
        assert abs(res.stats["energy"] - st["energy"]) <= 1e-6 * st["energy"]
    summary = serve.latency_summary(results)
    assert summary["count"] == len(reqs) and summary["p99_s"] >= summary["p50_s"] > 0
