"""Host-side parts of the serving loop that need no GPU: the latency summary
(time-to-result = finish - arrival, percentiles by linear interpolation),
each request's flow descriptor, and its seeded host inputs."""
import numpy as np
import pytest

from paper_2607_17836_b300 import inputs, serve


def result(rid, arrival, finished):
    return serve.Result(rid=rid, arrival=arrival, admitted=arrival, finished=finished, steps=1,
                        particles=1, n=32, stats={})


def test_latency_summary():
    # latencies 1, 2, ..., 100 s: p50 = 50.5, p99 = 99.01 (linear interpolation)
    res = [result(k, 10.0 * k, 10.0 * k + (k + 1)) for k in range(100)]
    s = serve.latency_summary(res)
    assert s["count"] == 100
    assert s["p50_s"] == pytest.approx(50.5)
    assert s["p99_s"] == pytest.approx(99.01)
    assert s["mean_s"] == pytest.approx(50.5)
    assert s["max_s"] == pytest.approx(100.0)
    assert serve.latency_summary([]) == {"count": 0}


def test_latency_splits_into_queue_wait_and_service():
    # request k waits k s for admission, then runs 2 s: wait p50 = 49.5,
    # service 2 everywhere, and wait + service = time-to-result
    res = [serve.Result(rid=k, arrival=5.0 * k, admitted=6.0 * k, finished=6.0 * k + 2.0, steps=1,
                        particles=1, n=32, stats={}) for k in range(100)]
    s = serve.latency_summary(res)
    assert s["queue_wait"]["p50_s"] == pytest.approx(49.5)
    assert s["queue_wait"]["max_s"] == pytest.approx(99.0)
    assert s["service"]["p50_s"] == pytest.approx(2.0) and s["service"]["p99_s"] == pytest.approx(2.0)
    assert s["p50_s"] == pytest.approx(51.5)
    for r in res:
        assert r.queue_wait + r.service == pytest.approx(r.latency)


def test_request_descriptor_and_inputs():
    req = inputs.served_requests(count=5, seed=321)[3]
    d = serve.request_desc(req)
    wl = req.workload
    assert (d.n, d.interp, d.max_species, d.max_particles) == (wl.n, req.scheme, 1, wl.particles)
    assert (d.nu, d.dt) == (wl.nu, wl.dt)
    w0, xy = serve.prepare_inputs(req)
    np.testing.assert_array_equal(w0, wl.omega0())
    sp = wl.species[0]
    np.testing.assert_array_equal(xy, inputs.uniform_positions(sp.count, sp.seed))
