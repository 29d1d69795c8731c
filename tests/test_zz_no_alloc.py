"""el_dispersion_noalloc: the dispersion statistics without any allocation.

Callers that cannot allocate device memory when they need these numbers (a
loop that must not stall, since cudaMalloc and cudaFree can synchronise the
whole device, or an application whose device memory is all reserved up front
by another allocator) call this entry point: its scratch is a fixed device
array inside the library.  This file checks, through the C ABI, that it
returns what el_get_stats returns for the same particles, on two calls in a
row (the shared scratch keeps the previous call's contents, so the second
call, on a different particle count, must not see them).  It is collected
last so that a run stopping at the first failure has run everything else.
"""
import numpy as np
import pytest

from paper_2607_17836_b300 import elpath, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

MSD_RTOL = 1e-12        # same FP64 terms, same fixed reduction order
CLUSTER_TOL = 1e-3      # as in the statistics parity tests


def _run_flow():
    n = 64
    w0 = inputs.decaying_turbulence(n, seed=31, k0=6.0)
    counts, sts = (5000, 3001), (1.0, 0.0)
    g = elpath.Flow(n, 1e-3, 1e-2, w0, interp=1, max_species=2, max_particles=sum(counts),
                    sort_every=5)
    xys = [inputs.uniform_positions(c, seed=40 + k) for k, c in enumerate(counts)]
    for k, (xy, st) in enumerate(zip(xys, sts)):
        g.set_particles(k, xy, st)
    g.step(60)
    return g, counts, xys


def test_noalloc_matches_get_stats_on_two_calls():
    g, counts, xys = _run_flow()
    stats = g.stats()
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    for k in (0, 1):          # two calls in a row, different particle counts
        pos, _ = g.particles(k, counts[k])
        xy = torch.from_numpy(pos).cuda()
        xy0 = torch.from_numpy(np.ascontiguousarray(xys[k])).cuda()
        elpath.dispersion_noalloc(xy, xy0, out=out)
        torch.cuda.synchronize()
        msd_x, msd_y, cluster = out.cpu().numpy()
        ref_x, ref_y = stats["msd"][k]
        assert abs(msd_x - ref_x) <= MSD_RTOL * ref_x
        assert abs(msd_y - ref_y) <= MSD_RTOL * ref_y
        assert abs(cluster - stats["cluster"][k]) <= CLUSTER_TOL * max(1.0, abs(stats["cluster"][k]))
    g.close()


def test_noalloc_replayed_from_a_captured_graph():
    """Called inside a stream capture (torch's default, global mode), after a
    first plain call: the graph's replay gives the plain call's bits (the
    scratch address is looked up in the capturing context, nothing is
    allocated)."""
    g, counts, xys = _run_flow()
    pos, _ = g.particles(0, counts[0])
    g.close()
    xy = torch.from_numpy(pos).cuda()
    xy0 = torch.from_numpy(np.ascontiguousarray(xys[0])).cuda()
    ref = elpath.dispersion_noalloc(xy, xy0).clone()
    torch.cuda.synchronize()
    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        elpath.dispersion_noalloc(xy, xy0, out=out)
    for _ in range(2):
        out.fill_(float("nan"))
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, ref)


def test_noalloc_empty_set_gives_zeros():
    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    xy = torch.zeros((0, 2), dtype=torch.float64, device="cuda")
    elpath.dispersion_noalloc(xy, xy, out=out)
    torch.cuda.synchronize()
    assert out.cpu().tolist() == [0.0, 0.0, 0.0]


def test_noalloc_positions_whole_periods_away():
    # Unwrapped positions several periods away from [0, 2 pi): the same
    # displacement from the same x(0) shifted alike, so the mean-square
    # displacement agrees to rounding, and the wrapped box counts (integers)
    # are the same, so the clustering index is bit-identical.
    g, counts, xys = _run_flow()
    pos, _ = g.particles(0, counts[0])
    g.close()
    rng = np.random.default_rng(7)
    shift = 2.0 * np.pi * rng.integers(-4, 5, size=(counts[0], 2)).astype(np.float64)
    outs = []
    for dx in (0.0, shift):
        xy = torch.from_numpy(np.ascontiguousarray(pos + dx)).cuda()
        xy0 = torch.from_numpy(np.ascontiguousarray(xys[0] + dx)).cuda()
        out = torch.empty(3, dtype=torch.float64, device="cuda")
        elpath.dispersion_noalloc(xy, xy0, out=out)
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy())
    np.testing.assert_allclose(outs[1][:2], outs[0][:2], rtol=1e-9)
    assert outs[1][2] == outs[0][2]


def test_noalloc_refuses_misaligned_positions():
    # Refused on the host before any launch: the kernels read 16-byte pairs.
    flat = torch.zeros(2 * 64 + 1, dtype=torch.float64, device="cuda")
    xy = flat[1:].view(64, 2)
    assert xy.data_ptr() % 16 == 8
    with pytest.raises(elpath.ElpathError) as e:
        elpath.dispersion_noalloc(xy, xy)
    assert e.value.status == 1
    assert "aligned" in str(e.value)


def test_noalloc_rejects_more_particles_than_its_scratch():
    n_big = elpath.NOALLOC_MAX_PARTICLES + 1
    xy = torch.zeros((n_big, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(elpath.ElpathError) as e:
        elpath.dispersion_noalloc(xy, xy)
    assert e.value.status == 1
    assert "scratch" in str(e.value)
