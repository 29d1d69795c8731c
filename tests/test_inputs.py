"""The seeded synthetic inputs against their stated recipes (CPU only): the
decaying-turbulence field's shell spectrum is k^4 exp(-(k/k0)^2) up to
random-phase noise, with no energy outside the 2/3 band and zero mean; the
double shear layer's x-averaged vorticity is -du/dy of its tanh velocity
profile; particle positions are uniform on the periodic square; the served
stream's arrivals are Poisson with the stated rate and its draws come from
the stated sets and ranges, as do the ensemble members'."""
import math

import numpy as np
import pytest

from paper_2607_17836_b300 import inputs


def test_decaying_turbulence_spectrum_band_and_mean():
    n, k0 = 256, 10.0
    w = inputs.decaying_turbulence(n, seed=21, k0=k0)
    wh = np.fft.fft2(w) / (n * n)
    k = np.fft.fftfreq(n, d=1.0 / n)
    KX, KY = np.meshgrid(k, k, indexing="xy")
    kmag = np.hypot(KX, KY)
    band = (3 * np.abs(KX) < n) & (3 * np.abs(KY) < n)
    assert abs(wh[0, 0]) < 1e-12 * np.max(np.abs(wh))                  # zero mean
    assert np.max(np.abs(wh[~band])) < 1e-12 * np.max(np.abs(wh))      # nothing outside 2/3
    e = np.where(kmag > 0, np.abs(wh) ** 2 / (2 * np.maximum(kmag, 1e-30) ** 2), 0.0)
    # per mode the recipe puts energy E(k) / (pi k) with E(k) = k^4 exp(-(k/k0)^2)
    target = np.where((kmag > 0) & band,
                      kmag ** 4 * np.exp(-(kmag / k0) ** 2) / (np.pi * np.maximum(kmag, 1e-30)), 0.0)
    shell = np.rint(kmag).astype(int)
    meas, want, count = (np.bincount(shell.ravel(), weights=a.ravel()) for a in
                         (e, target, np.ones_like(e)))
    scale = meas[1:40].sum() / want[1:40].sum()
    checked = 0
    for s in range(1, 40):
        if count[s] < 50 or want[s] < 1e-3 * want.max():
            continue
        ratio = meas[s] / (scale * want[s])
        assert abs(ratio - 1.0) < 5.0 / math.sqrt(count[s]), (s, ratio, count[s])
        checked += 1
    assert checked >= 15
    # and the steep fall beyond the peak, shell 30 against shell 16: a shell
    # holds E(s) = s^4 exp(-(s/k0)^2) times (its lattice modes) / (2 pi s)
    shell_e = lambda s: s ** 4 * math.exp(-(s / k0) ** 2) * count[s] / (2 * math.pi * s)
    assert meas[30] / meas[16] == pytest.approx(shell_e(30) / shell_e(16), rel=0.4)


def test_shear_layer_vorticity_is_minus_du_dy():
    n, delta, amp = 512, math.pi / 50, 1e-3
    w = inputs.kelvin_helmholtz(n, seed=7, delta=delta, amp=amp)
    y = np.arange(n) * (2 * math.pi / n)
    u = lambda yy: np.tanh((yy - math.pi / 2) / delta) - np.tanh((yy - 3 * math.pi / 2) / delta) - 1.0
    h = 1e-6
    minus_dudy = -(u(y + h) - u(y - h)) / (2 * h)           # by differencing, not by formula
    mean_x = w.mean(axis=1)                                # rows are y, columns x
    # the sin(4x) part averages to 0 over the row; the U[-1, 1] part to
    # about amp/delta * 3/sqrt(n)
    assert np.max(np.abs(mean_x - minus_dudy)) < amp / delta * 6.0 / math.sqrt(n) + 1e-6 / delta
    assert np.max(np.abs(minus_dudy)) == pytest.approx(1.0 / delta, rel=1e-3)


def test_positions_are_uniform_on_the_square():
    xy = inputs.uniform_positions(400_000, seed=5)
    assert xy.shape == (400_000, 2)
    assert xy.min() >= 0.0 and xy.max() < 2 * math.pi
    counts, _, _ = np.histogram2d(xy[:, 0], xy[:, 1], bins=4, range=[[0, 2 * math.pi]] * 2)
    expect = 400_000 / 16
    assert np.max(np.abs(counts - expect)) < 5 * math.sqrt(expect)
    a, b = inputs.uniform_positions(1000, 9), inputs.uniform_positions(1000, 9)
    np.testing.assert_array_equal(a, b)                                  # seeded
    assert not np.array_equal(a, inputs.uniform_positions(1000, 10))


def test_served_stream_recipe():
    # Poisson arrivals at 20/s: exponential gaps of mean 1/20 (the mean of
    # 2000 gaps within 5 standard errors); grids, schemes, Stokes numbers from
    # their sets; particle counts log-uniform in [1e3, 1e7]; steps in range
    reqs = inputs.served_requests(count=2000)
    t = np.array([r.arrival for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert abs(gaps.mean() - 0.05) < 5 * 0.05 / math.sqrt(len(gaps))
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1          # exponential: std = mean
    assert {r.workload.n for r in reqs} == {128, 256, 512, 1024, 2048}
    assert {r.scheme for r in reqs} == {0, 1}
    assert {r.workload.species[0].st for r in reqs} == {0.0, 0.1, 1.0, 10.0}
    lg = np.log10([r.workload.species[0].count for r in reqs])
    assert lg.min() >= 3.0 - 1e-9 and lg.max() <= 7.0 + 1e-9
    assert abs(lg.mean() - 5.0) < 5 * (4 / math.sqrt(12)) / math.sqrt(len(lg))
    steps = np.array([r.workload.steps for r in reqs])
    assert steps.min() >= 100 and steps.max() <= 2000
    assert [r.rid for r in reqs] == list(range(2000))


def test_ensemble_members_recipe():
    ms = inputs.ensemble_members(64)
    assert len(ms) == 64
    assert {m.n for m in ms} <= {256, 512, 1024} and len({m.n for m in ms}) == 3
    assert [m.ic_seed for m in ms] == [1000 + k for k in range(64)]     # per-member seeds
    counts = np.array([m.species[0].count for m in ms])
    assert counts.min() >= 10_000 and counts.max() <= 1_000_000
    assert {m.species[0].st for m in ms} <= {0.0, 0.1, 1.0, 10.0}


def _decaying_turbulence_plain(n, seed, k0=10.0, energy=1.0):
    # the recipe over the full (n, n) arrays, as decaying_turbulence states it
    rng = np.random.Generator(np.random.PCG64(seed))
    k = np.fft.fftfreq(n, d=1.0 / n)
    KX, KY = np.meshgrid(k, k, indexing="xy")
    kmag = np.hypot(KX, KY)
    band = (3 * np.abs(KX) < n) & (3 * np.abs(KY) < n) & (kmag > 0)
    shell = np.where(band, kmag ** 4 * np.exp(-(kmag / k0) ** 2), 0.0)
    amp = np.where(band, kmag * np.sqrt(shell / (np.pi * np.maximum(kmag, 1.0))), 0.0)
    z = amp * np.exp(1j * rng.uniform(0.0, 2 * math.pi, size=(n, n)))
    zneg = z[(-np.arange(n)) % n][:, (-np.arange(n)) % n]
    zr = 0.5 * (z + np.conj(zneg))
    zr *= math.sqrt(energy / (4 * math.pi ** 2) / (0.5 * np.sum(np.abs(zr[band]) ** 2 / kmag[band] ** 2)))
    return np.real(np.fft.ifft2(zr)) * (n * n)


@pytest.mark.parametrize("n, seed, k0", [(64, 3, 6.0), (128, 7, 10.0), (256, 1005, 10.0)])
def test_decaying_turbulence_equals_its_plain_recipe(n, seed, k0):
    # the generator draws only the 2/3 band and caches what depends on the
    # grid alone; the field is the plain recipe's, bit for bit (the stored
    # oracle statistics were computed from it)
    a = inputs.decaying_turbulence(n, seed, k0=k0)
    b = _decaying_turbulence_plain(n, seed, k0)
    assert np.array_equal(a, b) and np.array_equal(np.signbit(a), np.signbit(b))
    assert np.array_equal(inputs.decaying_turbulence(n, seed, k0=k0), a)   # again, from the cache
