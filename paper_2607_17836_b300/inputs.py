"""Seeded synthetic inputs for the coupled Eulerian-Lagrangian workloads.

This module only draws and shapes input data: initial vorticity fields,
particle positions, ensembles and request streams.  It holds none of the
method's arithmetic (no time stepping, no interpolation, no diagnostics), so
both the CUDA path and the FP64 oracle can consume its output.  Every field
is FP64 on the host, row-major [j][i] (y slow, x fast) on the periodic square
[0, 2 pi)^2 with nodes x_i = i * 2 pi / n.  Randomness comes from numpy's
PCG64 generator seeded explicitly per call.
"""
from __future__ import annotations

import functools
import math
from dataclasses import dataclass, field

import numpy as np

TWO_PI = 2.0 * math.pi


def grid(n: int):
    """Node coordinates (X, Y), each n x n, X varying along the fast axis."""
    x = np.arange(n, dtype=np.float64) * (TWO_PI / n)
    return np.meshgrid(x, x, indexing="xy")


def taylor_green(n: int, amplitude: float = 2.0) -> np.ndarray:
    """omega = amplitude * sin(x) sin(y) (Taylor-Green vortex)."""
    X, Y = grid(n)
    return amplitude * np.sin(X) * np.sin(Y)


def _wavenumbers(n: int):
    k = np.fft.fftfreq(n, d=1.0 / n)
    KX, KY = np.meshgrid(k, k, indexing="xy")
    return KX, KY


def decaying_turbulence(n: int, seed: int, k0: float = 10.0, energy: float = 1.0) -> np.ndarray:
    """Random-phase vorticity with shell energy spectrum E(k) ~ k^4 exp(-(k/k0)^2).

    Mode amplitudes |omega_k| = |k| sqrt(E(|k|) / (pi |k|)) give E(k) per unit
    shell width; phases are uniform.  Only modes with 3|kx| < n and 3|ky| < n
    are drawn, so the field is unchanged by a 2/3 projection.  The real part
    of the synthesised field is taken and rescaled so that the kinetic energy
    integrated over the periodic domain, (2 pi)^2 * 1/2 <u^2 + v^2>, equals
    `energy` (the mean density 1/2 <u^2+v^2> = sum_{k != 0} |omega_k|^2 /
    (2 |k|^2) is then energy / (2 pi)^2).  With unit energy per unit area
    instead, max |u| ~ 4.8 at n = 1024 and dt = 5e-4 puts the highest kept
    modes at an advective CFL number ~1.5, outside the stability region of
    the AB2 scheme: the FP64 solve overflows within ~200 steps.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    band, amp_band, k2_band = _shell_spectrum(n, float(k0))
    phase = rng.uniform(0.0, TWO_PI, size=(n, n))
    z = np.zeros((n, n), dtype=np.complex128)  # zero outside the band
    z[band] = amp_band * np.exp(1j * phase[band])
    # Coefficients of the real part: (z_k + conj(z_{-k})) / 2, with
    # z_{-k}[j][i] = z[-j mod n][-i mod n].
    zneg = np.roll(z[::-1, ::-1], 1, axis=(0, 1))
    zr = 0.5 * (z + np.conj(zneg))
    e_mean = 0.5 * np.sum(np.abs(zr[band]) ** 2 / k2_band)
    zr *= math.sqrt(energy / (TWO_PI * TWO_PI) / e_mean)
    omega = np.real(np.fft.ifft2(zr)) * (n * n)
    return np.ascontiguousarray(omega)


@functools.lru_cache(maxsize=8)
def _shell_spectrum(n: int, k0: float):
    """The parts of decaying_turbulence that depend on (n, k0) only, computed
    once per grid: the drawn band (3|kx| < n, 3|ky| < n, k != 0), the mode
    amplitudes |k| sqrt(E(|k|) / (pi |k|)) on it and |k|^2 on it (read-only)."""
    KX, KY = _wavenumbers(n)
    kmag = np.hypot(KX, KY)
    band = (3 * np.abs(KX) < n) & (3 * np.abs(KY) < n) & (kmag > 0)
    shell = np.where(band, kmag ** 4 * np.exp(-(kmag / k0) ** 2), 0.0)
    amp = np.where(band, kmag * np.sqrt(shell / (np.pi * np.maximum(kmag, 1.0))), 0.0)
    out = (band, amp[band], kmag[band] ** 2)
    for a in out:
        a.setflags(write=False)
    return out


def kelvin_helmholtz(n: int, seed: int, delta: float = math.pi / 50, amp: float = 1e-3,
                     kx: int = 4) -> np.ndarray:
    """Double shear layer u = tanh((y - pi/2)/delta) - tanh((y - 3pi/2)/delta) - 1.

    Its vorticity is omega = -du/dy = -(1/delta)[sech^2((y - pi/2)/delta)
    - sech^2((y - 3pi/2)/delta)].  Added perturbation, relative to the peak
    shear vorticity 1/delta: amp * (sin(kx x) + r), r ~ U[-1, 1] per node.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    X, Y = grid(n)
    sech2 = lambda s: 1.0 / np.cosh(s) ** 2
    base = -(1.0 / delta) * (sech2((Y - math.pi / 2) / delta) - sech2((Y - 3 * math.pi / 2) / delta))
    r = rng.uniform(-1.0, 1.0, size=(n, n))
    return np.ascontiguousarray(base + amp * (1.0 / delta) * (np.sin(kx * X) + r))


def uniform_positions(count: int, seed: int) -> np.ndarray:
    """count x 2 FP64 positions, uniform on [0, 2 pi)^2."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(0.0, TWO_PI, size=(int(count), 2))


# --- workload descriptions -----------------------------------------------------
@dataclass
class SpeciesSpec:
    count: int
    st: float
    seed: int


@dataclass
class Workload:
    name: str
    n: int
    nu: float
    dt: float
    steps: int
    ic: str                   # "taylor_green" | "decaying_turbulence" | "kelvin_helmholtz"
    ic_seed: int
    species: list = field(default_factory=list)
    schemes: tuple = (0,)     # interpolation schemes run on this workload

    def omega0(self) -> np.ndarray:
        if self.ic == "taylor_green":
            return taylor_green(self.n)
        if self.ic == "decaying_turbulence":
            return decaying_turbulence(self.n, self.ic_seed)
        if self.ic == "kelvin_helmholtz":
            return kelvin_helmholtz(self.n, self.ic_seed)
        raise ValueError(self.ic)

    @property
    def particles(self) -> int:
        return sum(s.count for s in self.species)


def taylor_green_64() -> Workload:
    """64^2 Taylor-Green, nu=0.01, dt=1e-3, 200 steps, 4096 tracers, bilinear."""
    return Workload("taylor_green_64", 64, 0.01, 1e-3, 200, "taylor_green", 0,
                    [SpeciesSpec(4096, 0.0, 1)], (0,))


def decaying_turbulence_1024(scale: float = 1.0) -> Workload:
    """1024^2 decaying turbulence, nu=1e-4, dt=5e-4, 2000 steps; 1M tracers and
    1M inertial particles at each St in {0.1, 1, 10}; all three schemes.
    `scale` shrinks the particle counts (for tests)."""
    c = max(1, int(round(1_000_000 * scale)))
    return Workload("decaying_turbulence_1024", 1024, 1e-4, 5e-4, 2000, "decaying_turbulence", 2,
                    [SpeciesSpec(c, 0.0, 3), SpeciesSpec(c, 0.1, 4), SpeciesSpec(c, 1.0, 5),
                     SpeciesSpec(c, 10.0, 6)], (0, 1, 2))


def kelvin_helmholtz_2048(scale: float = 1.0) -> Workload:
    """2048^2 double shear layer, nu=5e-5, dt=2.5e-4, 4000 steps, 16M inertial
    particles at St=1, Catmull-Rom."""
    c = max(1, int(round(16_000_000 * scale)))
    return Workload("kelvin_helmholtz_2048", 2048, 5e-5, 2.5e-4, 4000, "kelvin_helmholtz", 7,
                    [SpeciesSpec(c, 1.0, 8)], (1,))


def ensemble_members(count: int = 64, seed: int = 1000):
    """Independent decaying-turbulence members: n from {256, 512, 1024},
    particle count log-uniform in [1e4, 1e6], St from {0, 0.1, 1, 10};
    member m uses IC seed 1000 + m."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for m in range(count):
        n = int(rng.choice([256, 512, 1024]))
        npart = int(round(10 ** rng.uniform(4.0, 6.0)))
        st = float(rng.choice([0.0, 0.1, 1.0, 10.0]))
        out.append(Workload(f"member{m}", n, 1e-4, 5e-4, 0, "decaying_turbulence", 1000 + m,
                            [SpeciesSpec(npart, st, 2000 + m)], (0,)))
    return out


@dataclass
class Request:
    rid: int
    arrival: float            # seconds after the stream starts
    workload: Workload
    scheme: int


def served_requests(count: int = 2000, rate: float = 20.0, seed: int = 5000,
                    grids=(128, 256, 512, 1024, 2048), max_particles: float = 1e7,
                    steps=(100, 2000)):
    """Poisson arrival stream of coupled simulations: n from `grids`, particle
    count log-uniform in [1e3, max_particles], St from {0, 0.1, 1, 10},
    bilinear or Catmull-Rom, steps uniform in `steps`."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for r in range(count):
        t += float(rng.exponential(1.0 / rate))
        n = int(rng.choice(list(grids)))
        npart = int(round(10 ** rng.uniform(3.0, math.log10(max_particles))))
        st = float(rng.choice([0.0, 0.1, 1.0, 10.0]))
        scheme = int(rng.choice([0, 1]))
        nsteps = int(rng.integers(steps[0], steps[1] + 1))
        wl = Workload(f"req{r}", n, 1e-4, 5e-4, nsteps, "decaying_turbulence", seed + 1 + r,
                      [SpeciesSpec(npart, st, seed + 100000 + r)], (scheme,))
        out.append(Request(r, t, wl, scheme))
    return out
