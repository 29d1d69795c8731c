"""FP64 CPU oracle for the coupled Eulerian-Lagrangian method (arxiv 2607.17836).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
restatement of the method that the CUDA library is checked against.  Only the
test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline /
reference leg may import it; the product path never does.  It shares no code
with the CUDA library: the arithmetic lives in ``oracle.c`` (its own radix-2
FFT, direct stencils, RK4), compiled here with gcc, and this module only
marshals arrays and adds the particle statistics.

Readings of the paper that the oracle takes (where the paper is silent):
  * first AB2 step is forward Euler;
  * 2/3 rule = square mask 3|kx| < N and 3|ky| < N;
  * the Nyquist mode gets a zero derivative;
  * cubic stencils wrap periodically (no bilinear fallback at the seam);
  * B-spline weights act on interpolating coefficients (prefilter) unless
    ``bspline_prefilter=False`` (raw samples, as the paper's Eq. 21 reads);
  * zero slip: an inertial particle starts with the interpolated fluid
    velocity at its start position;
  * MSD = <|x(t) - x(0)|^2> over unwrapped positions, per axis;
  * clustering index = Var(n)/mean(n) - 1 of the counts n on a 64 x 64 box
    grid (0 for a Poisson distribution).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

BILINEAR, CATMULL_ROM, BSPLINE = 0, 1, 2
TWO_PI = 2.0 * np.pi


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, OpenMP); return its path."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        D = ctypes.POINTER(ctypes.c_double)
        I64 = ctypes.c_int64
        lib.orc_fft1.argtypes = [D, D, ctypes.c_int, ctypes.c_int]
        lib.orc_fft2.argtypes = [D, D, ctypes.c_int, ctypes.c_int]
        lib.orc_flow_new.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, D]
        lib.orc_flow_new.restype = ctypes.c_void_p
        lib.orc_flow_free.argtypes = [ctypes.c_void_p]
        lib.orc_flow_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
        lib.orc_flow_step_count.argtypes = [ctypes.c_void_p]
        lib.orc_flow_step_count.restype = I64
        lib.orc_flow_fields.argtypes = [ctypes.c_void_p, D, D, D, D, D]
        lib.orc_flow_get_spectrum.argtypes = [ctypes.c_void_p, D, D]
        lib.orc_flow_nonlinear.argtypes = [ctypes.c_void_p, D]
        lib.orc_flow_diagnostics.argtypes = [ctypes.c_void_p, D]
        lib.orc_interp.argtypes = [ctypes.c_int, D, ctypes.c_int, ctypes.c_double, ctypes.c_double]
        lib.orc_interp.restype = ctypes.c_double
        lib.orc_interp_many.argtypes = [ctypes.c_int, D, ctypes.c_int, I64, D, D, D]
        lib.orc_bspline_prefilter.argtypes = [ctypes.c_int, D]
        lib.orc_particles_rk4.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                          D, D, D, D, I64, D, D, D, D]
        lib.orc_flow_psi.argtypes = [ctypes.c_void_p, D]
        lib.orc_psi_velocity_many.argtypes = [ctypes.c_int, ctypes.c_int, D, I64, D, D, D, D]
        lib.orc_tracers_rk4_psi.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, D, D, I64,
                                            D, D]
        lib.orc_num_threads.restype = ctypes.c_int
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        _lib = lib
        return lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return _load().orc_num_threads()


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


# --- FFT ------------------------------------------------------------------
def fft1(x, sign=-1):
    """Radix-2 transform of a 1-D complex array: sum_j x_j exp(sign 2 pi i jk/n)."""
    x = np.asarray(x, dtype=np.complex128)
    re, im = _f64(x.real.copy()), _f64(x.imag.copy())
    _load().orc_fft1(_p(re), _p(im), int(x.shape[0]), int(sign))
    return re + 1j * im


def fft2(x, sign=-1):
    """Radix-2 2-D transform (rows, then columns) of an n x n complex array."""
    x = np.asarray(x, dtype=np.complex128)
    re, im = _f64(x.real.copy()), _f64(x.imag.copy())
    _load().orc_fft2(_p(re), _p(im), int(x.shape[0]), int(sign))
    return re + 1j * im


# --- interpolation ----------------------------------------------------------
def interp(f, scheme, x, y):
    """Interpolate the periodic n x n grid function f ([j][i]) at points (x, y)."""
    f = _f64(f)
    x, y = _f64(np.atleast_1d(x)), _f64(np.atleast_1d(y))
    out = np.empty_like(x)
    _load().orc_interp_many(int(f.shape[0]), _p(f), int(scheme), int(x.size), _p(x), _p(y), _p(out))
    return out


def bspline_prefilter(f):
    """Interpolating cubic B-spline coefficients of the periodic grid function f."""
    c = _f64(f).copy()
    _load().orc_bspline_prefilter(int(c.shape[0]), _p(c))
    return c


def particles_rk4(scheme, dt, st, un, vn, un1, vn1, x, y, vx=None, vy=None):
    """One RK4 step in place on unwrapped positions (and velocities if st > 0)."""
    n = int(un.shape[0])
    arrs = [_f64(a) for a in (un, vn, un1, vn1)]
    for a in (x, y) + ((vx, vy) if st > 0 else ()):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    _load().orc_particles_rk4(n, int(scheme), float(dt), float(st), *[_p(a) for a in arrs],
                              int(x.size), _p(x), _p(y), _p(vx) if st > 0 else None,
                              _p(vy) if st > 0 else None)


def psi_velocity(psi, scheme, x, y):
    """Tracer velocity from the streamfunction grid function by Eq. 11."""
    psi = _f64(psi)
    x, y = _f64(np.atleast_1d(x)), _f64(np.atleast_1d(y))
    u, v = np.empty_like(x), np.empty_like(x)
    _load().orc_psi_velocity_many(int(psi.shape[0]), int(scheme), _p(psi), int(x.size), _p(x),
                                  _p(y), _p(u), _p(v))
    return u, v


def tracers_rk4_psi(scheme, dt, psin, psin1, x, y):
    """One RK4 step in place of tracers driven by the streamfunction (Eq. 11)."""
    a, b = _f64(psin), _f64(psin1)
    assert x.dtype == np.float64 and y.dtype == np.float64
    _load().orc_tracers_rk4_psi(int(a.shape[0]), int(scheme), float(dt), _p(a), _p(b), int(x.size),
                                _p(x), _p(y))


# --- fluid --------------------------------------------------------------------
class Flow:
    """Pseudospectral AB2 vorticity solver on the periodic [0, 2 pi)^2 grid."""

    def __init__(self, n, nu, dt, omega0, ab2_mode=0):
        self.n, self.nu, self.dt, self.ab2_mode = int(n), float(nu), float(dt), int(ab2_mode)
        if self.n < 4 or self.n & (self.n - 1):
            raise ValueError("n must be a power of two >= 4")
        w0 = _f64(omega0)
        assert w0.shape == (self.n, self.n)
        self._lib = _load()
        self._h = self._lib.orc_flow_new(self.n, self.nu, self.dt, self.ab2_mode, _p(w0))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_flow_free(h)
            self._h = None

    @property
    def step_count(self) -> int:
        return int(self._lib.orc_flow_step_count(self._h))

    def step(self, nsteps=1):
        self._lib.orc_flow_step(self._h, int(nsteps))

    def fields(self, which=("u", "v", "w")):
        n = self.n
        out = {k: np.empty((n, n)) for k in which}
        ptrs = [_p(out.get(k)) for k in ("u", "v", "w", "wx", "wy")]
        self._lib.orc_flow_fields(self._h, *ptrs)
        return out

    def psi(self):
        out = np.empty((self.n, self.n))
        self._lib.orc_flow_psi(self._h, _p(out))
        return out

    def spectrum(self):
        n = self.n
        re, im = np.empty((n, n)), np.empty((n, n))
        self._lib.orc_flow_get_spectrum(self._h, _p(re), _p(im))
        return re + 1j * im

    def nonlinear(self):
        out = np.empty((self.n, self.n))
        self._lib.orc_flow_nonlinear(self._h, _p(out))
        return out

    def diagnostics(self):
        out = np.empty(3)
        self._lib.orc_flow_diagnostics(self._h, _p(out))
        return float(out[0]), float(out[1]), float(out[2])


# --- statistics ------------------------------------------------------------------
def msd(x, y, x0, y0):
    """Mean-square displacement of unwrapped trajectories, per axis (x, y)."""
    dx, dy = np.asarray(x) - np.asarray(x0), np.asarray(y) - np.asarray(y0)
    return float(np.mean(dx * dx)), float(np.mean(dy * dy))


def msd_sem(x, y, x0, y0):
    """Standard error of the per-axis mean-square displacement (Sec. 5.5):
    the sample standard deviation of the squared displacements over the
    particles divided by sqrt(np); two-pass (mean first, then the squared
    deviations).  0 for fewer than two particles."""
    out = []
    for a, a0 in ((x, x0), (y, y0)):
        d = np.asarray(a, dtype=np.float64) - np.asarray(a0, dtype=np.float64)
        q = d * d
        m = q.size
        if m < 2:
            out.append(0.0)
            continue
        mean = q.sum() / m
        var = ((q - mean) ** 2).sum() / (m - 1)
        out.append(float(np.sqrt(var / m)))
    return tuple(out)


def diffusivity(msd_xy, t):
    """D_i = <(x_i - x_i0)^2> / (2 t) per axis (Sec. 5.5, Sec. 6), 0 at t = 0."""
    return tuple((m / (2.0 * t)) if t > 0 else 0.0 for m in msd_xy)


def cluster_index(x, y, boxes=64):
    """Var(n)/mean(n) - 1 of particle counts on a boxes x boxes grid of the
    periodic domain (0 for uniformly random positions)."""
    xw = np.mod(np.asarray(x, dtype=np.float64), TWO_PI)
    yw = np.mod(np.asarray(y, dtype=np.float64), TWO_PI)
    bx = np.minimum((xw * (boxes / TWO_PI)).astype(np.int64), boxes - 1)
    by = np.minimum((yw * (boxes / TWO_PI)).astype(np.int64), boxes - 1)
    counts = np.bincount(by * boxes + bx, minlength=boxes * boxes).astype(np.float64)
    m = counts.mean()
    return float(counts.var() / m - 1.0) if m > 0 else 0.0


# --- the prescribed kinematic flow (Sec. 5.2) -------------------------------------
# psi = (alpha/k) sin(k[x - eps sin(omega t)]) sin(k[y - eps sin(omega t + phi)]),
# u = d psi/dy, v = -d psi/dx, written out term by term.
def kinematic_velocity(x, y, t, alpha, k, eps, omega, phi=0.0):
    """(u, v) of the oscillating Taylor-Green flow at points (x, y), time t."""
    ax = k * (np.asarray(x, dtype=np.float64) - eps * np.sin(omega * t))
    ay = k * (np.asarray(y, dtype=np.float64) - eps * np.sin(omega * t + phi))
    return alpha * np.sin(ax) * np.cos(ay), -alpha * np.cos(ax) * np.sin(ay)


def kinematic_fields(n, t, alpha, k, eps, omega, phi=0.0):
    """u, v, psi and omega = -laplacian(psi) on the n x n grid ([j][i]) at time t."""
    xs = np.arange(n) * (TWO_PI / n)
    x, y = np.meshgrid(xs, xs)  # x varies along i (columns), y along j (rows)
    ax = k * (x - eps * np.sin(omega * t))
    ay = k * (y - eps * np.sin(omega * t + phi))
    psi = (alpha / k) * np.sin(ax) * np.sin(ay)
    u = alpha * np.sin(ax) * np.cos(ay)
    v = -alpha * np.cos(ax) * np.sin(ay)
    return {"u": u, "v": v, "psi": psi, "omega": 2.0 * k * k * psi}


def tracers_rk4_analytic(dt, t, x, y, alpha, k, eps, omega, phi=0.0):
    """One classical RK4 step (Eq. 12) of tracers in the prescribed field,
    stages at t, t + dt/2, t + dt/2, t + dt; returns the new (x, y)."""
    vel = lambda px, py, tt: kinematic_velocity(px, py, tt, alpha, k, eps, omega, phi)
    k1 = vel(x, y, t)
    k2 = vel(x + 0.5 * dt * k1[0], y + 0.5 * dt * k1[1], t + 0.5 * dt)
    k3 = vel(x + 0.5 * dt * k2[0], y + 0.5 * dt * k2[1], t + 0.5 * dt)
    k4 = vel(x + dt * k3[0], y + dt * k3[1], t + dt)
    return (x + dt / 6.0 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0]),
            y + dt / 6.0 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1]))


class KinematicRun:
    """Tracers in the prescribed kinematic flow by one of the three routes of
    Sec. 5.2: "analytic" (the field at the particle), "velocity" (u, v on the
    grid, interpolated in space and blended in time) or "psi" (the
    streamfunction on the grid, interpolated, Eq. 11)."""

    def __init__(self, n, dt, params, xy, approach="analytic", scheme=BILINEAR, prefilter=True):
        self.n, self.dt, self.p = int(n), float(dt), dict(params)
        self.p.setdefault("phi", 0.0)
        self.approach, self.scheme, self.prefilter = approach, int(scheme), bool(prefilter)
        xy = np.asarray(xy, dtype=np.float64).reshape(-1, 2)
        self.x, self.y = xy[:, 0].copy(), xy[:, 1].copy()
        self.x0, self.y0 = self.x.copy(), self.y.copy()
        self.step_count = 0
        self._level = self._grid(0.0) if approach != "analytic" else None

    def _grid(self, t):
        f = kinematic_fields(self.n, t, **self.p)
        pre = self.scheme == BSPLINE and self.prefilter
        fix = (lambda a: bspline_prefilter(a)) if pre else (lambda a: a)
        if self.approach == "psi":
            return fix(f["psi"])
        return fix(f["u"]), fix(f["v"])

    @property
    def t(self):
        return self.step_count * self.dt

    def step(self, nsteps=1):
        for _ in range(int(nsteps)):
            t0 = self.t
            if self.approach == "analytic":
                self.x, self.y = tracers_rk4_analytic(self.dt, t0, self.x, self.y, **self.p)
            else:
                nxt = self._grid(t0 + self.dt)
                if self.approach == "psi":
                    tracers_rk4_psi(self.scheme, self.dt, self._level, nxt, self.x, self.y)
                else:
                    particles_rk4(self.scheme, self.dt, 0.0, self._level[0], self._level[1], nxt[0],
                                  nxt[1], self.x, self.y)
                self._level = nxt
            self.step_count += 1


# --- coupled driver (Algorithm 1) -------------------------------------------------
class Species:
    def __init__(self, xy, st, v0):
        xy = np.asarray(xy, dtype=np.float64).reshape(-1, 2)
        self.st = float(st)
        self.x = np.ascontiguousarray(xy[:, 0].copy())
        self.y = np.ascontiguousarray(xy[:, 1].copy())
        self.x0, self.y0 = self.x.copy(), self.y.copy()
        if self.st > 0:
            self.vx = np.ascontiguousarray(v0[0], dtype=np.float64)
            self.vy = np.ascontiguousarray(v0[1], dtype=np.float64)
        else:
            self.vx = self.vy = None


class Coupled:
    """One-way coupled step of Algorithm 1: advance the fluid n -> n+1, then
    every particle species by one RK4 step between the two field levels."""

    def __init__(self, n, nu, dt, omega0, scheme=BILINEAR, ab2_mode=0, bspline_prefilter=True,
                 tracer_velocity=0):
        self.flow = Flow(n, nu, dt, omega0, ab2_mode)
        self.n, self.dt, self.scheme = int(n), float(dt), int(scheme)
        self.prefilter = bool(bspline_prefilter)
        self.tracer_psi = bool(tracer_velocity)
        self.species: list[Species] = []
        self._level = self._stencil_fields()
        self._psi = self._psi_field()

    def _psi_field(self):
        if not self.tracer_psi:
            return None
        p = self.flow.psi()
        return bspline_prefilter(p) if self.scheme == BSPLINE and self.prefilter else p

    def _stencil_fields(self):
        f = self.flow.fields(("u", "v"))
        u, v = f["u"], f["v"]
        if self.scheme == BSPLINE and self.prefilter:
            u, v = bspline_prefilter(u), bspline_prefilter(v)
        return u, v

    @property
    def t(self):
        return self.flow.step_count * self.dt

    def add_species(self, xy, st, vxy=None):
        xy = np.asarray(xy, dtype=np.float64).reshape(-1, 2)
        if st > 0:
            if vxy is None:
                u, v = self._level
                v0 = (interp(u, self.scheme, xy[:, 0], xy[:, 1]), interp(v, self.scheme, xy[:, 0], xy[:, 1]))
            else:
                vxy = np.asarray(vxy, dtype=np.float64).reshape(-1, 2)
                v0 = (vxy[:, 0].copy(), vxy[:, 1].copy())
        else:
            v0 = None
        self.species.append(Species(xy, st, v0))
        return len(self.species) - 1

    def step(self, nsteps=1):
        for _ in range(int(nsteps)):
            un, vn = self._level
            pn = self._psi
            self.flow.step(1)
            un1, vn1 = self._stencil_fields()
            pn1 = self._psi_field()
            for s in self.species:
                if s.st == 0 and self.tracer_psi:
                    tracers_rk4_psi(self.scheme, self.dt, pn, pn1, s.x, s.y)
                else:
                    particles_rk4(self.scheme, self.dt, s.st, un, vn, un1, vn1, s.x, s.y, s.vx, s.vy)
            self._level = (un1, vn1)
            self._psi = pn1

    def stats(self):
        e, z, p = self.flow.diagnostics()
        out = {"t": self.t, "step": self.flow.step_count, "energy": e, "enstrophy": z,
               "palinstrophy": p, "msd": [], "cluster": [], "np": []}
        for s in self.species:
            out["msd"].append(msd(s.x, s.y, s.x0, s.y0))
            out["cluster"].append(cluster_index(s.x, s.y))
            out["np"].append(int(s.x.size))
        return out
