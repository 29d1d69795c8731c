"""ctypes binding of libelpath.so (include/elpath.h), same names as the C ABI.

Argument marshalling only: every step of the coupled path runs in the CUDA
library.  PyTorch provides the device workspace (a uint8 tensor) and the
CUDA stream.  If the library is missing this module raises; there is no
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libelpath.so")

BILINEAR, CATMULL_ROM, BSPLINE, ANALYTIC = 0, 1, 2, 3
MAX_SPECIES = 8
STATUS = {0: "EL_OK", 1: "EL_EINVAL", 2: "EL_ENOMEM", 3: "EL_ECUDA", 4: "EL_ECUFFT",
          5: "EL_ESTATE", 6: "EL_ENONFINITE", 7: "EL_ETIMEOUT"}

# Public C symbols, in include/elpath.h order.
SYMBOLS = ("el_workspace_bytes", "el_create_flow", "el_create_kinematic", "el_set_particles",
           "el_step_coupled",
           "el_get_stats", "el_get_particles", "el_get_field", "el_sample_velocity",
           "el_profile_step", "el_get_tuning", "el_set_tuning", "el_autotune",
           "el_kernel_launches", "el_flow_fused", "el_batch_workspace_bytes", "el_batch_create", "el_batch_add",
           "el_batch_remove", "el_batch_step", "el_batch_autotune", "el_batch_size",
           "el_batch_kernel_launches", "el_batch_last_error", "el_batch_destroy",
           "el_batch_fft_pool_bytes", "el_batch_add_fft_pool", "el_dispersion_noalloc", "el_save_state", "el_load_state", "el_destroy_flow",
           "el_last_error")
NOALLOC_MAX_PARTICLES = 262144


class ElpathError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class el_flow_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("interp", ctypes.c_int32), ("nu", ctypes.c_double),
                ("dt", ctypes.c_double), ("ab2_mode", ctypes.c_int32),
                ("bspline_prefilter", ctypes.c_int32), ("max_species", ctypes.c_int32),
                ("sort_every", ctypes.c_int32), ("max_particles", ctypes.c_int64),
                ("tracer_velocity", ctypes.c_int32)]


class el_tuning(ctypes.Structure):
    _fields_ = [("rk4_threads", ctypes.c_int32), ("sort_every", ctypes.c_int32),
                ("sort_shift", ctypes.c_int32), ("gather", ctypes.c_int32),
                ("ms_per_step", ctypes.c_double)]


GATHER_AUTO, GATHER_REGISTERS, GATHER_SHARED = 0, 1, 2


class el_kinematic(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("k", ctypes.c_double), ("eps", ctypes.c_double),
                ("omega", ctypes.c_double), ("phi", ctypes.c_double)]


class el_stats(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("step", ctypes.c_int64), ("energy", ctypes.c_double),
                ("enstrophy", ctypes.c_double), ("palinstrophy", ctypes.c_double),
                ("msd", (ctypes.c_double * 2) * MAX_SPECIES),
                ("cluster", ctypes.c_double * MAX_SPECIES), ("np", ctypes.c_int64 * MAX_SPECIES),
                ("finite", ctypes.c_int32), ("msd_sem", (ctypes.c_double * 2) * MAX_SPECIES),
                ("diffusivity", (ctypes.c_double * 2) * MAX_SPECIES)]


_lib = None


def load(path: str = LIB_PATH):
    """Open libelpath.so and declare the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FileNotFoundError(f"{path} is missing: build it with "
                                "`python -m paper_2607_17836_b300.build` (no fallback path exists)")
    lib = ctypes.CDLL(path)
    P, D, I32, I64, V = (ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int32,
                         ctypes.c_int64, ctypes.c_void_p)
    lib.el_workspace_bytes.argtypes = [ctypes.POINTER(el_flow_desc)]
    lib.el_workspace_bytes.restype = ctypes.c_size_t
    lib.el_create_flow.argtypes = [ctypes.POINTER(el_flow_desc), D, V, ctypes.c_size_t, V,
                                   ctypes.POINTER(P)]
    lib.el_create_kinematic.argtypes = [ctypes.POINTER(el_flow_desc), ctypes.POINTER(el_kinematic),
                                        V, ctypes.c_size_t, V, ctypes.POINTER(P)]
    lib.el_create_kinematic.restype = ctypes.c_int
    lib.el_set_particles.argtypes = [P, I32, I64, ctypes.c_double, D, D]
    lib.el_step_coupled.argtypes = [P, I32]
    lib.el_get_stats.argtypes = [P, ctypes.POINTER(el_stats)]
    lib.el_get_particles.argtypes = [P, I32, D, D]
    lib.el_get_field.argtypes = [P, I32, D]
    lib.el_sample_velocity.argtypes = [P, I64, V, ctypes.c_double, V]
    lib.el_profile_step.argtypes = [P, D, I32]
    lib.el_kernel_launches.argtypes = [P]
    lib.el_kernel_launches.restype = I64
    lib.el_flow_fused.argtypes = [P]
    lib.el_flow_fused.restype = I32
    T = ctypes.POINTER(el_tuning)
    lib.el_get_tuning.argtypes = [P, T]
    lib.el_set_tuning.argtypes = [P, T]
    lib.el_autotune.argtypes = [P, I32, T]
    lib.el_batch_workspace_bytes.argtypes = [I32]
    lib.el_batch_workspace_bytes.restype = ctypes.c_size_t
    lib.el_batch_create.argtypes = [I32, V, ctypes.c_size_t, V, ctypes.POINTER(P)]
    lib.el_batch_add.argtypes = [P, P]
    lib.el_batch_remove.argtypes = [P, P]
    lib.el_batch_step.argtypes = [P, I32]
    lib.el_batch_autotune.argtypes = [P, I32, T]
    lib.el_batch_size.argtypes = [P]
    lib.el_batch_size.restype = I32
    lib.el_batch_kernel_launches.argtypes = [P]
    lib.el_batch_kernel_launches.restype = I64
    lib.el_batch_last_error.argtypes = [P]
    lib.el_batch_last_error.restype = ctypes.c_char_p
    lib.el_batch_destroy.argtypes = [P]
    lib.el_batch_fft_pool_bytes.argtypes = [ctypes.POINTER(el_flow_desc), I32]
    lib.el_batch_fft_pool_bytes.restype = ctypes.c_size_t
    lib.el_batch_add_fft_pool.argtypes = [P, ctypes.POINTER(el_flow_desc), I32, V, ctypes.c_size_t]
    lib.el_batch_add_fft_pool.restype = ctypes.c_int
    for name in ("el_get_tuning", "el_set_tuning", "el_autotune", "el_batch_create",
                 "el_batch_add", "el_batch_remove", "el_batch_step", "el_batch_autotune",
                 "el_batch_destroy"):
        getattr(lib, name).restype = ctypes.c_int
    lib.el_dispersion_noalloc.argtypes = [V, V, I64, V, V]
    lib.el_dispersion_noalloc.restype = ctypes.c_int
    lib.el_save_state.argtypes = [P, V, ctypes.POINTER(ctypes.c_size_t)]
    lib.el_load_state.argtypes = [P, V, ctypes.c_size_t]
    lib.el_destroy_flow.argtypes = [P]
    lib.el_last_error.argtypes = [P]
    lib.el_last_error.restype = ctypes.c_char_p
    for name in ("el_create_flow", "el_set_particles", "el_step_coupled", "el_get_stats",
                 "el_get_particles", "el_get_field", "el_sample_velocity", "el_profile_step",
                 "el_save_state", "el_load_state", "el_destroy_flow"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _host_f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def make_desc(n, nu, dt, interp=BILINEAR, ab2_mode=0, bspline_prefilter=True, max_species=0,
              max_particles=0, sort_every=0, tracer_velocity=0) -> el_flow_desc:
    return el_flow_desc(int(n), int(interp), float(nu), float(dt), int(ab2_mode),
                        1 if bspline_prefilter else 0, int(max_species), int(sort_every),
                        int(max_particles), int(tracer_velocity))


def workspace_bytes(desc: el_flow_desc) -> int:
    return int(load().el_workspace_bytes(ctypes.byref(desc)))


def dispersion_noalloc(xy_dev, xy0_dev, out=None, stream=None):
    """el_dispersion_noalloc: (msd_x, msd_y, cluster) of device positions,
    with no allocation inside the library (its scratch is a fixed device
    array).  xy_dev, xy0_dev: CUDA float64 tensors (np, 2); out: CUDA float64
    tensor of 3 (allocated here if None, by the caller's allocator)."""
    import torch
    lib = load()
    assert xy_dev.is_cuda and xy_dev.dtype == torch.float64 and xy_dev.is_contiguous()
    assert xy0_dev.shape == xy_dev.shape and xy0_dev.dtype == torch.float64
    if out is None:
        out = torch.empty(3, dtype=torch.float64, device=xy_dev.device)
    s = stream if stream is not None else torch.cuda.current_stream(xy_dev.device)
    st = lib.el_dispersion_noalloc(ctypes.c_void_p(xy_dev.data_ptr()),
                                   ctypes.c_void_p(xy0_dev.data_ptr()), int(xy_dev.shape[0]),
                                   ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(s.cuda_stream))
    if st != 0:
        raise ElpathError(st, lib.el_last_error(None).decode())
    return out


class Flow:
    """One coupled simulation (el_flow) on a CUDA device."""

    def __init__(self, n, nu, dt, omega0, interp=BILINEAR, ab2_mode=0, bspline_prefilter=True,
                 max_species=0, max_particles=0, sort_every=0, stream=None, device=None,
                 workspace=None, tracer_velocity=0, kinematic=None):
        """omega0: initial vorticity (n x n) of a solved flow; or, with
        kinematic = dict(alpha=, k=, eps=, omega=, phi=), the prescribed
        oscillating Taylor-Green field (el_create_kinematic; omega0 unused)."""
        import torch
        lib = load()
        self._lib = lib
        self.desc = make_desc(n, nu, dt, interp, ab2_mode, bspline_prefilter, max_species,
                              max_particles, sort_every, tracer_velocity)
        self.n = int(n)
        self.device = torch.device(device if device is not None else "cuda")
        nbytes = workspace_bytes(self.desc)
        if nbytes == 0:
            raise ElpathError(1, "invalid flow description (or no CUDA device)")
        if workspace is None:
            workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.workspace = workspace
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        h = ctypes.c_void_p()
        if kinematic is not None:
            kin = el_kinematic(float(kinematic["alpha"]), float(kinematic["k"]),
                               float(kinematic["eps"]), float(kinematic["omega"]),
                               float(kinematic.get("phi", 0.0)))
            with torch.cuda.device(self.device):
                st = lib.el_create_kinematic(ctypes.byref(self.desc), ctypes.byref(kin),
                                             ctypes.c_void_p(workspace.data_ptr()),
                                             ctypes.c_size_t(workspace.numel()),
                                             ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        else:
            w0 = _host_f64(omega0)
            if w0.shape != (self.n, self.n):
                raise ValueError(f"omega0 must be {self.n}x{self.n}")
            with torch.cuda.device(self.device):
                st = lib.el_create_flow(ctypes.byref(self.desc), _dptr(w0),
                                        ctypes.c_void_p(workspace.data_ptr()),
                                        ctypes.c_size_t(workspace.numel()),
                                        ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if st != 0:
            raise ElpathError(st, lib.el_last_error(None).decode())
        self._h = h

    # -- helpers
    def _check(self, st):
        if st != 0:
            raise ElpathError(st, self._lib.el_last_error(self._h).decode())

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.el_destroy_flow(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- ABI calls
    def set_particles(self, species, xy, st, vxy=None):
        xy = _host_f64(xy, (-1, 2))
        v = _host_f64(vxy, (-1, 2)) if vxy is not None else None
        if v is not None and v.shape != xy.shape:
            raise ValueError("vxy must match xy")
        self._check(self._lib.el_set_particles(self._h, int(species), int(xy.shape[0]),
                                               float(st), _dptr(xy), _dptr(v)))

    def step(self, nsteps=1):
        self._check(self._lib.el_step_coupled(self._h, int(nsteps)))

    def stats(self, allow_nonfinite=False) -> dict:
        s = el_stats()
        st = self._lib.el_get_stats(self._h, ctypes.byref(s))
        if st != 0 and not (allow_nonfinite and st == 6):
            self._check(st)
        return {"t": s.t, "step": s.step, "energy": s.energy, "enstrophy": s.enstrophy,
                "palinstrophy": s.palinstrophy,
                "msd": [(s.msd[k][0], s.msd[k][1]) for k in range(MAX_SPECIES)],
                "cluster": [s.cluster[k] for k in range(MAX_SPECIES)],
                "np": [s.np[k] for k in range(MAX_SPECIES)], "finite": bool(s.finite),
                "msd_sem": [(s.msd_sem[k][0], s.msd_sem[k][1]) for k in range(MAX_SPECIES)],
                "diffusivity": [(s.diffusivity[k][0], s.diffusivity[k][1])
                                for k in range(MAX_SPECIES)]}

    def particles(self, species, count):
        xy = np.empty((count, 2))
        vxy = np.empty((count, 2))
        self._check(self._lib.el_get_particles(self._h, int(species), _dptr(xy), _dptr(vxy)))
        return xy, vxy

    def particles_into(self, species, xy=None, vxy=None):
        """el_get_particles into caller-owned (e.g. pinned) float64 host arrays."""
        self._check(self._lib.el_get_particles(self._h, int(species), _dptr(xy), _dptr(vxy)))

    def field(self, which):
        out = np.empty((self.n, self.n))
        self._check(self._lib.el_get_field(self._h, int(which), _dptr(out)))
        return out

    def sample_velocity(self, xy_dev, theta=1.0, out=None):
        """xy_dev: CUDA float64 tensor (np, 2).  Returns a CUDA float64 (np, 2) tensor."""
        import torch
        assert xy_dev.is_cuda and xy_dev.dtype == torch.float64 and xy_dev.is_contiguous()
        if out is None:
            out = torch.empty_like(xy_dev)
        self._check(self._lib.el_sample_velocity(self._h, int(xy_dev.shape[0]),
                                                 ctypes.c_void_p(xy_dev.data_ptr()),
                                                 float(theta), ctypes.c_void_p(out.data_ptr())))
        return out

    def profile_step(self):
        """One coupled step with per-stage CUDA-event times (ms):
        {"fluid": ms, "particles": ms (all species, one launch), "sort": ms}."""
        buf = np.zeros(3)
        self._check(self._lib.el_profile_step(self._h, _dptr(buf), int(buf.size)))
        return {"fluid": float(buf[0]), "particles": float(buf[1]), "sort": float(buf[2])}

    def kernel_launches(self) -> int:
        return int(self._lib.el_kernel_launches(self._h))

    @property
    def fused(self) -> bool:
        """The fluid step runs the library's fused transforms (el_flow_fused)."""
        return bool(self._lib.el_flow_fused(self._h))

    def tuning(self) -> dict:
        t = el_tuning()
        self._check(self._lib.el_get_tuning(self._h, ctypes.byref(t)))
        return {"rk4_threads": t.rk4_threads, "sort_every": t.sort_every,
                "sort_shift": t.sort_shift, "gather": t.gather}

    def set_tuning(self, rk4_threads=256, sort_every=20, sort_shift=0, gather=GATHER_AUTO):
        t = el_tuning(int(rk4_threads), int(sort_every), int(sort_shift), int(gather), 0.0)
        self._check(self._lib.el_set_tuning(self._h, ctypes.byref(t)))

    def autotune(self, trial_steps=10) -> dict:
        """el_autotune: the trial steps are real steps of this simulation."""
        t = el_tuning()
        self._check(self._lib.el_autotune(self._h, int(trial_steps), ctypes.byref(t)))
        return {"rk4_threads": t.rk4_threads, "sort_every": t.sort_every,
                "sort_shift": t.sort_shift, "gather": t.gather,
                "ms_per_step": t.ms_per_step}

    def save_state(self) -> bytes:
        """el_save_state: the flow's complete state at its current step."""
        size = ctypes.c_size_t(0)
        self._check(self._lib.el_save_state(self._h, None, ctypes.byref(size)))
        buf = ctypes.create_string_buffer(size.value)
        self._check(self._lib.el_save_state(self._h, buf, ctypes.byref(size)))
        return buf.raw[:size.value]

    def load_state(self, image: bytes):
        """el_load_state: replace the flow's state by a saved image."""
        image = bytes(image)
        self._check(self._lib.el_load_state(self._h, ctypes.c_char_p(image), len(image)))

    def synchronize(self):
        self.stream.synchronize()


class Batch:
    """el_batch: flows advanced together by one kernel per stage over all of them."""

    def __init__(self, max_members, stream=None, device=None):
        import torch
        lib = load()
        self._lib = lib
        self.device = torch.device(device if device is not None else "cuda")
        nbytes = int(lib.el_batch_workspace_bytes(int(max_members)))
        if nbytes == 0:
            raise ElpathError(1, "max_members out of range")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            st = lib.el_batch_create(int(max_members), ctypes.c_void_p(self.workspace.data_ptr()),
                                     ctypes.c_size_t(nbytes),
                                     ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if st != 0:
            raise ElpathError(st, lib.el_last_error(None).decode())
        self._h = h
        self.members = []
        self.pools = []

    def _check(self, st):
        if st != 0:
            raise ElpathError(st, self._lib.el_batch_last_error(self._h).decode())

    def add_fft_pool(self, n, slots, interp=BILINEAR, bspline_prefilter=True, tracer_velocity=0):
        """An FFT pool for `slots` members of grid n (and the plane count the
        scheme / prefilter / tracer-velocity options imply); members added
        afterwards take its slots.  Its device memory is held here until close."""
        import torch
        desc = make_desc(n, 0.0, 1.0, interp=interp, bspline_prefilter=bspline_prefilter,
                         tracer_velocity=tracer_velocity)
        nbytes = int(self._lib.el_batch_fft_pool_bytes(ctypes.byref(desc), int(slots)))
        if nbytes == 0:
            raise ElpathError(1, "invalid pool class or slot count")
        mem = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        with torch.cuda.device(self.device):
            self._check(self._lib.el_batch_add_fft_pool(self._h, ctypes.byref(desc), int(slots),
                                                        ctypes.c_void_p(mem.data_ptr()),
                                                        ctypes.c_size_t(nbytes)))
        self.pools.append(mem)
        return nbytes

    def add(self, flow):
        self._check(self._lib.el_batch_add(self._h, flow._h))
        self.members.append(flow)

    def remove(self, flow):
        self._check(self._lib.el_batch_remove(self._h, flow._h))
        self.members.remove(flow)

    def step(self, nsteps=1):
        self._check(self._lib.el_batch_step(self._h, int(nsteps)))

    def autotune(self, trial_steps=10) -> dict:
        t = el_tuning()
        self._check(self._lib.el_batch_autotune(self._h, int(trial_steps), ctypes.byref(t)))
        return {"rk4_threads": t.rk4_threads, "sort_every": t.sort_every,
                "sort_shift": t.sort_shift, "gather": t.gather,
                "ms_per_step": t.ms_per_step}

    def size(self) -> int:
        return int(self._lib.el_batch_size(self._h))

    def kernel_launches(self) -> int:
        return int(self._lib.el_batch_kernel_launches(self._h))

    def synchronize(self):
        self.stream.synchronize()

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.el_batch_destroy(h)
            self._h = None
            self.members = []
            self.pools = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
