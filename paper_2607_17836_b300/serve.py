"""Continuous-batching server of coupled simulations on one GPU.

Requests (a grid size, a particle species, an interpolation scheme and a
step count; see ``inputs.served_requests``) arrive over time.  The server
keeps every admitted simulation's fields and particles on the device and
advances all of them together in one ``el_batch`` (one kernel per stage over
all of them).  Between batch ticks it

  * admits waiting requests while their device footprint
    (``el_workspace_bytes``) fits the HBM budget and a batch slot is free,
  * retires finished ones: their statistics (and, if asked, final particle
    positions) are read back, the member leaves the batch and its workspace
    is released.

A tick advances the batch by min(tick_steps, fewest steps any member still
needs), so a request finishes exactly at its step count.  Time-to-result is
measured from the request's arrival to the moment its result is on the host.
A request's host inputs (initial vorticity, particle positions) are prepared
on a thread pool from the moment it arrives, so the device loop never waits
for them; the oldest request whose inputs are ready is admitted first (one
still being prepared does not hold back the requests behind it, and one that
is ready but does not fit the memory left does).
Everything numerical runs in the CUDA library; this module only schedules.
"""
from __future__ import annotations

import collections
import time
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

from . import elpath, inputs


@dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    steps: int
    particles: int
    n: int
    stats: dict
    positions: np.ndarray | None = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival

    @property
    def queue_wait(self) -> float:
        """Arrival to admission: waiting for inputs, memory or a batch slot."""
        return self.admitted - self.arrival

    @property
    def service(self) -> float:
        """Admission to the result on the host: the steps in the shared batch."""
        return self.finished - self.admitted


@dataclass
class _Active:
    request: inputs.Request
    flow: elpath.Flow
    workspace_bytes: int
    steps_left: int
    admitted: float


def request_desc(req: inputs.Request):
    wl = req.workload
    return elpath.make_desc(wl.n, wl.nu, wl.dt, interp=req.scheme, max_species=1,
                            max_particles=wl.particles, sort_every=20)


def prepare_inputs(req: inputs.Request):
    """The request's host inputs: initial vorticity and particle positions."""
    wl = req.workload
    sp = wl.species[0]
    return wl.omega0(), inputs.uniform_positions(sp.count, sp.seed)


# The served flows' particle-step block size and re-binning cadence.  On the
# served stream's first 200 requests at 20 requests/s: 128 threads and every
# 40 steps 1.61e10 particle-steps/s (p50 2.93 s) against 1.55e10 (p50 3.3 s)
# for the library's 256 threads and every 20 steps; 128 / 20 and 128 / 80
# 1.59e10 / 1.61e10, 256 / 40 and 256 / 80 1.57e10 / 1.59e10.
SERVE_RK4_THREADS = 128
SERVE_SORT_EVERY = 40


def build_flow(req: inputs.Request, stream, device, prepared=None, rk4_threads=SERVE_RK4_THREADS,
               sort_every=SERVE_SORT_EVERY) -> elpath.Flow:
    """The request's simulation from its (prepared) initial vorticity and
    particles; rk4_threads: the particle step's block size (None: the
    library's default), sort_every: its re-binning cadence in steps."""
    wl = req.workload
    sp = wl.species[0]
    omega0, xy = prepared if prepared is not None else prepare_inputs(req)
    g = elpath.Flow(wl.n, wl.nu, wl.dt, omega0, interp=req.scheme, max_species=1,
                    max_particles=wl.particles, sort_every=sort_every, stream=stream, device=device)
    if rk4_threads is not None:
        g.set_tuning(rk4_threads, sort_every, 0, elpath.GATHER_AUTO)
    g.set_particles(0, xy, sp.st)
    return g


@dataclass
class Server:
    hbm_budget: int                  # bytes of device memory the simulations may hold
    max_members: int = 64
    tick_steps: int = 20
    keep_positions: bool = False
    device: str = "cuda"
    prep_workers: int = 8            # threads preparing arrived requests' host inputs
    prep_ahead: int = 16             # waiting requests (oldest first) whose inputs are prepared
    fft_pool_slots: dict = None      # grid n -> FFT-pool slots (None: per-member transforms)
    rk4_threads: int = SERVE_RK4_THREADS  # the batch's particle-step block size (None: the library's)
    sort_every: int = SERVE_SORT_EVERY    # each member's re-binning cadence in steps
    results: list = field(default_factory=list)

    def __post_init__(self):
        import torch
        self._torch = torch
        self.batch = elpath.Batch(self.max_members, device=self.device)
        self.waiting: collections.deque = collections.deque()  # [request, inputs future or None]
        self.pool = ThreadPoolExecutor(max_workers=max(1, self.prep_workers))
        self.active: list[_Active] = []
        self.used = 0
        # FFT pools (bilinear and Catmull-Rom requests share one class per
        # grid size): their memory is held for the server's lifetime and
        # counted against the budget
        for n, slots in sorted((self.fft_pool_slots or {}).items()):
            self.used += self.batch.add_fft_pool(int(n), int(slots))
        self.peak_used = self.used
        self.particle_steps = 0
        self.t0 = time.perf_counter()

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def submit(self, req: inputs.Request):
        need = elpath.workspace_bytes(request_desc(req))
        if need == 0 or need > self.hbm_budget:
            raise ValueError(f"request {req.rid} needs {need} B, over the {self.hbm_budget} B budget")
        self.waiting.append([req, None])
        self._prepare_ahead()

    def _prepare_ahead(self):
        for k, entry in enumerate(self.waiting):
            if k >= self.prep_ahead:
                break
            if entry[1] is None:
                entry[1] = self.pool.submit(prepare_inputs, entry[0])

    def _admit(self):
        self._prepare_ahead()
        while self.waiting and len(self.active) < self.max_members:
            # the oldest request whose inputs are ready (one whose inputs are
            # still being prepared does not hold back those behind it)
            k = next((k for k, (_, prep) in enumerate(self.waiting)
                      if prep is not None and prep.done()), None)
            if k is None:
                break
            req, prep = self.waiting[k]
            need = elpath.workspace_bytes(request_desc(req))
            if self.used + need > self.hbm_budget:
                break                                # oldest ready first: wait for memory
            del self.waiting[k]
            self._prepare_ahead()
            g = build_flow(req, None, self.device, prep.result(), self.rk4_threads, self.sort_every)
            self.batch.add(g)
            self.active.append(_Active(req, g, need, req.workload.steps, self.now()))
            self.used += need
            self.peak_used = max(self.peak_used, self.used)

    def _retire(self):
        still = []
        for a in self.active:
            if a.steps_left > 0:
                still.append(a)
                continue
            st = a.flow.stats()
            pos = None
            if self.keep_positions:
                pos, _ = a.flow.particles(0, a.request.workload.particles)
            self.batch.remove(a.flow)
            a.flow.close()
            self.used -= a.workspace_bytes
            wl = a.request.workload
            self.results.append(Result(a.request.rid, a.request.arrival, a.admitted, self.now(),
                                       wl.steps, wl.particles, wl.n, st, pos))
        self.active = still

    def tick(self) -> int:
        """Admit, advance the batch, retire; returns the steps advanced."""
        self._admit()
        if not self.active:
            return 0
        k = min(self.tick_steps, min(a.steps_left for a in self.active))
        self.batch.step(k)
        for a in self.active:
            a.steps_left -= k
            self.particle_steps += k * a.request.workload.particles
        if any(a.steps_left == 0 for a in self.active):
            self._retire()
        return k

    def run(self, requests, time_scale: float = 1.0, timeout: float | None = None):
        """Serve a stream: request r arrives at r.arrival * time_scale seconds
        after the start (wall clock).  Returns the list of results."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        self.t0 = time.perf_counter()
        for r in pending:
            r.arrival = r.arrival * time_scale
        while pending or self.waiting or self.active:
            t = self.now()
            while pending and pending[0].arrival <= t:
                self.submit(pending.popleft())
            if timeout is not None and t > timeout:
                break
            if self.active:
                self.tick()
            elif self.waiting:
                self._admit()
                if not self.active:
                    time.sleep(0.001)                # inputs still being prepared
            elif pending:
                time.sleep(max(0.0, min(0.01, pending[0].arrival - t)))
        return self.results

    def close(self):
        for a in self.active:
            self.batch.remove(a.flow)
            a.flow.close()
        self.active = []
        self.batch.close()
        self.pool.shutdown(wait=True, cancel_futures=True)


def latency_summary(results) -> dict:
    """Time-to-result percentiles (linear interpolation), and the same for its
    two parts: the queue wait (arrival to admission) and the service time
    (admission to the result on the host)."""
    lat = np.array([r.latency for r in results])
    if lat.size == 0:
        return {"count": 0}
    out = {"count": int(lat.size), "p50_s": float(np.percentile(lat, 50)),
           "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()),
           "max_s": float(lat.max())}
    for name in ("queue_wait", "service"):
        x = np.array([getattr(r, name) for r in results])
        out[name] = {"p50_s": float(np.percentile(x, 50)), "p99_s": float(np.percentile(x, 99)),
                     "mean_s": float(x.mean()), "max_s": float(x.max())}
    return out
