"""Continuous-batching server of coupled simulations on one GPU.

Requests (a grid size, a particle species, an interpolation scheme and a
step count; see ``inputs.served_requests``) arrive over time.  The server
keeps every admitted simulation's fields and particles on the device and
advances all of them together in one ``el_batch`` (one persistent kernel per
stage).  Between batch ticks it

  * admits waiting requests while their device footprint
    (``el_workspace_bytes``) fits the HBM budget and a batch slot is free,
  * retires finished ones: their statistics (and, if asked, final particle
    positions) are read back, the member leaves the batch and its workspace
    is released.

A tick advances the batch by min(tick_steps, fewest steps any member still
needs), so a request finishes exactly at its step count.  Time-to-result is
measured from the request's arrival to the moment its result is on the host.
Everything numerical runs in the CUDA library; this module only schedules.
"""
from __future__ import annotations

import collections
import time
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


def build_flow(req: inputs.Request, stream, device) -> elpath.Flow:
    """The request's simulation: its initial vorticity and particles."""
    wl = req.workload
    sp = wl.species[0]
    g = elpath.Flow(wl.n, wl.nu, wl.dt, wl.omega0(), interp=req.scheme, max_species=1,
                    max_particles=wl.particles, sort_every=20, stream=stream, device=device)
    g.set_particles(0, inputs.uniform_positions(sp.count, sp.seed), sp.st)
    return g


@dataclass
class Server:
    hbm_budget: int                  # bytes of device memory the simulations may hold
    max_members: int = 64
    tick_steps: int = 20
    keep_positions: bool = False
    device: str = "cuda"
    results: list = field(default_factory=list)

    def __post_init__(self):
        import torch
        self._torch = torch
        self.batch = elpath.Batch(self.max_members, device=self.device)
        self.waiting: collections.deque = collections.deque()
        self.active: list[_Active] = []
        self.used = 0
        self.peak_used = 0
        self.particle_steps = 0
        self.t0 = time.perf_counter()

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def submit(self, req: inputs.Request):
        need = elpath.workspace_bytes(request_desc(req))
        if need == 0 or need > self.hbm_budget:
            raise ValueError(f"request {req.rid} needs {need} B, over the {self.hbm_budget} B budget")
        self.waiting.append(req)

    def _admit(self):
        while self.waiting and len(self.active) < self.max_members:
            req = self.waiting[0]
            need = elpath.workspace_bytes(request_desc(req))
            if self.used + need > self.hbm_budget:
                break                                # oldest first: wait for memory
            self.waiting.popleft()
            g = build_flow(req, None, self.device)
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
            if self.waiting or self.active:
                self.tick()
            elif pending:
                time.sleep(max(0.0, min(0.01, pending[0].arrival - t)))
        return self.results

    def close(self):
        for a in self.active:
            self.batch.remove(a.flow)
            a.flow.close()
        self.active = []
        self.batch.close()


def latency_summary(results) -> dict:
    lat = np.array([r.latency for r in results])
    if lat.size == 0:
        return {"count": 0}
    return {"count": int(lat.size), "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()),
            "max_s": float(lat.max())}
