"""Benchmark of the coupled Eulerian-Lagrangian hot path on one B300.

Workload (one "step" = one coupled step of Algorithm 1 over the whole batch):
decaying 2-D turbulence on a 1024^2 grid (nu = 1e-4, dt = 5e-4), 1M passive
tracers and 1M inertial particles at each of St = 0.1, 1, 10, all resident
in HBM, interpolation scheme selectable (bilinear by default, the paper's
production scheme).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--scheme bilinear|catmull_rom|bspline]
                  [--impl ours|reference]

Prints one JSON line.  `value` is particle-steps/s of the whole coupled step
(fluid included), timed with CUDA events on the flow's stream around calls of
10 steps (inside a call the fluid step of n+1 overlaps the particle step of
n).  Each step touches more bytes than L2 holds (about 153 MiB at 1024^2
with 4M particles against 126 MiB), and a 256 MiB write flushes L2 before
every call, outside its event pair.  The solve latency (p50/p99) is taken
over 200 single-step calls, each after an L2 flush.  `--impl reference`
times the FP64 CPU oracle instead.
Under torchrun (N > 1) each rank runs an independent replica (weak scaling;
the path has no exchange step) and rank 0 prints the aggregate.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2607_17836_b300 import inputs  # noqa: E402

SCHEMES = {"bilinear": 0, "catmull_rom": 1, "bspline": 2}
METRIC = "particle-steps/s (RK4+interp) & fluid steps/s at 1024^2; p50/p99 solve latency"
SORT_EVERY = 20
# Algorithmic bytes per particle-step of the RK4 kernel as the method's
# state counts them: an 8-byte periodic image count, an 8-byte cell index,
# an 8-byte offset pair and (inertial particles) an 8-byte velocity pair,
# each read and written once; plus one read of the level pair (u, v at two
# time levels, 16 N^2 bytes) per launch.
BYTES_TRACER = 2 * (8 + 8 + 8)
BYTES_INERTIAL = 2 * (8 + 8 + 8 + 8)
FIELD_PAIR_BYTES_PER_NODE = 16
# Compulsory bytes of this library's layout: the 4-byte packed cell and the
# offset pair (and velocity pair) are read and written every step; the image
# count is written only when a particle crosses the periodic boundary.
COMPULSORY_TRACER = 2 * (4 + 8)
COMPULSORY_INERTIAL = 2 * (4 + 8 + 8)
FLUSH_BYTES = 256 << 20
L2_BYTES = 126 << 20
LATENCY_SAMPLES = 200
# Snapshot bytes one particle-step gathers, per interpolation width W (W x W
# nodes of (u, v) in FP32): the plain form fetches the nodes at each of its 6
# snapshot evaluations (levels n and n+1 at stages 1 and 4, both at stages 2
# and 3); the kernel here fetches each node once as one 16-byte level pair.
GATHER_PLAIN = {0: 6 * 4 * 8, 1: 6 * 16 * 8, 2: 6 * 16 * 8}
GATHER_CACHED = {0: 4 * 16, 1: 16 * 16, 2: 16 * 16}
CHUNK = 10          # coupled steps per el_step_coupled call in the timed region


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for rel in ("paper_2607_17836_b300/csrc/rk4.cu", "paper_2607_17836_b300/csrc/interp.cuh",
                "paper_2607_17836_b300/csrc/stages.cuh"):
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_profile(scheme_name):
    """Figures of the RK4 kernel from the committed ncu summary
    (profiles/k_rk4_<scheme>_traffic.txt), if they were taken on the current
    kernel source; else an empty dict."""
    p = os.path.join(ROOT, "profiles", f"k_rk4_{scheme_name}_traffic.txt")
    if not os.path.exists(p):
        return {}
    vals = {}
    with open(p) as fh:
        for line in fh:
            if "=" in line and not line.startswith("#"):
                k, v = line.strip().split("=", 1)
                vals[k.strip()] = v.strip()
    if vals.get("source_hash") != kernel_source_hash():
        return {}
    return vals


def recorded_traffic(scheme_name):
    """DRAM bytes per particle-step of the RK4 kernel from the committed ncu
    summary, if it was taken on the current kernel source; else None."""
    try:
        return float(recorded_profile(scheme_name)["dram_bytes_per_particle_step"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """SM clocks and clock-event (throttle) reasons sampled during the timed
    region: through NVML every 5 ms (read-only queries of the driver's
    libnvidia-ml), else nvidia-smi every 50 ms."""

    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index, device=None):
        self.index = index
        self.device = device
        self.rows = []          # (sm_mhz, max_mhz, set of reason names)
        self.proc = None
        self.nvml = None
        self.stop = threading.Event()

    def _nvml_handle(self):
        """Read-only NVML queries for this process's CUDA device (matched by
        UUID, else by PCI bus id, else the only device), through ctypes on the
        driver's libnvidia-ml: returns a function giving (sm MHz, max sm MHz,
        clock-event reason bits)."""
        import ctypes
        import torch
        nv = ctypes.CDLL("libnvidia-ml.so.1")
        if nv.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        prop = torch.cuda.get_device_properties(self.device if self.device is not None else self.index)
        h = ctypes.c_void_p()
        found = False
        uuid = getattr(prop, "uuid", None)
        if uuid is not None:
            found = nv.nvmlDeviceGetHandleByUUID(f"GPU-{uuid}".encode(), ctypes.byref(h)) == 0
        if not found:
            bus = f"{prop.pci_domain_id:08X}:{prop.pci_bus_id:02X}:{prop.pci_device_id:02X}.0"
            found = nv.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(h)) == 0
        if not found:
            cnt = ctypes.c_uint(0)
            if nv.nvmlDeviceGetCount_v2(ctypes.byref(cnt)) == 0 and cnt.value == 1:
                found = nv.nvmlDeviceGetHandleByIndex_v2(0, ctypes.byref(h)) == 0
        if not found:
            raise RuntimeError("no NVML handle for this device")
        reasons_fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            nv.nvmlDeviceGetCurrentClocksThrottleReasons
        sm, mx, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()

        def read():
            if (nv.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(sm)) != 0 or      # 1: NVML_CLOCK_SM
                    nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) != 0 or
                    reasons_fn(h, ctypes.byref(rs)) != 0):
                raise RuntimeError("NVML query failed")
            return float(sm.value), float(mx.value), int(rs.value)
        read()
        return read

    def __enter__(self):
        self.nvml_error = None
        try:
            self.nvml = self._nvml_handle()
            self.thread = threading.Thread(target=self._poll_nvml, daemon=True)
            self.thread.start()
            return self
        except Exception as e:
            self.nvml = None
            self.nvml_error = repr(e)[:200]
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    # NVML clock-event reason bits of NAMES: HW slowdown, HW thermal, SW thermal, SW power cap
    BITS = (0x8, 0x40, 0x20, 0x4)

    def _poll_nvml(self):
        read = self.nvml
        while not self.stop.is_set():
            try:
                sm, mx, r = read()
            except Exception:
                break
            self.rows.append((sm, mx, {n for n, b in zip(self.NAMES, self.BITS) if r & b}))
            self.stop.wait(0.005)

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7 and parts[0].replace(".", "").isdigit():
                self.rows.append((float(parts[0]), float(parts[1]),
                                  {n for n, v in zip(self.NAMES, parts[3:]) if v == "Active"}))

    def __exit__(self, *exc):
        self.stop.set()
        if self.nvml:
            self.thread.join(timeout=2)
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(r[0] for r in self.rows),
                "sm_max_mhz": max(r[1] for r in self.rows),
                "reasons": sorted(set().union(*(r[2] for r in self.rows))),
                "samples": len(self.rows), "source": "nvml" if self.nvml else "nvidia-smi",
                **({"nvml_error": self.nvml_error} if self.nvml_error else {})}


def max_over_ranks(x: float, world: int, device=None) -> float:
    """Largest value of x over the ranks (x itself when world == 1)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Whole-job rate: the units every rank processed over the slowest rank's time."""
    return units_per_rank * world / seconds_max


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ----------------------------------------------------------------------------------
class OracleSample:
    """The FP64 oracle as it stands, on a bounded sample of the workload: the
    full-grid fluid solve plus every `subsample`-th particle of each species,
    started as the GPU arm starts them (zero slip: an inertial particle takes
    the interpolated fluid velocity at its start, from the interpolating
    spline coefficients for the B-spline scheme).  Built once; each step()
    times one coupled step (fluid step, then the particle step between the
    two levels) and returns (fluid seconds, particle seconds)."""

    def __init__(self, wl, scheme, subsample=64):
        import oracle
        self.oracle, self.wl, self.scheme, self.subsample = oracle, wl, scheme, subsample
        self.flow = oracle.Flow(wl.n, wl.nu, wl.dt, wl.omega0())
        f = self.flow.fields(("u", "v"))
        self.level = (f["u"], f["v"])
        su, sv = self._stencil(*self.level)
        self.sets = []
        for sp in wl.species:
            xy = inputs.uniform_positions(sp.count, sp.seed)[::subsample]
            x, y = xy[:, 0].copy(), xy[:, 1].copy()
            vx = vy = None
            if sp.st > 0:
                vx, vy = oracle.interp(su, scheme, x, y), oracle.interp(sv, scheme, x, y)
            self.sets.append((sp, x, y, vx, vy))
        self.sampled = sum(len(s[1]) for s in self.sets)

    def _stencil(self, u, v):
        if self.scheme == 2:
            return self.oracle.bspline_prefilter(u), self.oracle.bspline_prefilter(v)
        return u, v

    def step(self):
        o = self.oracle
        t0 = time.perf_counter()
        self.flow.step(1)
        f = self.flow.fields(("u", "v"))
        un1, vn1 = f["u"], f["v"]
        a, b = self._stencil(*self.level)
        c, d = self._stencil(un1, vn1)
        t1 = time.perf_counter()
        for sp, x, y, vx, vy in self.sets:
            o.particles_rk4(self.scheme, self.wl.dt, sp.st, a, b, c, d, x, y, vx, vy)
        t2 = time.perf_counter()
        self.level = (un1, vn1)
        return t1 - t0, t2 - t1

    def rate(self, t_fluid, t_part):
        """Particle-steps/s of the full workload for one step that took
        t_fluid + t_part (particle time scaled up by the subsample)."""
        return self.wl.particles / (t_fluid + t_part * self.subsample)

    def describe(self, steps):
        return (f"{steps} coupled steps of the {self.wl.n}^2 fluid solve plus every "
                f"{self.subsample}th particle of each species ({self.sampled} particles, zero slip "
                f"as on the GPU); particle time scaled x{self.subsample} to the full "
                f"{self.wl.particles} particles")


def cpu_oracle_rate(wl, scheme, budget_s=12.0, subsample=64, max_steps=40):
    """The oracle on a bounded sample (OracleSample), stepped until max_steps
    or budget_s.  Returns (particle-steps/s, fluid steps/s, cores, description)."""
    import oracle
    smp = OracleSample(wl, scheme, subsample)
    t_fluid = t_part = 0.0
    steps = 0
    t_start = time.perf_counter()
    while steps < max_steps and (time.perf_counter() - t_start) < budget_s:
        a, b = smp.step()
        t_fluid += a
        t_part += b
        steps += 1
    ps = smp.rate(t_fluid / steps, t_part / steps)
    return ps, steps / t_fluid, oracle.num_threads(), smp.describe(steps)


def cpu_oracle_config1():
    """The FP64 oracle on the Taylor-Green case in full (64^2, 200 steps,
    4096 tracers, bilinear): wall seconds and rates on this host's cores."""
    import oracle
    wl = inputs.taylor_green_64()
    sp = wl.species[0]
    t0 = time.perf_counter()
    flow = oracle.Flow(wl.n, wl.nu, wl.dt, wl.omega0())
    f = flow.fields(("u", "v"))
    lvl = (f["u"], f["v"])
    xy = inputs.uniform_positions(sp.count, sp.seed)
    x, y = xy[:, 0].copy(), xy[:, 1].copy()
    t_fluid = 0.0
    for _ in range(wl.steps):
        a = time.perf_counter()
        flow.step(1)
        f = flow.fields(("u", "v"))
        t_fluid += time.perf_counter() - a
        oracle.particles_rk4(0, wl.dt, 0.0, lvl[0], lvl[1], f["u"], f["v"], x, y)
        lvl = (f["u"], f["v"])
    wall = time.perf_counter() - t0
    return {"workload": "taylor_green_64 in full: 64^2, 200 steps, 4096 tracers, bilinear",
            "seconds": wall, "particle_steps_per_s": sp.count * wl.steps / wall,
            "fluid_steps_per_s": wl.steps / t_fluid, "cores": oracle.num_threads()}


def run_reference(args, wl, scheme, world, rank):
    """The reference arm: the FP64 oracle on the host cores, on the bounded
    sample of OracleSample (set up once), W untimed coupled steps, then K
    timed ones; value = the workload's particle-steps over the K steps' time."""
    if rank != 0:
        return
    import oracle
    smp = OracleSample(wl, scheme)
    for _ in range(args.warmup):
        smp.step()
    t_fluid = t_part = 0.0
    for _ in range(args.steps):
        a, b = smp.step()
        t_fluid += a
        t_part += b
    value = smp.rate(t_fluid / args.steps, t_part / args.steps)
    cores = oracle.num_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "particle-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * wl.particles / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(wl, args.scheme),
            "fluid_steps_per_s": args.steps / t_fluid,
            "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": cores,
                             "kind": "oracle", "sample": smp.describe(args.steps)},
            "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def step_working_set_bytes(wl):
    """Distinct device bytes one coupled step touches: the particle state it
    streams (cell + offset, + velocity for inertial particles), the spectral
    half-planes (omega-hat high and low parts, AB2 history, N-hat and the four
    derivative planes), the five physical planes (u, v, omega_x, omega_y, N)
    and the two level pairs."""
    n = wl.n
    state = sum(s.count * (COMPULSORY_INERTIAL if s.st > 0 else COMPULSORY_TRACER) // 2
                for s in wl.species)
    return state + 8 * 8 * n * (n // 2 + 1) + 5 * 4 * n * n + 2 * 16 * n * n


def config_of(wl, scheme_name):
    ws = step_working_set_bytes(wl)
    return {"workload": wl.name, "n": wl.n, "nu": wl.nu, "dt": wl.dt,
            "species": [{"count": s.count, "st": s.st} for s in wl.species],
            "particles": wl.particles, "scheme": scheme_name, "sort_every": SORT_EVERY,
            "positions": "split precision: int32 image + cell index + fp32 offset",
            "l2": (f"inputs larger than L2: each coupled step touches {ws / 2**20:.0f} MiB "
                   f"(particle state + fluid planes + level pairs) against a {L2_BYTES >> 20} MiB "
                   f"L2; a {FLUSH_BYTES >> 20} MiB write also flushes L2 before every call of "
                   f"{CHUNK} timed steps, outside the events"),
            "parallelism": "replicas (one independent simulation per GPU)"}


def roofline_point(species, n, launch_ms, peak, traffic=None):
    """Roofline figures of one particle-step launch over `species` (list of
    (count, st)) on an n^2 field, launch_ms long: the algorithmic bytes
    (48 / 64 B per particle-step plus the field pair), this layout's
    compulsory bytes (24 / 40 B plus the field pair) and, if known, the DRAM
    bytes ncu measured for one launch."""
    t = launch_ms * 1e-3
    pair = FIELD_PAIR_BYTES_PER_NODE * n * n
    alg = sum(c * (BYTES_INERTIAL if st > 0 else BYTES_TRACER) for c, st in species) + pair
    comp = sum(c * (COMPULSORY_INERTIAL if st > 0 else COMPULSORY_TRACER) for c, st in species) + pair
    out = {"launch_ms": launch_ms, "particle_steps_per_s": sum(c for c, _ in species) / t,
           "achieved": alg / t / 1e9, "frac": alg / t / 1e9 / peak, "bytes_per_launch": alg,
           "compulsory": {"bytes_per_launch": comp, "achieved": comp / t / 1e9,
                          "frac": comp / t / 1e9 / peak},
           "dram": None}
    if traffic is not None:
        out["dram"] = {"bytes_per_launch": traffic, "achieved": traffic / t / 1e9,
                       "frac": traffic / t / 1e9 / peak,
                       "source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch "
                                 "(committed profile of the current kernel source)"}
    return out


def run_ensemble(args, dev, members=64, steps=20):
    """Config 4: independent decaying-turbulence members of uneven sizes, the
    batched engine (autotuned) against one-simulation-at-a-time launches of
    the same members on one stream.  Particle-steps/s of both."""
    import torch
    from paper_2607_17836_b300 import elpath
    wls = inputs.ensemble_members(members)
    stream = torch.cuda.Stream(dev)
    flows = []
    for wl in wls:
        sp = wl.species[0]
        g = elpath.Flow(wl.n, wl.nu, wl.dt, wl.omega0(), interp=0, max_species=1,
                        max_particles=sp.count, sort_every=SORT_EVERY, stream=stream, device=dev)
        g.set_particles(0, inputs.uniform_positions(sp.count, sp.seed), sp.st)
        flows.append(g)
    total = sum(wl.particles for wl in wls)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for g in flows:                      # warm-up: graphs captured, first re-binning done
        g.step(3)
    stream.synchronize()
    ev[0].record(stream)
    for _ in range(steps):
        for g in flows:
            g.step(1)
    ev[1].record(stream)
    stream.synchronize()
    seq_ms = ev[0].elapsed_time(ev[1])
    batch = elpath.Batch(members, device=dev)
    for g in flows:
        batch.add(g)
    tuning = batch.autotune(trial_steps=4)
    batch.step(3)
    launches0 = batch.kernel_launches()
    ev[2].record(batch.stream)
    batch.step(steps)
    ev[3].record(batch.stream)
    batch.synchronize()
    bat_ms = ev[2].elapsed_time(ev[3])
    launches = (batch.kernel_launches() - launches0) / steps
    batch.close()
    # the same members in a batch with one FFT pool per grid size of the
    # members on cuFFT transforms (each member's transforms batched with the
    # others of its size; the fused members share the fused kernels' launches)
    sizes = {n: sum(1 for w in wls if w.n == n) for n in (256, 512, 1024)}
    cufft_sizes = {n: sum(1 for w, g in zip(wls, flows) if w.n == n and not g.fused) for n in sizes}
    pooled = elpath.Batch(members, device=dev)
    pool_bytes = sum(pooled.add_fft_pool(n, c) for n, c in cufft_sizes.items() if c > 0)
    for g in flows:
        pooled.add(g)
    pooled.step(3)
    ev[2].record(pooled.stream)
    pooled.step(steps)
    ev[3].record(pooled.stream)
    pooled.synchronize()
    pool_ms = ev[2].elapsed_time(ev[3])
    pooled.close()
    out = {"workload": f"{members} decaying-turbulence members, n in {{256, 512, 1024}}, "
                       f"1e4-1e6 particles each (log-uniform), St in {{0, 0.1, 1, 10}}",
           "members": members, "particles": total, "steps": steps,
           "sizes": {str(n): c for n, c in sizes.items()},
           "batched_particle_steps_per_s": total * steps / (pool_ms * 1e-3),
           "sequential_particle_steps_per_s": total * steps / (seq_ms * 1e-3),
           "speedup": seq_ms / pool_ms, "batched_ms_per_step": pool_ms / steps,
           "sequential_ms_per_step": seq_ms / steps,
           "batched_launches_per_step": launches,
           "fft_pools": {"bytes": pool_bytes,
                         "without_pools_particle_steps_per_s": total * steps / (bat_ms * 1e-3),
                         "without_pools_ms_per_step": bat_ms / steps},
           "tuning": tuning}
    for g in flows:
        g.close()
    torch.cuda.empty_cache()
    return out


def run_serving(dev, count=200, rate=20.0, budget_gb=120.0, timeout=None):
    """Config 5: the served stream (grids 128^2-2048^2, 1e3-1e7 particles,
    St in {0, 0.1, 1, 10}, bilinear or Catmull-Rom, 100-2000 steps), its
    first `count` requests, arriving as the configured 20/s Poisson stream
    with its clock scaled to `rate` requests/s; HBM-footprint admission."""
    import torch
    from paper_2607_17836_b300 import serve
    reqs = inputs.served_requests(count=count)
    pools = {128: 4}   # FFT-pool slots per grid size whose bilinear / Catmull-Rom flows use cuFFT
    srv = serve.Server(hbm_budget=int(budget_gb * 2**30), max_members=64, tick_steps=50,
                       device=dev, fft_pool_slots=pools)
    t0 = time.perf_counter()
    results = srv.run(reqs, time_scale=20.0 / rate, timeout=timeout)
    wall = time.perf_counter() - t0
    srv.close()
    torch.cuda.empty_cache()
    lat = serve.latency_summary(results)
    span = max(r.arrival for r in reqs)
    work = sum(r.workload.particles * r.workload.steps for r in reqs)
    return {"workload": f"first {count} of the 2000 requests of the served stream, Poisson "
                        f"arrivals at {rate:g} requests/s (the 20/s stream's clock scaled)",
            "requests": count, "arrival_rate_per_s": rate, "completed": len(results),
            "arrivals_span_s": span, "wall_s": wall, "latency": lat,
            "particle_steps_per_s": srv.particle_steps / wall,
            "offered_particle_steps_per_s": work / span if span > 0 else None,
            "requests_per_s": len(results) / wall, "peak_hbm_gb": srv.peak_used / 2**30,
            "hbm_budget_gb": budget_gb, "fft_pool_slots": {str(n): k for n, k in pools.items()}}


def run_serving_vs_sequential(dev, count=32, budget_gb=120.0):
    """The served form against one simulation at a time, on the same work:
    the served stream's first `count` requests, all present at the start,
    (a) served together (continuous batching, FFT pools, host inputs
    prepared on the server's thread pool) and (b) run one after another, each
    alone (inputs, flow creation, its steps, statistics, teardown).
    Particle-steps/s of both over their wall time; each result is the same
    alone and in the mix (tests/test_gpu_configs.py)."""
    import torch
    from paper_2607_17836_b300 import serve
    reqs = inputs.served_requests(count=count)
    work = sum(r.workload.particles * r.workload.steps for r in reqs)
    pools = {128: 4}
    srv = serve.Server(hbm_budget=int(budget_gb * 2**30), max_members=64, tick_steps=50,
                       device=dev, fft_pool_slots=pools)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    srv.run(inputs.served_requests(count=count), time_scale=0.0)
    served_s = time.perf_counter() - t0
    srv.close()
    torch.cuda.empty_cache()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for req in reqs:
        g = serve.build_flow(req, None, dev)
        g.step(req.workload.steps)
        g.stats()
        g.close()
    seq_s = time.perf_counter() - t0
    return {"workload": f"first {count} requests of the served stream, all present at the start",
            "particle_steps": work, "served_s": served_s, "one_at_a_time_s": seq_s,
            "served_particle_steps_per_s": work / served_s,
            "one_at_a_time_particle_steps_per_s": work / seq_s, "speedup": seq_s / served_s}


# Sec. 5.2 with the paper's 2 km domain mapped onto [0, 2 pi): lengths and
# speeds scale by pi (k = 1, alpha = 3.6 pi, eps = 0.3 L = 0.6 pi), times stay.
KINEMATIC_PAPER = dict(alpha=3.6 * math.pi, k=1.0, eps=0.6 * math.pi, omega=1.8, phi=0.0)


def run_kinematic(count=1000, n=128, dt=1e-3, marks=(1000, 10_000, 100_000)):
    """The tracer benchmark of Sec. 5.2 at the paper's size: 1000 tracers in
    the oscillating Taylor-Green flow for 100 h (1e5 steps of 1e-3 h), by the
    three routes; msd in km^2 (lengths / pi) at 1, 10 and 100 h."""
    import torch
    from paper_2607_17836_b300 import elpath
    xy = inputs.uniform_positions(count, 7)
    routes = {"analytic": (elpath.ANALYTIC, 0), "velocity_bilinear": (0, 0),
              "streamfunction_bilinear": (0, 1)}
    out = {"workload": f"oscillating Taylor-Green (Sec. 5.2), {count} tracers, {n}^2 grid "
                       f"(the paper's 100^2 rounded up to a power of two), dt = {dt} h, "
                       f"{marks[-1]} steps", "routes": {}}
    scale = 1.0 / math.pi ** 2  # (2 pi / L)^2 with L = 2 km
    for name, (interp, tv) in routes.items():
        g = elpath.Flow(n, 0.0, dt, None, interp=interp, max_species=1, max_particles=count,
                        tracer_velocity=tv, kinematic=KINEMATIC_PAPER, sort_every=0)
        g.set_particles(0, xy, 0.0)
        st = g.stream
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        done, series, ms = 0, [], 0.0
        for mark in marks:
            e0.record(st)
            g.step(mark - done)
            e1.record(st)
            st.synchronize()
            ms += e0.elapsed_time(e1)
            done = mark
            s = g.stats()
            series.append({"t_h": s["t"], "msd_km2": (s["msd"][0][0] + s["msd"][0][1]) * scale,
                           "msd_sem_km2": math.hypot(*s["msd_sem"][0]) * scale,
                           "diffusivity_km2_per_h": (s["diffusivity"][0][0] + s["diffusivity"][0][1]) * scale})
        out["routes"][name] = {"ms_per_step": ms / done, "particle_steps_per_s": count * done / (ms / 1e3),
                               "series": series}
        g.close()
    a = out["routes"]["analytic"]["series"][-1]["msd_km2"]
    out["msd_rel_diff_vs_analytic_at_end"] = {
        k: abs(v["series"][-1]["msd_km2"] - a) / a for k, v in out["routes"].items() if k != "analytic"}
    return out


def run_transport(wl, steps=(500, 1000, 2000)):
    """Particle-number convergence (Sec. 5.5) on the 1024^2 decaying field:
    100, 500, 1000 and 2000 tracers in one flow; msd, its standard error and
    D = msd / 2t per count, and the largest pairwise msd gap in units of the
    combined standard error."""
    from paper_2607_17836_b300 import elpath
    sets = [(100, 31), (500, 32), (1000, 33), (2000, 34)]
    g = elpath.Flow(wl.n, wl.nu, wl.dt, wl.omega0(), interp=0, max_species=len(sets),
                    max_particles=sum(c for c, _ in sets), sort_every=20)
    for k, (c, seed) in enumerate(sets):
        g.set_particles(k, inputs.uniform_positions(c, seed), 0.0)
    done, rows = 0, []
    for mark in steps:
        g.step(mark - done)
        done = mark
        s = g.stats()
        z = 0.0
        for i in range(len(sets)):
            for j in range(i + 1, len(sets)):
                for a in range(2):
                    bound = math.hypot(s["msd_sem"][i][a], s["msd_sem"][j][a])
                    if bound > 0:
                        z = max(z, abs(s["msd"][i][a] - s["msd"][j][a]) / bound)
        rows.append({"t": s["t"], "max_gap_in_sem": z,
                     "by_count": {str(c): {"msd": list(s["msd"][k]), "msd_sem": list(s["msd_sem"][k]),
                                           "diffusivity": list(s["diffusivity"][k])}
                                  for k, (c, _) in enumerate(sets)}})
    g.close()
    return {"workload": "decaying turbulence 1024^2 (the config-2 field), tracers 100/500/1000/2000",
            "series": rows}


def run_ours(args, wl, scheme, world, rank, local):
    import torch
    import torch.distributed as dist
    from paper_2607_17836_b300 import elpath

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w0 = wl.omega0()
    flow = elpath.Flow(wl.n, wl.nu, wl.dt, w0, interp=scheme, max_species=len(wl.species),
                       max_particles=wl.particles, sort_every=SORT_EVERY, device=dev)
    xys = [inputs.uniform_positions(s.count, s.seed + 1000 * rank) for s in wl.species]
    for k, s in enumerate(wl.species):
        flow.set_particles(k, xys[k], s.st)
    stream = flow.stream
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)

    # Warm-up: the autotuner's trial windows (real steps; no result depends on
    # the settings it picks), then W plain steps.
    tuning = flow.autotune(trial_steps=5) if not args.no_autotune else flow.tuning()
    for _ in range(args.warmup):
        flow.step(1)
    stream.synchronize()

    # Timed region: K coupled steps, issued as calls of CHUNK steps (inside a
    # call the fluid step of n+1 overlaps the particle step of n); an L2 flush
    # (256 MiB write) precedes every call, outside its event pair.
    chunks = [CHUNK] * (args.steps // CHUNK) + ([args.steps % CHUNK] if args.steps % CHUNK else [])
    starts = [torch.cuda.Event(enable_timing=True) for _ in chunks]
    ends = [torch.cuda.Event(enable_timing=True) for _ in chunks]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    launches0 = flow.kernel_launches()
    with ClockSampler(local, dev) as clocks:
        t_wall0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for k, c in enumerate(chunks):
                flush.fill_(k & 0xFF)
                starts[k].record(stream)
                flow.step(c)
                ends[k].record(stream)
        stream.synchronize()
        t_wall = time.perf_counter() - t_wall0
    torch.cuda.synchronize(dev)
    launches = flow.kernel_launches() - launches0
    chunk_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = max_over_ranks(float(sum(chunk_ms)), world, dev)
    if world > 1:
        dist.barrier()

    # Solve latency of one coupled step: LATENCY_SAMPLES calls of one step
    # each (fluid step, then particle step: nothing to overlap inside a call
    # of one), every one preceded by an L2 flush outside its event pair.
    lat_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(LATENCY_SAMPLES)]
    with torch.cuda.stream(stream):
        for k, (e0, e1) in enumerate(lat_ev):
            flush.fill_((k + 1) & 0xFF)
            e0.record(stream)
            flow.step(1)
            e1.record(stream)
    stream.synchronize()
    lat_ms = sorted(e0.elapsed_time(e1) for e0, e1 in lat_ev)

    # Per-stage times (direct launches with events between the stages).
    prof = [flow.profile_step() for _ in range(20)]
    fluid_ms = statistics.mean(p["fluid"] for p in prof)
    part_ms = statistics.mean(p["particles"] for p in prof)
    peak, peak_kind = measured_peaks()
    traffic_pps = recorded_traffic(args.scheme)
    traffic = traffic_pps * wl.particles if traffic_pps is not None else None
    mix = [(s.count, s.st) for s in wl.species]
    point4 = roofline_point(mix, wl.n, part_ms, peak, traffic)

    # The fluid solver alone as it runs inside el_step_coupled (captured
    # graphs): a flow with no particles, CUDA events around 500 steps.
    solo = elpath.Flow(wl.n, wl.nu, wl.dt, w0, interp=scheme, max_species=0)
    solo.step(10)
    fe0, fe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fe0.record(solo.stream)
    solo.step(500)
    fe1.record(solo.stream)
    solo.stream.synchronize()
    fluid_graph_ms = fe0.elapsed_time(fe1) / 500
    solo.close()

    # The roofline workload of the particle stage: 1024^2 with 16M inertial
    # particles at St = 1 in one species (same fluid, same scheme).
    point16 = None
    if not args.no_roofline16:
        big = 16_000_000
        g16 = elpath.Flow(wl.n, wl.nu, wl.dt, w0, interp=scheme, max_species=1,
                          max_particles=big, sort_every=SORT_EVERY, device=dev)
        g16.set_particles(0, inputs.uniform_positions(big, 99 + rank), 1.0)
        g16.autotune(trial_steps=4)
        for _ in range(3):
            g16.step(1)
        pr = [g16.profile_step() for _ in range(10)]
        ms16 = statistics.mean(p["particles"] for p in pr)
        t16 = recorded_profile(args.scheme).get("dram_bytes_per_particle_step_16M")
        point16 = roofline_point([(big, 1.0)], wl.n, ms16, peak,
                                 float(t16) * big if t16 is not None else None)
        point16["workload"] = "1024^2 fluid, 16M inertial particles (St = 1), one species"
        g16.close()
        del g16
        torch.cuda.empty_cache()
    del flush

    # End to end through the public API: particles from pinned host memory,
    # K coupled steps, statistics and every particle state back to pinned
    # memory.  The pinned buffers are allocated once and used by one untimed
    # round first: the first DMA into freshly pinned pages is several times
    # slower (16 MB: 5.1 ms the first time, 0.30 ms after), a one-time cost a
    # caller that keeps its buffers pays once.
    pinned_in = [torch.from_numpy(xy).pin_memory() for xy in xys]
    pinned_xy = [torch.empty((s.count, 2), dtype=torch.float64).pin_memory() for s in wl.species]
    pinned_v = [torch.empty((s.count, 2), dtype=torch.float64).pin_memory() for s in wl.species]

    def e2e_round():
        t0 = time.perf_counter()
        for k, s in enumerate(wl.species):
            flow.set_particles(k, pinned_in[k].numpy(), s.st)
        t1 = time.perf_counter()
        flow.step(args.steps)
        st = flow.stats()                 # waits for the steps
        t2 = time.perf_counter()
        for k, s in enumerate(wl.species):
            flow.particles_into(k, pinned_xy[k].numpy(), pinned_v[k].numpy() if s.st > 0 else None)
        t3 = time.perf_counter()
        return t3 - t0, st, {"upload_ms": 1e3 * (t1 - t0), "steps_and_stats_ms": 1e3 * (t2 - t1),
                             "readback_ms": 1e3 * (t3 - t2)}

    e2e_round()                           # untimed: first touch of the pinned buffers
    torch.cuda.synchronize(dev)
    e2e_s, st, e2e_phases = e2e_round()
    h2d = sum(xy.nbytes for xy in xys)
    d2h = sum(s.count * 16 * (2 if s.st > 0 else 1) for s in wl.species)
    e2e_value = aggregate_rate(wl.particles * args.steps, world, max_over_ranks(e2e_s, world, dev))

    if rank != 0:
        return
    # The gather's L2 side (the level pair, 16 N^2 B, is L2-resident): snapshot
    # bytes per particle-step over the particle stage's time, and the L2
    # throughput ncu measured for the same kernel (percent of the hardware's
    # peak; a library copy or reduction does not reach that peak, so none is
    # timed here as a denominator).
    parts_per_s = wl.particles / (part_ms * 1e-3)
    try:
        lts_pct = float(recorded_profile(args.scheme)["lts_throughput_pct"])
    except (KeyError, ValueError):
        lts_pct = None
    gather = {"scheme": args.scheme, "unit": "GB/s",
              "plain_bytes_per_particle_step": GATHER_PLAIN[scheme],
              "cached_bytes_per_particle_step": GATHER_CACHED[scheme],
              "achieved_plain": GATHER_PLAIN[scheme] * parts_per_s / 1e9,
              "achieved_cached": GATHER_CACHED[scheme] * parts_per_s / 1e9,
              "l2_throughput_pct_of_peak": lts_pct,
              "l2_source": "ncu lts__throughput of the same kernel and workload "
                           "(profiles/k_rk4_<scheme>_traffic.txt), null if the kernel changed since"}
    value = aggregate_rate(wl.particles * args.steps, world, total_ms * 1e-3)
    p50 = lat_ms[len(lat_ms) // 2]
    p99 = lat_ms[min(len(lat_ms) - 1, int(math.ceil(0.99 * len(lat_ms))) - 1)]
    roofline = {"bound": "hbm", "achieved": point4["achieved"], "peak": peak, "unit": "GB/s",
                "frac": point4["frac"], "traffic": traffic,
                "kernel": "k_rk4 (one launch: every species of one step)",
                "peak_kind": peak_kind, "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth)",
                "bytes_per_particle_step": {"tracer": BYTES_TRACER, "inertial": BYTES_INERTIAL,
                                            "plus_per_launch": "16 N^2 (level pair)"},
                "compulsory_bytes_per_particle_step": {"tracer": COMPULSORY_TRACER,
                                                       "inertial": COMPULSORY_INERTIAL},
                "at_4M_mix": point4, "at_16M_inertial": point16}
    line = {"metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": config_of(wl, args.scheme),
            "fluid_steps_per_s": 1e3 / fluid_graph_ms,
            "fluid_steps_per_s_direct_launches": 1e3 / fluid_ms,
            "coupled_steps_per_s": 1e3 * args.steps / total_ms,
            "latency_ms": {"p50": p50, "p99": p99, "samples": len(lat_ms), "min": lat_ms[0],
                           "max": lat_ms[-1],
                           "what": "device time of one coupled step called alone (fluid step, "
                                   "then particle step), L2 flushed before each sample"},
            "stage_ms": {"fluid": fluid_ms, "particles": part_ms},
            "roofline": roofline,
            "e2e": {"value": e2e_value, "unit": "particle-steps/s",
                    "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                    "what": "set_particles from pinned host + K steps + stats + particles back "
                            "into pinned host buffers (allocated once, used by one untimed round)",
                    "phases": e2e_phases},
            "l2_gather": gather, "tuning": tuning,
            "gpu_launches": launches, "wall_s": t_wall,
            "clocks": clocks.summary(), "energy": st["energy"]}
    if not args.no_ensemble:
        line["ensemble"] = run_ensemble(args, dev)
    if not args.no_kinematic:
        line["kinematic_tg"] = run_kinematic()
    if not args.no_transport:
        line["transport"] = run_transport(wl)
    if not args.no_serving:
        line["serving"] = run_serving(dev, count=args.serving_requests, rate=args.serving_rate)
        line["serving_overload"] = run_serving(dev, count=args.overload_requests, rate=20.0)
        line["serving_vs_one_at_a_time"] = run_serving_vs_sequential(dev)
        line["serving_overload"]["note"] = ("the configured 20/s asks for about twice what one "
                                            "GPU serves: queues grow, so its latency describes "
                                            "a backlog, not the service")
    if not args.no_cpu_baseline:
        ps, fsps, cores, desc = cpu_oracle_rate(wl, scheme)
        line["cpu_baseline"] = {"value": ps, "unit": "particle-steps/s", "cores": cores,
                                "kind": "oracle", "sample": desc, "fluid_steps_per_s": fsps,
                                "config1_full": cpu_oracle_config1()}
    print(json.dumps(line), flush=True)


def run_profile_launch(args, wl, scheme):
    """A fixed launch of k_rk4 for ncu: the bench workload ("mix": 4 species
    x 1M) or the roofline point ("16M": 16M inertial particles at St = 1),
    1024^2 ("shear": the 2048^2 shear layer's 16M at St = 1 instead),
    128-thread blocks, re-binning every 20 steps in single cells,
    the stencil gather of --gather (default: automatic); 21 steps (re-binned at step 20), then three
    steps with per-stage CUDA events.  `ncu -k regex:k_rk4 -s 21 -c 1`
    captures the first of those three particle launches.  "batch16M": the
    16M flow alone in a batch (el_batch), 21 batched steps, then 3 more;
    `ncu -k regex:k_batch_rk4 -s 21 -c 1` captures the batched kernel at
    the same point."""
    from paper_2607_17836_b300 import elpath
    if args.profile_launch in ("16M", "batch16M"):
        species = [(16_000_000, 1.0, 99)]
    elif args.profile_launch == "shear":  # the 2048^2 shear layer, 16M at St = 1
        wl = inputs.kelvin_helmholtz_2048()
        species = [(s.count, s.st, s.seed) for s in wl.species]
    else:
        species = [(s.count, s.st, s.seed) for s in wl.species]
    g = elpath.Flow(wl.n, wl.nu, wl.dt, wl.omega0(), interp=scheme, max_species=len(species),
                    max_particles=sum(c for c, _, _ in species), sort_every=SORT_EVERY)
    for k, (c, st, seed) in enumerate(species):
        g.set_particles(k, inputs.uniform_positions(c, seed), st)
    gather = {"auto": elpath.GATHER_AUTO, "registers": elpath.GATHER_REGISTERS,
              "shared": elpath.GATHER_SHARED}[args.gather]
    g.set_tuning(128, SORT_EVERY, 0, gather)
    if args.profile_launch == "batch16M":
        batch = elpath.Batch(2)
        batch.add(g)
        batch.step(21)
        batch.step(3)
        batch.synchronize()
        print(json.dumps({"batched_steps": 24, "particles": sum(c for c, _, _ in species)}), flush=True)
        batch.remove(g)
        batch.close()
        g.close()
        return
    g.step(21)
    for _ in range(3):
        print(json.dumps(g.profile_step()), flush=True)
    g.close()


def run_profile_ensemble(args):
    """A fixed run of the 64-member ensemble for ncu: the batch as the bench
    builds it (one FFT pool per grid size of members on cuFFT transforms, no
    autotuning), 3 steps, then 2 more.  Its steps run inside the NVTX range
    el_batch_step, so `ncu --nvtx --nvtx-include "el_batch_step/"` captures
    only their kernels."""
    import torch
    from paper_2607_17836_b300 import elpath
    wls = inputs.ensemble_members(64)
    batch = elpath.Batch(64)
    flows = []
    for wl in wls:
        sp = wl.species[0]
        g = elpath.Flow(wl.n, wl.nu, wl.dt, wl.omega0(), interp=0, max_species=1,
                        max_particles=sp.count, sort_every=SORT_EVERY)
        g.set_particles(0, inputs.uniform_positions(sp.count, sp.seed), sp.st)
        flows.append(g)
    for n in (256, 512, 1024):
        k = sum(1 for w, g in zip(wls, flows) if w.n == n and not g.fused)
        if k:
            batch.add_fft_pool(n, k)
    for g in flows:
        batch.add(g)
    batch.step(3)
    batch.synchronize()
    batch.step(2)
    batch.synchronize()
    print(json.dumps({"members": len(flows), "steps": 5,
                      "sizes": {str(n): sum(1 for w in wls if w.n == n) for n in (256, 512, 1024)}}))
    batch.close()
    for g in flows:
        g.close()


def run_profile_served(args):
    """A fixed batch of the served stream's first 32 requests for ncu: their
    flows as the server builds them, one FFT pool of 4 slots for the 128^2
    members (as the server holds it), 3 steps, then 2 more.  The steps run
    inside the NVTX range el_batch_step, so `ncu --nvtx --nvtx-include
    "el_batch_step/"` captures only their kernels."""
    import torch
    from paper_2607_17836_b300 import elpath, serve
    reqs = inputs.served_requests(count=32)
    dev = torch.device("cuda:0")
    batch = elpath.Batch(64)
    batch.add_fft_pool(128, 4)
    flows = [serve.build_flow(r, None, dev) for r in reqs]
    for g in flows:
        batch.add(g)
    batch.step(3)
    batch.synchronize()
    batch.step(2)
    batch.synchronize()
    print(json.dumps({"members": len(flows), "steps": 5,
                      "grids": {str(n): sum(1 for r in reqs if r.workload.n == n)
                                for n in (128, 256, 512, 1024, 2048)},
                      "schemes": {str(k): sum(1 for r in reqs if r.scheme == k) for k in (0, 1)},
                      "particles": sum(r.workload.particles for r in reqs)}))
    batch.close()
    for g in flows:
        g.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--scheme", default="bilinear", choices=sorted(SCHEMES))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-roofline16", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-kinematic", action="store_true")
    ap.add_argument("--no-transport", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=200,
                    help="requests of the served stream to run (its first N of 2000)")
    ap.add_argument("--serving-rate", type=float, default=6.0,
                    help="arrival rate (requests/s) of the sustained serving run")
    ap.add_argument("--overload-requests", type=int, default=200,
                    help="requests of the served stream run at its configured 20/s")
    ap.add_argument("--profile-launch", choices=["mix", "16M", "batch16M", "shear", "ensemble", "served"], default=None,
                    help="only a fixed k_rk4 launch for ncu (see run_profile_launch), the "
                         "64-member ensemble's batched steps (run_profile_ensemble), or a batch "
                         "of the served stream's first 32 requests (run_profile_served)")
    ap.add_argument("--gather", choices=["auto", "registers", "shared"], default="auto",
                    help="stencil gather of the cubic schemes in --profile-launch")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world, rank, local = dist_setup()
    wl = inputs.decaying_turbulence_1024()
    scheme = SCHEMES[args.scheme]
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend)
    if args.profile_launch:
        import torch
        torch.cuda.set_device(local)
        if args.profile_launch == "ensemble":
            run_profile_ensemble(args)
        elif args.profile_launch == "served":
            run_profile_served(args)
        else:
            run_profile_launch(args, wl, scheme)
        return
    try:
        if args.impl == "reference":
            run_reference(args, wl, scheme, world, rank)
        else:
            run_ours(args, wl, scheme, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
