"""Shared helpers for the GPU-vs-oracle parity tests (test code only)."""
from __future__ import annotations

import json
import os

import numpy as np

import oracle
from paper_2607_17836_b300 import elpath, inputs

TWO_PI = 2.0 * np.pi

# Tolerances (relative to the FP64 oracle):
GATHER_RTOL = 2e-6        # interpolated velocity: max |err| / max |u|
OMEGA_RTOL = 1e-5         # vorticity L-inf after 100 steps: max |err| / max |omega|
POS_ATOL = 1e-5 * TWO_PI  # particle positions after 200 steps
STATS_RTOL = 1e-2         # long chaotic runs: dispersion and clustering


SCHEME_NAMES = {0: "bilinear", 1: "Catmull-Rom", 2: "B-spline"}


def record(workload, scheme, quantity, value, bound):
    """Append an achieved error (and the bound the test asserts, or None for
    a figure that is reported but not asserted) as one JSON line to the file
    named by EL_PARITY_LOG, when that is set."""
    path = os.environ.get("EL_PARITY_LOG")
    if not path:
        return
    name = SCHEME_NAMES.get(scheme, scheme) if scheme is not None else "-"
    with open(path, "a") as fh:
        fh.write(json.dumps({"workload": workload, "scheme": name, "quantity": quantity,
                             "value": float(value),
                             "bound": None if bound is None else float(bound)}) + "\n")


def write_table(log_path, out_path):
    """Render the recorded errors as a markdown table (worst value per
    workload, scheme and quantity)."""
    rows = {}
    with open(log_path) as fh:
        for line in fh:
            r = json.loads(line)
            key = (r["workload"], r["scheme"], r["quantity"])
            if key not in rows or r["value"] > rows[key]["value"]:
                rows[key] = r
    lines = ["# Achieved errors of the CUDA path against the FP64 oracle",
             "",
             "Written by the GPU parity tests (tests/conftest.py, EL_PARITY_LOG and",
             "EL_PARITY_TABLE): the worst value each test measured, beside the bound it asserts.",
             "",
             "| workload | scheme | quantity | achieved | bound |",
             "|---|---|---|---|---|"]
    for key in sorted(rows):
        r = rows[key]
        bound = "reported" if r["bound"] is None else f"{r['bound']:.3g}"
        lines.append(f"| {r['workload']} | {r['scheme']} | {r['quantity']} | {r['value']:.3g} | "
                     f"{bound} |")
    with open(out_path, "w") as fh:
        fh.write("\n".join(lines) + "\n")


def rel_linf(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def oracle_stencil(u, v, scheme, prefilter=True):
    if scheme == oracle.BSPLINE and prefilter:
        return oracle.bspline_prefilter(u), oracle.bspline_prefilter(v)
    return u, v


class OracleRun:
    """Oracle fluid + any number of (scheme, st, positions) particle sets,
    all driven by one FP64 fluid solve (the fluid does not depend on the
    particles or on the interpolation scheme)."""

    def __init__(self, n, nu, dt, omega0, ab2_mode=0, prefilter=True):
        self.flow = oracle.Flow(n, nu, dt, omega0, ab2_mode)
        self.prefilter = prefilter
        self.sets = []
        f = self.flow.fields(("u", "v"))
        self.level = (f["u"], f["v"])
        self.psi_level = self.flow.psi()

    def add(self, scheme, st, xy, vxy=None, psi=False):
        xy = np.asarray(xy, dtype=np.float64).reshape(-1, 2)
        x, y = xy[:, 0].copy(), xy[:, 1].copy()
        if st > 0:
            if vxy is None:
                su, sv = oracle_stencil(*self.level, scheme, self.prefilter)
                vx, vy = oracle.interp(su, scheme, x, y), oracle.interp(sv, scheme, x, y)
            else:
                vxy = np.asarray(vxy, dtype=np.float64).reshape(-1, 2)
                vx, vy = vxy[:, 0].copy(), vxy[:, 1].copy()
        else:
            vx = vy = None
        self.sets.append({"scheme": scheme, "st": float(st), "x": x, "y": y, "vx": vx, "vy": vy,
                          "x0": x.copy(), "y0": y.copy(), "psi": bool(psi) and st == 0})
        return len(self.sets) - 1

    def step(self, nsteps):
        for _ in range(nsteps):
            un, vn = self.level
            pn = self.psi_level
            self.flow.step(1)
            f = self.flow.fields(("u", "v"))
            un1, vn1 = f["u"], f["v"]
            pn1 = self.flow.psi()
            cache = {}
            for s in self.sets:
                sc = s["scheme"]
                if s["psi"]:
                    key = ("psi", sc)
                    if key not in cache:
                        pre = sc == oracle.BSPLINE and self.prefilter
                        cache[key] = ((oracle.bspline_prefilter(pn) if pre else pn),
                                      (oracle.bspline_prefilter(pn1) if pre else pn1))
                    a, b = cache[key]
                    oracle.tracers_rk4_psi(sc, self.flow.dt, a, b, s["x"], s["y"])
                    continue
                if sc not in cache:
                    cache[sc] = (oracle_stencil(un, vn, sc, self.prefilter),
                                 oracle_stencil(un1, vn1, sc, self.prefilter))
                (a, b), (c, d) = cache[sc]
                oracle.particles_rk4(sc, self.flow.dt, s["st"], a, b, c, d, s["x"], s["y"],
                                     s["vx"], s["vy"])
            self.level = (un1, vn1)
            self.psi_level = pn1

    def positions(self, k):
        s = self.sets[k]
        return np.stack([s["x"], s["y"]], axis=1)

    def velocities(self, k):
        s = self.sets[k]
        return np.stack([s["vx"], s["vy"]], axis=1)


def gpu_flow(n, nu, dt, omega0, interp=0, max_species=1, max_particles=0, sort_every=0,
             ab2_mode=0, prefilter=True, tracer_velocity=0):
    return elpath.Flow(n, nu, dt, omega0, interp=interp, ab2_mode=ab2_mode,
                       bspline_prefilter=prefilter, max_species=max_species,
                       max_particles=max_particles, sort_every=sort_every,
                       tracer_velocity=tracer_velocity)


def decaying(n, seed=2, k0=10.0):
    return inputs.decaying_turbulence(n, seed, k0=k0)
