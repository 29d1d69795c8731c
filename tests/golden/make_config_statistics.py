"""Write the FP64 oracle's long-run particle statistics of the two large workloads.

    python tests/golden/make_config_statistics.py [decaying_turbulence_1024] [kelvin_helmholtz_2048]

Only the FP64 oracle (oracle/) and the seeded input generators run here; the
CUDA library is never loaded.  The output files hold what the GPU's long
chaotic runs are compared with (dispersion and clustering within 1 %):

  * decaying turbulence, 1024^2, 2000 steps (nu = 1e-4, dt = 5e-4): the four
    species (tracers and St = 0.1, 1, 10), every 16th particle of each (62,500
    of 1M), under each of the three interpolation schemes, all driven by one
    FP64 fluid solve (the fluid depends on neither the particles nor the
    scheme); zero-slip start, as the library does;
  * double shear layer, 2048^2, 4000 steps (nu = 5e-5, dt = 2.5e-4): every
    64th of the 16M inertial particles at St = 1 (250,000), Catmull-Rom.

At each checkpoint step the file records, per scheme and species, the
per-axis mean-square displacement (Sec. 5.5) and the clustering index of the
sampled particles and the fluid's E, Z, P; at the last checkpoint also the
unwrapped positions of about 120 particles per species (every 8192nd, or
131072nd, of the species) for a position-error figure.  Running
the first takes about 10 minutes on 8 host cores, the second about 45.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2607_17836_b300 import inputs  # noqa: E402

PLANS = {
    "decaying_turbulence_1024": dict(workload=inputs.decaying_turbulence_1024, stride=16,
                                     position_stride=8192, schemes=(0, 1, 2),
                                     checkpoints=(200, 1000, 2000)),
    "kelvin_helmholtz_2048": dict(workload=inputs.kelvin_helmholtz_2048, stride=64,
                                  position_stride=131072, schemes=(1,),
                                  checkpoints=(200, 1000, 2000, 4000)),
}


def stencil_levels(u, v, scheme):
    """The grid values a scheme's weights act on: interpolating B-spline
    coefficients for the B-spline, the samples themselves otherwise."""
    if scheme == oracle.BSPLINE:
        return oracle.bspline_prefilter(u), oracle.bspline_prefilter(v)
    return u, v


def run(name):
    plan = PLANS[name]
    wl = plan["workload"]()
    stride, pstride = plan["stride"], plan["position_stride"]
    w0 = wl.omega0()
    flow = oracle.Flow(wl.n, wl.nu, wl.dt, w0)
    f = flow.fields(("u", "v"))
    level = (f["u"], f["v"])
    sets = []
    for scheme in plan["schemes"]:
        su, sv = stencil_levels(*level, scheme)
        for k, sp in enumerate(wl.species):
            xy = inputs.uniform_positions(sp.count, sp.seed)[::stride]
            x, y = xy[:, 0].copy(), xy[:, 1].copy()
            vx = vy = None
            if sp.st > 0:  # zero slip: the interpolated fluid velocity at x(0)
                vx, vy = oracle.interp(su, scheme, x, y), oracle.interp(sv, scheme, x, y)
            sets.append(dict(scheme=scheme, species=k, st=sp.st, x=x, y=y, vx=vx, vy=vy,
                             x0=x.copy(), y0=y.copy()))
    out = {"workload": name, "n": wl.n, "nu": wl.nu, "dt": wl.dt, "ic_seed": wl.ic_seed,
           "species": [{"count": s.count, "st": s.st, "seed": s.seed} for s in wl.species],
           "stride": stride, "position_stride": pstride,
           "written_by": "tests/golden/make_config_statistics.py (FP64 oracle only)",
           "oracle_threads": oracle.num_threads(), "checkpoints": {}}
    t0 = time.time()
    done = 0
    for mark in plan["checkpoints"]:
        while done < mark:
            un, vn = level
            flow.step(1)
            f = flow.fields(("u", "v"))
            un1, vn1 = f["u"], f["v"]
            for scheme in plan["schemes"]:
                a, b = stencil_levels(un, vn, scheme)
                c, d = stencil_levels(un1, vn1, scheme)
                for s in sets:
                    if s["scheme"] == scheme:
                        oracle.particles_rk4(scheme, wl.dt, s["st"], a, b, c, d, s["x"], s["y"],
                                             s["vx"], s["vy"])
            level = (un1, vn1)
            done += 1
        e, z, p = flow.diagnostics()
        rows = []
        for s in sets:
            mx, my = oracle.msd(s["x"], s["y"], s["x0"], s["y0"])
            row = {"scheme": s["scheme"], "species": s["species"], "st": s["st"],
                   "msd": [mx, my], "cluster": oracle.cluster_index(s["x"], s["y"]),
                   "sampled": int(s["x"].size)}
            if mark == plan["checkpoints"][-1]:
                pick = slice(0, None, pstride // stride)
                row["positions"] = np.stack([s["x"][pick], s["y"][pick]], 1).tolist()
            rows.append(row)
        out["checkpoints"][str(mark)] = {"energy": e, "enstrophy": z, "palinstrophy": p,
                                         "sets": rows}
        print(f"{name}: step {mark} after {time.time() - t0:.0f} s", flush=True)
    out["seconds"] = time.time() - t0
    path = os.path.join(HERE, f"{name}_statistics.json")
    with open(path, "w") as fh:
        json.dump(out, fh)
        fh.write("\n")
    print("wrote", path)


if __name__ == "__main__":
    for name in (sys.argv[1:] or list(PLANS)):
        run(name)
