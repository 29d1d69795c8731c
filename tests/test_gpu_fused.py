"""The fused 256^2-2048^2 fluid steps (fused_fluid.cu: pruned transforms
of our own, fused with the AB2 update and the nonlinear term) against the
cuFFT path (ELPATH_FLUID_CUFFT=1, run in a child process), and against the
oracle.

At 1024^2 every plane configuration the step has: 4 planes (bilinear,
Catmull-Rom, raw B-spline), 6 (prefiltered B-spline), 5 and 7 (with the
streamfunction plane of tracer_velocity = 1), each AB2 form; at 2048^2, 512^2
and 256^2 the ones it serves (4 and 6 planes; a 2048-point transform is two
1024-point ones on a warp pair, a 512- or 256-point one is held by a group of
16 or 8 lanes).  The two paths differ only by the rounding of their
transforms, so after 100 steps the vorticity agrees to a few 1e-7 and
positions to a few 1e-8; the physical velocity planes, which the fused step
does not keep, are rebuilt on request.
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from paper_2607_17836_b300 import elpath, inputs
from parity import OMEGA_RTOL, POS_ATOL, OracleRun, record, rel_linf

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N = 1024
CASES = [  # (n, interp, bspline_prefilter, tracer_velocity, ab2_mode): planes
    (N, 0, 1, 0, 0),     # 4
    (N, 1, 1, 0, 1),     # 4, explicit AB2
    (N, 2, 0, 0, 0),     # 4 (raw B-spline)
    (N, 2, 1, 0, 0),     # 6
    (N, 0, 1, 1, 0),     # 5
    (N, 2, 1, 1, 1),     # 7, explicit AB2
    (2048, 0, 1, 0, 0),  # 4
    (2048, 1, 1, 0, 1),  # 4, explicit AB2
    (2048, 2, 1, 0, 0),  # 6
    (512, 0, 1, 0, 0),   # 4
    (512, 2, 1, 0, 1),   # 6, explicit AB2
    (256, 1, 1, 0, 0),   # 4
    (256, 2, 0, 0, 1),   # 4 (raw B-spline), explicit AB2
]

CHILD = textwrap.dedent("""
    import sys, numpy as np
    sys.path.insert(0, {root!r})
    from paper_2607_17836_b300 import elpath, inputs
    n, interp, pre, tv, mode = {case!r}
    w0 = inputs.decaying_turbulence(n, 2)
    g = elpath.Flow(n, 1e-4, 5e-4 * 1024 / n, w0, interp=interp, bspline_prefilter=pre, tracer_velocity=tv,
                    ab2_mode=mode, max_species=2, max_particles=40000, sort_every=20)
    g.set_particles(0, inputs.uniform_positions(20000, 3), 0.0)
    g.set_particles(1, inputs.uniform_positions(20000, 4), 1.0)
    g.step(100)
    st = g.stats()
    np.savez({out!r}, w=g.field(0), u=g.field(1), v=g.field(2), p0=g.particles(0, 20000)[0],
             p1=g.particles(1, 20000)[0], e=np.array([st["energy"], st["enstrophy"], st["palinstrophy"]]))
""")


def run_child(case, out, cufft):
    script = CHILD.format(root=ROOT, case=case, out=out)
    env = dict(os.environ)
    env.pop("ELPATH_FLUID_CUFFT", None)
    if cufft:
        env["ELPATH_FLUID_CUFFT"] = "1"
    r = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True, env=env,
                       timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    return np.load(out)


@pytest.mark.parametrize("case", CASES, ids=["bilinear", "catmull_rom_explicit", "bspline_raw",
                                             "bspline", "psi", "bspline_psi_explicit",
                                             "2048_bilinear", "2048_catmull_rom_explicit", "2048_bspline",
                                             "512_bilinear", "512_bspline_explicit", "256_catmull_rom",
                                             "256_bspline_raw_explicit"])
def test_fused_step_matches_the_cufft_path(case, tmp_path):
    a = run_child(case, str(tmp_path / "fused.npz"), cufft=False)
    b = run_child(case, str(tmp_path / "cufft.npz"), cufft=True)
    name = f"fused vs cuFFT fluid step, {case[0]}^2, case {case[1:]}"
    for key in ("w", "u", "v"):
        d = rel_linf(a[key], b[key])
        record(name, case[1], f"{key} L-inf rel. difference, 100 steps", d, 2e-6)
        assert d < 2e-6, (key, d)
    for key in ("p0", "p1"):
        d = float(np.max(np.abs(a[key] - b[key])))
        record(name, case[1], "max position difference, 100 steps", d, 1e-6)
        assert d < 1e-6, (key, d)
    np.testing.assert_allclose(a["e"], b["e"], rtol=1e-6)


@pytest.mark.parametrize("n", [256, 512, 1024])
def test_fused_step_against_the_oracle_with_the_velocity_planes(n):
    # the fused path is the default at these sizes (4 planes): vorticity and
    # the rebuilt physical velocity against the FP64 oracle after 100 steps
    w0 = inputs.decaying_turbulence(n, 2)
    dt = 5e-4 * 1024 / n
    g = elpath.Flow(n, 1e-4, dt, w0, interp=1, max_species=0)
    assert g.fused
    o = OracleRun(n, 1e-4, dt, w0)
    g.step(100)
    o.step(100)
    f = o.flow.fields(("u", "v", "w"))
    for which, key in ((0, "w"), (1, "u"), (2, "v")):
        d = rel_linf(g.field(which), f[key])
        record(f"fused fluid step, decaying {n}^2", None, f"{key} L-inf rel., 100 steps", d, OMEGA_RTOL)
        assert d < OMEGA_RTOL, (key, d)
    g.close()


def test_fused_step_resumes_bit_for_bit():
    w0 = inputs.decaying_turbulence(N, 5)
    xy = inputs.uniform_positions(30000, 6)

    def make():
        g = elpath.Flow(N, 1e-4, 5e-4, w0, interp=2, max_species=1, max_particles=30000,
                        sort_every=9)
        g.set_particles(0, xy, 1.0)
        return g

    ref = make()
    ref.step(17)
    image = ref.save_state()
    ref.step(23)
    other = make()
    other.step(3)
    other.load_state(image)
    other.step(23)
    np.testing.assert_array_equal(other.field(0), ref.field(0))
    np.testing.assert_array_equal(other.particles(0, 30000)[0], ref.particles(0, 30000)[0])
    np.testing.assert_array_equal(other.field(1), ref.field(1))
    ref.close()
    other.close()
