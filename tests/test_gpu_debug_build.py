"""The EL_CHECK_BOUNDS debug build: the particle kernel checks every
particle's split state (cell index below n, offsets in [0, 1)) and counts
violations in a device word, reported by el_get_stats as EL_ESTATE, with no
trap.  A clean chaotic run must count none; a state image whose particle
offset was altered on the host (checksum recomputed) must be caught.  The
debug library is compiled into a temporary directory and driven from a child
process, so this process keeps the production library."""
import os
import struct
import subprocess
import sys
import textwrap

import pytest

from paper_2607_17836_b300 import build

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import struct, sys
    sys.path.insert(0, {root!r})
    from paper_2607_17836_b300 import elpath, inputs
    elpath.load({lib!r})

    def fnv1a(data):
        h = 1469598103934665603
        for b in data:
            h = ((h ^ b) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
        return h

    # a clean chaotic run, every scheme, tracers and inertial particles
    for interp in (0, 1, 2):
        g = elpath.Flow(64, 1e-3, 1e-3, inputs.decaying_turbulence(64, 5, k0=6.0), interp=interp,
                        max_species=2, max_particles=4000, sort_every=9)
        g.set_particles(0, inputs.uniform_positions(2000, 1), 0.0)
        g.set_particles(1, inputs.uniform_positions(2000, 2), 1.0)
        g.step(150)
        assert g.stats()["finite"]
        g.close()

    # a state image with one particle's offset moved outside [0, 1)
    n, np_ = 32, 100
    g = elpath.Flow(n, 1e-3, 1e-3, inputs.decaying_turbulence(n, 5, k0=4.0), interp=0,
                    max_species=1, max_particles=np_)
    g.set_particles(0, inputs.uniform_positions(np_, 3), 0.0)
    g.step(3)
    img = bytearray(g.save_state())
    hdr = struct.unpack_from("<I", img, 12)[0]
    pad8 = lambda x: (x + 7) // 8 * 8
    nm = n * (n // 2 + 1)
    off = pad8(hdr) + 4 * pad8(nm * 8) + pad8(n * n * 16) + pad8(np_ * 4)  # first offset (x)
    struct.pack_into("<f", img, off, 1.5)
    struct.pack_into("<Q", img, len(img) - 8, fnv1a(bytes(img[:-8])))
    h = elpath.Flow(n, 1e-3, 1e-3, inputs.decaying_turbulence(n, 5, k0=4.0), interp=0,
                    max_species=1, max_particles=np_)
    h.load_state(bytes(img))
    h.step(1)
    try:
        h.stats()
        print("NOT CAUGHT")
    except elpath.ElpathError as e:
        assert e.status == 5, e
        assert "invariant" in str(e), e
        print("CAUGHT", e)
""")


def test_debug_build_counts_invariant_violations(tmp_path):
    lib = str(tmp_path / "libelpath_check.so")
    build.build_to(lib, ["-DEL_CHECK_BOUNDS=1"])  # raises on a compile error
    script = tmp_path / "child.py"
    script.write_text(CHILD.format(root=ROOT, lib=lib))
    out = subprocess.run([sys.executable, str(script)], capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stdout[-2000:] + out.stderr[-2000:]
    assert "CAUGHT" in out.stdout, out.stdout
    assert "particle 0 of species 0" in out.stdout, out.stdout
