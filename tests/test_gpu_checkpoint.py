"""Checkpoint and resume through the C ABI (el_save_state / el_load_state).

The state image holds everything a coupled step reads, so a run that is
saved, loaded into another flow (or rewound in place) and stepped on must
reproduce the uninterrupted run bit for bit: vorticity, every particle's
position and velocity, and the FP64 statistics.  Damaged or mismatched
images are refused with the flow left as it was.
"""
import ctypes
import struct

import numpy as np
import pytest

from paper_2607_17836_b300 import elpath, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = [  # (n, interp, tracer_velocity, [(count, St)], nu, dt)
    (64, 0, 0, [(3001, 0.0), (2000, 1.0)], 1e-3, 1e-3),
    (64, 1, 0, [(1500, 0.1)], 5e-4, 1e-3),
    (128, 2, 1, [(2500, 0.0), (777, 10.0)], 1e-4, 5e-4),
]


def make(case, seed, sort_every=7):
    n, interp, tv, species, nu, dt = case
    g = elpath.Flow(n, nu, dt, inputs.decaying_turbulence(n, seed), interp=interp,
                    max_species=len(species), max_particles=sum(c for c, _ in species),
                    sort_every=sort_every, tracer_velocity=tv)
    for k, (c, st) in enumerate(species):
        g.set_particles(k, inputs.uniform_positions(c, seed * 10 + k), st)
    return g


def state(g, case):
    out = [g.field(0)]
    for k, (c, _) in enumerate(case[3]):
        out.extend(g.particles(k, c))
    s = g.stats()
    out.append(np.array([s["energy"], s["enstrophy"], s["palinstrophy"], s["step"]]
                        + [m for pair in s["msd"] for m in pair] + s["cluster"]))
    return out


def assert_bitwise(a, b):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("case", CASES, ids=["bilinear", "catmull_rom", "bspline_psi"])
def test_resume_in_another_flow_is_bitwise(case):
    k_before, k_after = 23, 31
    ref = make(case, 5)
    ref.step(k_before)
    image = ref.save_state()
    u_at_save = ref.field(1)
    ref.step(k_after)
    expect = state(ref, case)
    # a flow with another initial field and other particles (and another
    # re-binning cadence, which enters no result) takes the image over
    other = make(case, 9, sort_every=3)
    other.step(4)
    other.load_state(image)
    assert other.stats()["step"] == k_before
    np.testing.assert_allclose(other.field(1), u_at_save, rtol=0,
                               atol=1e-6 * np.max(np.abs(u_at_save)))
    other.step(k_after)
    assert_bitwise(state(other, case), expect)
    ref.close()
    other.close()


def test_rewind_in_place_and_save_at_step_zero():
    case = CASES[0]
    g = make(case, 3)
    image0 = g.save_state()
    g.step(12)
    image12 = g.save_state()
    g.step(9)
    first = state(g, case)
    g.load_state(image12)
    g.step(9)
    assert_bitwise(state(g, case), first)
    g.load_state(image0)
    g.step(21)
    assert_bitwise(state(g, case), first)
    g.close()


def test_bad_images_are_refused_and_leave_the_flow_unchanged():
    case = CASES[1]
    g = make(case, 4)
    g.step(6)
    image = bytearray(g.save_state())
    good = make(case, 4)
    good.step(6)
    for bad in (bytes(image[:-9]),                                  # truncated
                bytes(image[:100]),
                bytes(image[:200]) + bytes([image[200] ^ 1]) + bytes(image[201:]),  # altered
                b"\0" * len(image)):                                # not an image
        with pytest.raises(elpath.ElpathError) as e:
            g.load_state(bad)
        assert e.value.status == 1
    # another descriptor (dt differs)
    n, interp, tv, species, nu, dt = case
    alien = make((n, interp, tv, species, nu, dt * 0.5), 4)
    with pytest.raises(elpath.ElpathError) as e:
        alien.load_state(bytes(image))
    assert e.value.status == 1
    # a flow too small for the image's particles
    small = elpath.Flow(n, nu, dt, inputs.decaying_turbulence(n, 4), interp=interp,
                        max_species=1, max_particles=100)
    with pytest.raises(elpath.ElpathError) as e:
        small.load_state(bytes(image))
    assert e.value.status == 1
    # a buffer that is too small reports the size it needs
    need = ctypes.c_size_t(16)
    buf = ctypes.create_string_buffer(16)
    lib = elpath.load()
    assert lib.el_save_state(g._h, buf, ctypes.byref(need)) == 1
    assert need.value == len(image)
    # nothing above changed g: it still runs exactly like its twin
    g.step(10)
    good.step(10)
    assert_bitwise(state(g, case), state(good, case))
    for f in (g, good, alien, small):
        f.close()


def test_batch_members_save_but_do_not_load():
    case = CASES[0]
    a = make(case, 6)
    batch = elpath.Batch(2)
    batch.add(a)
    batch.step(5)
    image = a.save_state()
    with pytest.raises(elpath.ElpathError) as e:
        a.load_state(image)
    assert e.value.status == 5
    batch.remove(a)
    b = make(case, 8)
    b.load_state(image)
    ref = make(case, 6)
    ref.step(5)
    a.step(7)
    b.step(7)
    ref.step(7)
    sa, sb, sr = state(a, case), state(b, case), state(ref, case)
    assert_bitwise(sb, sa)       # the image carried the member's state exactly
    assert np.max(np.abs(sa[0] - sr[0])) <= 1e-5 * np.max(np.abs(sr[0]))
    for x, y in zip(sa[1:-1], sr[1:-1]):
        assert np.max(np.abs(x - y)) <= 1e-5 * 2 * np.pi
    batch.close()
    for f in (a, b, ref):
        f.close()


def _fnv1a(data):
    h = 1469598103934665603
    for b in data:
        h = ((h ^ b) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def test_invalid_particle_state_is_refused_before_any_upload():
    # Images whose checksum is valid (recomputed after the edit) but whose
    # particle state is not: cells that index past the grid, offsets outside
    # [0, 1), non-finite velocities or x(0), ids that are not a permutation,
    # counts that the image does not hold.  The library checks them on the
    # host before anything reaches the device, so each is refused with
    # EL_EINVAL and the flow keeps running exactly like its twin.
    case = CASES[0]                       # n = 64: 3001 tracers, 2000 at St = 1
    n = case[0]
    g = make(case, 4)
    g.step(6)
    image = bytes(g.save_state())
    twin = make(case, 4)
    twin.step(6)
    pad8 = lambda x: (x + 7) // 8 * 8
    hdr = struct.unpack_from("<I", image, 12)[0]
    nm = n * (n // 2 + 1)
    at = pad8(hdr) + 4 * pad8(nm * 8) + pad8(n * n * 16)
    sec = {}
    for k, (m, st) in enumerate(case[3]):
        for name, size in (("cell", 4), ("off", 8), ("vel", 8 if st > 0 else 0), ("img", 8),
                           ("id", 4), ("x0", 16)):
            if size:
                sec[(k, name)] = at
                at += pad8(m * size)
    assert at + 8 == len(image)

    def edited(*edits):
        b = bytearray(image)
        for fmt, where, value in edits:
            struct.pack_into(fmt, b, where, value)
        struct.pack_into("<Q", b, len(b) - 8, _fnv1a(bytes(b[:-8])))
        return bytes(b)

    cell5 = struct.unpack_from("<I", image, sec[(0, "cell")] + 4 * 5)[0]
    id10 = struct.unpack_from("<I", image, sec[(0, "id")] + 4 * 10)[0]
    np_at = 24 + ctypes.sizeof(elpath.el_flow_desc) + 16      # header: ... step, since_sort, np[]
    assert struct.unpack_from("<q", image, np_at)[0] == case[3][0][0]
    bad = {
        "cell i = n": edited(("<I", sec[(0, "cell")] + 4 * 5, (cell5 & 0xFFFF0000) | n)),
        "cell j >= n": edited(("<I", sec[(1, "cell")] + 4 * 3, (70 << 16) | 1)),
        "offset 1.5": edited(("<f", sec[(0, "off")] + 8 * 7, 1.5)),
        "offset -0.25": edited(("<f", sec[(1, "off")] + 8 * 2 + 4, -0.25)),
        "offset NaN": edited(("<f", sec[(0, "off")], float("nan"))),
        "velocity inf": edited(("<f", sec[(1, "vel")] + 8 * 3, float("inf"))),
        "duplicate id": edited(("<I", sec[(0, "id")] + 4 * 9, id10)),
        "id = np": edited(("<I", sec[(1, "id")], case[3][1][0])),
        "x0 NaN": edited(("<d", sec[(1, "x0")] + 16 * 4 + 8, float("nan"))),
        "count beyond the image": edited(("<q", np_at, case[3][0][0] + 1)),
    }
    for what, img in bad.items():
        with pytest.raises(elpath.ElpathError) as e:
            g.load_state(img)
        assert e.value.status == 1, what
    # the unedited image still loads (the offsets above were computed right)
    g.load_state(edited())
    g.step(10)
    twin.step(10)
    assert_bitwise(state(g, case), state(twin, case))
    g.close()
    twin.close()
