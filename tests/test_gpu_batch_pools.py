"""FFT pools of the batched engine (through the C ABI): members of one class
(grid n and inverse-transform plane count) transform together in one batched
cuFFT call per transform.  Their results equal their solo runs within the
parity tolerances (only cuFFT's batched kernels round differently); members
that find no free slot, or no pool of their class, transform alone; N-hat,
carried between steps, follows a member into and out of its slot, and a state
image saved while it sits in a slot resumes bit for bit."""
import ctypes

import numpy as np
import pytest

from paper_2607_17836_b300 import elpath, inputs
from parity import OMEGA_RTOL, POS_ATOL, rel_linf

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# (n, scheme, [(count, St)], nu, dt): three members of the 64^2 bilinear
# class, two of the 128^2 B-spline class (6 planes with the prefilter), one
# 32^2 member with no pool
SPECS = [
    (64, 0, [(3000, 0.0), (1000, 1.0)], 5e-4, 1e-3),
    (64, 0, [(2000, 0.1)], 5e-4, 1e-3),
    (64, 0, [(500, 10.0)], 5e-4, 1e-3),
    (128, 2, [(4000, 1.0)], 1e-4, 5e-4),
    (128, 2, [(1500, 0.0), (700, 0.1)], 1e-4, 5e-4),
    (32, 1, [(800, 1.0)], 1e-3, 2e-3),
]


def make(spec, seed, sort_every=9):
    n, scheme, species, nu, dt = spec
    g = elpath.Flow(n, nu, dt, inputs.decaying_turbulence(n, seed, k0=min(10.0, n / 8)),
                    interp=scheme, max_species=len(species),
                    max_particles=sum(c for c, _ in species), sort_every=sort_every)
    for k, (c, st) in enumerate(species):
        g.set_particles(k, inputs.uniform_positions(c, seed * 10 + k), st)
    return g


def state(g, spec):
    out = [g.field(0)]
    for k, (c, _) in enumerate(spec[2]):
        out.extend(g.particles(k, c))
    return out


def assert_close(a, b):
    assert rel_linf(a[0], b[0]) < OMEGA_RTOL
    for x, y in zip(a[1:], b[1:]):
        assert np.max(np.abs(x - y)) <= POS_ATOL


def solo_states(steps):
    out = []
    for m, spec in enumerate(SPECS):
        g = make(spec, 200 + m)
        g.step(steps)
        out.append(state(g, spec))
        g.close()
    return out


def test_pooled_members_match_their_solo_runs():
    steps = 40
    ref = solo_states(steps)
    batch = elpath.Batch(8)
    batch.add_fft_pool(64, 4)                                  # one slot stays free
    batch.add_fft_pool(128, 1, interp=elpath.BSPLINE)          # the second member finds it full
    flows = [make(spec, 200 + m) for m, spec in enumerate(SPECS)]
    for g in flows:
        batch.add(g)
    batch.step(steps)
    for g, spec, r in zip(flows, SPECS, ref):
        assert g.stats()["step"] == steps
        assert_close(state(g, spec), r)
    l0 = batch.kernel_launches()
    batch.step(2)
    assert batch.kernel_launches() - l0 == 2 * 6                 # our kernels per step unchanged
    batch.close()


def test_slots_are_reused_and_n_hat_follows_the_member():
    # A sits in the pool's only slot for 20 steps and leaves; B then takes
    # the slot.  A state image of B saved while it sits in the slot (its N-hat
    # read from the slot) resumes bit for bit like B itself after B leaves
    # (its N-hat copied back): both continue on per-member transforms.
    a_spec, b_spec = SPECS[0], SPECS[1]
    ref_a = make(a_spec, 31)
    ref_a.step(35)
    ref_b = make(b_spec, 32)
    ref_b.step(30)
    a, b = make(a_spec, 31), make(b_spec, 32)
    batch = elpath.Batch(4)
    batch.add_fft_pool(64, 1)
    batch.add(a)
    batch.step(20)
    batch.remove(a)
    a.step(15)                                                  # alone again, own transforms
    b.step(5)
    batch.add(b)                                                # B takes the freed slot
    batch.step(15)
    image = b.save_state()
    batch.remove(b)
    b.step(10)
    assert_close(state(a, a_spec), state(ref_a, a_spec))
    assert_close(state(b, b_spec), state(ref_b, b_spec))
    c = make(b_spec, 99)
    c.load_state(image)
    c.step(10)
    for x, y in zip(state(b, b_spec), state(c, b_spec)):
        np.testing.assert_array_equal(x, y)
    batch.close()


def test_pool_arguments():
    lib = elpath.load()
    batch = elpath.Batch(2)
    with pytest.raises(elpath.ElpathError):
        batch.add_fft_pool(64, 0)                               # no slots
    with pytest.raises(elpath.ElpathError):
        batch.add_fft_pool(48, 2)                               # not a power of two
    desc = elpath.make_desc(64, 0.0, 1.0)
    need = int(lib.el_batch_fft_pool_bytes(ctypes.byref(desc), 2))
    assert need > 2 * 2 * 4 * 64 * 64 * 4                       # at least the physical planes
    small = torch.empty(need - 4096, dtype=torch.uint8, device="cuda")
    st = lib.el_batch_add_fft_pool(batch._h, ctypes.byref(desc), 2,
                                   ctypes.c_void_p(small.data_ptr()), ctypes.c_size_t(need - 4096))
    assert st == 2                                              # EL_ENOMEM
    batch.close()
