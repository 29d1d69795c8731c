"""CPU checks of the C ABI: the library builds and loads, exports every
symbol include/elpath.h declares, and the ctypes structs match the C layout.
No compute call is made (no GPU here)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2607_17836_b300 import build, elpath

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "elpath.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return elpath.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(el_\w+)\s*\(", text)))


def test_header_declares_the_binding_symbols():
    assert declared_functions() == sorted(elpath.SYMBOLS)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", elpath.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (el_\w+)$", out, flags=re.M))
    for name in declared_functions():
        assert name in exported, name
        assert getattr(lib, name) is not None




def test_struct_layouts_match_c(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(f"""
#include <stdio.h>
#include <stddef.h>
#include "{HEADER}"
int main(void) {{
  printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(el_flow_desc), offsetof(el_flow_desc, nu),
         offsetof(el_flow_desc, dt), offsetof(el_flow_desc, max_particles),
         offsetof(el_flow_desc, sort_every), offsetof(el_flow_desc, tracer_velocity));
  printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(el_stats), offsetof(el_stats, msd),
         offsetof(el_stats, cluster), offsetof(el_stats, np), offsetof(el_stats, finite),
         offsetof(el_stats, msd_sem), offsetof(el_stats, diffusivity));
  return 0;
}}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-o", str(exe), str(src)], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    d = [int(x) for x in lines[0].split()]
    s = [int(x) for x in lines[1].split()]
    D, S = elpath.el_flow_desc, elpath.el_stats
    assert d == [ctypes.sizeof(D), D.nu.offset, D.dt.offset, D.max_particles.offset,
                 D.sort_every.offset, D.tracer_velocity.offset]
    assert s == [ctypes.sizeof(S), S.msd.offset, S.cluster.offset, S.np.offset, S.finite.offset,
                 S.msd_sem.offset, S.diffusivity.offset]


def test_calls_without_device_fail_cleanly(lib):
    bad = elpath.make_desc(100, 1e-3, 1e-3)      # n not a power of two
    assert lib.el_workspace_bytes(ctypes.byref(bad)) == 0
    h = ctypes.c_void_p()
    st = lib.el_create_flow(ctypes.byref(bad), None, None, 0, None, ctypes.byref(h))
    assert st == 1 and not h.value
    assert b"n must be" in lib.el_last_error(None)
    assert lib.el_step_coupled(None, 1) == 1
    assert lib.el_kernel_launches(None) == 0
    assert lib.el_flow_fused(None) == 0
    size = ctypes.c_size_t(0)
    assert lib.el_save_state(None, None, ctypes.byref(size)) == 1
    assert lib.el_load_state(None, None, 0) == 1
