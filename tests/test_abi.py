"""The C-ABI library builds for sm_103a, loads, and exports every entry point include/sweep.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2207_12848_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sweep.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ctypes.CDLL(build.OUT)


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sweep_[a-z_]+)\s*\(", src)))


def test_header_declares_the_binding_exports():
    assert declared_functions() == sorted(_lib.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_struct_layout_matches_header(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "sweep.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\\n", sizeof(sweep_opts), offsetof(sweep_opts, tol_pbc), offsetof(sweep_opts, spin_budget),
         sizeof(sweep_stats), offsetof(sweep_stats, schedule_used));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    vals = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert vals == [ctypes.sizeof(_lib.sweep_opts), _lib.sweep_opts.tol_pbc.offset, _lib.sweep_opts.spin_budget.offset,
                    ctypes.sizeof(_lib.sweep_stats), _lib.sweep_stats.schedule_used.offset]


def test_host_only_entry_points(lib):
    lib.sweep_status_string.restype = ctypes.c_char_p
    assert lib.sweep_status_string(2) == b"dependency graph is cyclic"
    o = _lib.sweep_opts()
    lib.sweep_default_opts(ctypes.byref(o))
    assert o.precision == 32 and o.tol_pbc == 1e-6 and o.max_it_scat == 100


def test_create_without_a_usable_device_fails_cleanly(lib):
    # device index far out of range: an error status, never a crash or a fallback
    h = ctypes.c_void_p()
    assert lib.sweep_create(ctypes.byref(h), 4096, None) != 0
    assert not h.value
