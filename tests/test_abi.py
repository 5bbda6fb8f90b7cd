"""Host-only checks of the C ABI: the library builds for sm_103a, loads, and
exports every function include/pint.h declares; ctypes struct layouts match
the C compiler's.  No GPU computation is called."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pint.h")


@pytest.fixture(scope="module")
def libpint():
    from paper_2411_09244_gb300 import _lib, build
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    return _lib.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pint_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_five_stage_calls():
    names = declared_functions()
    for n in ("pint_setup_fine_grid", "pint_build_multiscale_spaces", "pint_assemble_reduced",
              "pint_parareal_solve", "pint_adjoint"):
        assert n in names


def test_every_declared_symbol_is_exported(libpint):
    for name in declared_functions():
        assert hasattr(libpint, name), name


def test_struct_layouts_match_header(libpint):
    from paper_2411_09244_gb300 import _lib
    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "pint.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(pint_space_info), sizeof(pint_stats),
         offsetof(pint_stats, jumps), offsetof(pint_stats, solve_ms), offsetof(pint_stats, launches),
         sizeof(pint_batch_item), offsetof(pint_batch_item, wr_tol), offsetof(pint_batch_item, stats),
         offsetof(pint_batch_item, status));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(src, "w").write(prog)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    got = [C.sizeof(_lib.SpaceInfo), C.sizeof(_lib.Stats), _lib.Stats.jumps.offset,
           _lib.Stats.solve_ms.offset, _lib.Stats.launches.offset, C.sizeof(_lib.BatchItem),
           _lib.BatchItem.wr_tol.offset, _lib.BatchItem.stats.offset, _lib.BatchItem.status.offset]
    assert [int(x) for x in out] == got


def test_null_context_is_rejected_without_gpu(libpint):
    # argument checks happen before any device work
    from paper_2411_09244_gb300._lib import SpaceInfo
    info = SpaceInfo()
    assert libpint.pint_build_multiscale_spaces(None, 4, 2, 1, C.byref(info)) == -1
    assert libpint.pint_destroy(None) == 0
    assert b"NULL" in libpint.pint_last_error()


def test_wait_limit_control_without_gpu(libpint):
    # process-wide setting, no device state: usable without a GPU
    default = libpint.pint_set_wait_limit(-1)
    assert default == 1 << 22
    assert libpint.pint_set_wait_limit(7) == default
    assert libpint.pint_set_wait_limit(-1) == 7
    assert libpint.pint_set_wait_limit(-1) == default


def test_sweep_smem_control_without_gpu(libpint):
    default = libpint.pint_set_sweep_smem(-1)
    assert default == 200 * 1024
    assert libpint.pint_set_sweep_smem(0) == default
    assert libpint.pint_set_sweep_smem(-1) == 0
    assert libpint.pint_set_sweep_smem(-1) == default


def test_flag_and_status_constants_match_the_header():
    """The binding's enum constants are the header's values."""
    from paper_2411_09244_gb300 import _lib
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    defined = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(PINT_[A-Z0-9_]+)\s*=\s*(-?\d+)", src)}
    assert defined
    for name, value in defined.items():
        if hasattr(_lib, name):
            assert getattr(_lib, name) == value, name
    for name in ("PINT_FP64", "PINT_MIXED", "PINT_COARSE_FP64", "PINT_REFINE_FP64", "PINT_COARSE_GRID"):
        assert name in defined and hasattr(_lib, name), name
