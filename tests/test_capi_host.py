"""Host-side checks of the C ABI (no GPU needed): the library builds, loads,
exports every entry point that include/kbc.h declares, the Python binding
covers exactly those names, and argument validation fails cleanly before any
device work."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

from paper_1507_02509_gb300 import build as kbuild
from paper_1507_02509_gb300 import capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "kbc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kbc_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    kbuild.build()
    return capi.load()


def test_header_declares_the_paper_path():
    names = declared_functions()
    for required in ("kbc_create", "kbc_init", "kbc_step", "kbc_moments", "kbc_destroy",
                     "kbc_diagnostics", "kbc_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_binding_covers_exactly_the_header():
    assert sorted(capi.SIGNATURES) == declared_functions()
    for name in declared_functions():
        assert callable(getattr(capi, name)), name


def test_arguments_rejected_before_device_work(lib):
    h = ctypes.c_void_p()
    assert lib.kbc_create(0, 8, 1, 0.9, 1, ctypes.byref(h)) == capi.KBC_ERR_ARG
    assert h.value is None
    assert "grid" in lib.kbc_last_error(None).decode()
    assert lib.kbc_create(8, 8, 9, 0.9, 1, ctypes.byref(h)) == capi.KBC_ERR_ARG
    assert lib.kbc_create(8, 8, 1, 0.0, 1, ctypes.byref(h)) == capi.KBC_ERR_ARG
    assert lib.kbc_create(8, 8, 1, 1.01, 1, ctypes.byref(h)) == capi.KBC_ERR_ARG
    assert lib.kbc_create(8, 8, 1, 0.9, 5, ctypes.byref(h)) == capi.KBC_ERR_ARG
    assert lib.kbc_create(65536, 65536, 1, 0.9, 1, ctypes.byref(h)) == capi.KBC_ERR_ARG
    assert lib.kbc_create(8, 8, 1, 0.9, 1, None) == capi.KBC_ERR_ARG
    # NULL handles never crash
    assert lib.kbc_step(None, 1) == capi.KBC_ERR_ARG
    assert lib.kbc_destroy(None) == capi.KBC_ERR_ARG
    assert lib.kbc_set_stream(None, None) == capi.KBC_ERR_ARG


def test_allocator_hook_pairs(lib):
    # one hook without the other is rejected; resetting to the default works
    assert lib.kbc_set_allocator(capi.ALLOC_FN(lambda *a: None), capi.FREE_FN(0), None) == \
        capi.KBC_ERR_ARG
    assert lib.kbc_set_allocator(capi.ALLOC_FN(0), capi.FREE_FN(0), None) == capi.KBC_OK


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(RuntimeError):
        capi._lib_backup = capi._lib
        try:
            capi._lib = None
            capi.load(str(tmp_path / "nope.so"))
        finally:
            capi._lib = capi._lib_backup


def test_table3_definitions():
    """Re = N sqrt(2E)/nu and t_e ~ Z^(-1/2) reproduce the printed columns of
    Table 3 (tests/golden/table3_turbulence.txt)."""
    from paper_1507_02509_gb300 import viscosity_for_reynolds

    rows = []
    with open(os.path.join(ROOT, "tests", "golden", "table3_turbulence.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    assert len(rows) == 9
    for re_, n, e0, z0, nu, te in rows:
        assert viscosity_for_reynolds(int(n), e0, re_) == pytest.approx(nu, rel=2e-3)
        assert z0 ** -0.5 == pytest.approx(te, rel=3e-3)


C_CALLER = r"""
#include <stdio.h>
#include <string.h>
#include "kbc.h"

int main(void)
{
    kbc_handle h = 0;
    double bytes = 0.0;
    /* an empty grid is rejected before any device work */
    if (kbc_create(0, 8, KBC_B, 0.9, KBC_F32_DEV, &h) != KBC_ERR_ARG || h != 0) return 1;
    if (strlen(kbc_last_error(0)) == 0) return 2;
    if (kbc_bytes_per_update(0, &bytes) != KBC_ERR_ARG) return 3;
    printf("%s\n", kbc_last_error(0));
    return 0;
}
"""


def test_header_compiles_as_c_and_links(lib, tmp_path):
    """A plain C99 caller (no C++) compiles against include/kbc.h with all
    warnings as errors, links against the in-tree library and gets the
    documented status codes."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "caller.c"
    src.write_text(C_CALLER)
    exe = tmp_path / "caller"
    libdir = os.path.dirname(kbuild.LIB)
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-L", libdir, "-lkbc_gb300", f"-Wl,-rpath,{libdir}", "-o", str(exe)],
                   check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert "grid" in r.stdout
