"""Host-side checks of the C ABI (no GPU work): build, exported symbols, tables, argument checks."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_1801_01201_gb300 import _lib as L
from paper_1801_01201_gb300 import solver as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "misdc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(misdc_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_function():
    lib = L.load()
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(L.EXPORTS)


@pytest.mark.parametrize("n_nodes", [2, 3, 4, 5])
def test_library_tables_equal_oracle_tables(n_nodes):
    tau, Q, QI, QE = S.lobatto(n_nodes)
    t2, Q2, S2, QI2, QE2 = O.lobatto(n_nodes - 1)
    np.testing.assert_allclose(tau, t2, atol=1e-15)
    np.testing.assert_allclose(Q, Q2, atol=1e-15)
    np.testing.assert_allclose(QI, QI2, atol=1e-15)
    np.testing.assert_allclose(QE, QE2, atol=1e-15)


def test_invalid_arguments_are_rejected_before_device_work():
    lib = L.load()
    assert lib.misdc_lobatto(1, None, None, None, None) == L.E_INVALID
    assert lib.misdc_lobatto(12, None, None, None, None) == L.E_INVALID
    h = C.c_void_p()
    assert lib.misdc_create(None, None, None, None, C.byref(h)) == L.E_INVALID
    assert b"null" in lib.misdc_last_error()
    assert lib.misdc_step(None, None, None, 1e-6, 1, None) == L.E_INVALID
    assert lib.misdc_lincomb(0, 1, None, None, None, 0, None) == L.E_INVALID
    o = L.Opts()
    lib.misdc_default_opts(C.byref(o))
    assert (o.n_nodes, o.n_sweeps, o.nu, o.scheme) == (3, 4, 2, L.SCHEMES["CISDCQ"])


def test_pde_entry_point_checks_arguments_on_the_host():
    """misdc_pde_step rejects bad arguments before any device work; n = 0 is a no-op."""
    lib = L.load()
    vp = C.c_void_p(1)
    assert lib.misdc_pde_step(7, 5, 4, 1, 0.05, 1, 200, 20.0, 1, vp, vp, vp, None, None, None) == L.E_INVALID
    assert lib.misdc_pde_step(2, 5, 4, 1, 0.05, 1, 4, 20.0, 1, vp, vp, vp, None, None, None) == L.E_INVALID
    assert b"nx" in lib.misdc_last_error()
    assert lib.misdc_pde_step(2, 5, 0, 1, 0.05, 1, 200, 20.0, 1, vp, vp, vp, None, None, None) == L.E_INVALID
    assert lib.misdc_pde_step(2, 5, 4, 1, -0.05, 1, 200, 20.0, 1, vp, vp, vp, None, None, None) == L.E_INVALID
    assert lib.misdc_pde_step(2, 5, 4, 1, 0.05, 1, 200, 20.0, 0, None, None, None, None, None, None) == L.OK
    # shared memory of one instance: (4 + 12 M + 5 + 7 M) nx + 33 doubles and M nx pivot bytes
    for n_nodes, nx in ((5, 200), (3, 53)):
        M = n_nodes - 1
        assert S.pde_smem_bytes(n_nodes, nx) == 8 * ((9 + 19 * M) * nx + 33) + M * nx


STRUCTS = {"MechDesc": "misdc_mech_desc", "GridDesc": "misdc_grid_desc", "Opts": "misdc_opts",
           "Stats": "misdc_stats", "LowMachDesc": "misdc_lowmach_desc", "Tuning": "misdc_tuning"}


def test_struct_layouts_match_header(tmp_path):
    """Every structure the binding passes through the C ABI has, field by field,
    the offset and the size the header gives it (a C program compiled against
    include/misdc.h prints them), so no field added on one side only can shift
    the others."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "misdc.h"', "int main(void) {"]
    for py, cname in STRUCTS.items():
        cls = getattr(L, py)
        lines.append('  printf("%s size %%zu\\n", sizeof(%s));' % (py, cname))
        for f, _ in cls._fields_:
            lines.append('  printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (py, f, cname, f))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                         check=True).stdout.splitlines())
    for py in STRUCTS:
        cls = getattr(L, py)
        assert int(got[py + " size"]) == C.sizeof(cls), py
        for f, _ in cls._fields_:
            assert int(got["%s.%s" % (py, f)]) == getattr(cls, f).offset, (py, f)
