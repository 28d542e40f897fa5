"""The C-ABI library builds, loads and exports every symbol include/sem.h declares.

Also checks the library's host-side GLL rule and D_hat (no GPU needed) against
the oracle and the golden closed forms.
"""
import os
import re

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2104_05829_gb300 import _lib, build
    build.build()
    return _lib.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "sem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sem_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("sem_setup", "sem_ax", "sem_gs", "sem_solve", "sem_free", "sem_grad_h1"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2104_05829_gb300 import _lib
    for n in _declared():
        assert hasattr(lib, n), n
        assert n in _lib.SIGNATURES, f"{n} missing from the Python binding"


def test_no_cpu_fallback_without_library(tmp_path, monkeypatch):
    """Loading fails loudly when the built library is absent."""
    from paper_2104_05829_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "lib_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        _lib.load()


@pytest.mark.parametrize("N", range(1, 12))
def test_library_gll_matches_oracle(lib, N):
    from paper_2104_05829_gb300 import gll
    xi, rho, D = gll(N)
    xo, ro = O.gll(N)
    np.testing.assert_allclose(xi, xo, atol=2e-16)
    np.testing.assert_allclose(rho, ro, rtol=2e-15)
    np.testing.assert_allclose(D, O.deriv_matrix(N), atol=1e-13 * N * N)


def test_library_rejects_bad_order(lib):
    import ctypes as C
    assert lib.sem_gll(0, None, None, None) == -1
    assert lib.sem_gll(12, None, None, None) == -1
    assert "outside" in lib.sem_last_error_detail().decode()


def test_setup_argument_validation_on_host(lib):
    """Invalid meshes are rejected before any device work."""
    import ctypes as C
    from paper_2104_05829_gb300 import _lib as L
    h = C.c_void_p()
    assert lib.sem_setup(None, None, C.byref(h)) == L.SEM_EINVAL
    x = np.zeros(8)
    g = np.array([1, 2, 3, 4, 5, 6, 7, -8], dtype=np.int64)
    m = L.SemMesh(1, 1, x.ctypes.data, x.ctypes.data, x.ctypes.data, g.ctypes.data, None)
    assert lib.sem_setup(C.byref(m), None, C.byref(h)) == L.SEM_EINVAL
    m = L.SemMesh(1, 12, x.ctypes.data, x.ctypes.data, x.ctypes.data, g.ctypes.data, None)
    assert lib.sem_setup(C.byref(m), None, C.byref(h)) == L.SEM_EINVAL
    m = L.SemMesh(0, 1, x.ctypes.data, x.ctypes.data, x.ctypes.data, g.ctypes.data, None)
    assert lib.sem_setup(C.byref(m), None, C.byref(h)) == L.SEM_EINVAL
    assert not h.value


def test_projection_entry_points_reject_null_on_host(lib):
    import ctypes as C
    from paper_2104_05829_gb300 import _lib as L
    h = C.c_void_p()
    assert lib.sem_proj_create(None, 4, C.byref(h)) == L.SEM_EINVAL and not h.value
    assert lib.sem_proj_count(None) == L.SEM_EINVAL
    assert lib.sem_proj_reset(None) == L.SEM_EINVAL
    assert lib.sem_proj_vectors(None, 0, None, None) == L.SEM_EINVAL
    assert lib.sem_proj_project(None, None, None, None, None) == L.SEM_EINVAL
    assert lib.sem_proj_update(None, None, 0, None, None, None, None) == L.SEM_EINVAL
    assert lib.sem_solve_proj(None, None, None, None, 1e-8, 10, 0, 0, 0, None, None, None) == L.SEM_EINVAL
    lib.sem_proj_free(None)


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structures have the field offsets and sizes the C compiler
    gives the header's structures (gcc on this host; no GPU)."""
    import ctypes
    import shutil
    import subprocess

    from paper_2104_05829_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"sem_mesh": _lib.SemMesh, "sem_opts": _lib.SemOpts, "sem_coef": _lib.SemCoef,
               "sem_info": _lib.SemInfo, "sem_level_desc": _lib.SemLevelDesc}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "sem.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line.strip():
            parts = line.split()
            got[(parts[0], parts[1])] = int(parts[2])
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
