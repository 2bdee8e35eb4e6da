"""The C-ABI library builds, loads and exports every entry point declared in include/*.h (no GPU calls)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"^\s*(?!typedef)[A-Za-z_][A-Za-z0-9_ ]*[ *]+([A-Za-z_][A-Za-z0-9_]*)\s*\([^;{}]*\)\s*;",
                             src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2210_08816_gb300 import build
    return build.build()


def test_header_declares_the_hot_path_calls():
    d = _declared()
    for name in ("fv_residual", "fv_jvp", "fv_project", "fv_jvp_project", "newton_steady", "arnoldi_leading",
                 "fv_grid_create", "fv_grid_destroy", "fv_strerror"):
        assert name in d


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header(libpath):
    from paper_2210_08816_gb300 import fv
    assert set(fv.EXPORTED) == _declared()
    L = fv.lib()
    assert L.fv_strerror(0).decode() == "ok"
    assert L.fv_strerror(-4).decode().startswith("iteration")


def test_struct_layouts_match_header(libpath):
    # sizes derived from the C declarations (x86-64 / aarch64 LP64 ABI)
    from paper_2210_08816_gb300 import fv
    assert ctypes.sizeof(fv.fv_grid_desc) == 3 * 4 + 4 + 3 * 8 + 2 * 8
    # precond, forcing, then the pseudo-time step (double)
    assert ctypes.sizeof(fv.fv_newton_opts) == 4 + 4 + 2 * 8 + 3 * 4 + 4 + 2 * 8 + 4 + 4 + 8
    # ..., euler_dt, inner_m, inner_max, inner_tol, vecs_fp64 (+4 padding)
    assert ctypes.sizeof(fv.fv_arnoldi_opts) == 4 + 4 + 8 + 4 * 4 + 8 + 8 + 8 + 4 + 4 + 8 + 4 + 4 + 8 + 4 + 4
    # ..., seconds, restarts_low (+4 padding), matvecs_low, matvecs_fp64, solves, solves_short, solve_worst
    assert ctypes.sizeof(fv.fv_arnoldi_report) == (4 + 4 + 4 + 4 + 8 + 3 * 64 * 8 + 256 * 4 + 8 + 4 + 4 + 8 + 8
                                                   + 4 + 4 + 8)


def test_struct_offsets_match_the_c_compiler(tmp_path):
    """Every field offset of the binding's ctypes structs equals the C compiler's offsetof for the header."""
    import shutil
    import subprocess
    from paper_2210_08816_gb300 import fv
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [fv.fv_grid_desc, fv.fv_newton_opts, fv.fv_newton_report, fv.fv_arnoldi_opts, fv.fv_arnoldi_report,
               fv.fv_critical_opts, fv.fv_critical_report]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cube_fv.h"', "int main(void) {"]
    for st in structs:
        lines.append(f'printf("{st.__name__} size %zu\\n", sizeof({st.__name__}));')
        for name, _ in st._fields_:
            lines.append(f'printf("{st.__name__} {name} %zu\\n", offsetof({st.__name__}, {name}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(ln.split()[:2]): int(ln.split()[2]) for ln in out if ln.strip()}
    for st in structs:
        assert got[(st.__name__, "size")] == ctypes.sizeof(st), st.__name__
        for name, _ in st._fields_:
            assert got[(st.__name__, name)] == getattr(st, name).offset, (st.__name__, name)


def test_richardson_extrapolation_is_the_least_squares_line(libpath):
    """fv_richardson (host arithmetic, no GPU): exact for values linear in h^2, least squares otherwise."""
    import numpy as np
    from paper_2210_08816_gb300 import fv
    h2 = [1 / 100.0 ** 2, 1 / 128.0 ** 2, 1 / 256.0 ** 2]
    lim, sl = fv.fv_richardson(h2, [4.5e7 + 3e10 * x for x in h2])
    assert lim == pytest.approx(4.5e7, rel=1e-13) and sl == pytest.approx(3e10, rel=1e-10)
    vals = [4.61e7, 4.57e7, 4.52e7]
    ref = np.polyfit(h2, vals, 1)
    lim, sl = fv.fv_richardson(h2, vals)
    assert lim == pytest.approx(ref[1], rel=1e-12) and sl == pytest.approx(ref[0], rel=1e-9)
    with pytest.raises(fv.FvError):
        fv.fv_richardson([1.0], [2.0])
