"""Host-side behaviour of the C-ABI and its binding that needs no GPU.

* The option structs that `fv_*_default_opts` fill carry the defaults that include/cube_fv.h documents
  beside each field ("(default X)" or "X (default)"): the header is the user's only statement of them.
* The binding refuses what the library could not dereference (host tensors, wrong dtype or size) before
  any call reaches the device, with FvError(FV_EINVAL).
* fv_grid_create refuses sizes outside [2, 1024] per axis or with 4 N >= 2^31, a non-positive Pr, and
  caller faces that do not run strictly increasing from 0 to 1, before any device allocation.
"""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cube_fv.h")

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fv():
    from paper_2210_08816_gb300 import build
    build.build()
    from paper_2210_08816_gb300 import fv as _fv
    _fv.lib()
    return _fv


def _documented_defaults(struct):
    """{field: value} for every field of `struct` whose comment states a default."""
    src = open(HEADER).read()
    end = re.search(r"\}\s*" + struct + r"\s*;", src)
    assert end, struct
    body = src[src.rindex("typedef struct", 0, end.start()):end.start()]
    out = {}
    for f in re.finditer(r"(?:int|double|long long)\s+(\w+);\s*/\*(.*?)\*/", body, flags=re.S):
        name, comment = f.group(1), f.group(2)
        a = re.search(r"\(default ([-+0-9.eE]+)", comment)
        b = re.search(r"(?:^|[\s:;])([-+0-9.eE]+) \(default\)", comment)
        if a:
            out[name] = float(a.group(1))
        elif b:
            out[name] = float(b.group(1))
    return out


@pytest.mark.parametrize("struct,fn", [("fv_newton_opts", "fv_newton_default_opts"),
                                       ("fv_arnoldi_opts", "fv_arnoldi_default_opts"),
                                       ("fv_critical_opts", "fv_critical_default_opts")])
def test_default_options_match_the_header(fv, struct, fn):
    documented = _documented_defaults(struct)
    assert len(documented) >= 2, (struct, documented)
    opts = getattr(fv, fn)()
    for name, value in documented.items():
        assert getattr(opts, name) == pytest.approx(value, rel=1e-15), (struct, name)


def test_binding_refuses_host_and_mistyped_tensors(fv):
    cpu = torch.zeros(16, dtype=torch.float64)
    with pytest.raises(fv.FvError) as e:
        fv._ptr(cpu, torch.float64, 16, "x")
    assert e.value.status == fv.FV_EINVAL
    with pytest.raises(fv.FvError):
        fv.fv_dot_noalloc(fv.FV_FP64, cpu, cpu, torch.zeros(1, dtype=torch.float64))


def test_status_strings_cover_every_code(fv):
    L = fv.lib()
    codes = [getattr(fv, n) for n in dir(fv) if re.fullmatch(r"FV_E[A-Z]+", n)] + [fv.FV_OK]
    texts = {c: L.fv_strerror(c).decode() for c in codes}
    assert all(texts.values()), texts
    assert len(set(texts.values())) == len(codes), texts


@pytest.mark.parametrize("nx,ny,nz,Pr", [(1, 8, 8, 0.71), (8, 1025, 8, 0.71), (8, 8, 8, 0.0), (8, 8, 8, -1.0),
                                         (1024, 1024, 1024, 0.71)])
def test_grid_create_refuses_bad_sizes(fv, nx, ny, nz, Pr):
    import ctypes as C
    desc = fv.fv_grid_desc(nx=nx, ny=ny, nz=nz, stretch=1.5, Pr=Pr)
    h = C.c_void_p()
    assert fv.lib().fv_grid_create(C.byref(desc), None, C.byref(h)) == fv.FV_EINVAL
    assert not h.value


@pytest.mark.parametrize("faces", [[0.1, 0.5, 1.0], [0.0, 0.5, 0.9], [0.0, 0.5, 0.5, 1.0], [0.0, 0.7, 0.4, 1.0]])
def test_grid_create_refuses_bad_faces(fv, faces):
    import ctypes as C
    n = len(faces) - 1
    arr = (C.c_double * len(faces))(*faces)
    ok = (C.c_double * (n + 1))(*[i / n for i in range(n + 1)])
    desc = fv.fv_grid_desc(nx=n, ny=n, nz=n, stretch=0.0, Pr=0.71)
    desc.xf = C.cast(arr, C.POINTER(C.c_double))
    desc.yf = desc.zf = C.cast(ok, C.POINTER(C.c_double))
    h = C.c_void_p()
    assert fv.lib().fv_grid_create(C.byref(desc), None, C.byref(h)) == fv.FV_EINVAL
    assert not h.value
