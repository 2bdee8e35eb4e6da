"""Python binding of the C-ABI in include/cube_fv.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does nothing but check the
arguments, pass device pointers of torch tensors (torch owns device memory and streams) and
turn status codes into exceptions.  All arithmetic runs in libcubefv.so; if the library is
missing this module raises instead of computing anything itself.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libcubefv.so")

FV_OK, FV_EINVAL, FV_ENOMEM, FV_ECUDA, FV_ENOCONV, FV_ENAN, FV_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
FV_FP64, FV_FP32 = 0, 1


class FvError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: {detail} (status {status})")
        self.status = status


class fv_grid_desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("xf", C.POINTER(C.c_double)), ("yf", C.POINTER(C.c_double)), ("zf", C.POINTER(C.c_double)),
                ("stretch", C.c_double), ("Pr", C.c_double)]


class fv_newton_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("tol", C.c_double), ("krylov_tol", C.c_double),
                ("max_newton", C.c_int), ("max_matvec", C.c_int), ("gmres_m", C.c_int),
                ("gr_start", C.c_double), ("gr_ratio", C.c_double), ("precond", C.c_int),
                ("forcing", C.c_int), ("ptc_dt0", C.c_double)]


class fv_newton_report(C.Structure):
    _fields_ = [("status", C.c_int), ("newton_steps", C.c_int), ("matvecs", C.c_int),
                ("gmres_fallbacks", C.c_int), ("continuation_steps", C.c_int),
                ("residual0", C.c_double), ("residual", C.c_double), ("history", C.c_double * 64)]


class fv_arnoldi_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("m", C.c_int), ("tol", C.c_double), ("max_restarts", C.c_int),
                ("max_degree", C.c_int), ("min_degree", C.c_int), ("guard", C.c_int),
                ("seed", C.c_ulonglong), ("sigma", C.c_double), ("low_tol", C.c_double),
                ("low_max_restarts", C.c_int), ("euler_dt", C.c_double), ("inner_m", C.c_int),
                ("inner_max", C.c_int), ("inner_tol", C.c_double), ("vecs_fp64", C.c_int)]


class fv_arnoldi_report(C.Structure):
    _fields_ = [("status", C.c_int), ("nconv", C.c_int), ("restarts", C.c_int), ("matvecs", C.c_longlong),
                ("residual", C.c_double * 64), ("lam_scaled_re", C.c_double * 64),
                ("lam_scaled_im", C.c_double * 64), ("degrees", C.c_int * 256), ("seconds", C.c_double),
                ("restarts_low", C.c_int), ("matvecs_low", C.c_longlong), ("matvecs_fp64", C.c_longlong),
                ("solves", C.c_int), ("solves_short", C.c_int), ("solve_worst", C.c_double)]


class fv_critical_opts(C.Structure):
    _fields_ = [("gr_a", C.c_double), ("gr_b", C.c_double), ("tol", C.c_double), ("max_iter", C.c_int),
                ("mode", C.c_int)]


class fv_critical_report(C.Structure):
    _fields_ = [("status", C.c_int), ("evaluations", C.c_int), ("gr_cr", C.c_double), ("lam_re", C.c_double),
                ("lam_im", C.c_double), ("omega_scaled", C.c_double), ("gr", C.c_double * 40),
                ("re", C.c_double * 40), ("im", C.c_double * 40)]


FV_MODE_LEADING, FV_MODE_REAL, FV_MODE_OSCILLATORY = 0, 1, 2

# int (*fv_tracked_fn)(double gr, void* ctx, double* re, double* im)
TRACKED_FN = C.CFUNCTYPE(C.c_int, C.c_double, C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double))

_lib = None


def lib():
    """Load libcubefv.so (built by paper_2210_08816_gb300.build.build()); raise if it is absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise FvError(FV_EINVAL, "load", f"{LIB_PATH} is missing; build it with paper_2210_08816_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp, d, i = C.c_void_p, C.c_double, C.c_int
        sig = {
            "fv_grid_create": (i, [C.POINTER(fv_grid_desc), vp, C.POINTER(vp)]),
            "fv_grid_destroy": (i, [vp]),
            "fv_set_stream": (i, [vp, vp]),
            "fv_state_elems": (C.c_longlong, [vp]),
            "fv_set_wait_limit": (i, [vp, C.c_longlong]),
            "fv_sync": (i, [vp]),
            "fv_residual": (i, [vp, d, vp, vp]),
            "fv_jvp": (i, [vp, i, d, vp, vp, vp]),
            "fv_project": (i, [vp, i, vp, i, d, C.POINTER(i), C.POINTER(d)]),
            "fv_jvp_project": (i, [vp, i, d, d, vp, vp, vp]),
            "fv_jvp_project_lincomb": (i, [vp, i, d, d, vp, vp, vp, d, d, d, vp, C.POINTER(d)]),
            "fv_jvp_project_lincomb_dev": (i, [vp, i, d, d, vp, vp, vp, d, d, d, vp, vp]),
            "fv_dot": (i, [vp, i, vp, vp, C.POINTER(d)]),
            "fv_dot_noalloc": (i, [i, C.c_longlong, vp, vp, vp, vp]),
            "fv_axpby": (i, [vp, i, d, vp, d, vp]),
            "fv_convert": (i, [vp, i, vp, vp]),
            "fv_diffusion_solve": (i, [vp, i, vp, vp]),
            "fv_transfer": (i, [vp, vp, vp, vp]),
            "fv_diagnostics": (i, [vp, vp, C.POINTER(d), C.POINTER(d)]),
            "fv_time_step": (i, [vp, d, d, i, vp, C.POINTER(d), C.POINTER(d)]),
            "fv_jvp_project_batch": (i, [vp, i, d, d, vp, i, vp, vp, i]),
            "fv_get_tuning": (i, [vp, C.POINTER(i), C.POINTER(i)]),
            "fv_batch_plan_create": (i, [i, C.POINTER(vp), i, C.POINTER(d), C.POINTER(d), C.POINTER(vp),
                                         C.POINTER(i), C.POINTER(vp), C.POINTER(vp), i, C.POINTER(vp)]),
            "fv_batch_plan_launch": (i, [vp, vp]),
            "fv_batch_plan_destroy": (i, [vp]),
            "fv_newton_default_opts": (None, [C.POINTER(fv_newton_opts)]),
            "newton_steady": (i, [vp, d, vp, C.POINTER(fv_newton_opts), C.POINTER(fv_newton_report)]),
            "fv_arnoldi_default_opts": (None, [C.POINTER(fv_arnoldi_opts)]),
            "arnoldi_leading": (i, [vp, i, d, vp, C.POINTER(fv_arnoldi_opts), C.POINTER(d), C.POINTER(d), vp,
                                    C.POINTER(fv_arnoldi_report)]),
            "fv_critical_default_opts": (None, [C.POINTER(fv_critical_opts)]),
            "fv_critical_gr": (i, [vp, i, vp, C.POINTER(fv_newton_opts), C.POINTER(fv_arnoldi_opts),
                                   C.POINTER(fv_critical_opts), C.POINTER(fv_critical_report)]),
            "fv_critical_root": (i, [C.POINTER(fv_critical_opts), TRACKED_FN, vp, C.POINTER(fv_critical_report)]),
            "fv_richardson": (i, [i, C.POINTER(d), C.POINTER(d), C.POINTER(d), C.POINTER(d)]),
            "fv_profile": (i, [vp, i]),
            "fv_profile_read": (i, [vp, C.POINTER(d), C.POINTER(C.c_longlong)]),
            "fv_strerror": (C.c_char_p, [i]),
            "fv_last_error": (C.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


EXPORTED = ["fv_grid_create", "fv_grid_destroy", "fv_set_stream", "fv_state_elems", "fv_set_wait_limit", "fv_sync",
            "fv_residual", "fv_jvp",
            "fv_project", "fv_jvp_project", "fv_jvp_project_lincomb", "fv_jvp_project_lincomb_dev", "fv_dot",
            "fv_dot_noalloc", "fv_axpby", "fv_convert", "fv_diffusion_solve", "fv_jvp_project_batch",
            "fv_get_tuning", "fv_transfer", "fv_diagnostics", "fv_time_step", "fv_batch_plan_create", "fv_batch_plan_launch", "fv_batch_plan_destroy",
            "fv_newton_default_opts", "newton_steady", "fv_arnoldi_default_opts", "arnoldi_leading", "fv_critical_default_opts", "fv_critical_gr", "fv_critical_root", "fv_richardson", "fv_profile",
            "fv_profile_read", "fv_strerror", "fv_last_error"]

FV_PROF_CLASSES = 7
PROF_NAMES = ["stencil", "divergence", "transform", "correct", "reduce", "vector", "transform_tc"]


def _check(status: int, where: str, ok=(FV_OK,)):
    if status not in ok:
        L = lib()
        raise FvError(status, where, f"{L.fv_strerror(status).decode()}: {L.fv_last_error().decode()}")
    return status


def _ptr(t, dtype, n, where):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise FvError(FV_EINVAL, where, "expected a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous() or t.numel() != n:
        raise FvError(FV_EINVAL, where, f"expected a contiguous {dtype} tensor of {n} elements, got "
                                        f"{t.dtype} {tuple(t.shape)}")
    return C.c_void_p(t.data_ptr())


class Grid:
    """Owner of an fv_grid handle (fv_grid_create / fv_grid_destroy)."""

    def __init__(self, nx, ny, nz, stretch=0.0, Pr=0.71, faces=None, stream=None):
        import torch
        desc = fv_grid_desc(nx=nx, ny=ny, nz=nz, stretch=float(stretch), Pr=float(Pr))
        self._keep = []
        if faces is not None:
            ptrs = []
            for f in faces:
                arr = (C.c_double * len(f))(*[float(x) for x in f])
                self._keep.append(arr)
                ptrs.append(C.cast(arr, C.POINTER(C.c_double)))
            desc.xf, desc.yf, desc.zf = ptrs
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        h = C.c_void_p()
        _check(lib().fv_grid_create(C.byref(desc), C.c_void_p(stream), C.byref(h)), "fv_grid_create")
        self.h = h
        self.shape = (nz, ny, nx)
        self.n = 4 * nx * ny * nz

    def close(self):
        if getattr(self, "h", None):
            lib().fv_grid_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def dtype(self, prec):
        import torch
        return torch.float64 if prec == FV_FP64 else torch.float32


def fv_grid_create(nx, ny, nz, stretch=0.0, Pr=0.71, faces=None, stream=None) -> Grid:
    return Grid(nx, ny, nz, stretch=stretch, Pr=Pr, faces=faces, stream=stream)


def fv_grid_destroy(g: Grid):
    g.close()


def fv_set_stream(g: Grid, stream):
    _check(lib().fv_set_stream(g.h, C.c_void_p(stream)), "fv_set_stream")


def fv_set_wait_limit(g: Grid, spins: int):
    """Polls of every device-side wait of the handle's kernels before it gives up (< 0: the default)."""
    _check(lib().fv_set_wait_limit(g.h, int(spins)), "fv_set_wait_limit")


def fv_sync(g: Grid) -> int:
    """Synchronise the handle's stream; returns FV_OK or FV_ETIMEOUT (a device-side wait gave up)."""
    return _check(lib().fv_sync(g.h), "fv_sync", ok=(FV_OK, FV_ETIMEOUT))


def fv_residual(g: Grid, Gr, q, F):
    import torch
    _check(lib().fv_residual(g.h, float(Gr), _ptr(q, torch.float64, g.n, "q"), _ptr(F, torch.float64, g.n, "F")),
           "fv_residual")
    return F


def fv_jvp(g: Grid, prec, Gr, q, v, Jv):
    dt = g.dtype(prec)
    _check(lib().fv_jvp(g.h, prec, float(Gr), _ptr(q, dt, g.n, "q"), _ptr(v, dt, g.n, "v"), _ptr(Jv, dt, g.n, "Jv")),
           "fv_jvp")
    return Jv


def fv_project(g: Grid, prec, v, max_it=1, tol=0.0, want_div=False):
    it = C.c_int(0)
    dv = C.c_double(0.0)
    _check(lib().fv_project(g.h, prec, _ptr(v, g.dtype(prec), g.n, "v"), int(max_it), float(tol), C.byref(it),
                            C.byref(dv) if want_div else None), "fv_project")
    return it.value, (dv.value if want_div else None)


FV_BATCH_GRAPH = 1
FV_BATCH_AUTOTUNE = 2


def fv_jvp_project_batch(g: Grid, prec, Gr, sigma, q, V, W, nvec, use_graph=False, autotune=False):
    """W_i = P (J V_i - sigma V_i) + sigma V_i for nvec vectors stored back to back in V and W."""
    dt = g.dtype(prec)
    flags = (FV_BATCH_GRAPH if use_graph else 0) | (FV_BATCH_AUTOTUNE if autotune else 0)
    _check(lib().fv_jvp_project_batch(g.h, prec, float(Gr), float(sigma), _ptr(q, dt, g.n, "q"), int(nvec),
                                      _ptr(V, dt, g.n * nvec, "V"), _ptr(W, dt, g.n * nvec, "W"), flags),
           "fv_jvp_project_batch")
    return W


def fv_get_tuning(g: Grid):
    """(z-chunk of the block stencil picked by the autotuner (0 = default), block size it was timed on)."""
    zc, nv = C.c_int(0), C.c_int(0)
    _check(lib().fv_get_tuning(g.h, C.byref(zc), C.byref(nv)), "fv_get_tuning")
    return zc.value, nv.value


class BatchPlan:
    """Several problems (grid handle, Gr, sigma, q, block V -> W) captured into one CUDA graph whose branches
    run concurrently (fv_batch_plan_create); launch() replays it on a stream.  Keeps references to the
    tensors and grids so that they outlive the plan."""

    def __init__(self, problems, prec, autotune=False):
        n = len(problems)
        dt = None
        hs, grs, sig, qs, nv, vs, ws = [], [], [], [], [], [], []
        for (g, Gr, sigma, q, V, W, nvec) in problems:
            dt = g.dtype(prec)
            hs.append(g.h)
            grs.append(float(Gr))
            sig.append(float(sigma))
            qs.append(_ptr(q, dt, g.n, "q"))
            vs.append(_ptr(V, dt, g.n * nvec, "V"))
            ws.append(_ptr(W, dt, g.n * nvec, "W"))
            nv.append(int(nvec))
        self._keep = problems
        arr = lambda t, xs: (t * n)(*xs)
        h = C.c_void_p()
        _check(lib().fv_batch_plan_create(n, arr(C.c_void_p, hs), prec, arr(C.c_double, grs), arr(C.c_double, sig),
                                          arr(C.c_void_p, qs), arr(C.c_int, nv), arr(C.c_void_p, vs),
                                          arr(C.c_void_p, ws), FV_BATCH_AUTOTUNE if autotune else 0, C.byref(h)),
               "fv_batch_plan_create")
        self.h = h

    def launch(self, stream=None):
        _check(lib().fv_batch_plan_launch(self.h, C.c_void_p(stream)), "fv_batch_plan_launch")

    def close(self):
        if getattr(self, "h", None):
            lib().fv_batch_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fv_diffusion_solve(g: Grid, prec, x, out):
    """out = L^-1 x (the diffusion operator of J, per field); x and out may be the same tensor."""
    dt = g.dtype(prec)
    _check(lib().fv_diffusion_solve(g.h, prec, _ptr(x, dt, g.n, "x"), _ptr(out, dt, g.n, "out")),
           "fv_diffusion_solve")
    return out


def fv_transfer(g_from: Grid, q_from, g_to: Grid, q_to):
    """q_to = the FP64 state q_from of grid g_from interpolated onto grid g_to (then projected there)."""
    import torch
    _check(lib().fv_transfer(g_from.h, _ptr(q_from, torch.float64, g_from.n, "q_from"), g_to.h,
                             _ptr(q_to, torch.float64, g_to.n, "q_to")), "fv_transfer")
    return q_to


def fv_diagnostics(g: Grid, q):
    """(E_kin, Nu) of the FP64 state q (Eqs. 12 and 13)."""
    import torch
    e, nu = C.c_double(0.0), C.c_double(0.0)
    _check(lib().fv_diagnostics(g.h, _ptr(q, torch.float64, g.n, "q"), C.byref(e), C.byref(nu)), "fv_diagnostics")
    return e.value, nu.value


def fv_time_step(g: Grid, Gr, dt, nsteps, q):
    """Advance the FP64 state q in place by nsteps semi-implicit steps; returns the (E_kin, Nu) histories
    (nsteps + 1 values each, before the first step and after every step)."""
    import torch
    e = (C.c_double * (nsteps + 1))()
    nu = (C.c_double * (nsteps + 1))()
    _check(lib().fv_time_step(g.h, float(Gr), float(dt), int(nsteps), _ptr(q, torch.float64, g.n, "q"), e, nu),
           "fv_time_step")
    return list(e), list(nu)


def fv_jvp_project(g: Grid, prec, Gr, sigma, q, v, out):
    dt = g.dtype(prec)
    _check(lib().fv_jvp_project(g.h, prec, float(Gr), float(sigma), _ptr(q, dt, g.n, "q"), _ptr(v, dt, g.n, "v"),
                                _ptr(out, dt, g.n, "out")), "fv_jvp_project")
    return out


def fv_jvp_project_lincomb_dev(g: Grid, prec, Gr, sigma, q, v, w, alpha, beta, gamma, out, norm2=None):
    """The same step, stream-ordered: ||out||^2 into the device float64 tensor norm2 (one element) if given."""
    import torch
    dt = g.dtype(prec)
    wp = _ptr(w, dt, g.n, "w") if w is not None else None
    np_ = _ptr(norm2, torch.float64, 1, "norm2") if norm2 is not None else None
    _check(lib().fv_jvp_project_lincomb_dev(g.h, prec, float(Gr), float(sigma), _ptr(q, dt, g.n, "q"),
                                            _ptr(v, dt, g.n, "v"), wp, float(alpha), float(beta), float(gamma),
                                            _ptr(out, dt, g.n, "out"), np_), "fv_jvp_project_lincomb_dev")
    return out


def fv_jvp_project_lincomb(g: Grid, prec, Gr, sigma, q, v, w, alpha, beta, gamma, out, want_norm=False):
    """out = alpha (P (J v - sigma v) + sigma v) + beta v + gamma w; returns ||out||^2 if want_norm."""
    dt = g.dtype(prec)
    wp = _ptr(w, dt, g.n, "w") if w is not None else None
    nrm = C.c_double(0.0)
    _check(lib().fv_jvp_project_lincomb(g.h, prec, float(Gr), float(sigma), _ptr(q, dt, g.n, "q"),
                                        _ptr(v, dt, g.n, "v"), wp, float(alpha), float(beta), float(gamma),
                                        _ptr(out, dt, g.n, "out"), C.byref(nrm) if want_norm else None),
           "fv_jvp_project_lincomb")
    return nrm.value if want_norm else out


def fv_dot(g: Grid, prec, a, b) -> float:
    dt = g.dtype(prec)
    r = C.c_double(0.0)
    _check(lib().fv_dot(g.h, prec, _ptr(a, dt, g.n, "a"), _ptr(b, dt, g.n, "b"), C.byref(r)), "fv_dot")
    return r.value


def fv_dot_noalloc(prec, a, b, result, stream=None):
    """<a, b> into the device FP64 tensor `result` (one element), with no allocation in the library.
    a, b and result must sit on one device; the call runs with that device current (and, by default, on
    its current stream)."""
    import torch
    dt = torch.float64 if prec == FV_FP64 else torch.float32
    n = a.numel()
    for name, t in (("b", b), ("result", result)):
        if isinstance(t, torch.Tensor) and t.device != a.device:
            raise FvError(FV_EINVAL, "fv_dot_noalloc", f"{name} is on {t.device}, a is on {a.device}")
    pa = _ptr(a, dt, n, "a")
    with torch.cuda.device(a.device):
        if stream is None:
            stream = torch.cuda.current_stream(a.device).cuda_stream
        _check(lib().fv_dot_noalloc(int(prec), n, pa, _ptr(b, dt, n, "b"), _ptr(result, torch.float64, 1, "result"),
                                    C.c_void_p(stream)), "fv_dot_noalloc")
    return result


def fv_axpby(g: Grid, prec, alpha, x, beta, y):
    dt = g.dtype(prec)
    _check(lib().fv_axpby(g.h, prec, float(alpha), _ptr(x, dt, g.n, "x"), float(beta), _ptr(y, dt, g.n, "y")),
           "fv_axpby")
    return y


def fv_convert(g: Grid, src, dst):
    import torch
    to32 = src.dtype == torch.float64
    _check(lib().fv_convert(g.h, 1 if to32 else 0,
                            _ptr(src, torch.float64 if to32 else torch.float32, g.n, "src"),
                            _ptr(dst, torch.float32 if to32 else torch.float64, g.n, "dst")), "fv_convert")
    return dst


def fv_profile(g: Grid, enable: bool):
    _check(lib().fv_profile(g.h, 1 if enable else 0), "fv_profile")


def fv_profile_read(g: Grid):
    """{class name: (milliseconds, launches)} accumulated since fv_profile(g, True)."""
    ms = (C.c_double * FV_PROF_CLASSES)()
    n = (C.c_longlong * FV_PROF_CLASSES)()
    _check(lib().fv_profile_read(g.h, ms, n), "fv_profile_read")
    return {PROF_NAMES[k]: (ms[k], n[k]) for k in range(FV_PROF_CLASSES)}


def fv_newton_default_opts() -> fv_newton_opts:
    o = fv_newton_opts()
    lib().fv_newton_default_opts(C.byref(o))
    return o


def newton_steady(g: Grid, Gr, q_inout, opts: fv_newton_opts | None = None):
    """Returns (status, report); status FV_ENOCONV is returned, not raised."""
    import torch
    o = opts or fv_newton_default_opts()
    rep = fv_newton_report()
    st = lib().newton_steady(g.h, float(Gr), _ptr(q_inout, torch.float64, g.n, "q"), C.byref(o), C.byref(rep))
    _check(st, "newton_steady", ok=(FV_OK, FV_ENOCONV))
    return st, rep


def fv_arnoldi_default_opts() -> fv_arnoldi_opts:
    o = fv_arnoldi_opts()
    lib().fv_arnoldi_default_opts(C.byref(o))
    return o


def arnoldi_leading(g: Grid, k, Gr, q, opts: fv_arnoldi_opts | None = None, vecs=None):
    """Returns (status, eigenvalues (complex list), report)."""
    import torch
    o = opts or fv_arnoldi_default_opts()
    re = (C.c_double * (k + 1))()
    im = (C.c_double * (k + 1))()
    rep = fv_arnoldi_report()
    vp = None
    if vecs is not None:
        vp = _ptr(vecs, g.dtype(FV_FP64 if o.vecs_fp64 else o.precision), (k + 1) * g.n, "vecs")
    st = lib().arnoldi_leading(g.h, int(k), float(Gr), _ptr(q, torch.float64, g.n, "q"), C.byref(o), re, im, vp,
                               C.byref(rep))
    _check(st, "arnoldi_leading", ok=(FV_OK, FV_ENOCONV))
    lam = [complex(re[i], im[i]) for i in range(rep.nconv)]
    return st, lam, rep


def fv_critical_default_opts() -> fv_critical_opts:
    o = fv_critical_opts()
    lib().fv_critical_default_opts(C.byref(o))
    return o


def fv_critical_gr(g: Grid, k, q, copts: fv_critical_opts, nopts: fv_newton_opts | None = None,
                   aopts: fv_arnoldi_opts | None = None):
    """Returns (status, report); q (FP64, in place) ends as the steady state at the critical Gr."""
    import torch
    rep = fv_critical_report()
    st = lib().fv_critical_gr(g.h, int(k), _ptr(q, torch.float64, g.n, "q"), C.byref(nopts) if nopts else None,
                              C.byref(aopts) if aopts else None, C.byref(copts), C.byref(rep))
    _check(st, "fv_critical_gr", ok=(FV_OK, FV_ENOCONV))
    return st, rep


def fv_critical_root(copts: fv_critical_opts, f):
    """The root iteration of fv_critical_gr on a host function f(gr) -> the tracked eigenvalue (complex or
    real).  Returns (status, report); FV_ENOCONV is returned, not raised; an exception raised by f ends the
    iteration and is raised again here."""
    raised = []

    def tracked(gr, ctx, re, im):
        try:
            lam = complex(f(gr))
        except Exception as e:  # noqa: BLE001 -- raised again after the call returns
            raised.append(e)
            return FV_EINVAL
        re[0], im[0] = lam.real, lam.imag
        return FV_OK

    cb = TRACKED_FN(tracked)
    rep = fv_critical_report()
    st = lib().fv_critical_root(C.byref(copts), cb, None, C.byref(rep))
    if raised:
        raise raised[0]
    _check(st, "fv_critical_root", ok=(FV_OK, FV_ENOCONV))
    return st, rep


def fv_richardson(h2, values):
    """(limit, slope) of the least-squares line values = limit + slope h2 (Richardson extrapolation)."""
    n = len(h2)
    a = (C.c_double * n)(*[float(x) for x in h2])
    b = (C.c_double * n)(*[float(x) for x in values])
    lim, sl = C.c_double(0.0), C.c_double(0.0)
    _check(lib().fv_richardson(n, a, b, C.byref(lim), C.byref(sl)), "fv_richardson")
    return lim.value, sl.value
