"""GPU parity: every entry point of libcubefv.so against the FP64 oracle on identical seeded inputs.

Tolerances (norm-wise, per field: max|gpu - oracle| / max|oracle|):
* FP64 paths: 1e-12 for the stencils and the projection (different summation order only; the
  worst cancellation is the diffusion term ~ 4 max|v| / h_min^2 against results of the same order).
* FP32 paths: inputs are rounded to FP32 first and the oracle runs in FP64 on the rounded values.
  The stencil sums ~40 products with unit round-off u = 2^-24; the fast-diagonalisation solve applies
  six dense n x n transforms whose rounding grows like sqrt(n) u each, so the projected fields carry
  ~6 sqrt(n) u ~ 6e-6 at n = 256.  Bounds: 2e-5 (stencil), 5e-5 (projection / fused path).
"""
import numpy as np
import pytest

import oracle.discretisation as D
from oracle.projection import Projector
from paper_2210_08816_gb300 import seeded

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PR = 0.71
TOL64 = 1e-12
TOL32_STENCIL = 2e-5
TOL32_PROJ = 5e-5


@pytest.fixture(scope="module")
def fv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_08816_gb300 import build
    build.build()
    from paper_2210_08816_gb300 import fv as _fv
    _fv.lib()
    return _fv


def dev(api, dtype):
    return torch.tensor(np.stack(api), dtype=dtype, device="cuda").contiguous().view(-1)


def host(t, shape):
    a = t.view(4, *shape).double().cpu().numpy()
    return [a[c] for c in range(4)]


def rel(a, b):
    return max(float(np.max(np.abs(a[c] - b[c]))) / max(float(np.max(np.abs(b[c]))), 1e-300) for c in range(4))


def state(og, seed, sigma=0.5, project=True):
    """Seeded base state: conduction + projected N(0, sigma^2) perturbation (exchange layout)."""
    q = D.from_api(og, seeded.normal_fields(seed, og.shape, sigma))
    if project:
        q = Projector(og).full(q)
    q[3] = q[3] + (1.0 - og.axes[0].xc)[None, None, :]
    return D.to_api(og, q)


def vector(og, seed, sigma=1.0):
    return D.to_api(og, D.from_api(og, seeded.normal_fields(seed, og.shape, sigma)))


def round32(api):
    return [a.astype(np.float32).astype(np.float64) for a in api]


GRIDS = [((7, 5, 3), 0.0), ((17, 13, 11), 1.5), ((32, 32, 32), 1.5), ((2, 2, 2), 0.0), ((64, 48, 40), 1.5),
         ((130, 3, 5), 0.0), ((128, 16, 20), 0.0), ((192, 17, 35), 1.5)]


@pytest.mark.parametrize("shape,stretch", GRIDS)
def test_residual_fp64(fv, shape, stretch):
    og = D.Grid(*shape, stretch=stretch, Pr=PR)
    g = fv.Grid(*shape, stretch=stretch, Pr=PR)
    q = state(og, 1)
    Gr = 3.0e4
    F = torch.empty(g.n, dtype=torch.float64, device="cuda")
    fv.fv_residual(g, Gr, dev(q, torch.float64), F)
    assert rel(host(F, og.shape), D.residual(og, Gr, q)) <= TOL64


@pytest.mark.parametrize("shape,stretch", GRIDS)
def test_jvp_fp64_and_fp32(fv, shape, stretch):
    og = D.Grid(*shape, stretch=stretch, Pr=PR)
    g = fv.Grid(*shape, stretch=stretch, Pr=PR)
    q, v = state(og, 2), vector(og, 3)
    Gr = 5.0e4
    out = torch.empty(g.n, dtype=torch.float64, device="cuda")
    fv.fv_jvp(g, fv.FV_FP64, Gr, dev(q, torch.float64), dev(v, torch.float64), out)
    assert rel(host(out, og.shape), D.jvp(og, Gr, q, v)) <= TOL64
    q32, v32 = round32(q), round32(v)
    out32 = torch.empty(g.n, dtype=torch.float32, device="cuda")
    fv.fv_jvp(g, fv.FV_FP32, Gr, dev(q32, torch.float32), dev(v32, torch.float32), out32)
    assert rel(host(out32, og.shape), D.jvp(og, Gr, q32, v32)) <= TOL32_STENCIL


@pytest.mark.parametrize("shape,stretch", GRIDS)
def test_project_fp64_and_fp32(fv, shape, stretch):
    og = D.Grid(*shape, stretch=stretch, Pr=PR)
    g = fv.Grid(*shape, stretch=stretch, Pr=PR)
    v = vector(og, 4)
    ref = Projector(og).api(v)
    t = dev(v, torch.float64)
    it, div = fv.fv_project(g, fv.FV_FP64, t, max_it=1, want_div=True)
    assert it == 1 and div <= 1e-12
    assert rel(host(t, og.shape), ref) <= TOL64
    v32 = round32(v)
    ref32 = Projector(og).api(v32)
    t32 = dev(v32, torch.float32)
    it, div = fv.fv_project(g, fv.FV_FP32, t32, max_it=1, want_div=True)
    assert div <= 1e-4
    assert rel(host(t32, og.shape), ref32) <= TOL32_PROJ


@pytest.mark.parametrize("shape,stretch", [((17, 13, 11), 1.5), ((40, 40, 40), 1.5), ((3, 4, 5), 0.0)])
@pytest.mark.parametrize("sigma", [0.0, -750.0])
def test_jvp_project_fused(fv, shape, stretch, sigma):
    og = D.Grid(*shape, stretch=stretch, Pr=PR)
    g = fv.Grid(*shape, stretch=stretch, Pr=PR)
    q, v = state(og, 5), vector(og, 6)
    Gr = 1.0e5
    P = Projector(og)
    qf, vf = D.from_api(og, q), D.from_api(og, v)
    J = D.jvp_full(og, Gr, qf, vf)
    ref = P.full([J[c] - sigma * vf[c] for c in range(4)])
    ref = D.to_api(og, [ref[c] + sigma * vf[c] for c in range(4)])
    out = torch.empty(g.n, dtype=torch.float64, device="cuda")
    fv.fv_jvp_project(g, fv.FV_FP64, Gr, sigma, dev(q, torch.float64), dev(v, torch.float64), out)
    assert rel(host(out, og.shape), ref) <= TOL64
    q32, v32 = round32(q), round32(v)
    qf, vf = D.from_api(og, q32), D.from_api(og, v32)
    J = D.jvp_full(og, Gr, qf, vf)
    ref = P.full([J[c] - sigma * vf[c] for c in range(4)])
    ref = D.to_api(og, [ref[c] + sigma * vf[c] for c in range(4)])
    out32 = torch.empty(g.n, dtype=torch.float32, device="cuda")
    fv.fv_jvp_project(g, fv.FV_FP32, Gr, sigma, dev(q32, torch.float32), dev(v32, torch.float32), out32)
    assert rel(host(out32, og.shape), ref) <= TOL32_PROJ


def _one_sided(n, a):
    """Caller faces clustered towards one wall only (no mirror symmetry): (e^(a i/n) - 1) / (e^a - 1)."""
    xf = np.expm1(a * np.arange(n + 1) / n) / np.expm1(a)
    xf[0], xf[-1] = 0.0, 1.0
    return xf


@pytest.mark.parametrize("shape", [(64, 32, 64), (17, 13, 11)])
def test_caller_faces_without_mirror_symmetry(fv, shape):
    """Grids built from caller faces that are not mirror-symmetric, against the oracle on the same faces:
    the FP64 fused J.v + projection (bound as for the 256-point axis: summation-order round-off amplified by
    the smallest centre spacing) and the FP32 projection.  (64, 32, 64) has tensor-core sizes: its FP32
    solve must take the CUDA-core passes, since the half-size eigenproblem split needs a symmetric axis."""
    faces = (_one_sided(shape[0], 1.2), _one_sided(shape[1], -0.8), _one_sided(shape[2], 0.6))
    og = D.Grid(*shape, Pr=PR, xyz_faces=faces)
    g = fv.Grid(*shape, Pr=PR, faces=faces)
    q, v = state(og, 12), vector(og, 13)
    Gr = 1.0e5
    P = Projector(og)
    qf, vf = D.from_api(og, q), D.from_api(og, v)
    J = D.jvp_full(og, Gr, qf, vf)
    ref = D.to_api(og, P.full(J))
    scale = D.to_api(og, J)
    out = torch.empty(g.n, dtype=torch.float64, device="cuda")
    fv.fv_jvp_project(g, fv.FV_FP64, Gr, 0.0, dev(q, torch.float64), dev(v, torch.float64), out)
    got = host(out, og.shape)
    err = max(float(np.max(np.abs(got[c] - ref[c]))) / max(float(np.max(np.abs(scale[c]))),
                                                             float(np.max(np.abs(ref[c]))), 1e-300)
              for c in range(4))
    dcmin = min(float(np.min(a.dc)) for a in og.axes)
    assert err <= max(TOL64, np.finfo(np.float64).eps * np.sqrt(max(shape)) / dcmin), err
    v32 = round32(v)
    ref32 = P.api(v32)
    t32 = dev(v32, torch.float32)
    _, div = fv.fv_project(g, fv.FV_FP32, t32, max_it=1, want_div=True)
    assert div <= 1e-4
    assert rel(host(t32, og.shape), ref32) <= TOL32_PROJ


def test_dot_axpby_deterministic(fv):
    shape = (33, 17, 9)
    og = D.Grid(*shape)
    g = fv.Grid(*shape)
    a, b = vector(og, 7), vector(og, 8)
    ta, tb = dev(a, torch.float64), dev(b, torch.float64)
    r1 = fv.fv_dot(g, fv.FV_FP64, ta, tb)
    r2 = fv.fv_dot(g, fv.FV_FP64, ta, tb)
    assert r1 == r2
    ref = sum(float(np.sum(a[c] * b[c])) for c in range(4))
    assert abs(r1 - ref) <= 1e-12 * sum(float(np.sum(np.abs(a[c] * b[c]))) for c in range(4))
    fv.fv_axpby(g, fv.FV_FP64, 2.0, ta, -0.5, tb)
    got = host(tb, og.shape)
    assert rel(got, [2.0 * a[c] - 0.5 * b[c] for c in range(4)]) <= 1e-15
    t32 = dev(a, torch.float32)
    assert fv.fv_dot(g, fv.FV_FP32, t32, t32) == pytest.approx(sum(float(np.sum(a[c] ** 2)) for c in range(4)),
                                                               rel=1e-6)


def test_full_size_256_fp32_fused_matches_oracle(fv):
    """256^3 tanh-stretched, Gr = 2e8: the bench's workload and launch configuration."""
    shape, Gr = (256, 256, 256), 2.0e8
    og = D.Grid(*shape, stretch=1.5, Pr=PR)
    g = fv.Grid(*shape, stretch=1.5, Pr=PR)
    q = state(og, 100, sigma=50.0, project=False)   # synthetic base flow (divergence not required for J.v)
    v = vector(og, 101)
    q32, v32 = round32(q), round32(v)
    out = torch.empty(g.n, dtype=torch.float32, device="cuda")
    fv.fv_jvp_project(g, fv.FV_FP32, Gr, 0.0, dev(q32, torch.float32), dev(v32, torch.float32), out)
    got = host(out, og.shape)
    del out
    ref = Projector(og).api(D.jvp(og, Gr, q32, v32))
    assert rel(got, ref) <= TOL32_PROJ


@pytest.mark.parametrize("shape", [(256, 12, 10), (10, 256, 12), (12, 10, 256)])
def test_fp64_paths_on_a_256_cell_axis(fv, shape):
    """The plain FP64 form (the comparison form of the 256^3 workload) along an axis of 256 stretched cells,
    Gr = 2e8: J.v and the projection each against the oracle at 1e-12 of their results.  The fused
    J.v + projection is measured against its input J.v: P removes the hydrostatic part of Gr T_v e_z, so
    the pressure potential phi is of the size of J.v (times the unit length) while the result is the
    remainder.  Each side rounds phi to a relative eps sqrt(n) (n-term sums of the fast-diagonalisation
    passes) and differences it over the centre spacing, so the bound is eps sqrt(n) / min(dc) of |J.v|:
    3e-12 for 256 cells stretched with s = 1.5 (min(dc) = 1.2e-3)."""
    og = D.Grid(*shape, stretch=1.5, Pr=PR)
    g = fv.Grid(*shape, stretch=1.5, Pr=PR)
    q, v = state(og, 12, sigma=30.0), vector(og, 13)
    Gr = 2.0e8
    P = Projector(og)
    qd, vd = dev(q, torch.float64), dev(v, torch.float64)
    out = torch.empty(g.n, dtype=torch.float64, device="cuda")
    fv.fv_jvp(g, fv.FV_FP64, Gr, qd, vd, out)
    jv_ref = D.jvp(og, Gr, q, v)
    assert rel(host(out, og.shape), jv_ref) <= TOL64
    t = vd.clone()
    fv.fv_project(g, fv.FV_FP64, t)
    assert rel(host(t, og.shape), P.api(v)) <= TOL64
    qf, vf = D.from_api(og, q), D.from_api(og, v)
    J = D.jvp_full(og, Gr, qf, vf)
    for sigma in (0.0, -2.0e5):
        Jin = [J[c] - sigma * vf[c] for c in range(4)]
        ref = P.full(Jin)
        ref = D.to_api(og, [ref[c] + sigma * vf[c] for c in range(4)])
        scale = D.to_api(og, Jin)
        fv.fv_jvp_project(g, fv.FV_FP64, Gr, sigma, qd, vd, out)
        got = host(out, og.shape)
        err = max(float(np.max(np.abs(got[c] - ref[c]))) / max(float(np.max(np.abs(scale[c]))),
                                                                 float(np.max(np.abs(ref[c]))), 1e-300)
                  for c in range(4))
        dcmin = min(float(np.min(a.dc)) for a in og.axes if a.n > 1)
        tol = max(TOL64, np.finfo(np.float64).eps * np.sqrt(max(shape)) / dcmin)
        assert err <= tol, (sigma, err, tol)


def test_full_size_256_fp64_fused_matches_oracle(fv):
    """256^3 tanh-stretched, Gr = 2e8 in plain FP64: the fused J.v + projection of the comparison form
    against the oracle at 1e-12, every element."""
    shape, Gr = (256, 256, 256), 2.0e8
    og = D.Grid(*shape, stretch=1.5, Pr=PR)
    g = fv.Grid(*shape, stretch=1.5, Pr=PR)
    q = state(og, 100, sigma=50.0, project=False)
    v = vector(og, 101)
    out = torch.empty(g.n, dtype=torch.float64, device="cuda")
    fv.fv_jvp_project(g, fv.FV_FP64, Gr, 0.0, dev(q, torch.float64), dev(v, torch.float64), out)
    got = host(out, og.shape)
    del out
    ref = Projector(og).api(D.jvp(og, Gr, q, v))
    assert rel(got, ref) <= TOL64
    g.close()


def test_errors_are_status_codes(fv):
    with pytest.raises(fv.FvError) as e:
        fv.Grid(1, 4, 4)
    assert e.value.status == fv.FV_EINVAL
    g = fv.Grid(4, 4, 4)
    a = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    with pytest.raises(fv.FvError) as e:
        fv.fv_jvp_project(g, fv.FV_FP64, 1.0, 0.0, a, a, a)
    assert e.value.status == fv.FV_EINVAL
    with pytest.raises(fv.FvError):
        fv.fv_jvp(g, 7, 1.0, a, a, torch.zeros_like(a))


@pytest.mark.parametrize("prec_name", ["fp64", "fp32"])
def test_fused_recurrence_step(fv, prec_name):
    shape, Gr, sigma = (20, 14, 9), 8.0e4, -900.0
    og = D.Grid(*shape, stretch=1.5, Pr=PR)
    g = fv.Grid(*shape, stretch=1.5, Pr=PR)
    q, v, w = state(og, 9), vector(og, 10), vector(og, 11)
    prec, dt, tol = ((fv.FV_FP64, torch.float64, TOL64) if prec_name == "fp64"
                     else (fv.FV_FP32, torch.float32, TOL32_PROJ))
    if prec_name == "fp32":
        q, v, w = round32(q), round32(v), round32(w)
    alpha, beta, gamma = 0.37, -1.9, 0.55
    P = Projector(og)
    qf, vf, wf = D.from_api(og, q), D.from_api(og, v), D.from_api(og, w)
    J = D.jvp_full(og, Gr, qf, vf)
    A = P.full([J[c] - sigma * vf[c] for c in range(4)])
    ref = D.to_api(og, [alpha * (A[c] + sigma * vf[c]) + beta * vf[c] + gamma * wf[c] for c in range(4)])
    tw = dev(w, dt)
    nrm = fv.fv_jvp_project_lincomb(g, prec, Gr, sigma, dev(q, dt), dev(v, dt), tw, alpha, beta, gamma, tw,
                                    want_norm=True)
    got = host(tw, og.shape)
    assert rel(got, ref) <= tol
    ref_n2 = sum(float(np.sum(a * a)) for a in got)   # the fused norm is that of the stored result
    assert nrm == pytest.approx(ref_n2, rel=1e-12)


@pytest.mark.parametrize("shape,stretch", [((17, 13, 11), 1.5), ((16, 12, 10), 0.0), ((2, 2, 3), 0.0)])
def test_diffusion_solve_inverts_the_oracle_diffusion(fv, shape, stretch):
    """fv_diffusion_solve (L^-1 of the Newton preconditioner): the oracle's diffusion operator with
    homogeneous wall data maps the FP64 output back onto the input (1e-10: the check goes through L,
    whose condition number here is ~1e4); the FP32 output matches the FP64 one within the projection's
    FP32 bound."""
    og = D.Grid(*shape, stretch=stretch, Pr=PR)
    g = fv.Grid(*shape, stretch=stretch, Pr=PR)
    x = D.to_api(og, D.from_api(og, seeded.normal_fields(41, og.shape)))  # wall slots zero
    x64 = dev(x, torch.float64)
    out64 = torch.empty_like(x64)
    fv.fv_diffusion_solve(g, fv.FV_FP64, x64, out64)
    got = host(out64, og.shape)
    back = D.diffusion(og, D.from_api(og, got), 0.0)
    full = D.from_api(og, x)
    interior = [full[0][:, :, 1:-1], full[1][:, 1:-1, :], full[2][1:-1, :, :], full[3]]
    assert rel(back, interior) <= 1e-10
    for c in range(3):  # wall slots stay zero
        assert np.all(np.take(got[c], 0, axis=2 - c) == 0.0)
    x32 = dev(x, torch.float32)
    out32 = torch.empty_like(x32)
    fv.fv_diffusion_solve(g, fv.FV_FP32, x32, out32)
    assert rel(host(out32, og.shape), got) <= TOL32_PROJ
    fv.fv_diffusion_solve(g, fv.FV_FP64, x64, x64)  # in place
    assert rel(host(x64, og.shape), got) <= 1e-14


def test_stream_ordered_step_matches_the_synchronous_one(fv):
    """fv_jvp_project_lincomb_dev (norm left on the device) computes the same step and the same norm as
    fv_jvp_project_lincomb (norm read back to the host)."""
    shape = (64, 48, 40)
    og = D.Grid(*shape, stretch=1.5, Pr=PR)
    g = fv.Grid(*shape, stretch=1.5, Pr=PR)
    q = dev(state(og, 7), torch.float32)
    v = dev(vector(og, 8), torch.float32)
    w = dev(vector(og, 9), torch.float32)
    a = torch.empty_like(v)
    nrm = fv.fv_jvp_project_lincomb(g, fv.FV_FP32, 2e5, -50.0, q, v, w, 0.3, -1.2, 0.7, a, want_norm=True)
    b = torch.empty_like(v)
    n2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    fv.fv_jvp_project_lincomb_dev(g, fv.FV_FP32, 2e5, -50.0, q, v, w, 0.3, -1.2, 0.7, b, norm2=n2)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert float(n2.item()) == nrm


@pytest.mark.parametrize("prec_name,shape", [("fp32", (64, 48, 40)), ("fp64", (17, 13, 11))])
def test_batched_fused_path_eager_and_graph(fv, prec_name, shape):
    """fv_jvp_project_batch gives exactly the per-vector fv_jvp_project results, eagerly and through its
    captured graph (first call captures, later calls replay it on new vector contents)."""
    prec = fv.FV_FP32 if prec_name == "fp32" else fv.FV_FP64
    dt = torch.float32 if prec_name == "fp32" else torch.float64
    og = D.Grid(*shape, stretch=1.5, Pr=PR)
    g = fv.Grid(*shape, stretch=1.5, Pr=PR)
    nvec, Gr, sigma = 5, 3e5, -60.0
    q = dev(state(og, 21), dt)
    V = torch.cat([dev(vector(og, 30 + i), dt) for i in range(nvec)])
    ref = torch.empty_like(V)
    for i in range(nvec):
        fv.fv_jvp_project(g, prec, Gr, sigma, q, V[i * g.n:(i + 1) * g.n], ref[i * g.n:(i + 1) * g.n])
    W = torch.empty_like(V)
    fv.fv_jvp_project_batch(g, prec, Gr, sigma, q, V, W, nvec, use_graph=False)
    assert torch.equal(W, ref)
    for _ in range(2):  # capture, then replay
        W.zero_()
        fv.fv_jvp_project_batch(g, prec, Gr, sigma, q, V, W, nvec, use_graph=True)
        torch.cuda.synchronize()
        assert torch.equal(W, ref)
    # the replay reads the vectors' current contents
    V.mul_(2.0)
    fv.fv_jvp_project_batch(g, prec, Gr, sigma, q, V, W, nvec, use_graph=True)
    torch.cuda.synchronize()
    assert torch.allclose(W, 2.0 * ref, rtol=1e-5 if prec_name == "fp32" else 1e-12, atol=0)
    # a different argument set is captured anew
    fv.fv_jvp_project_batch(g, prec, 2 * Gr, sigma, q, V, W, nvec, use_graph=True)
    torch.cuda.synchronize()
    ref2 = torch.empty_like(V[:g.n])
    fv.fv_jvp_project(g, prec, 2 * Gr, sigma, q, V[:g.n], ref2)
    assert torch.equal(W[:g.n], ref2)


def test_block_path_tensorcore_autotuned(fv):
    """A block of FP32 vectors on a grid where every stage has its block form (two-cell stencil, quad
    divergence and correction, tcgen05 passes over the stacked fields), with the z-chunk autotuner on:
    the per-vector results of fv_jvp_project to FP32 round-off (each cell's arithmetic is the same; only
    the grouping of cells into CTAs and tiles differs), and the oracle within the fused-path bound."""
    shape = (64, 64, 64)
    og = D.Grid(*shape, stretch=1.5, Pr=PR)
    g = fv.Grid(*shape, stretch=1.5, Pr=PR)
    nvec, Gr, sigma = 6, 1.0e5, -750.0
    q = dev(state(og, 41), torch.float32)
    vs = [round32(vector(og, 50 + i)) for i in range(nvec)]
    V = torch.cat([dev(v, torch.float32) for v in vs])
    ref = torch.empty_like(V)
    for i in range(nvec):
        fv.fv_jvp_project(g, fv.FV_FP32, Gr, sigma, q, V[i * g.n:(i + 1) * g.n], ref[i * g.n:(i + 1) * g.n])
    W = torch.empty_like(V)
    for graph in (False, True, True):
        W.zero_()
        fv.fv_jvp_project_batch(g, fv.FV_FP32, Gr, sigma, q, V, W, nvec, use_graph=graph, autotune=True)
        torch.cuda.synchronize()
        for i in range(nvec):
            a, b = W[i * g.n:(i + 1) * g.n], ref[i * g.n:(i + 1) * g.n]
            assert float((a - b).abs().max()) <= 1e-6 * float(b.abs().max()), (graph, i)
    zc, nv = fv.fv_get_tuning(g)
    assert zc in (4, 8, 16, 32, 64) and nv == nvec
    # one vector of the block against the oracle (FP32-rounded inputs, FP64 oracle)
    qa = round32(state(og, 41))
    P = Projector(og)
    i = 3
    qf, vf = D.from_api(og, qa), D.from_api(og, vs[i])
    J = D.jvp_full(og, Gr, qf, vf)
    r = P.full([J[c] - sigma * vf[c] for c in range(4)])
    exp = D.to_api(og, [r[c] + sigma * vf[c] for c in range(4)])
    assert rel(host(W[i * g.n:(i + 1) * g.n], og.shape), exp) <= TOL32_PROJ
    g.close()


def test_batch_plan_several_grids_one_graph(fv):
    """fv_batch_plan: three continuation points on grids of different sizes (one of them without the
    block stencil) in one captured graph with concurrent branches give the per-vector results, and the
    last vector of every problem matches the oracle within the fused-path FP32 bound; a replay
    reads the vectors' current contents; growing a handle's block buffers invalidates the plan."""
    probs = [((64, 64, 64), 3.0e7, 3), ((40, 36, 32), 7.4e7, 2), ((96, 32, 48), 2.5e8, 2)]
    keep, oracle_ref = [], []
    for k, (shape, Gr, nvec) in enumerate(probs):
        og = D.Grid(*shape, stretch=1.5, Pr=PR)
        g = fv.Grid(*shape, stretch=1.5, Pr=PR)
        qa = round32(state(og, 60 + k))
        va = [round32(vector(og, 70 + 10 * k + i)) for i in range(nvec)]
        q = dev(qa, torch.float32)
        V = torch.cat([dev(v, torch.float32) for v in va])
        W = torch.empty_like(V)
        sigma = -100.0 * (k + 1)
        ref = torch.empty_like(V)
        for i in range(nvec):
            fv.fv_jvp_project(g, fv.FV_FP32, Gr, sigma, q, V[i * g.n:(i + 1) * g.n], ref[i * g.n:(i + 1) * g.n])
        keep.append((g, Gr, sigma, q, V, W, nvec, ref))
        # the oracle's result for the last vector of this problem (FP32-rounded inputs, FP64 oracle)
        qf, vf = D.from_api(og, qa), D.from_api(og, va[-1])
        J = D.jvp_full(og, Gr, qf, vf)
        r = Projector(og).full([J[c] - sigma * vf[c] for c in range(4)])
        oracle_ref.append((og, D.to_api(og, [r[c] + sigma * vf[c] for c in range(4)])))
    plan = fv.BatchPlan([k[:7] for k in keep], fv.FV_FP32, autotune=True)
    for (g, Gr, sigma, q, V, W, nvec, ref), (og, exp) in zip(keep, oracle_ref):
        assert rel(host(W[(nvec - 1) * g.n:nvec * g.n], og.shape), exp) <= TOL32_PROJ, og.shape

    def check(scale):
        torch.cuda.synchronize()
        for (g, Gr, sigma, q, V, W, nvec, ref) in keep:
            err = float((W - scale * ref).abs().max())
            assert err <= 1e-5 * float(ref.abs().max()) * scale, (g.shape, err)

    check(1.0)
    for (_, _, _, _, _, W, _, _) in keep:
        W.zero_()
    plan.launch(torch.cuda.current_stream().cuda_stream)
    check(1.0)
    for (_, _, _, _, V, W, _, _) in keep:
        V.mul_(2.0)
        W.zero_()
    plan.launch(torch.cuda.current_stream().cuda_stream)
    check(2.0)
    # a larger block on the first handle reallocates its block buffers: the plan refuses to replay
    g0, Gr0, s0, q0 = keep[0][:4]
    V2 = torch.cat([keep[0][4]] * 2)
    W2 = torch.empty_like(V2)
    fv.fv_jvp_project_batch(g0, fv.FV_FP32, Gr0, s0, q0, V2, W2, 2 * keep[0][6])
    with pytest.raises(fv.FvError):
        plan.launch(torch.cuda.current_stream().cuda_stream)
    plan.close()
    for k in keep:
        k[0].close()


@pytest.mark.parametrize("src,dst", [((20, 16, 12), (33, 27, 21)), ((64, 64, 64), (96, 80, 72)), ((33, 27, 21), (20, 16, 12))])
def test_grid_transfer_matches_oracle(fv, src, dst):
    """fv_transfer (grid sequencing) against the oracle's trilinear transfer and projection, FP64, 1e-12."""
    from oracle import transfer as TR
    oa, ob = D.Grid(*src, stretch=1.5, Pr=PR), D.Grid(*dst, stretch=1.5, Pr=PR)
    ga, gb = fv.Grid(*src, stretch=1.5, Pr=PR), fv.Grid(*dst, stretch=1.5, Pr=PR)
    qa = state(oa, 91, sigma=3.0)
    ref = D.to_api(ob, TR.transfer(oa, D.from_api(oa, qa), ob))
    out = torch.empty(gb.n, dtype=torch.float64, device="cuda")
    fv.fv_transfer(ga, dev(qa, torch.float64), gb, out)
    torch.cuda.synchronize()
    assert rel(host(out, ob.shape), ref) <= TOL64
    ga.close()
    gb.close()
