"""GPU Newton and Chebyshev-Arnoldi drivers (through the C-ABI) against the oracle.

* FP64 Newton, with and without its optional diffusion preconditioner, reaches the oracle's steady
  state (both solve P F = 0 to round-off; the states agree to 1e-9 in max-norm, the residual tolerance
  divided by the smallest eigenvalue magnitude); so does pseudo-transient continuation, with no Gr ladder.
* Mixed Newton (FP32 Krylov, FP64 residual) refines to the FP64 state within 1e-8 max-norm.
* FP64 Arnoldi: Gr = 0 closed-form temperature spectrum, and agreement with the oracle's
  Chebyshev-Arnoldi at Gr > 0 (both converged to 1e-9 residual: eigenvalues to 1e-8).
* Mixed Arnoldi: leading eigenvalue within 1e-6 of the FP64 one; its Ritz vectors certified by the
  oracle's own FP64 residual ||P J x - lam x|| / (|lam| ||x||).
* The 32^3, Gr = 1e5 workload: GPU Newton, then the four leading eigenvalues of both forms against
  the oracle's stored ones (tests/golden/config0_eigs_32.txt), with the Chebyshev filter and with the
  implicit-Euler transform.
"""
import os

import numpy as np
import pytest

import oracle.discretisation as D
from oracle import diagnostics as DG
from oracle import solvers as SV
from oracle.projection import Projector

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
PR = 0.71


@pytest.fixture(scope="module")
def fv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_08816_gb300 import build
    build.build()
    from paper_2210_08816_gb300 import fv as _fv
    _fv.lib()
    return _fv


def dev(api):
    return torch.tensor(np.stack(api), dtype=torch.float64, device="cuda").contiguous().view(-1)


def host(t, shape):
    a = t.view(4, *shape).double().cpu().numpy()
    return [a[c] for c in range(4)]


def maxrel(a, b):
    return max(float(np.max(np.abs(a[c] - b[c]))) for c in range(4)) / max(float(np.max(np.abs(b[c]))) for c in range(4))


def conduction_api(og):
    return D.to_api(og, D.conduction_state(og))


@pytest.mark.parametrize("precond", [0, 1])
def test_newton_fp64_matches_oracle(fv, precond):
    """With and without the diffusion preconditioner: the same steady state as the (unpreconditioned)
    oracle Newton."""
    shape, Gr = (10, 8, 6), 1.2e4
    og = D.Grid(*shape, stretch=1.5, Pr=PR)
    q_ref, rep_ref = SV.newton_steady(og, Gr, D.conduction_state(og), tol=1e-11)
    assert rep_ref["status"] == "converged"
    g = fv.Grid(*shape, stretch=1.5, Pr=PR)
    q = dev(conduction_api(og))
    o = fv.fv_newton_default_opts()
    o.tol = 1e-11
    o.precond = precond
    st, rep = fv.newton_steady(g, Gr, q, o)
    assert st == fv.FV_OK, rep.history[:rep.newton_steps + 1]
    got = host(q, og.shape)
    assert maxrel(got, D.to_api(og, q_ref)) <= 1e-9
    assert max(DG.symmetry_measures(og, got[3])) <= 1e-9      # Section 2: symmetric steady flow


def test_newton_mixed_refines_to_fp64(fv):
    shape, Gr = (16, 16, 16), 1.0e5
    og = D.Grid(*shape, stretch=1.5, Pr=PR)
    g = fv.Grid(*shape, stretch=1.5, Pr=PR)
    res = {}
    for prec in (fv.FV_FP64, fv.FV_FP32):
        q = dev(conduction_api(og))
        o = fv.fv_newton_default_opts()
        o.precision = prec
        o.tol = 1e-12
        o.max_newton = 30
        o.gr_start = 1.25e4
        o.gr_ratio = 2.0
        st, rep = fv.newton_steady(g, Gr, q, o)
        assert st == fv.FV_OK, (prec, list(rep.history[:rep.newton_steps + 1]))
        res[prec] = host(q, og.shape)
    assert maxrel(res[fv.FV_FP32], res[fv.FV_FP64]) <= 1e-8
    # certificate with the oracle's own operators
    P = Projector(og)
    r = P.full(D.residual_full(og, Gr, D.from_api(og, res[fv.FV_FP32])))
    scale = max(float(np.max(np.abs(a))) for a in D.residual_full(og, Gr, D.conduction_state(og)))
    assert max(float(np.max(np.abs(a))) for a in r) <= 1e-9 * scale


@pytest.fixture(scope="module")
def cube32(fv):
    """32^3 uniform, Pr = 0.71, Gr = 1e5: GPU Newton from conduction (continuation from 1.25e4)."""
    shape, Gr = (32, 32, 32), 1.0e5
    og = D.Grid(*shape, stretch=0.0, Pr=PR)
    g = fv.Grid(*shape, stretch=0.0, Pr=PR)
    q = dev(conduction_api(og))
    o = fv.fv_newton_default_opts()
    o.gr_start, o.gr_ratio = 1.25e4, 2.0
    st, rep = fv.newton_steady(g, Gr, q, o)
    return og, g, Gr, q, st, rep


def test_newton_32cube_uniform_config(fv, cube32):
    """32^3 uniform, Pr = 0.71, Gr = 1e5 (continuation from 1.25e4), inner solves to 1e-10."""
    og, g, Gr, q, st, rep = cube32
    assert st == fv.FV_OK
    got = host(q, og.shape)
    P = Projector(og)
    r = P.full(D.residual_full(og, Gr, D.from_api(og, got)))
    assert max(float(np.max(np.abs(a))) for a in r) <= 1e-9 * rep.residual0
    assert max(DG.symmetry_measures(og, got[3])) <= 1e-9
    assert DG.nusselt_hot(og, got[3]) < -1.0


def _golden_eigs(name):
    rows = [ln.split() for ln in open(os.path.join(os.path.dirname(__file__), "golden", name))
            if ln.strip() and not ln.startswith("#")]
    return np.array([float(a) + 1j * float(b) for a, b in rows])


def test_arnoldi_32cube_matches_stored_oracle_eigenvalues(fv, cube32):
    """The 32^3 Gr = 1e5 workload: four leading eigenvalues (k = 4, m = 20) by the FP64 and the mixed
    GPU forms against the oracle's, stored by tests/golden/make_config0_eigs.py (tol 1e-9)."""
    og, g, Gr, q, st, rep = cube32
    assert st == fv.FV_OK
    ref = _golden_eigs("config0_eigs_32.txt")
    o = fv.fv_arnoldi_default_opts()
    o.tol = 1e-9
    st, lam, r64 = fv.arnoldi_leading(g, 4, Gr, q, o)
    assert st == fv.FV_OK
    assert len(lam) == len(ref) and np.allclose(np.array(lam), ref, rtol=1e-8, atol=0), (lam, ref)
    o.precision = fv.FV_FP32
    o.tol = 1e-6
    st, lam32, r32 = fv.arnoldi_leading(g, 4, Gr, q, o)
    assert st == fv.FV_OK
    assert np.allclose(np.array(lam32[:len(ref)]), ref, rtol=1e-6, atol=0), (lam32, ref)


def test_arnoldi_euler_transform_32cube_matches_stored_oracle_eigenvalues(fv, cube32):
    """Arnoldi on the implicit-Euler propagator (I - dt P J)^-1 instead of the Chebyshev polynomial:
    the same four leading eigenvalues of the 32^3, Gr = 1e5 workload as the oracle's stored ones (FP64
    to 1e-8; the mixed form, whose FP64 cycles solve by iterative refinement around FP32 GMRES, to 1e-6)."""
    og, g, Gr, q, st, rep = cube32
    assert st == fv.FV_OK
    ref = _golden_eigs("config0_eigs_32.txt")
    o = fv.fv_arnoldi_default_opts()
    o.tol = 1e-9
    # shift s = 1/dt = 333: the pair -65.85 +- 198i ranks by |lam - s| among the twelve kept values (with
    # s = 100 it would rank behind -97.5 +- 140i and -103 and not be kept); -67.95 and -72.77 lie within
    # 1.2 % of each other in |lam - s|, which takes the cycles below
    o.euler_dt = 3e-3
    o.m = 40
    o.max_restarts = 30
    st, lam, r64 = fv.arnoldi_leading(g, 4, Gr, q, o)
    assert st == fv.FV_OK, (lam, list(r64.residual[:4]))
    assert len(lam) == len(ref) and np.allclose(np.array(lam), ref, rtol=1e-8, atol=0), (lam, ref)
    assert all(d == 0 for d in r64.degrees[:r64.restarts + 1])   # no Chebyshev filter ran
    o.precision = fv.FV_FP32
    o.tol = 1e-6
    st, lam32, r32 = fv.arnoldi_leading(g, 4, Gr, q, o)
    assert st == fv.FV_OK, (lam32, list(r32.residual[:4]))
    assert np.allclose(np.array(lam32[:len(ref)]), ref, rtol=1e-6, atol=0), (lam32, ref)


def test_arnoldi_fp64_gr0_closed_form(fv):
    shape = (10, 8, 6)
    og = D.Grid(*shape, stretch=0.0, Pr=PR)
    g = fv.Grid(*shape, stretch=0.0, Pr=PR)
    q = dev(conduction_api(og))
    o = fv.fv_arnoldi_default_opts()
    o.tol = 1e-10
    st, lam, rep = fv.arnoldi_leading(g, 4, 0.0, q, o)
    assert st == fv.FV_OK
    l1 = lambda n, j: 4.0 * n * n * np.sin(j * np.pi / (2 * n)) ** 2
    expect = sorted((-(l1(10, a) + l1(8, b) + l1(6, c)) / PR for a in range(1, 4) for b in range(4) for c in range(4)),
                    reverse=True)[:4]
    assert np.allclose([z.real for z in lam[:4]], expect, rtol=1e-9, atol=0)


def test_arnoldi_fp64_and_mixed_vs_oracle(fv):
    shape, Gr = (8, 7, 6), 1.2e4
    og = D.Grid(*shape, stretch=1.5, Pr=PR)
    q_ref, _ = SV.newton_steady(og, Gr, D.conduction_state(og), tol=1e-11)
    x0 = np.random.default_rng(3).standard_normal(D.n_unknowns(og))
    lam_ref, _, info = SV.leading_eigenvalues(og, Gr, q_ref, k=4, m=20, seed_vector=x0, tol=1e-9)
    assert info["converged"]
    g = fv.Grid(*shape, stretch=1.5, Pr=PR)
    q = dev(D.to_api(og, q_ref))
    o = fv.fv_arnoldi_default_opts()
    o.tol = 1e-9
    st, lam, rep = fv.arnoldi_leading(g, 4, Gr, q, o)
    assert st == fv.FV_OK
    k = min(len(lam), len(lam_ref))
    assert np.allclose(np.array(lam[:k]), lam_ref[:k], rtol=1e-8, atol=0), (lam, lam_ref)
    # mixed: FP32 Krylov vectors, FP64 Hessenberg / Gram-Schmidt coefficients
    o.precision = fv.FV_FP32
    o.tol = 1e-6
    vecs = torch.empty((4 + 1) * g.n, dtype=torch.float32, device="cuda")
    st, lam32, rep32 = fv.arnoldi_leading(g, 4, Gr, q, o, vecs=vecs)
    assert st == fv.FV_OK
    assert abs(lam32[0] - lam_ref[0]) <= 1e-6 * abs(lam_ref[0])
    # certify the leading Ritz vector with the oracle's FP64 operator
    x = host(vecs[:g.n], og.shape)
    A = SV.projected_jacobian(og, Gr, q_ref)
    xv = D.pack(D.from_api(og, x))
    if lam32[0].imag == 0.0:
        r = A(xv) - lam32[0].real * xv
        assert np.linalg.norm(r) <= 1e-5 * abs(lam32[0]) * np.linalg.norm(xv)


def test_newton_pseudo_transient_from_conduction(fv):
    """Pseudo-transient continuation (ptc_dt0 > 0) reaches Gr = 1e5 on a 16^3 stretched grid straight
    from conduction, with no Gr ladder, and lands on the same steady state as plain Newton along a
    ladder (a globalisation changes the path, not the converged state); certified by the oracle's FP64
    residual."""
    shape, Gr = (16, 16, 16), 1.0e5
    og = D.Grid(*shape, stretch=1.5, Pr=PR)
    g = fv.Grid(*shape, stretch=1.5, Pr=PR)
    res = {}
    for name in ("ladder", "ptc"):
        q = dev(conduction_api(og))
        o = fv.fv_newton_default_opts()
        o.tol = 1e-12
        if name == "ladder":
            o.max_newton = 30
            o.gr_start, o.gr_ratio = 1.25e4, 2.0
        else:
            o.max_newton = 60
            o.ptc_dt0 = 1e-2
        st, rep = fv.newton_steady(g, Gr, q, o)
        assert st == fv.FV_OK, (name, list(rep.history[:min(rep.newton_steps + 1, 64)]))
        if name == "ptc":
            assert rep.continuation_steps == 0
        res[name] = host(q, og.shape)
    assert maxrel(res["ptc"], res["ladder"]) <= 1e-9
    P = Projector(og)
    r = P.full(D.residual_full(og, Gr, D.from_api(og, res["ptc"])))
    scale = max(float(np.max(np.abs(a))) for a in D.residual_full(og, Gr, D.conduction_state(og)))
    assert max(float(np.max(np.abs(a))) for a in r) <= 1e-9 * scale


@pytest.fixture(scope="module")
def cube16_high_gr(fv):
    """16^3 tanh-stretched (s = 1.5), Gr = 1.6e6: GPU Newton by pseudo-transient continuation from conduction."""
    shape, Gr = (16, 16, 16), 1.6e6
    og = D.Grid(*shape, stretch=1.5, Pr=PR)
    g = fv.Grid(*shape, stretch=1.5, Pr=PR)
    q = dev(conduction_api(og))
    o = fv.fv_newton_default_opts()
    o.tol = 1e-12
    o.max_newton = 60
    o.ptc_dt0 = 1e-3
    o.gr_start, o.gr_ratio = 1e5, 4.0
    st, rep = fv.newton_steady(g, Gr, q, o)
    return og, g, Gr, q, st, rep


@pytest.mark.parametrize("prec_name", ["fp64", "mixed"])
def test_shift_invert_arnoldi_matches_independent_oracle_at_high_gr(fv, cube16_high_gr, prec_name):
    """The implicit-Euler (shift-invert) Arnoldi with thick restarts against eigenvalues that the oracle
    computed by a different method: Newton with sparse-LU corrections and ARPACK shift-invert on the saddle
    pencil at several shifts along the imaginary axis (tests/golden/make_high_gr_eigs.py).  With the shift
    s = 1/dt = 100 the four values nearest s are the four leading real eigenvalues, golden values 1, 2, 3
    and 6 (the pair -108.5 +- 820i between them lies 850 from s and ranks behind others): FP64 to 1e-8, the
    mixed form to 1e-6; the GPU steady state is certified by the oracle's residual first."""
    og, g, Gr, q, st, rep = cube16_high_gr
    assert st == fv.FV_OK, list(rep.history[:rep.newton_steps + 1])
    got = host(q, og.shape)
    P = Projector(og)
    r = P.full(D.residual_full(og, Gr, D.from_api(og, got)))
    assert max(float(np.max(np.abs(a))) for a in r) <= 1e-8 * rep.residual0
    gold = _golden_eigs("eigs_16_stretched_gr1.6e6.txt")
    ref = gold[[0, 1, 2, 5]]
    assert np.all(ref.imag == 0.0)
    o = fv.fv_arnoldi_default_opts()
    o.euler_dt = 1e-2
    o.m = 30
    o.max_restarts = 12
    o.tol = 1e-9 if prec_name == "fp64" else 1e-6
    o.precision = fv.FV_FP64 if prec_name == "fp64" else fv.FV_FP32
    st, lam, r64 = fv.arnoldi_leading(g, 4, Gr, q, o)
    assert st == fv.FV_OK, (lam, list(r64.residual[:r64.nconv]))
    rtol = 1e-8 if prec_name == "fp64" else 1e-6
    assert np.allclose(np.array(lam[:4]), ref, rtol=rtol, atol=0), (lam, ref)


def test_small_dt_detects_the_high_frequency_pair(fv, cube16_high_gr):
    """With s = 1/dt = 3333 the distance |lam - s| ranks nearly by real part, and the oracle's pair
    -108.47 +- 820.34i (4th and 5th by real part) is among the returned values (FP64, six values, 14
    cycles): detected, within 1e-4 of the oracle, its residual below 1e-2.  The convergence is slow at
    such a shift (the wanted values of B = (A - s)^-1 lie within a factor 1.1 of each other), so this
    checks detection, not the polished value."""
    og, g, Gr, q, st, rep = cube16_high_gr
    assert st == fv.FV_OK
    pair = _golden_eigs("eigs_16_stretched_gr1.6e6.txt")[3]
    o = fv.fv_arnoldi_default_opts()
    o.euler_dt = 3e-4
    o.m = 30
    o.max_restarts = 14
    o.tol = 1e-6
    st, lam, r64 = fv.arnoldi_leading(g, 6, Gr, q, o)
    i = int(np.argmin([abs(z - pair) for z in lam]))
    assert abs(lam[i] - pair) <= 1e-4 * abs(pair), (lam, pair)
    assert r64.residual[i] <= 1e-2, list(r64.residual[:r64.nconv])
