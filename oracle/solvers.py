"""Newton with BiCGstab(2)/GMRES inner solves, and Chebyshev-preconditioned Arnoldi (FP64, numpy).

Test infrastructure only (see the package docstring).

Section 1 (methods paragraph): steady flows by Newton's method whose
corrections come from BiCGstab(2) combined with GMRES; leading eigenvalues by
the Chebyshev-preconditioned Arnoldi iteration (its ref. 21: Saad's Chebyshev
acceleration of Arnoldi's method); every Krylov vector divergence free.
Section 4.1: four leading eigenvalues are needed to separate two close modes.

Readings where the paper is silent:
* BiCGstab(2) (Sleijpen & Fokkema 1993) runs first; GMRES(m) takes over from
  the current iterate on a breakdown (rho or gamma = 0) or when the residual
  has not halved over 20 cycles.
* Krylov inner products are Euclidean over the unknowns.
* The Chebyshev filter uses an ellipse symmetric about the real axis that
  contains the unwanted Ritz values; it is picked from a confocal family by a
  small scan that maximises the slowest wanted damping rate.  The polynomial is
  T_n((z - d)/c) / T_n((lam_ref - d)/c), applied by its three-term recurrence in
  real arithmetic with c^2 (which may be negative).  The ellipse contains this
  cycle's unwanted Ritz values and the far end of the spectrum (the Rayleigh
  quotient of a short power iteration, pushed out by 5%): filtered restarts no
  longer show that end, and T_n grows fast outside its ellipse.
* P J vanishes on the gradient complement range(G), so on the full unknown
  space it has a spurious eigenvalue 0 that lies to the right of every wanted
  eigenvalue of a stable flow; round-off gradient components would be
  amplified by the filter.  The Krylov methods therefore apply
      A_sigma x = P (J x - sigma x) + sigma x ,
  which equals P J x on divergence-free x and moves the complement to the
  eigenvalue sigma < 0 inside the damped part of the spectrum (sigma = half
  the largest diffusion eigenvalue estimate, `default_shift`).
"""
from __future__ import annotations

import numpy as np

from .discretisation import (Grid, jvp_full, residual_full, pack, unpack)
from .projection import Projector


# ----------------------------------------------------------------------------- linear solvers
def bicgstab2(A, b, x0=None, tol=1e-10, max_matvec=20000, stall_cycles=20):
    """BiCGstab(l) with l = 2.  Returns (x, info) with info['status'] in
    {'converged', 'breakdown', 'stalled', 'maxit'} and the residual history."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A(x) if x0 is not None else b.copy()
    nmv = 1 if x0 is not None else 0
    rt = r.copy()
    u = np.zeros_like(b)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, {"status": "converged", "history": [0.0], "matvecs": nmv}
    rho0, alpha, omega = 1.0, 0.0, 1.0
    hist = [np.linalg.norm(r) / bnorm]
    best_at = 0
    while True:
        if hist[-1] <= tol:
            return x, {"status": "converged", "history": hist, "matvecs": nmv}
        if nmv + 4 > max_matvec:
            return x, {"status": "maxit", "history": hist, "matvecs": nmv}
        rho0 = -omega * rho0
        R = [r, None, None]
        U = [u, None, None]
        for j in range(2):                      # BiCG part
            rho1 = float(np.dot(R[j], rt))
            if rho0 == 0.0 or rho1 == 0.0:
                return x, {"status": "breakdown", "history": hist, "matvecs": nmv}
            beta = alpha * rho1 / rho0
            rho0 = rho1
            for i in range(j + 1):
                U[i] = R[i] - beta * U[i]
            U[j + 1] = A(U[j])
            gamma = float(np.dot(U[j + 1], rt))
            if gamma == 0.0:
                return x, {"status": "breakdown", "history": hist, "matvecs": nmv + 1}
            alpha = rho0 / gamma
            for i in range(j + 1):
                R[i] = R[i] - alpha * U[i + 1]
            R[j + 1] = A(R[j])
            x = x + alpha * U[0]
            nmv += 2
        # minimal-residual part: min || R0 - g1 R1 - g2 R2 ||
        G = np.array([[np.dot(R[1], R[1]), np.dot(R[1], R[2])],
                      [np.dot(R[2], R[1]), np.dot(R[2], R[2])]])
        c = np.array([np.dot(R[1], R[0]), np.dot(R[2], R[0])])
        try:
            g = np.linalg.solve(G, c)
        except np.linalg.LinAlgError:
            return x, {"status": "breakdown", "history": hist, "matvecs": nmv}
        x = x + g[0] * R[0] + g[1] * R[1]
        r = R[0] - g[0] * R[1] - g[1] * R[2]
        u = U[0] - g[0] * U[1] - g[1] * U[2]
        omega = float(g[1])
        hist.append(np.linalg.norm(r) / bnorm)
        if hist[-1] <= 0.5 * hist[best_at]:
            best_at = len(hist) - 1
        elif len(hist) - 1 - best_at >= stall_cycles:
            return x, {"status": "stalled", "history": hist, "matvecs": nmv}


def gmres(A, b, x0=None, tol=1e-10, m=30, max_matvec=20000):
    """Restarted GMRES(m) with repeated classical Gram-Schmidt and a small least-squares solve."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, {"status": "converged", "history": [0.0], "matvecs": 0}
    nmv = 0
    hist = []
    while True:
        r = b - A(x)
        nmv += 1
        beta = np.linalg.norm(r)
        hist.append(beta / bnorm)
        if beta <= tol * bnorm:
            return x, {"status": "converged", "history": hist, "matvecs": nmv}
        if nmv >= max_matvec:
            return x, {"status": "maxit", "history": hist, "matvecs": nmv}
        V = np.zeros((m + 1, b.size))
        H = np.zeros((m + 1, m))
        V[0] = r / beta
        k_used = m
        for j in range(m):
            w = A(V[j])
            nmv += 1
            for _ in range(2):
                h = V[:j + 1] @ w
                w = w - V[:j + 1].T @ h
                H[:j + 1, j] += h
            H[j + 1, j] = np.linalg.norm(w)
            e1 = np.zeros(j + 2)
            e1[0] = beta
            y, *_ = np.linalg.lstsq(H[:j + 2, :j + 1], e1, rcond=None)
            res = np.linalg.norm(H[:j + 2, :j + 1] @ y - e1)
            if H[j + 1, j] == 0.0 or res <= tol * bnorm or nmv >= max_matvec:
                k_used = j + 1
                break
            V[j + 1] = w / H[j + 1, j]
        e1 = np.zeros(k_used + 1)
        e1[0] = beta
        y, *_ = np.linalg.lstsq(H[:k_used + 1, :k_used], e1, rcond=None)
        x = x + V[:k_used].T @ y


def solve_linear(A, b, tol=1e-10, max_matvec=20000):
    """BiCGstab(2) combined with GMRES: GMRES(30) continues from BiCGstab(2)'s iterate
    after a breakdown or stagnation."""
    x, info = bicgstab2(A, b, tol=tol, max_matvec=max_matvec)
    info["solver"] = "bicgstab2"
    if info["status"] in ("breakdown", "stalled"):
        x, info2 = gmres(A, b, x0=x, tol=tol, max_matvec=max_matvec - info["matvecs"])
        info2["solver"] = "bicgstab2+gmres"
        info2["matvecs"] += info["matvecs"]
        info = info2
    return x, info


# ----------------------------------------------------------------------------- Newton
def newton_steady(grid: Grid, Gr: float, q0, tol=1e-10, krylov_tol=1e-10, max_newton=20,
                  max_matvec=20000, projector: Projector | None = None):
    """Newton's method for P F(q) = 0 on divergence-free q (full arrays in and out).

    Each correction solves (P J(q)) delta = -P F(q) on the divergence-free
    subspace.  Stops when ||P F||_inf <= tol * max(1, ||P F(q0)||_inf) or when
    ||delta||_inf <= 1e-12 * max(1, ||q||_inf).
    """
    P = projector or Projector(grid)
    q = [np.array(a, dtype=np.float64, copy=True) for a in q0]
    report = {"residual": [], "krylov": [], "status": "maxit"}
    r0 = None
    for _ in range(max_newton + 1):
        r = pack(P.full(residual_full(grid, Gr, q)))
        rn = float(np.max(np.abs(r)))
        report["residual"].append(rn)
        r0 = rn if r0 is None else r0
        if rn <= tol * max(1.0, r0):
            report["status"] = "converged"
            break
        if len(report["krylov"]) >= max_newton:
            break
        A = shifted_operator(grid, Gr, q, default_shift(grid), P)

        delta, info = solve_linear(A, -r, tol=krylov_tol, max_matvec=max_matvec)
        report["krylov"].append({k: info[k] for k in ("status", "solver", "matvecs")})
        d = unpack(grid, delta)
        q = [q[c] + d[c] for c in range(4)]
        qn = max(float(np.max(np.abs(pack(q)))), 1.0)
        if float(np.max(np.abs(delta))) <= 1e-12 * qn:
            r = pack(P.full(residual_full(grid, Gr, q)))
            report["residual"].append(float(np.max(np.abs(r))))
            report["status"] = "converged"
            break
    return q, report


# ----------------------------------------------------------------------------- Arnoldi
def arnoldi(A, v0, m):
    """m steps of Arnoldi with classical Gram-Schmidt applied twice.  Returns V (m+1 rows) and H."""
    n = v0.size
    V = np.zeros((m + 1, n))
    H = np.zeros((m + 1, m))
    V[0] = v0 / np.linalg.norm(v0)
    for j in range(m):
        w = A(V[j])
        for _ in range(2):
            h = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h
            H[:j + 1, j] += h
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] == 0.0:
            return V[:j + 1], H[:j + 1, :j + 1], j + 1
        V[j + 1] = w / H[j + 1, j]
    return V, H, m


def order_eigs(lam: np.ndarray) -> np.ndarray:
    """Indices ordering eigenvalues by real part descending, then |Im| descending, +Im first."""
    return np.array(sorted(range(len(lam)), key=lambda i: (-lam[i].real, -abs(lam[i].imag), -lam[i].imag)))


def _level(z, d, c2):
    """|w| with w = xi + sqrt(xi^2 - 1), xi = (z - d)/c, |w| >= 1: the confocal-ellipse level of z."""
    z = np.asarray(z, dtype=complex)
    if abs(c2) < 1e-300:
        return np.abs(z - d)
    c = np.sqrt(complex(c2))
    xi = (z - d) / c
    s = np.sqrt(xi * xi - 1.0)
    w1, w2 = np.abs(xi + s), np.abs(xi - s)
    return np.maximum(w1, w2)


def ellipse_right_end(d, c2, level):
    """Rightmost real point of the confocal ellipse of the given level: z = d + c (w + 1/w) / 2 with
    |w| = level; w = level for real foci (c^2 > 0), w = -i level for imaginary foci, a circle of radius
    `level` about d for c^2 = 0."""
    if abs(c2) < 1e-300:
        return d + level
    if c2 > 0.0:
        return d + np.sqrt(c2) * (level + 1.0 / level) / 2.0
    return d + np.sqrt(-c2) * (level - 1.0 / level) / 2.0


def best_ellipse(wanted, unwanted):
    """Scan a family of real-centred ellipses; return (d, c2, rate) maximising the slowest
    wanted damping rate min_w level(w)/max_u level(u), among the ellipses (through the outermost
    unwanted value) whose rightmost real point stays left of every wanted real part: anything on the
    real axis further right would rank among the wanted and must not be damped (at high Gr the first
    Ritz values are far-off ones with large imaginary parts, and an ellipse around them can cover the
    leading eigenvalues near the origin).  Without such an ellipse in the scan, the best of all."""
    ur = np.real(unwanted)
    a_min, a_max = float(np.min(ur)), float(np.max(ur))
    span = max(a_max - a_min, 1e-12 * max(1.0, abs(a_max)))
    b_max = float(np.max(np.abs(np.imag(unwanted)))) if len(unwanted) else 0.0
    w_left = float(np.min(np.real(wanted)))
    best, best_ok = None, None
    for fd in np.linspace(0.2, 0.8, 13):
        d = a_min + fd * span
        a0 = max(a_max - d, d - a_min)
        for t in np.linspace(-1.0, 1.0, 41):
            c2 = t * max(a0 * a0, b_max * b_max)
            lu = float(np.max(_level(unwanted, d, c2)))
            lw = float(np.min(_level(wanted, d, c2)))
            rate = lw / lu if lu > 0 else np.inf
            if best is None or rate > best[2]:
                best = (d, c2, rate)
            if ellipse_right_end(d, c2, lu) <= w_left and (best_ok is None or rate > best_ok[2]):
                best_ok = (d, c2, rate)
    return best_ok if best_ok is not None else best


def chebyshev_filter(A, y0, d, c2, lam_ref, degree):
    """y = T_n((A - d)/c) y0 / T_n((lam_ref - d)/c) by the three-term recurrence (real arithmetic).

    With tau_1 = 1/(lam_ref - d) and tau_{j+1} = 1/(2 (lam_ref - d) - c^2 tau_j):
        y_1 = tau_1 (A - d) y_0,   y_{j+1} = 2 tau_{j+1} (A - d) y_j - c^2 tau_j tau_{j+1} y_{j-1}.
    """
    s = lam_ref - d
    tau = 1.0 / s
    y_prev = y0
    y = tau * (A(y0) - d * y0)
    for _ in range(1, degree):
        tau_n = 1.0 / (2.0 * s - c2 * tau)
        y_next = 2.0 * tau_n * (A(y) - d * y) - c2 * tau * tau_n * y_prev
        y_prev, y, tau = y, y_next, tau_n
        nrm = np.linalg.norm(y)
        if nrm > 1e100 or nrm < 1e-100:     # rescale both terms of the recurrence together
            y, y_prev = y / nrm, y_prev / nrm
    return y


def _real_parts(X, theta, idx):
    """Real vectors of the Ritz pairs idx: the real part for +Im (or real) values, the imaginary part
    for the -Im partner of a conjugate pair."""
    return [X[:, i].real if theta[i].imag >= 0 else X[:, i].imag for i in idx]


def chebyshev_arnoldi(A, x0, k=4, m=20, tol=1e-10, max_restarts=50, max_degree=200, min_degree=10,
                      guard=2, power_steps=30, project=None, refresh=None, seed=12345, trace=None,
                      amplification=1e2):
    """Leading k eigenpairs (largest real part) of A by Chebyshev-preconditioned Arnoldi.

    Returns (lam, X, info): lam complex (k or k+1 values when a conjugate pair
    straddles the cut), X the Ritz vectors (complex, unit norm), info with the
    residual norms ||A x - lam x|| and the restart history.

    Cycle 0 runs m Arnoldi steps on A itself; every later cycle runs m Arnoldi
    steps, from p(A) applied to its start vector, on the preconditioned
    operator B = p(A), the Chebyshev polynomial
    p(z) = T_n((z - d)/c) / T_n((lam_ref - d)/c) of the current ellipse, which
    is small on the unwanted part of the spectrum and large on the wanted part.
    The eigenvalues of A come from the Rayleigh-Ritz projection G = V^T A V on
    the Krylov basis V (m more products with A); the k with the largest real
    part are tested by their true residuals ||A x - theta x|| <= tol |theta|.
    The next ellipse holds the unwanted Ritz values of G and the far end of the
    spectrum (power iteration), with `guard` Ritz values beyond the k wanted
    ones outside it; its degree gives the slowest guard value an advantage
    `amplification` over the ellipse.  The next cycle starts from the sum of
    the normalised wanted Ritz vectors plus a random component of relative
    weight `refresh` (default tol / 100, made divergence free by `project`), so
    that a mode the start lacked is present in the Krylov space of B, while the
    noise it brings stays below the tolerance.

    Running the Arnoldi on B rather than on A matters for this stiff operator:
    with ||A|| / |lam_wanted| ~ 1e2 .. 1e4 every Arnoldi step on A multiplies
    the round-off in the stiff directions by that ratio, so that after a few
    steps the Krylov vectors hold little but amplified round-off and the Ritz
    pairs stall far above the tolerance; B maps the stiff part into the small
    interior of the ellipse instead.
    """
    rng = np.random.default_rng(seed)
    refresh = 0.01 * tol if refresh is None else refresh
    x = x0 / np.linalg.norm(x0)
    info = {"restarts": 0, "matvecs": 0, "degrees": []}
    nmv = [0]

    def Af(v):
        nmv[0] += 1
        return A(v)

    # the far end of the spectrum: the largest-magnitude eigenvalue by power iteration (its Rayleigh
    # quotient); the Krylov spaces of B stop showing it, and T_n grows fast outside the ellipse
    z = x.copy()
    lam_far = 0.0
    for _ in range(power_steps):
        y = Af(z)
        lam_far = float(np.dot(z, y))
        z = y / np.linalg.norm(y)
    info["lam_far"] = lam_far

    filt = None
    for it in range(max_restarts + 1):
        if filt is None:
            V, H, mm = arnoldi(Af, x, m)
            G = H[:mm, :mm]                      # V^T A V for a Krylov basis of A
        else:
            # start from p(A) x: the restart vector's error in the stiff directions would otherwise sit in
            # v_1 alone, where no later Krylov vector of B (which damps those directions) can cancel it
            x = chebyshev_filter(Af, x, *filt)
            V, _, mm = arnoldi(lambda v: chebyshev_filter(Af, v, *filt), x / np.linalg.norm(x), m)
            AV = np.array([Af(V[j]) for j in range(mm)])
            G = V[:mm] @ AV.T                    # G[i, j] = v_i . A v_j
        theta, S = np.linalg.eig(G)
        idx = order_eigs(theta)
        theta, S = theta[idx], S[:, idx]
        S = S / np.linalg.norm(S, axis=0)
        nw = min(k, mm)
        if nw < mm and abs(theta[nw - 1].imag) > 0 and np.isclose(theta[nw], np.conj(theta[nw - 1])):
            nw += 1
        X = V[:mm].T @ S[:, :nw]
        res = np.array([np.linalg.norm(A(X[:, i].real) + 1j * A(X[:, i].imag) - theta[i] * X[:, i])
                        for i in range(nw)])
        conv = bool(np.all(res <= tol * np.maximum(np.abs(theta[:nw]), 1e-300)))
        if conv or mm < m or it == max_restarts:
            info.update(restarts=it, matvecs=nmv[0], residual=res, converged=conv or mm < m)
            return theta[:nw], X, info
        nf = min(nw + guard, mm - 2)
        if nf < mm and abs(theta[nf - 1].imag) > 0 and np.isclose(theta[nf], np.conj(theta[nf - 1])):
            nf += 1
        nf = max(nf, nw)
        wanted = theta[:nf]
        # the ellipse contains this cycle's unwanted Ritz values and the far end of the spectrum
        left = min(float(np.min(theta[nf:].real)), lam_far) if nf < mm else lam_far
        unwanted = np.concatenate([theta[nf:], [complex(1.05 * left, 0.0)]])
        d, c2, rate = best_ellipse(wanted, unwanted)
        lam_ref = float(np.max(wanted.real))
        if rate > 1.0:
            deg = int(np.clip(np.ceil(np.log(amplification) / np.log(rate)), min_degree, max_degree))
        else:
            deg = max_degree
        info["degrees"].append(deg)
        filt = (d, c2, lam_ref, deg)
        if trace is not None:
            trace(it, theta[:nw], res, d, c2, rate, deg)
        z = np.zeros(x.size)
        for y in _real_parts(X, theta, range(nw)):
            z += y / max(np.linalg.norm(y), 1e-300)
        if refresh > 0.0:
            r = rng.standard_normal(x.size)
            r = project(r) if project is not None else r
            z += refresh * np.linalg.norm(z) * r / np.linalg.norm(r)
        x = z / np.linalg.norm(z)
    raise AssertionError("unreachable")


def default_shift(grid: Grid) -> float:
    """sigma = -1/2 max(1, 1/Pr) sum_d 4 / min(width_d)^2, inside the diffusive part of the spectrum."""
    return -0.5 * max(1.0, 1.0 / grid.Pr) * sum(4.0 / float(a.dx.min()) ** 2 for a in grid.axes)


def shifted_operator(grid: Grid, Gr: float, q, sigma: float, projector: Projector | None = None):
    """x -> P (J(q) x - sigma x) + sigma x on unknown vectors (equal to P J x when D x = 0)."""
    P = projector or Projector(grid)

    def A(x):
        f = unpack(grid, x)
        J = jvp_full(grid, Gr, q, f)
        return pack(P.full([J[c] - sigma * f[c] for c in range(4)])) + sigma * x
    return A


def projected_jacobian(grid: Grid, Gr: float, q, projector: Projector | None = None):
    """The operator x -> pack(P J(q) unpack(x)) on unknown vectors (no shift)."""
    P = projector or Projector(grid)

    def A(x):
        return pack(P.full(jvp_full(grid, Gr, q, unpack(grid, x))))
    return A


def leading_eigenvalues(grid: Grid, Gr: float, q, k=4, m=20, seed_vector=None, tol=1e-10, **kw):
    """Leading k eigenvalues of P J(q) on the divergence-free subspace (start vector projected)."""
    P = Projector(grid)
    A = shifted_operator(grid, Gr, q, default_shift(grid), P)
    proj = lambda x: pack(P.full(unpack(grid, x)))
    x0 = proj(seed_vector)
    return chebyshev_arnoldi(A, x0, k=k, m=m, tol=tol, project=proj, **kw)
