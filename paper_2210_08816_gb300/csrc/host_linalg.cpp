// Small dense linear algebra on the host (FP64): the 1D generalised eigenproblems of the pressure
// solve, the Hessenberg eigenproblem of the Arnoldi iteration (m <= 200), Ritz vectors, the 2 x 2
// minimal-residual systems of BiCGstab(2) and the GMRES least-squares problem.
#include <algorithm>
#include <cmath>
#include <complex>
#include <limits>
#include <vector>

#include "fv_internal.h"

namespace fv {

using cd = std::complex<double>;

// Symmetric tridiagonal QR iteration with implicit Wilkinson shifts (Golub & Van Loan, "Matrix
// Computations", Sec. 8.3): chase the bulge of each shifted step with Givens rotations, deflate when an
// off-diagonal falls below eps (|d_k| + |d_k+1|), and accumulate the rotations into Q.
bool tridiag_eig(int n, std::vector<double>& d, std::vector<double>& e, std::vector<double>& Q) {
  Q.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
  if (n == 1) return true;
  const double eps = std::numeric_limits<double>::epsilon();
  int m = n - 1;
  int guard = 0;
  while (m > 0) {
    if (std::fabs(e[m - 1]) <= eps * (std::fabs(d[m - 1]) + std::fabs(d[m]))) {
      e[m - 1] = 0.0;
      --m;
      continue;
    }
    int l = m - 1;
    while (l > 0 && std::fabs(e[l - 1]) > eps * (std::fabs(d[l - 1]) + std::fabs(d[l]))) --l;
    if (++guard > 60 * n) return false;
    // Wilkinson shift: eigenvalue of the trailing 2x2 closer to d[m]
    const double t = 0.5 * (d[m - 1] - d[m]);
    const double b = e[m - 1];
    const double mu = d[m] - b * b / (t + std::copysign(std::hypot(t, b), t == 0.0 ? 1.0 : t));
    double x = d[l] - mu, z = e[l];
    for (int k = l; k < m; ++k) {
      const double r = std::hypot(x, z);
      const double c = (r == 0.0) ? 1.0 : x / r, s = (r == 0.0) ? 0.0 : z / r;
      if (k > l) e[k - 1] = r;
      const double dk = d[k], dk1 = d[k + 1], ek = e[k];
      d[k] = c * c * dk + 2.0 * c * s * ek + s * s * dk1;
      d[k + 1] = s * s * dk - 2.0 * c * s * ek + c * c * dk1;
      e[k] = c * s * (dk1 - dk) + (c * c - s * s) * ek;
      if (k < m - 1) {
        x = e[k];
        z = s * e[k + 1];
        e[k + 1] = c * e[k + 1];
      }
      for (int i = 0; i < n; ++i) {
        double* row = &Q[(size_t)i * n];
        const double qk = row[k], qk1 = row[k + 1];
        row[k] = c * qk + s * qk1;
        row[k + 1] = -s * qk + c * qk1;
      }
    }
  }
  return true;
}

// Eigenvalues of a real upper Hessenberg matrix by the complex single-shift QR algorithm: Wilkinson
// shift from the trailing 2x2 of the active block, Givens QR of H - mu I, RQ + mu I, deflation on small
// sub-diagonals, an exceptional shift after 10 steps without deflation.
bool hessenberg_eigvals(int m, const double* H, int ld, std::vector<double>& re, std::vector<double>& im) {
  std::vector<cd> A((size_t)m * m);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) A[(size_t)i * m + j] = (j >= i - 1) ? cd(H[(size_t)i * ld + j], 0.0) : cd(0.0);
  auto a = [&](int i, int j) -> cd& { return A[(size_t)i * m + j]; };
  re.assign(m, 0.0);
  im.assign(m, 0.0);
  const double eps = std::numeric_limits<double>::epsilon();
  std::vector<cd> cs(m), sn(m);
  int hi = m - 1, since = 0, total = 0;
  while (hi >= 0) {
    int l = hi;
    while (l > 0 && std::abs(a(l, l - 1)) > eps * (std::abs(a(l, l)) + std::abs(a(l - 1, l - 1)))) --l;
    if (l > 0) a(l, l - 1) = 0.0;
    if (l == hi) {
      re[hi] = a(hi, hi).real();
      im[hi] = a(hi, hi).imag();
      --hi;
      since = 0;
      continue;
    }
    if (++total > 100 * m) return false;
    cd mu;
    if (++since % 11 == 10) {
      mu = a(hi, hi) + std::abs(a(hi, hi - 1).real()) * 0.75;
    } else {
      const cd p = a(hi - 1, hi - 1), q = a(hi - 1, hi), r = a(hi, hi - 1), s = a(hi, hi);
      const cd half = 0.5 * (p - s);
      const cd disc = std::sqrt(half * half + q * r);
      const cd m1 = 0.5 * (p + s) + disc, m2 = 0.5 * (p + s) - disc;
      mu = (std::abs(m1 - s) < std::abs(m2 - s)) ? m1 : m2;
    }
    for (int k = l; k <= hi; ++k) a(k, k) -= mu;
    for (int k = l; k < hi; ++k) {
      const cd x = a(k, k), y = a(k + 1, k);
      const double r = std::sqrt(std::norm(x) + std::norm(y));
      const cd c = (r == 0.0) ? cd(1.0) : x / r, s = (r == 0.0) ? cd(0.0) : y / r;
      cs[k] = c;
      sn[k] = s;
      for (int j = k; j <= hi; ++j) {
        const cd t1 = a(k, j), t2 = a(k + 1, j);
        a(k, j) = std::conj(c) * t1 + std::conj(s) * t2;
        a(k + 1, j) = -s * t1 + c * t2;
      }
    }
    for (int k = l; k < hi; ++k) {
      const cd c = cs[k], s = sn[k];
      const int iend = std::min(k + 2, hi);
      for (int i = l; i <= iend; ++i) {
        const cd t1 = a(i, k), t2 = a(i, k + 1);
        a(i, k) = t1 * c + t2 * s;
        a(i, k + 1) = -t1 * std::conj(s) + t2 * std::conj(c);
      }
    }
    for (int k = l; k <= hi; ++k) a(k, k) += mu;
  }
  for (int i = 0; i < m; ++i)
    if (std::fabs(im[i]) <= 1e-13 * std::max(1.0, std::fabs(re[i]))) im[i] = 0.0;
  return true;
}

// Eigenvector of H for the eigenvalue lam by three steps of inverse iteration with (H - lam I) factored
// by Gaussian elimination with partial pivoting (complex); lam is nudged by a few eps ||H|| off exact
// singularity (the nudge is the residual ||H y - lam y|| the vector is left with, so it stays at round-off).
bool hessenberg_eigvec(int m, const double* H, int ld, double lre, double lim, std::vector<double>& y) {
  double hn = 0.0;
  for (int i = 0; i < m; ++i)
    for (int j = std::max(0, i - 1); j < m; ++j) hn = std::max(hn, std::fabs(H[(size_t)i * ld + j]));
  const cd lam(lre + 4.0 * std::numeric_limits<double>::epsilon() * std::max(hn, 1.0), lim);
  std::vector<cd> A((size_t)m * m);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) A[(size_t)i * m + j] = (j >= i - 1) ? cd(H[(size_t)i * ld + j]) : cd(0.0);
  for (int i = 0; i < m; ++i) A[(size_t)i * m + i] -= lam;
  std::vector<int> piv(m);
  for (int k = 0; k < m; ++k) {
    int p = k;
    for (int i = k + 1; i < m; ++i)
      if (std::abs(A[(size_t)i * m + k]) > std::abs(A[(size_t)p * m + k])) p = i;
    piv[k] = p;
    if (p != k)
      for (int j = 0; j < m; ++j) std::swap(A[(size_t)k * m + j], A[(size_t)p * m + j]);
    cd pk = A[(size_t)k * m + k];
    if (std::abs(pk) == 0.0) pk = A[(size_t)k * m + k] = cd(1e-300);
    for (int i = k + 1; i < m; ++i) {
      const cd f = A[(size_t)i * m + k] / pk;
      A[(size_t)i * m + k] = f;
      for (int j = k + 1; j < m; ++j) A[(size_t)i * m + j] -= f * A[(size_t)k * m + j];
    }
  }
  std::vector<cd> x(m, cd(1.0));
  for (int it = 0; it < 3; ++it) {
    for (int k = 0; k < m; ++k) {
      if (piv[k] != k) std::swap(x[k], x[piv[k]]);
      for (int i = k + 1; i < m; ++i) x[i] -= A[(size_t)i * m + k] * x[k];
    }
    for (int k = m - 1; k >= 0; --k) {
      cd s = x[k];
      for (int j = k + 1; j < m; ++j) s -= A[(size_t)k * m + j] * x[j];
      x[k] = s / A[(size_t)k * m + k];
    }
    double nrm = 0.0;
    for (auto& v : x) nrm += std::norm(v);
    nrm = std::sqrt(nrm);
    if (!(nrm > 0.0) || !std::isfinite(nrm)) return false;
    for (auto& v : x) v /= nrm;
  }
  // fix the phase: largest component real positive
  int imax = 0;
  for (int i = 1; i < m; ++i)
    if (std::abs(x[i]) > std::abs(x[imax])) imax = i;
  const cd ph = std::conj(x[imax]) / std::abs(x[imax]);
  y.resize(2 * (size_t)m);
  for (int i = 0; i < m; ++i) {
    const cd v = x[i] * ph;
    y[2 * i] = v.real();
    y[2 * i + 1] = (lim == 0.0) ? 0.0 : v.imag();
  }
  return true;
}

// Householder reduction of a general real matrix (m x m, row-major) to upper Hessenberg form:
// on return A holds H (zeros below the subdiagonal) and Q (m x m, row-major, orthogonal) with
// A_in = Q H Q^T, so that an eigenvector s of H gives the eigenvector Q s of A_in.
void hessenberg_reduce(int m, std::vector<double>& A, std::vector<double>& Q) {
  Q.assign((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) Q[(size_t)i * m + i] = 1.0;
  std::vector<double> v(m);
  for (int k = 0; k + 2 < m; ++k) {
    double alpha = 0.0;
    for (int i = k + 1; i < m; ++i) alpha += A[(size_t)i * m + k] * A[(size_t)i * m + k];
    alpha = std::sqrt(alpha);
    if (alpha == 0.0) continue;
    const double x0 = A[(size_t)(k + 1) * m + k];
    if (x0 > 0) alpha = -alpha;  // v = x - alpha e1 with alpha of the opposite sign: no cancellation
    double vn = 0.0;
    for (int i = 0; i < m; ++i) v[i] = 0.0;
    for (int i = k + 1; i < m; ++i) v[i] = A[(size_t)i * m + k];
    v[k + 1] -= alpha;
    for (int i = k + 1; i < m; ++i) vn += v[i] * v[i];
    if (vn == 0.0) continue;
    const double beta = 2.0 / vn;
    // A <- (I - beta v v^T) A
    for (int j = 0; j < m; ++j) {
      double s = 0.0;
      for (int i = k + 1; i < m; ++i) s += v[i] * A[(size_t)i * m + j];
      s *= beta;
      for (int i = k + 1; i < m; ++i) A[(size_t)i * m + j] -= s * v[i];
    }
    // A <- A (I - beta v v^T),  Q <- Q (I - beta v v^T)
    for (int i = 0; i < m; ++i) {
      double s = 0.0, t = 0.0;
      for (int j = k + 1; j < m; ++j) {
        s += A[(size_t)i * m + j] * v[j];
        t += Q[(size_t)i * m + j] * v[j];
      }
      s *= beta;
      t *= beta;
      for (int j = k + 1; j < m; ++j) {
        A[(size_t)i * m + j] -= s * v[j];
        Q[(size_t)i * m + j] -= t * v[j];
      }
    }
    for (int i = k + 2; i < m; ++i) A[(size_t)i * m + k] = 0.0;
  }
}

bool dense_solve(int n, std::vector<double> A, std::vector<double>& b) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[(size_t)i * n + k]) > std::fabs(A[(size_t)p * n + k])) p = i;
    if (A[(size_t)p * n + k] == 0.0) return false;
    if (p != k) {
      for (int j = 0; j < n; ++j) std::swap(A[(size_t)k * n + j], A[(size_t)p * n + j]);
      std::swap(b[k], b[p]);
    }
    for (int i = k + 1; i < n; ++i) {
      const double f = A[(size_t)i * n + k] / A[(size_t)k * n + k];
      for (int j = k; j < n; ++j) A[(size_t)i * n + j] -= f * A[(size_t)k * n + j];
      b[i] -= f * b[k];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    double s = b[k];
    for (int j = k + 1; j < n; ++j) s -= A[(size_t)k * n + j] * b[j];
    b[k] = s / A[(size_t)k * n + k];
  }
  return true;
}

// min || H y - beta e1 || for the (j+1) x j upper Hessenberg H by Givens rotations.
void hessenberg_lstsq(int j, const double* H, int ld, double beta, std::vector<double>& y, double* resid) {
  std::vector<double> R((size_t)(j + 1) * j);
  for (int r = 0; r <= j; ++r)
    for (int c = 0; c < j; ++c) R[(size_t)r * j + c] = H[(size_t)r * ld + c];
  std::vector<double> g(j + 1, 0.0);
  g[0] = beta;
  for (int k = 0; k < j; ++k) {
    const double x = R[(size_t)k * j + k], z = R[(size_t)(k + 1) * j + k];
    const double r = std::hypot(x, z);
    const double c = (r == 0.0) ? 1.0 : x / r, s = (r == 0.0) ? 0.0 : z / r;
    for (int col = k; col < j; ++col) {
      const double t1 = R[(size_t)k * j + col], t2 = R[(size_t)(k + 1) * j + col];
      R[(size_t)k * j + col] = c * t1 + s * t2;
      R[(size_t)(k + 1) * j + col] = -s * t1 + c * t2;
    }
    const double g1 = g[k], g2 = g[k + 1];
    g[k] = c * g1 + s * g2;
    g[k + 1] = -s * g1 + c * g2;
  }
  y.assign(j, 0.0);
  for (int k = j - 1; k >= 0; --k) {
    double s = g[k];
    for (int c = k + 1; c < j; ++c) s -= R[(size_t)k * j + c] * y[c];
    const double dkk = R[(size_t)k * j + k];
    y[k] = (dkk == 0.0) ? 0.0 : s / dkk;
  }
  if (resid) *resid = std::fabs(g[j]);
}

}  // namespace fv
