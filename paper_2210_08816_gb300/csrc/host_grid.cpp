// Host construction of one grid axis (FP64): the tanh-stretched, mirrored faces (Section 4.1 says only
// "stretched near the borders"; the library's reading is x_f = (1 + tanh(s (2 i / n - 1)) / tanh s) / 2
// with the lower half mirrored), the finite-volume metrics of the staggered grid, and the 1D
// eigen-decompositions behind the direct pressure solve (Neumann, cell-centred) and the Newton
// preconditioner's diffusion solves (Dirichlet, cell- and face-centred).
#include <algorithm>
#include <cmath>
#include <limits>
#include <numeric>
#include <string>
#include <vector>

#include "fv_internal.h"

namespace fv {
namespace {

int invalid(const std::string& msg) {
  set_error(msg);
  return FV_EINVAL;
}

}  // namespace

bool mirror_symmetric(const std::vector<double>& xf) {
  const int n = (int)xf.size() - 1;
  const double tol = 4.0 * std::numeric_limits<double>::epsilon();
  for (int i = 0; i <= n; ++i)
    if (std::fabs(xf[n - i] - (1.0 - xf[i])) > tol) return false;
  return true;
}

std::vector<double> tanh_faces(int n, double s) {
  std::vector<double> f(n + 1);
  for (int i = 0; i <= n; ++i)
    f[i] = (s == 0.0) ? (double)i / n : 0.5 * (1.0 + std::tanh(s * (2.0 * i / n - 1.0)) / std::tanh(s));
  for (int k = 0; k <= n / 2; ++k) f[n - k] = 1.0 - f[k];
  if (n % 2 == 0) f[n / 2] = 0.5;
  f[0] = 0.0;
  f[n] = 1.0;
  return f;
}


// Generalised eigen-decomposition of L = W^-1 K (K symmetric tridiagonal: diagonal kd, off-diagonal ko;
// W > 0 diagonal) through B = W^-1/2 K W^-1/2:  L = E diag(lam) Einv, E = W^-1/2 Q, Einv = Q^T W^1/2.
// The m x m result is written at offset `o` of n x n matrices (rows/columns o .. o+m-1).
static int tridiag_operator(int m, const std::vector<double>& kd, const std::vector<double>& ko,
                            const std::vector<double>& W, int n, int o, std::vector<double>& lam,
                            std::vector<double>& Einv, std::vector<double>& E) {
  if (m <= 0) return FV_OK;
  std::vector<double> d(m), e(std::max(m - 1, 1), 0.0), Q;
  for (int i = 0; i < m; ++i) d[i] = kd[i] / W[i];
  for (int i = 0; i + 1 < m; ++i) e[i] = ko[i] / std::sqrt(W[i] * W[i + 1]);
  if (!tridiag_eig(m, d, e, Q)) return invalid("tridiagonal eigensolver did not converge");
  for (int k = 0; k < m; ++k) {
    lam[o + k] = d[k];
    for (int i = 0; i < m; ++i) {
      const double qv = Q[(size_t)i * m + k];
      E[(size_t)(o + i) * n + (o + k)] = qv / std::sqrt(W[i]);
      Einv[(size_t)(o + k) * n + (o + i)] = qv * std::sqrt(W[i]);
    }
  }
  return FV_OK;
}

// The two Dirichlet diffusion operators of one axis (same flux form as the stencils' Laplacian).
static int build_dirichlet_ops(AxisHost& a) {
  const int n = a.n;
  // cell-centred: (L u)_i = [ (u_{i+1} - u_i) idc[i+1] - (u_i - u_{i-1}) idc[i] ] idx[i], u_{-1} = u_n = 0,
  // idc[0] = 2 / dx_0 and idc[n] = 2 / dx_{n-1} (walls half a cell away)
  std::vector<double> kd(n), ko(std::max(n - 1, 1), 0.0), W(n);
  for (int i = 0; i < n; ++i) {
    kd[i] = -(a.idc[i] + a.idc[i + 1]);
    if (i + 1 < n) ko[i] = a.idc[i + 1];
    W[i] = 1.0 / a.idx[i];
  }
  a.cd_lam.assign(n, 0.0);
  a.cd_Einv.assign((size_t)n * n, 0.0);
  a.cd_E.assign((size_t)n * n, 0.0);
  FV_TRY(tridiag_operator(n, kd, ko, W, n, 0, a.cd_lam, a.cd_Einv, a.cd_E));
  // face-centred on faces p = 1 .. n-1: (L u)_p = [ (u_{p+1} - u_p) idx[p] - (u_p - u_{p-1}) idx[p-1] ] idc[p],
  // u_0 = u_n = 0; control-volume width 1 / idc[p]
  const int mf = n - 1;
  std::vector<double> fd(std::max(mf, 1)), fo(std::max(mf, 1), 0.0), FW(std::max(mf, 1));
  for (int k = 0; k < mf; ++k) {
    const int p = k + 1;
    fd[k] = -(a.idx[p] + a.idx[p - 1]);
    if (k + 1 < mf) fo[k] = a.idx[p];
    FW[k] = 1.0 / a.idc[p];
  }
  a.fd_lam.assign(n, 0.0);
  a.fd_Einv.assign((size_t)n * n, 0.0);
  a.fd_E.assign((size_t)n * n, 0.0);
  a.fd_lam[0] = -1.0;  // dummy mode of the wall slot (its input is zero)
  a.fd_E[0] = 1.0;
  a.fd_Einv[0] = 1.0;
  return tridiag_operator(mf, fd, fo, FW, n, 1, a.fd_lam, a.fd_Einv, a.fd_E);
}

int build_axis(const std::vector<double>& xf, AxisHost& a) {
  const int n = (int)xf.size() - 1;
  a.n = n;
  std::vector<double> dx(n), xc(n);
  for (int i = 0; i < n; ++i) {
    dx[i] = xf[i + 1] - xf[i];
    xc[i] = 0.5 * (xf[i] + xf[i + 1]);
    if (!(dx[i] > 0.0)) return invalid("faces must be strictly increasing");
  }
  a.idx.assign(n + 1, 0.0);
  a.idc.assign(n + 1, 0.0);
  a.wl.assign(n + 1, 0.0);
  a.wr.assign(n + 1, 0.0);
  for (int i = 0; i < n; ++i) a.idx[i] = 1.0 / dx[i];
  a.idc[0] = 2.0 / dx[0];
  a.idc[n] = 2.0 / dx[n - 1];
  for (int f = 1; f < n; ++f) {
    a.idc[f] = 1.0 / (xc[f] - xc[f - 1]);
    a.wl[f] = dx[f] / (dx[f - 1] + dx[f]);
    a.wr[f] = dx[f - 1] / (dx[f - 1] + dx[f]);
  }
  // 1D Neumann operator A = W^-1 S; symmetric form B = W^-1/2 S W^-1/2 (tridiagonal)
  std::vector<double> d(n), e(std::max(n - 1, 1), 0.0);
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    if (i >= 1) s -= a.idc[i];
    if (i + 1 <= n - 1) s -= a.idc[i + 1];
    d[i] = s / dx[i];
    if (i + 1 <= n - 1) e[i] = a.idc[i + 1] / std::sqrt(dx[i] * dx[i + 1]);
  }
  std::vector<double> Q;
  if (!tridiag_eig(n, d, e, Q)) return invalid("tridiagonal eigensolver did not converge");
  std::vector<int> ord(n);
  std::iota(ord.begin(), ord.end(), 0);
  std::sort(ord.begin(), ord.end(), [&](int p, int q) { return d[p] > d[q]; });
  a.lam.assign(n, 0.0);
  a.Einv.assign((size_t)n * n, 0.0);
  a.E.assign((size_t)n * n, 0.0);
  for (int m = 0; m < n; ++m) {
    const int src = ord[m];
    a.lam[m] = (m == 0) ? 0.0 : d[src];  // the constant vector is an exact null vector
    for (int i = 0; i < n; ++i) {
      const double qv = Q[(size_t)i * n + src];
      a.E[(size_t)i * n + m] = qv / std::sqrt(dx[i]);
      a.Einv[(size_t)m * n + i] = qv * std::sqrt(dx[i]);
    }
  }
  return build_dirichlet_ops(a);
}

}  // namespace fv
