// Test-only C wrappers of the library's host-only code (paper_2210_08816_gb300/csrc/host_linalg.cpp,
// host_cheb.cpp, host_grid.cpp and host_tc.cpp), compiled together with those sources by the `host_shim` fixture of tests/conftest.py into
// a temporary shared object, so that the routines the eigen-solvers and the pressure solve rely on can be
// checked on the CPU.  Matrices are row-major double arrays; every wrapper copies in and out of the
// routines' std::vector arguments.
#include <cstring>
#include <string>
#include <vector>

#include "fv_internal.h"

// The library's error-message sink lives in its driver unit, which this object does not include.
namespace fv {
void set_error(const std::string&) {}
}  // namespace fv

extern "C" {

// d (n, in: diagonal, out: eigenvalues), e (n - 1), Q (n * n, column j = eigenvector j)
int shim_tridiag_eig(int n, double* d, const double* e, double* Q) {
  std::vector<double> dv(d, d + n), ev(n > 1 ? n - 1 : 1, 0.0), Qv;
  if (n > 1) std::memcpy(ev.data(), e, sizeof(double) * (n - 1));
  const bool ok = fv::tridiag_eig(n, dv, ev, Qv);
  std::memcpy(d, dv.data(), sizeof(double) * n);
  std::memcpy(Q, Qv.data(), sizeof(double) * n * n);
  return ok ? 1 : 0;
}

int shim_hessenberg_eigvals(int m, const double* H, double* re, double* im) {
  std::vector<double> r, i;
  const bool ok = fv::hessenberg_eigvals(m, H, m, r, i);
  if (ok) {
    std::memcpy(re, r.data(), sizeof(double) * m);
    std::memcpy(im, i.data(), sizeof(double) * m);
  }
  return ok ? 1 : 0;
}

// y: 2 m doubles, (re, im) interleaved
int shim_hessenberg_eigvec(int m, const double* H, double lre, double lim, double* y) {
  std::vector<double> yv;
  const bool ok = fv::hessenberg_eigvec(m, H, m, lre, lim, yv);
  if (ok) std::memcpy(y, yv.data(), sizeof(double) * 2 * m);
  return ok ? 1 : 0;
}

// A (m * m, in: general, out: Hessenberg H), Q (m * m) with A_in = Q H Q^T
void shim_hessenberg_reduce(int m, double* A, double* Q) {
  std::vector<double> Av(A, A + (size_t)m * m), Qv;
  fv::hessenberg_reduce(m, Av, Qv);
  std::memcpy(A, Av.data(), sizeof(double) * m * m);
  std::memcpy(Q, Qv.data(), sizeof(double) * m * m);
}

// H: (j + 1) x j with leading dimension ld; y: j
void shim_hessenberg_lstsq(int j, const double* H, int ld, double beta, double* y, double* resid) {
  std::vector<double> yv;
  fv::hessenberg_lstsq(j, H, ld, beta, yv, resid);
  std::memcpy(y, yv.data(), sizeof(double) * j);
}

int shim_dense_solve(int n, const double* A, double* b) {
  std::vector<double> Av(A, A + (size_t)n * n), bv(b, b + n);
  const bool ok = fv::dense_solve(n, Av, bv);
  if (ok) std::memcpy(b, bv.data(), sizeof(double) * n);
  return ok ? 1 : 0;
}

double shim_ellipse_level(double zr, double zi, double d, double c2) { return fv::ellipse_level(zr, zi, d, c2); }

double shim_ellipse_right_end(double d, double c2, double level) { return fv::ellipse_right_end(d, c2, level); }

void shim_best_ellipse(int nw, const double* wre, const double* wim, int nu, const double* ure, const double* uim,
                       double* d, double* c2, double* rate) {
  std::vector<fv::Ritz> w(nw), u(nu);
  for (int i = 0; i < nw; ++i) w[i] = {wre[i], wim[i]};
  for (int i = 0; i < nu; ++i) u[i] = {ure[i], uim[i]};
  fv::best_ellipse(w, u, *d, *c2, *rate);
}

void shim_tanh_faces(int n, double s, double* f) {
  const std::vector<double> v = fv::tanh_faces(n, s);
  std::memcpy(f, v.data(), sizeof(double) * (n + 1));
}

int shim_mirror_symmetric(int n, const double* xf) {
  return fv::mirror_symmetric(std::vector<double>(xf, xf + n + 1)) ? 1 : 0;
}

// xf: n + 1 faces; outputs: idx, idc, wl, wr (n + 1 each), lam, cd_lam, fd_lam (n), and the n x n
// matrices Einv, E, cd_Einv, cd_E, fd_Einv, fd_E
int shim_build_axis(int n, const double* xf, double* idx, double* idc, double* wl, double* wr, double* lam,
                    double* Einv, double* E, double* cd_lam, double* cd_Einv, double* cd_E, double* fd_lam,
                    double* fd_Einv, double* fd_E) {
  fv::AxisHost a;
  const int st = fv::build_axis(std::vector<double>(xf, xf + n + 1), a);
  if (st != FV_OK) return st;
  auto put = [](double* dst, const std::vector<double>& v) { std::memcpy(dst, v.data(), sizeof(double) * v.size()); };
  put(idx, a.idx);
  put(idc, a.idc);
  put(wl, a.wl);
  put(wr, a.wr);
  put(lam, a.lam);
  put(Einv, a.Einv);
  put(E, a.E);
  put(cd_lam, a.cd_lam);
  put(cd_Einv, a.cd_Einv);
  put(cd_E, a.cd_E);
  put(fd_lam, a.fd_lam);
  put(fd_Einv, a.fd_Einv);
  put(fd_E, a.fd_E);
  return FV_OK;
}

// Tensor-core operands of an nx x ny x nz grid with tanh stretching s (the library's faces and metrics).
// buf == NULL: returns the buffer length in floats.  Otherwise fills buf (cap floats), moff (24), loff (3)
// and soff (6) and returns the length; a negative value is the library's status.
long long shim_tc_operands(int nx, int ny, int nz, double s, float* buf, long long cap, long long* moff,
                           long long* loff, long long* soff) {
  const int ns[3] = {nx, ny, nz};
  std::vector<double> idx[3], idc[3];
  for (int d = 0; d < 3; ++d) {
    fv::AxisHost a;
    const int st = fv::build_axis(fv::tanh_faces(ns[d], s), a);
    if (st != FV_OK) return st;
    idx[d] = a.idx;
    idc[d] = a.idc;
  }
  fv::TcOperands op;
  const int st = fv::tc_host_operands(ns, idx, idc, op);
  if (st != FV_OK) return st;
  const long long len = (long long)op.buf.size();
  if (!buf) return len;
  if (cap < len) return FV_EINVAL;
  std::memcpy(buf, op.buf.data(), sizeof(float) * op.buf.size());
  for (int d = 0; d < 3; ++d) {
    for (int j = 0; j < 8; ++j) moff[d * 8 + j] = (long long)op.moff[d][j];
    loff[d] = (long long)op.loff[d];
    for (int dir = 0; dir < 2; ++dir) soff[d * 2 + dir] = (long long)op.soff[d][dir];
  }
  return len;
}

}  // extern "C"
