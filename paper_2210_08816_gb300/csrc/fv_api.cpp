// The C-ABI (include/cube_fv.h): grid set-up, the J.v + projection hot path, and the host drivers of
// Newton's method (BiCGstab(2) + GMRES) and the Chebyshev-preconditioned Arnoldi iteration (Section 1,
// methods paragraph).  Every vector operation runs in the library's CUDA kernels; the host holds only
// scalars and the small dense matrices (Hessenberg, 2 x 2 minimal-residual systems).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <type_traits>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "fv_internal.h"

namespace fv {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }
int cuda_status(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return FV_ECUDA;
}
static int cu_ok(cudaError_t e, const char* what) { return e == cudaSuccess ? FV_OK : cuda_status(e, what); }
static int invalid(const std::string& msg) {
  set_error(msg);
  return FV_EINVAL;
}

// ------------------------------------------------------------------ measurement
static cudaEvent_t pool_event(const fv_grid_s* g) {
  Profiler& p = g->prof;
  if (p.used == p.pool.size()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    p.pool.push_back(e);
  }
  return p.pool[p.used++];
}

ProfScope::ProfScope(const fv_grid_s* grid, int kind) : g(grid) {
  if (!g->prof.enabled) return;
  cudaEvent_t a = pool_event(g), b = pool_event(g);
  if (!a || !b) return;
  cudaEventRecord(a, g->stream);
  stop = b;
  g->prof.records.push_back({kind, a, b});
}

ProfScope::~ProfScope() {
  if (stop) cudaEventRecord(stop, g->stream);
}

// ------------------------------------------------------------------ device memory helper
template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  int alloc(size_t count) {
    if (p) cudaFree(p);
    p = nullptr;
    n = count;
    if (count == 0) return FV_OK;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
      return FV_ENOMEM;
    }
    return FV_OK;
  }
};

template <typename R>
static int upload_axes(fv_grid_s* g, const AxisHost* ax, int which, Geo<R>& geo, FdmDev<R>& fdm, FdmDev<R>& cd,
                       FdmDev<R>& fd) {
  size_t total = 0;
  for (int d = 0; d < 3; ++d) total += 4 * (size_t)(ax[d].n + 1) + 3 * ((size_t)ax[d].n + 2 * (size_t)ax[d].n * ax[d].n);
  std::vector<R> h(total);
  std::vector<size_t> off;
  size_t o = 0;
  auto put = [&](const std::vector<double>& v) {
    off.push_back(o);
    for (double x : v) h[o++] = (R)x;
  };
  for (int d = 0; d < 3; ++d) {
    put(ax[d].idx);
    put(ax[d].idc);
    put(ax[d].wl);
    put(ax[d].wr);
    put(ax[d].lam);
    put(ax[d].Einv);
    put(ax[d].E);
    put(ax[d].cd_lam);
    put(ax[d].cd_Einv);
    put(ax[d].cd_E);
    put(ax[d].fd_lam);
    put(ax[d].fd_Einv);
    put(ax[d].fd_E);
  }
  void* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, total * sizeof(R));
  if (e != cudaSuccess) {
    set_error(std::string("cudaMalloc metrics: ") + cudaGetErrorString(e));
    return FV_ENOMEM;
  }
  g->metric_buf[which] = buf;
  FV_CUDA(cudaMemcpy(buf, h.data(), total * sizeof(R), cudaMemcpyHostToDevice));
  const R* base = (const R*)buf;
  for (int d = 0; d < 3; ++d) {
    geo.n[d] = ax[d].n;
    const size_t* od = off.data() + 13 * d;
    geo.idx[d] = base + od[0];
    geo.idc[d] = base + od[1];
    geo.wl[d] = base + od[2];
    geo.wr[d] = base + od[3];
    fdm.lam[d] = base + od[4];
    fdm.Einv[d] = base + od[5];
    fdm.E[d] = base + od[6];
    cd.lam[d] = base + od[7];
    cd.Einv[d] = base + od[8];
    cd.E[d] = base + od[9];
    fd.lam[d] = base + od[10];
    fd.Einv[d] = base + od[11];
    fd.E[d] = base + od[12];
  }
  return FV_OK;
}

template <typename R>
static constexpr int prec_index() {
  return sizeof(R) == 8 ? 0 : 1;
}

template <typename R>
static int ensure_ws(fv_grid_s* g) {
  const int p = prec_index<R>();
  if (g->ws.Y[p]) return FV_OK;
  const size_t N = g->N;
  void *Y = nullptr, *t0 = nullptr, *t1 = nullptr;
  if (cudaMalloc(&Y, 4 * N * sizeof(R)) != cudaSuccess || cudaMalloc(&t0, N * sizeof(R)) != cudaSuccess ||
      cudaMalloc(&t1, N * sizeof(R)) != cudaSuccess) {
    if (Y) cudaFree(Y);
    if (t0) cudaFree(t0);
    cudaGetLastError();
    set_error("workspace allocation failed");
    return FV_ENOMEM;
  }
  g->ws.Y[p] = Y;
  g->ws.t0[p] = t0;
  g->ws.t1[p] = t1;
  return FV_OK;
}

// ------------------------------------------------------------------ the hot path
template <typename R>
int jvp_project(fv_grid_s* g, double Gr, double sigma, const R* q, const R* v, R* out) {
  FV_TRY(ensure_ws<R>(g));
  const int p = prec_index<R>();
  R* Y = (R*)g->ws.Y[p];
  R* phi = (R*)g->ws.t1[p];
  R* tmp = (R*)g->ws.t0[p];
  FV_TRY(launch_jvp<R>(g, Gr, sigma, q, v, Y));
  FV_TRY(launch_divergence<R>(g, Y, phi));
  FV_TRY(launch_poisson<R>(g, phi, phi, tmp));
  FV_TRY(launch_correct<R>(g, Y, phi, 1.0, sigma != 0.0 ? v : nullptr, sigma, nullptr, 0.0, out));
  return FV_OK;
}

// out = alpha (P(J y - sigma y)) + beta y + gamma yprev   (one step of a three-term recurrence in A)
template <typename R>
int chebyshev_step(fv_grid_s* g, double Gr, double sigma, const R* q, const R* y, const R* yprev, double alpha,
                   double beta, double gamma, R* out, int norm_slot) {
  FV_TRY(ensure_ws<R>(g));
  const int p = prec_index<R>();
  R* Y = (R*)g->ws.Y[p];
  R* phi = (R*)g->ws.t1[p];
  R* tmp = (R*)g->ws.t0[p];
  FV_TRY(launch_jvp<R>(g, Gr, sigma, q, y, Y));
  FV_TRY(launch_divergence<R>(g, Y, phi));
  FV_TRY(launch_poisson<R>(g, phi, phi, tmp));
  FV_TRY(launch_correct<R>(g, Y, phi, alpha, y, beta, yprev, gamma, out, norm_slot));
  return FV_OK;
}

template <typename R>
static int project_inplace(fv_grid_s* g, R* v, int max_it, double tol, int* iters, double* div_rel) {
  FV_TRY(ensure_ws<R>(g));
  const int p = prec_index<R>();
  R* phi = (R*)g->ws.t1[p];
  R* tmp = (R*)g->ws.t0[p];
  const bool want = (div_rel != nullptr) || max_it > 1;
  double d0 = 0.0, dn = 0.0;
  int it = 0;
  FV_TRY(launch_divergence<R>(g, v, phi));
  if (want) {
    FV_TRY(launch_dot<R>(g, phi, phi, g->N, 0));
    FV_TRY(read_scalars(g, 0, 1, &d0));
    d0 = std::sqrt(d0);
  }
  for (it = 1; it <= std::max(1, max_it); ++it) {
    FV_TRY(launch_poisson<R>(g, phi, phi, tmp));
    FV_TRY(launch_correct<R>(g, v, phi, 1.0, nullptr, 0.0, nullptr, 0.0, v));
    if (!want) break;
    FV_TRY(launch_divergence<R>(g, v, phi));
    FV_TRY(launch_dot<R>(g, phi, phi, g->N, 0));
    FV_TRY(read_scalars(g, 0, 1, &dn));
    dn = std::sqrt(dn);
    if (!(dn > tol * d0) || it == max_it) break;
  }
  if (iters) *iters = std::min(it, std::max(1, max_it));
  if (div_rel) *div_rel = (d0 > 0.0) ? dn / d0 : 0.0;
  return FV_OK;
}

// ------------------------------------------------------------------ small vector toolkit over device vectors
template <typename R>
struct Vec {
  fv_grid_s* g;
  size_t n;
  int dot(const R* a, const R* b, double* out) {
    FV_TRY(launch_dot<R>(g, a, b, n, 0));
    FV_TRY(read_scalars(g, 0, 1, out));
    if (!std::isfinite(*out)) {
      set_error("non-finite inner product");
      return FV_ENAN;
    }
    return FV_OK;
  }
  int lin(R* out, std::initializer_list<std::pair<double, const R*>> terms) {
    double c[4];
    const R* x[4];
    int k = 0;
    for (auto& t : terms) {
      c[k] = t.first;
      x[k] = t.second;
      ++k;
    }
    return launch_lincomb<R>(g, n, k, c, x, out);
  }
  int copy(R* dst, const R* src) {
    FV_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(R), cudaMemcpyDeviceToDevice, g->stream));
    return FV_OK;
  }
  int zero(R* dst) {
    FV_CUDA(cudaMemsetAsync(dst, 0, n * sizeof(R), g->stream));
    return FV_OK;
  }
};

// ------------------------------------------------------------------ Newton preconditioner
// out = L^-1 in, field by field (the diffusion operator of J with homogeneous wall data); in and out
// may alias.
template <typename R>
static int diffusion_solve(fv_grid_s* g, const R* in, R* out, double s = 0.0) {
  FV_TRY(ensure_ws<R>(g));
  R* tmp = (R*)g->ws.t0[prec_index<R>()];
  for (int f = 0; f < 4; ++f)
    FV_TRY(launch_field_solve<R>(g, f, in + (size_t)f * g->N, out + (size_t)f * g->N, tmp, s));
  return FV_OK;
}

// Right preconditioner M^-1 = P L^-1 (the diffusion part of J inverted, then projected): it removes
// the stiff diffusion eigenvalues (up to ~12 / h_min^2) from P J M^-1, but P and L do not commute at
// no-slip walls, so P J M^-1 is not a compact perturbation of P there.
// With a pseudo-time shift s: M^-1 = P (L - s I)^-1 for the operator P J - s I.
template <typename R>
static int apply_precond(fv_grid_s* g, const R* in, R* out, double s = 0.0) {
  FV_TRY(diffusion_solve<R>(g, in, out, s));
  return project_inplace<R>(g, out, 1, 0.0, nullptr, nullptr);
}

// ------------------------------------------------------------------ BiCGstab(2) and GMRES
// y = A x = P (J - sigma) x + sigma x - s x, or A M^-1 x when `pre` (a 4N scratch vector) is set; s is the
// reciprocal pseudo-time step (0: the Newton operator itself).
template <typename R>
struct Operator {
  fv_grid_s* g;
  double Gr, sigma;
  const R* q;
  long long* matvecs;
  R* pre = nullptr;
  double s = 0.0;
  int apply(const R* x, R* y) {
    ++*matvecs;
    const R* in = x;
    if (pre) {
      FV_TRY(apply_precond<R>(g, x, pre, s));
      in = pre;
    }
    FV_TRY(jvp_project<R>(g, Gr, sigma, q, in, y));
    if (s == 0.0) return FV_OK;
    Vec<R> V{g, 4 * g->N};
    return V.lin(y, {{1.0, y}, {-s, in}});
  }
};

struct SolveInfo {
  int status = FV_ENOCONV;  // FV_OK converged
  bool breakdown = false, stalled = false;
  int matvecs = 0;
  double rel = 1.0;
};

// BiCGstab(l), l = 2 (Sleijpen & Fokkema 1993): two BiCG steps, then the minimal-residual polynomial
// update min || r0 - g1 r1 - g2 r2 || by its 2 x 2 normal equations.
template <typename R>
static int bicgstab2(Operator<R>& A, const R* b, R* x, double tol, int max_mv, R* work, SolveInfo& info) {
  Vec<R> V{A.g, 4 * A.g->N};
  const size_t n = V.n;
  R *r = work, *rt = work + n, *u = work + 2 * n, *u1 = work + 3 * n, *u2 = work + 4 * n, *r1 = work + 5 * n,
    *r2 = work + 6 * n;
  FV_TRY(V.zero(x));
  FV_TRY(V.copy(r, b));
  FV_TRY(V.copy(rt, b));
  FV_TRY(V.zero(u));
  double bn2;
  FV_TRY(V.dot(b, b, &bn2));
  const double bn = std::sqrt(bn2);
  info = SolveInfo{};
  if (bn == 0.0) {
    info.status = FV_OK;
    info.rel = 0.0;
    return FV_OK;
  }
  double rho0 = 1.0, alpha = 0.0, omega = 1.0, best = 1.0;
  int best_cycle = 0, cycle = 0;
  const long long mv0 = *A.matvecs;
  for (;;) {
    info.matvecs = (int)(*A.matvecs - mv0);
    if (info.rel <= tol) {
      info.status = FV_OK;
      return FV_OK;
    }
    if (info.matvecs + 4 > max_mv) return FV_OK;
    rho0 = -omega * rho0;
    double rho1, gamma;
    // j = 0
    FV_TRY(V.dot(r, rt, &rho1));
    if (rho0 == 0.0 || rho1 == 0.0) {
      info.breakdown = true;
      return FV_OK;
    }
    double beta = alpha * rho1 / rho0;
    rho0 = rho1;
    FV_TRY(V.lin(u, {{1.0, r}, {-beta, u}}));
    FV_TRY(A.apply(u, u1));
    FV_TRY(V.dot(u1, rt, &gamma));
    if (gamma == 0.0) {
      info.breakdown = true;
      return FV_OK;
    }
    alpha = rho0 / gamma;
    FV_TRY(V.lin(r, {{1.0, r}, {-alpha, u1}}));
    FV_TRY(A.apply(r, r1));
    FV_TRY(V.lin(x, {{1.0, x}, {alpha, u}}));
    // j = 1
    FV_TRY(V.dot(r1, rt, &rho1));
    if (rho1 == 0.0) {
      info.breakdown = true;
      return FV_OK;
    }
    beta = alpha * rho1 / rho0;
    rho0 = rho1;
    FV_TRY(V.lin(u, {{1.0, r}, {-beta, u}}));
    FV_TRY(V.lin(u1, {{1.0, r1}, {-beta, u1}}));
    FV_TRY(A.apply(u1, u2));
    FV_TRY(V.dot(u2, rt, &gamma));
    if (gamma == 0.0) {
      info.breakdown = true;
      return FV_OK;
    }
    alpha = rho0 / gamma;
    FV_TRY(V.lin(r, {{1.0, r}, {-alpha, u1}}));
    FV_TRY(V.lin(r1, {{1.0, r1}, {-alpha, u2}}));
    FV_TRY(A.apply(r1, r2));
    FV_TRY(V.lin(x, {{1.0, x}, {alpha, u}}));
    // minimal residual part
    double g11, g12, g22, c1, c2;
    FV_TRY(V.dot(r1, r1, &g11));
    FV_TRY(V.dot(r1, r2, &g12));
    FV_TRY(V.dot(r2, r2, &g22));
    FV_TRY(V.dot(r1, r, &c1));
    FV_TRY(V.dot(r2, r, &c2));
    std::vector<double> G = {g11, g12, g12, g22}, c = {c1, c2};
    if (!dense_solve(2, G, c)) {
      info.breakdown = true;
      return FV_OK;
    }
    FV_TRY(V.lin(x, {{1.0, x}, {c[0], r}, {c[1], r1}}));
    FV_TRY(V.lin(r, {{1.0, r}, {-c[0], r1}, {-c[1], r2}}));
    FV_TRY(V.lin(u, {{1.0, u}, {-c[0], u1}, {-c[1], u2}}));
    omega = c[1];
    double rr;
    FV_TRY(V.dot(r, r, &rr));
    info.rel = std::sqrt(rr) / bn;
    ++cycle;
    if (info.rel <= 0.5 * best) {
      best = info.rel;
      best_cycle = cycle;
    } else if (cycle - best_cycle >= 20) {
      info.stalled = true;
      info.matvecs = (int)(*A.matvecs - mv0);
      return FV_OK;
    }
  }
}

// Restarted GMRES(m) from the initial guess in x, classical Gram-Schmidt applied twice.
template <typename R>
static int gmres(Operator<R>& A, const R* b, R* x, double tol, int m, int max_mv, R* basis, R* w, SolveInfo& info,
                 bool stop_on_stall = false) {
  Vec<R> V{A.g, 4 * A.g->N};
  const size_t n = V.n;
  fv_grid_s* g = A.g;
  double bn2;
  FV_TRY(V.dot(b, b, &bn2));
  const double bn = std::sqrt(bn2);
  const long long mv0 = *A.matvecs;
  info = SolveInfo{};
  if (bn == 0.0) {
    info.status = FV_OK;
    info.rel = 0.0;
    return FV_OK;
  }
  std::vector<double> H((size_t)(m + 1) * m), h(m + 1), h2(m + 1), y;
  double rel_cycle = 2.0;
  for (;;) {
    // r = b - A x into basis[0]
    FV_TRY(A.apply(x, w));
    FV_TRY(V.lin(basis, {{1.0, b}, {-1.0, w}}));
    double beta2;
    FV_TRY(V.dot(basis, basis, &beta2));
    const double beta = std::sqrt(beta2);
    info.rel = beta / bn;
    info.matvecs = (int)(*A.matvecs - mv0);
    if (info.rel <= tol) {
      info.status = FV_OK;
      return FV_OK;
    }
    if (info.matvecs >= max_mv) return FV_OK;
    // (stop_on_stall) a restart cycle that left the true residual nearly where it was: the solve sits at
    // its round-off floor (FP32 data) or stagnates; stop rather than spend the product budget
    if (stop_on_stall && info.rel > 0.9 * rel_cycle) {
      info.stalled = true;
      return FV_OK;
    }
    rel_cycle = info.rel;
    FV_TRY(V.lin(basis, {{1.0 / beta, basis}}));
    std::fill(H.begin(), H.end(), 0.0);
    int used = 0;
    for (int j = 0; j < m; ++j) {
      FV_TRY(A.apply(basis + (size_t)j * n, w));
      for (int pass = 0; pass < 2; ++pass) {
        FV_TRY(launch_multidot<R>(g, basis, n, j + 1, w, n, 1));
        FV_TRY(launch_subtract_basis<R>(g, basis, n, j + 1, g->ws.scalars + 1, w, n));
        FV_TRY(read_scalars(g, 1, j + 1, h.data()));
        for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] += h[i];
      }
      double wn2;
      FV_TRY(V.dot(w, w, &wn2));
      H[(size_t)(j + 1) * m + j] = std::sqrt(wn2);
      used = j + 1;
      double res;
      hessenberg_lstsq(used, H.data(), m, beta, y, &res);
      const bool done = res <= tol * bn || *A.matvecs - mv0 >= max_mv || wn2 == 0.0;
      if (!done) FV_TRY(V.lin(basis + (size_t)(j + 1) * n, {{1.0 / std::sqrt(wn2), w}}));
      if (done) break;
    }
    hessenberg_lstsq(used, H.data(), m, beta, y, nullptr);
    for (int i = 0; i < used; ++i) h2[i] = -y[i];
    FV_CUDA(cudaMemcpyAsync(g->ws.scalars + 1, h2.data(), sizeof(double) * used, cudaMemcpyHostToDevice, g->stream));
    FV_TRY(launch_subtract_basis<R>(g, basis, n, used, g->ws.scalars + 1, x, n));
    FV_CUDA(cudaStreamSynchronize(g->stream));
  }
}

}  // namespace fv

using namespace fv;

// ====================================================================== ABI
extern "C" {

const char* fv_strerror(int s) {
  switch (s) {
    case FV_OK: return "ok";
    case FV_EINVAL: return "invalid argument";
    case FV_ENOMEM: return "out of memory";
    case FV_ECUDA: return "CUDA error";
    case FV_ENOCONV: return "iteration did not converge";
    case FV_ENAN: return "NaN or Inf in a reduction";
    case FV_ETIMEOUT: return "device-side wait timed out";
    default: return "unknown status";
  }
}

const char* fv_last_error(void) { return g_last_error.c_str(); }

int fv_grid_create(const fv_grid_desc* desc, void* stream, fv_grid* out) {
  if (!desc || !out) return invalid("null argument");
  *out = nullptr;
  const int n[3] = {desc->nx, desc->ny, desc->nz};
  for (int d = 0; d < 3; ++d)
    if (n[d] < 2 || n[d] > kMaxN) return invalid("grid size out of range [2, 1024]");
  if (!(desc->Pr > 0.0)) return invalid("Pr must be positive");
  if (4.0 * n[0] * n[1] * (double)n[2] >= 2147483647.0) return invalid("4*nx*ny*nz must be below 2^31");
  const double* given[3] = {desc->xf, desc->yf, desc->zf};
  fv_grid_s* g = new fv_grid_s();
  g->nx = n[0];
  g->ny = n[1];
  g->nz = n[2];
  g->N = (size_t)n[0] * n[1] * n[2];
  g->Pr = desc->Pr;
  g->stream = (cudaStream_t)stream;
  AxisHost ax[3];
  int st = FV_OK;
  for (int d = 0; d < 3 && st == FV_OK; ++d) {
    if (given[d]) {
      g->xf[d].assign(given[d], given[d] + n[d] + 1);
      if (g->xf[d][0] != 0.0 || g->xf[d][n[d]] != 1.0) st = invalid("faces must start at 0 and end at 1");
    } else {
      g->xf[d] = tanh_faces(n[d], desc->stretch);
    }
    if (st == FV_OK) st = build_axis(g->xf[d], ax[d]);
    if (st == FV_OK) {
      double mw = 1.0;
      for (int i = 0; i < n[d]; ++i) mw = std::min(mw, g->xf[d][i + 1] - g->xf[d][i]);
      g->min_width[d] = mw;
    }
  }
  if (st == FV_OK) st = upload_axes<double>(g, ax, 0, g->geo64, g->fdm64, g->cd64, g->fd64);
  if (st == FV_OK) st = upload_axes<float>(g, ax, 1, g->geo32, g->fdm32, g->cd32, g->fd32);
  if (st == FV_OK && tc_eligible(g)) {
    std::vector<double> idx[3] = {ax[0].idx, ax[1].idx, ax[2].idx}, idc[3] = {ax[0].idc, ax[1].idc, ax[2].idc};
    if (tc_setup(g, idx, idc) != FV_OK) {  // keep the SIMT passes
      g->tc.ready = false;
      cudaGetLastError();
    }
  }
  if (st == FV_OK) {
    if (cudaMalloc(&g->ws.err, sizeof(int)) != cudaSuccess || cudaMemset(g->ws.err, 0, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&g->ws.partials, sizeof(double) * kReduceBlocks * 256) != cudaSuccess ||
        cudaMalloc(&g->ws.scalars, sizeof(double) * kMaxScalars) != cudaSuccess ||
        cudaMallocHost(&g->ws.host_scalars, sizeof(double) * kMaxScalars) != cudaSuccess) {
      cudaGetLastError();
      st = FV_ENOMEM;
      set_error("workspace allocation failed");
    }
  }
  if (st != FV_OK) {
    fv_grid_destroy(g);
    return st;
  }
  double s = 0.0;
  for (int d = 0; d < 3; ++d) s += 4.0 / (g->min_width[d] * g->min_width[d]);
  g->sigma_default = -0.5 * std::max(1.0, 1.0 / g->Pr) * s;
  *out = g;
  return FV_OK;
}

int fv_grid_destroy(fv_grid g) {
  if (!g) return FV_OK;
  for (int p = 0; p < 2; ++p) {
    if (g->metric_buf[p]) cudaFree(g->metric_buf[p]);
    if (g->ws.Y[p]) cudaFree(g->ws.Y[p]);
    if (g->ws.t0[p]) cudaFree(g->ws.t0[p]);
    if (g->ws.t1[p]) cudaFree(g->ws.t1[p]);
    if (g->ws.bY[p]) cudaFree(g->ws.bY[p]);
    if (g->ws.bt0[p]) cudaFree(g->ws.bt0[p]);
    if (g->ws.bt1[p]) cudaFree(g->ws.bt1[p]);
  }
  if (g->ws.partials) cudaFree(g->ws.partials);
  if (g->ws.scalars) cudaFree(g->ws.scalars);
  if (g->ws.host_scalars) cudaFreeHost(g->ws.host_scalars);
  for (cudaEvent_t e : g->prof.pool) cudaEventDestroy(e);
  if (g->tc.buf) cudaFree(g->tc.buf);
  if (g->ws.err) cudaFree(g->ws.err);
  if (g->batch_exec) cudaGraphExecDestroy(g->batch_exec);
  if (g->capture_stream) cudaStreamDestroy(g->capture_stream);
  delete g;
  return FV_OK;
}

int fv_set_stream(fv_grid g, void* stream) {
  if (!g) return invalid("null grid");
  g->stream = (cudaStream_t)stream;
  return FV_OK;
}

long long fv_state_elems(fv_grid g) { return g ? (long long)(4 * g->N) : -1; }

int fv_set_wait_limit(fv_grid g, long long spins) {
  if (!g) return invalid("null handle");
  g->wait_spins = spins < 0 ? -1 : spins;
  return FV_OK;
}

int fv_sync(fv_grid g) {
  if (!g) return invalid("null handle");
  int dev_err = 0;
  FV_CUDA(cudaMemcpyAsync(&dev_err, g->ws.err, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
  FV_CUDA(cudaStreamSynchronize(g->stream));
  if (dev_err != 0) {
    FV_CUDA(cudaMemsetAsync(g->ws.err, 0, sizeof(int), g->stream));
    FV_CUDA(cudaStreamSynchronize(g->stream));
    set_error("a bounded device-side wait expired (code " + std::to_string(dev_err) + ")");
    return FV_ETIMEOUT;
  }
  return FV_OK;
}

int fv_profile(fv_grid g, int enable) {
  if (!g) return invalid("null grid");
  FV_CUDA(cudaStreamSynchronize(g->stream));
  if (enable) {
    g->prof.records.clear();
    g->prof.used = 0;
  }
  g->prof.enabled = enable != 0;
  return FV_OK;
}

int fv_profile_read(fv_grid g, double* ms, long long* launches) {
  if (!g || !ms || !launches) return invalid("null argument");
  FV_CUDA(cudaStreamSynchronize(g->stream));
  for (int k = 0; k < FV_PROF_CLASSES; ++k) {
    ms[k] = 0.0;
    launches[k] = 0;
  }
  for (auto& r : g->prof.records) {
    float t = 0.0f;
    FV_CUDA(cudaEventElapsedTime(&t, r.start, r.stop));
    if (r.kind >= 0 && r.kind < FV_PROF_CLASSES) {
      ms[r.kind] += t;
      launches[r.kind] += 1;
    }
  }
  return FV_OK;
}

int fv_residual(fv_grid g, double Gr, const double* q, double* F) {
  if (!g || !q || !F) return invalid("null argument");
  return launch_residual<double>(g, Gr, q, F);
}

int fv_jvp(fv_grid g, int prec, double Gr, const void* q, const void* v, void* Jv) {
  if (!g || !q || !v || !Jv) return invalid("null argument");
  if (prec == FV_FP64) return launch_jvp<double>(g, Gr, 0.0, (const double*)q, (const double*)v, (double*)Jv);
  if (prec == FV_FP32) return launch_jvp<float>(g, Gr, 0.0, (const float*)q, (const float*)v, (float*)Jv);
  return invalid("precision must be FV_FP64 or FV_FP32");
}

int fv_project(fv_grid g, int prec, void* v, int max_it, double tol, int* iters, double* div_rel) {
  if (!g || !v) return invalid("null argument");
  if (prec == FV_FP64) return project_inplace<double>(g, (double*)v, max_it, tol, iters, div_rel);
  if (prec == FV_FP32) return project_inplace<float>(g, (float*)v, max_it, tol, iters, div_rel);
  return invalid("precision must be FV_FP64 or FV_FP32");
}

extern "C++" {
// block buffers for nvec vectors; a reallocation drops the handle's captured block (it refers to them)
template <typename R>
static int ensure_batch_ws(fv_grid_s* g, int nvec) {
  const int p = prec_index<R>();
  if (g->ws.bcap[p] >= nvec) return FV_OK;
  if (g->batch_exec) {
    cudaGraphExecDestroy(g->batch_exec);
    g->batch_exec = nullptr;
    g->batch_key = fv_grid_s::BatchKey();
  }
  void** bufs[3] = {&g->ws.bY[p], &g->ws.bt0[p], &g->ws.bt1[p]};
  for (void** b : bufs)
    if (*b) {
      cudaFree(*b);
      *b = nullptr;
    }
  g->ws.bcap[p] = 0;
  ++g->ws.bgen;
  const size_t N = g->N;
  const size_t sizes[3] = {4 * N * nvec * sizeof(R), N * nvec * sizeof(R), N * nvec * sizeof(R)};
  for (int i = 0; i < 3; ++i)
    if (cudaMalloc(bufs[i], sizes[i]) != cudaSuccess) {
      cudaGetLastError();
      for (void** b : bufs)
        if (*b) {
          cudaFree(*b);
          *b = nullptr;
        }
      set_error("block workspace allocation failed");
      return FV_ENOMEM;
    }
  g->ws.bcap[p] = nvec;
  return FV_OK;
}

// nvec fused J.v + projections, vector i at offset i * 4N of V and W: every stage is one launch over the
// whole block where its kernel has a block form (two-cell stencil, quad divergence and correction, all
// pressure-solve passes), else one launch per vector
template <typename R>
static int jvp_project_block(fv_grid_s* g, double Gr, double sigma, const R* q, int nvec, const R* V, R* W) {
  FV_TRY(ensure_ws<R>(g));
  FV_TRY(ensure_batch_ws<R>(g, nvec));
  const int p = prec_index<R>();
  R* Y = (R*)g->ws.bY[p];
  R* phi = (R*)g->ws.bt1[p];
  R* tmp = (R*)g->ws.bt0[p];
  const size_t n4 = 4 * g->N;
  bool pair = false;
  if constexpr (sizeof(R) == 4) pair = stencil_pair_eligible(g, q, V);
  if constexpr (sizeof(R) == 4) {
    if (pair) FV_TRY(launch_stencil_pair(g, Gr, sigma, q, V, Y, nvec));
  }
  (void)n4;
  if (!pair) FV_TRY(launch_jvp_block<R>(g, Gr, sigma, q, V, Y, nvec));
  FV_TRY(launch_divergence<R>(g, Y, phi, nvec));
  FV_TRY(launch_poisson_block<R>(g, phi, phi, tmp, nvec));
  FV_TRY(launch_correct_block<R>(g, Y, phi, sigma != 0.0 ? V : nullptr, sigma, W, nvec));
  return FV_OK;
}

// Autotuner of the block stencil's z-chunk: every candidate is timed with CUDA events on the handle's
// stream (one warm-up launch, then three) over the block it will run on; the fastest is kept.
static int autotune_pair(fv_grid_s* g, double Gr, double sigma, const float* q, int nvec, const float* V) {
  if (nvec < 2 || !stencil_pair_eligible(g, q, V) || g->tune.pair_zc_nvec == nvec) return FV_OK;
  FV_TRY(ensure_batch_ws<float>(g, nvec));
  float* Y = (float*)g->ws.bY[1];
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  FV_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_status(cudaErrorMemoryAllocation, "cudaEventCreate");
  }
  const bool prof = g->prof.enabled;
  g->prof.enabled = false;
  int st = FV_OK, best = 0, last_chunks = -1;
  float best_ms = 0.f;
  for (int zc : {4, 8, 16, 32, 64}) {
    const int chunks = (g->nz + zc - 1) / zc;
    if (chunks == last_chunks) continue;  // same launch as the previous candidate
    last_chunks = chunks;
    g->tune.pair_zc = zc;
    st = launch_stencil_pair(g, Gr, sigma, q, V, Y, nvec);
    if (st == FV_OK) st = cu_ok(cudaEventRecord(e0, g->stream), "cudaEventRecord");
    for (int r = 0; r < 3 && st == FV_OK; ++r) st = launch_stencil_pair(g, Gr, sigma, q, V, Y, nvec);
    if (st == FV_OK) st = cu_ok(cudaEventRecord(e1, g->stream), "cudaEventRecord");
    if (st == FV_OK) st = cu_ok(cudaEventSynchronize(e1), "cudaEventSynchronize");
    float ms = 0.f;
    if (st == FV_OK) st = cu_ok(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
    if (st != FV_OK) break;
    if (best == 0 || ms < best_ms) {
      best = zc;
      best_ms = ms;
    }
  }
  g->prof.enabled = prof;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  g->tune.pair_zc = (st == FV_OK) ? best : 0;
  g->tune.pair_zc_nvec = (st == FV_OK) ? nvec : 0;
  return st;
}

template <typename R>
static int block_launches(fv_grid_s* g, double Gr, double sigma, const void* q, int nvec, const void* V, void* W) {
  return jvp_project_block<R>(g, Gr, sigma, (const R*)q, nvec, (const R*)V, (R*)W);
}
}

// one eager pass over every problem (workspace, kernel attributes and tensor-core set-up happen outside any
// capture), optionally preceded by the autotuner
static int block_eager(fv_grid_s* g, int prec, double Gr, double sigma, const void* q, int nvec, const void* V,
                       void* W, int flags) {
  if (prec == FV_FP32 && (flags & FV_BATCH_AUTOTUNE))
    FV_TRY(autotune_pair(g, Gr, sigma, (const float*)q, nvec, (const float*)V));
  return prec == FV_FP64 ? block_launches<double>(g, Gr, sigma, q, nvec, V, W)
                         : block_launches<float>(g, Gr, sigma, q, nvec, V, W);
}

static int check_block(fv_grid_s* g, int prec, const void* q, int nvec, const void* V, const void* W) {
  if (!g || !q || !V || !W) return invalid("null argument");
  if (nvec < 1) return invalid("nvec must be at least 1");
  if (prec != FV_FP64 && prec != FV_FP32) return invalid("precision must be FV_FP64 or FV_FP32");
  const size_t bytes = 4 * g->N * (prec == FV_FP64 ? 8 : 4) * (size_t)nvec;
  const size_t qbytes = 4 * g->N * (prec == FV_FP64 ? 8 : 4);
  const char *v0 = (const char*)V, *w0 = (const char*)W, *q0 = (const char*)q;
  if ((w0 < v0 + bytes && v0 < w0 + bytes) || (w0 < q0 + qbytes && q0 < w0 + bytes))
    return invalid("W must not overlap V or q");
  return FV_OK;
}

// launches of one problem's block recorded on `s` (the handle's stream is swapped for the capture)
static int capture_block(fv_grid_s* g, cudaStream_t s, int prec, double Gr, double sigma, const void* q, int nvec,
                         const void* V, void* W) {
  cudaStream_t user = g->stream;
  const bool prof = g->prof.enabled;
  g->prof.enabled = false;
  g->stream = s;
  const int st = prec == FV_FP64 ? block_launches<double>(g, Gr, sigma, q, nvec, V, W)
                                 : block_launches<float>(g, Gr, sigma, q, nvec, V, W);
  g->stream = user;
  g->prof.enabled = prof;
  return st;
}

int fv_jvp_project_batch(fv_grid g, int prec, double Gr, double sigma, const void* q, int nvec, const void* V,
                         void* W, int flags) {
  FV_TRY(check_block(g, prec, q, nvec, V, W));
  if (!(flags & FV_BATCH_GRAPH)) return block_eager(g, prec, Gr, sigma, q, nvec, V, W, flags);
  fv_grid_s::BatchKey key;
  key.prec = prec;
  key.nvec = nvec;
  key.Gr = Gr;
  key.sigma = sigma;
  key.q = q;
  key.V = V;
  key.W = W;
  if (g->batch_exec && key == g->batch_key) {
    FV_CUDA(cudaGraphLaunch(g->batch_exec, g->stream));
    return FV_OK;
  }
  if (g->batch_exec) {
    cudaGraphExecDestroy(g->batch_exec);
    g->batch_exec = nullptr;
  }
  // the eager pass produces W for this call; then the same launches are captured for later calls
  FV_TRY(block_eager(g, prec, Gr, sigma, q, nvec, V, W, flags));
  if (!g->capture_stream) FV_CUDA(cudaStreamCreateWithFlags(&g->capture_stream, cudaStreamNonBlocking));
  FV_CUDA(cudaStreamSynchronize(g->stream));
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(g->capture_stream, cudaStreamCaptureModeThreadLocal);
  int st = (e == cudaSuccess) ? capture_block(g, g->capture_stream, prec, Gr, sigma, q, nvec, V, W)
                              : cuda_status(e, "cudaStreamBeginCapture");
  const cudaError_t e2 = cudaStreamEndCapture(g->capture_stream, &graph);
  if (st == FV_OK && e2 != cudaSuccess) st = cuda_status(e2, "cudaStreamEndCapture");
  if (st == FV_OK) {
    const cudaError_t e3 = cudaGraphInstantiate(&g->batch_exec, graph, 0);
    if (e3 != cudaSuccess) st = cuda_status(e3, "cudaGraphInstantiate");
  }
  if (graph) cudaGraphDestroy(graph);
  if (st != FV_OK) {
    g->batch_exec = nullptr;
    return st;
  }
  g->batch_key = key;
  return FV_OK;
}

int fv_get_tuning(fv_grid g, int* pair_zchunk, int* tuned_nvec) {
  if (!g) return invalid("null grid");
  if (pair_zchunk) *pair_zchunk = g->tune.pair_zc;
  if (tuned_nvec) *tuned_nvec = g->tune.pair_zc_nvec;
  return FV_OK;
}

// ------------------------------------------------------------------ several problems in one graph
struct fv_batch_plan_s {
  std::vector<fv_grid_s*> grids;
  std::vector<unsigned> gens;  // each handle's block-buffer generation at capture
  cudaGraphExec_t exec = nullptr;
};

int fv_batch_plan_create(int nprob, const fv_grid* grids, int prec, const double* Gr, const double* sigma,
                         const void* const* q, const int* nvec, const void* const* V, void* const* W, int flags,
                         fv_batch_plan* out) {
  if (!out) return invalid("null output");
  *out = nullptr;
  if (nprob < 1 || !grids || !Gr || !sigma || !q || !nvec || !V || !W) return invalid("null argument");
  for (int i = 0; i < nprob; ++i) {
    FV_TRY(check_block(grids[i], prec, q[i], nvec[i], V[i], W[i]));
    for (int j = 0; j < i; ++j)
      if (grids[j] == grids[i]) return invalid("every problem needs its own grid handle (workspaces run concurrently)");
  }
  for (int i = 0; i < nprob; ++i)
    FV_TRY(block_eager(grids[i], prec, Gr[i], sigma[i], q[i], nvec[i], V[i], W[i], flags));
  for (int i = 0; i < nprob; ++i) FV_CUDA(cudaStreamSynchronize(grids[i]->stream));
  // capture: a root stream forks one branch per problem and joins them, so the problems run concurrently
  std::vector<cudaStream_t> streams(nprob + 1, nullptr);
  std::vector<cudaEvent_t> events(nprob + 1, nullptr);
  int st = FV_OK;
  for (int i = 0; i <= nprob && st == FV_OK; ++i) {
    st = cu_ok(cudaStreamCreateWithFlags(&streams[i], cudaStreamNonBlocking), "cudaStreamCreateWithFlags");
    if (st == FV_OK) st = cu_ok(cudaEventCreateWithFlags(&events[i], cudaEventDisableTiming), "cudaEventCreate");
  }
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (st == FV_OK) {
    cudaStream_t root = streams[nprob];
    st = cu_ok(cudaStreamBeginCapture(root, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    if (st == FV_OK) {
      st = cu_ok(cudaEventRecord(events[nprob], root), "cudaEventRecord");
      for (int i = 0; i < nprob && st == FV_OK; ++i) {
        st = cu_ok(cudaStreamWaitEvent(streams[i], events[nprob], 0), "cudaStreamWaitEvent");
        if (st == FV_OK) st = capture_block(grids[i], streams[i], prec, Gr[i], sigma[i], q[i], nvec[i], V[i], W[i]);
        if (st == FV_OK) st = cu_ok(cudaEventRecord(events[i], streams[i]), "cudaEventRecord");
        if (st == FV_OK) st = cu_ok(cudaStreamWaitEvent(root, events[i], 0), "cudaStreamWaitEvent");
      }
      const cudaError_t e2 = cudaStreamEndCapture(root, &graph);
      if (st == FV_OK && e2 != cudaSuccess) st = cuda_status(e2, "cudaStreamEndCapture");
    }
  }
  if (st == FV_OK) st = cu_ok(cudaGraphInstantiate(&exec, graph, 0), "cudaGraphInstantiate");
  if (graph) cudaGraphDestroy(graph);
  for (int i = 0; i <= nprob; ++i) {
    if (events[i]) cudaEventDestroy(events[i]);
    if (streams[i]) cudaStreamDestroy(streams[i]);
  }
  if (st != FV_OK) {
    if (exec) cudaGraphExecDestroy(exec);
    return st;
  }
  fv_batch_plan_s* plan = new fv_batch_plan_s();
  plan->exec = exec;
  for (int i = 0; i < nprob; ++i) {
    plan->grids.push_back(grids[i]);
    plan->gens.push_back(grids[i]->ws.bgen);
  }
  *out = plan;
  return FV_OK;
}

int fv_batch_plan_launch(fv_batch_plan plan, void* stream) {
  if (!plan || !plan->exec) return invalid("null plan");
  for (size_t i = 0; i < plan->grids.size(); ++i)
    if (plan->grids[i]->ws.bgen != plan->gens[i])
      return invalid("a grid's block workspace was reallocated after the plan was captured; create the plan again");
  FV_CUDA(cudaGraphLaunch(plan->exec, (cudaStream_t)stream));
  return FV_OK;
}

int fv_batch_plan_destroy(fv_batch_plan plan) {
  if (!plan) return FV_OK;
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  delete plan;
  return FV_OK;
}

int fv_diagnostics(fv_grid g, const double* q, double* ekin, double* nu) {
  if (!g || !q) return invalid("null argument");
  FV_TRY(launch_ekin(g, q, 0));
  FV_TRY(launch_nusselt(g, q, 1));
  double v[2];
  FV_TRY(read_scalars(g, 0, 2, v));
  if (ekin) *ekin = v[0];
  if (nu) *nu = v[1];
  return FV_OK;
}

int fv_time_step(fv_grid g, double Gr, double dt, int nsteps, double* q, double* ekin, double* nu) {
  if (!g || !q) return invalid("null argument");
  if (!(dt > 0.0) || nsteps < 0) return invalid("need dt > 0 and nsteps >= 0");
  FV_TRY(ensure_ws<double>(g));
  const size_t n = 4 * g->N;
  DevBuf<double> F;
  FV_TRY(F.alloc(n));
  Vec<double> V{g, n};
  auto record = [&](int i) -> int {
    if (!ekin && !nu) return FV_OK;
    FV_TRY(launch_ekin(g, q, 0));
    FV_TRY(launch_nusselt(g, q, 1));
    double v[2];
    FV_TRY(read_scalars(g, 0, 2, v));
    if (ekin) ekin[i] = v[0];
    if (nu) nu[i] = v[1];
    if (!std::isfinite(v[0]) || !std::isfinite(v[1])) {
      set_error("non-finite diagnostics: the time step is unstable");
      return FV_ENAN;
    }
    return FV_OK;
  };
  FV_TRY(record(0));
  for (int it = 1; it <= nsteps; ++it) {
    // delta = (I - dt L)^-1 dt F(q) = -(L - I/dt)^-1 F(q); its velocity projected; q += delta
    FV_TRY(launch_residual<double>(g, Gr, q, F.p));
    FV_TRY(diffusion_solve<double>(g, F.p, F.p, 1.0 / dt));
    FV_TRY(project_inplace<double>(g, F.p, 1, 0.0, nullptr, nullptr));
    FV_TRY(V.lin(q, {{1.0, q}, {-1.0, F.p}}));
    FV_TRY(record(it));
  }
  return FV_OK;
}

int fv_transfer(fv_grid from, const double* q_from, fv_grid to, double* q_to) {
  if (!from || !to || !q_from || !q_to) return invalid("null argument");
  if ((const void*)q_from == (const void*)q_to) return invalid("q_to must not alias q_from");
  FV_TRY(ensure_ws<double>(to));
  FV_CUDA(cudaStreamSynchronize(from->stream));  // q_from is complete before the other stream reads it
  FV_TRY(launch_prolong(from, q_from, to, q_to));
  return project_inplace<double>(to, q_to, 1, 0.0, nullptr, nullptr);
}

int fv_diffusion_solve(fv_grid g, int prec, const void* in, void* out) {
  if (!g || !in || !out) return invalid("null argument");
  if (prec == FV_FP64) return diffusion_solve<double>(g, (const double*)in, (double*)out);
  if (prec == FV_FP32) return diffusion_solve<float>(g, (const float*)in, (float*)out);
  return invalid("precision must be FV_FP64 or FV_FP32");
}

int fv_jvp_project(fv_grid g, int prec, double Gr, double sigma, const void* q, const void* v, void* out) {
  if (!g || !q || !v || !out) return invalid("null argument");
  if (out == q || out == v) return invalid("out must not alias q or v");
  if (prec == FV_FP64) return jvp_project<double>(g, Gr, sigma, (const double*)q, (const double*)v, (double*)out);
  if (prec == FV_FP32) return jvp_project<float>(g, Gr, sigma, (const float*)q, (const float*)v, (float*)out);
  return invalid("precision must be FV_FP64 or FV_FP32");
}

int fv_jvp_project_lincomb_dev(fv_grid g, int prec, double Gr, double sigma, const void* q, const void* v,
                               const void* w, double alpha, double beta, double gamma, void* out,
                               double* norm2_dev) {
  if (!g || !q || !v || !out) return invalid("null argument");
  if (out == q || out == v) return invalid("out must not alias q or v");
  if (prec != FV_FP64 && prec != FV_FP32) return invalid("precision must be FV_FP64 or FV_FP32");
  const double b2 = alpha * sigma + beta;
  const int slot = norm2_dev ? 0 : -1;
  if (prec == FV_FP64)
    FV_TRY(chebyshev_step<double>(g, Gr, sigma, (const double*)q, (const double*)v, w ? (const double*)w : nullptr,
                                  alpha, b2, w ? gamma : 0.0, (double*)out, slot));
  else
    FV_TRY(chebyshev_step<float>(g, Gr, sigma, (const float*)q, (const float*)v, w ? (const float*)w : nullptr, alpha,
                                 b2, w ? gamma : 0.0, (float*)out, slot));
  if (norm2_dev)
    FV_CUDA(cudaMemcpyAsync(norm2_dev, g->ws.scalars, sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
  return FV_OK;
}

int fv_jvp_project_lincomb(fv_grid g, int prec, double Gr, double sigma, const void* q, const void* v,
                           const void* w, double alpha, double beta, double gamma, void* out, double* out_norm2) {
  if (!g || !q || !v || !out) return invalid("null argument");
  if (out == q || out == v) return invalid("out must not alias q or v");
  if (prec != FV_FP64 && prec != FV_FP32) return invalid("precision must be FV_FP64 or FV_FP32");
  // alpha (P(Jv - sigma v) + sigma v) + beta v + gamma w = alpha P(Jv - sigma v) + (alpha sigma + beta) v + gamma w
  const double b2 = alpha * sigma + beta;
  const int slot = out_norm2 ? 0 : -1;
  if (prec == FV_FP64)
    FV_TRY(chebyshev_step<double>(g, Gr, sigma, (const double*)q, (const double*)v, w ? (const double*)w : nullptr,
                                  alpha, b2, w ? gamma : 0.0, (double*)out, slot));
  else
    FV_TRY(chebyshev_step<float>(g, Gr, sigma, (const float*)q, (const float*)v, w ? (const float*)w : nullptr, alpha,
                                 b2, w ? gamma : 0.0, (float*)out, slot));
  if (out_norm2) {
    FV_TRY(read_scalars(g, 0, 1, out_norm2));
    if (!std::isfinite(*out_norm2)) {
      set_error("non-finite norm");
      return FV_ENAN;
    }
  }
  return FV_OK;
}

int fv_dot(fv_grid g, int prec, const void* a, const void* b, double* result) {
  if (!g || !a || !b || !result) return invalid("null argument");
  if (prec == FV_FP64) return Vec<double>{g, 4 * g->N}.dot((const double*)a, (const double*)b, result);
  if (prec == FV_FP32) return Vec<float>{g, 4 * g->N}.dot((const float*)a, (const float*)b, result);
  return invalid("precision must be FV_FP64 or FV_FP32");
}

int fv_axpby(fv_grid g, int prec, double alpha, const void* x, double beta, void* y) {
  if (!g || !x || !y) return invalid("null argument");
  if (prec == FV_FP64) return Vec<double>{g, 4 * g->N}.lin((double*)y, {{alpha, (const double*)x}, {beta, (const double*)y}});
  if (prec == FV_FP32) return Vec<float>{g, 4 * g->N}.lin((float*)y, {{alpha, (const float*)x}, {beta, (const float*)y}});
  return invalid("precision must be FV_FP64 or FV_FP32");
}

int fv_convert(fv_grid g, int to_fp32, const void* src, void* dst) {
  if (!g || !src || !dst) return invalid("null argument");
  if (to_fp32) return launch_convert(g, 4 * g->N, (const double*)src, (float*)dst);
  return launch_convert(g, 4 * g->N, (const float*)src, (double*)dst);
}

void fv_newton_default_opts(fv_newton_opts* o) {
  if (!o) return;
  o->precision = FV_FP64;
  o->tol = 1e-10;
  o->krylov_tol = 1e-10;
  o->max_newton = 20;
  o->max_matvec = 8000;
  o->gmres_m = 100;
  o->gr_start = 0.0;
  o->gr_ratio = 2.0;
  o->precond = 1;
  o->forcing = 1;
  o->ptc_dt0 = 0.0;
}

void fv_arnoldi_default_opts(fv_arnoldi_opts* o) {
  if (!o) return;
  o->precision = FV_FP64;
  o->m = 20;
  o->tol = 1e-9;
  o->max_restarts = 30;
  o->max_degree = 200;
  o->min_degree = 10;
  o->guard = 2;
  o->seed = 1;
  o->sigma = 0.0;
  o->low_tol = 1e-3;
  o->low_max_restarts = 20;
  o->euler_dt = 0.0;
  o->inner_m = 50;
  o->inner_max = 3000;
  o->inner_tol = 0.0;
  o->vecs_fp64 = 0;
}

}  // extern "C"

// ====================================================================== Newton
namespace fv {

template <typename R>
static int newton_at(fv_grid_s* g, double Gr, double* q, const fv_newton_opts& o, fv_newton_report* rep,
                     bool record) {
  const size_t n = 4 * g->N;
  Vec<double> V64{g, n};
  DevBuf<double> r64, d64;
  DevBuf<R> qR, rhs, x, work, basis, w;
  FV_TRY(r64.alloc(n));
  FV_TRY(d64.alloc(n));
  const bool mixed = !std::is_same<R, double>::value;
  if (mixed) FV_TRY(qR.alloc(n));
  FV_TRY(rhs.alloc(mixed ? n : 0));
  FV_TRY(x.alloc(n));
  FV_TRY(work.alloc(7 * n));
  FV_TRY(basis.alloc((size_t)(o.gmres_m + 1) * n));
  FV_TRY(w.alloc(n));
  DevBuf<R> pre;
  if (o.precond) FV_TRY(pre.alloc(n));
  const double sigma = g->sigma_default;
  // FP32 inner solves stall near u_32 times the stiffness ratio of what they apply: ~1e-5 unpreconditioned,
  // ~1e-3 through M^-1 = P L^-1 (L^-1 x is smooth, so J L^-1 x carries u_32 lam_max / lam_min of round-off);
  // the FP64 outer loop refines past either
  const double ktol = mixed ? std::max(o.krylov_tol, o.precond ? 1e-3 : 1e-5) : o.krylov_tol;
  double r0 = -1.0, r_prev = -1.0, eta_prev = 1e-2;
  // pseudo-transient continuation: step k solves (P J - I / dt_k) delta = -P F; after a step that lowered
  // the residual dt grows by (r_{k-1} / r_k)^2 clipped to [1.5, 10] (switched evolution relaxation with a
  // floor on the growth), after one that did not it halves (never below dt_0); plain Newton once
  // dt > 1e4 (|lambda| dt ~ 1e6 for the slowest modes of this problem)
  double dt = o.ptc_dt0;
  int steps = 0;
  DevBuf<double> qt;
  FV_TRY(qt.alloc(n));
  // ||P F(x)||_inf in FP64 (r64 holds P F(x) on return)
  auto proj_residual = [&](const double* xs, double* out) -> int {
    FV_TRY(launch_residual<double>(g, Gr, xs, r64.p));
    FV_TRY(project_inplace<double>(g, r64.p, 1, 0.0, nullptr, nullptr));
    FV_TRY(launch_maxabs<double>(g, r64.p, n, 0));
    FV_TRY(read_scalars(g, 0, 1, out));
    if (!std::isfinite(*out)) {
      set_error("non-finite Newton residual");
      return FV_ENAN;
    }
    return FV_OK;
  };
  for (int it = 0;; ++it) {
    double rn;
    FV_TRY(proj_residual(q, &rn));
    if (r0 < 0.0) r0 = rn;
    if (record) {
      if (it < 64) rep->history[it] = rn;
      rep->residual0 = r0;
      rep->residual = rn;
      rep->newton_steps = steps;
    }
    const double target = o.tol * std::max(1.0, r0);
    if (rn <= target) return FV_OK;
    // round-off floor: ||P F||_inf cannot fall below ~eps times its largest terms (buoyancy Gr T,
    // diffusion ~ sum_d 4 |q| / h_min,d^2) amplified by the projection's conditioning, which on fine
    // stretched grids lies above tol r0.  Floor estimate 1e3 eps max|q| (Gr + sum_d 4 / h_min,d^2)
    // (measured floors: ~1e-6 at 100^3, s = 1.5, Gr = 2.5e4, where this gives ~3e-6).
    double qmax;
    FV_TRY(launch_maxabs<double>(g, q, n, 0));
    FV_TRY(read_scalars(g, 0, 1, &qmax));
    double stiff = Gr;
    for (int d = 0; d < 3; ++d) stiff += 4.0 / (g->min_width[d] * g->min_width[d]);
    const double floor_est = 1e3 * std::numeric_limits<double>::epsilon() * qmax * stiff;
    if (rn <= floor_est) return FV_OK;
    if (steps >= o.max_newton) return FV_ENOCONV;
    // solve (P J(q)) delta = -P F(q)
    const R* qop;
    R* b;
    if (mixed) {
      FV_TRY(launch_convert(g, n, q, (float*)qR.p));
      FV_TRY(launch_convert(g, n, r64.p, (float*)rhs.p));
      qop = qR.p;
      b = rhs.p;
    } else {
      qop = (const R*)q;
      b = (R*)r64.p;
    }
    Vec<R> VR{g, n};
    FV_TRY(VR.lin(b, {{-1.0, b}}));
    long long mv = 0;
    Operator<R> A{g, Gr, sigma, qop, &mv};
    A.pre = o.precond ? pre.p : nullptr;
    if (dt > 0.0) {
      if (r_prev > 0.0)
        dt = (rn < r_prev) ? dt * std::min(10.0, std::max(1.5, (r_prev / rn) * (r_prev / rn)))
                           : std::max(o.ptc_dt0, 0.5 * dt);
      A.s = (dt < 1e4) ? 1.0 / dt : 0.0;
    }
    SolveInfo info;
    // inner tolerance: fixed krylov_tol, or Eisenstat-Walker (choice 2): eta = 0.9 (r_k / r_{k-1})^2,
    // at most 1e-2 (safeguard max(eta, 0.9 eta_{k-1}^2)), at least krylov_tol and half of what takes the
    // residual to the Newton target in this step (no over-solving near the round-off floor)
    double eta = ktol;
    if (o.forcing) {
      eta = (r_prev > 0.0) ? 0.9 * (rn / r_prev) * (rn / r_prev) : 1e-2;
      eta = std::max(eta, 0.9 * eta_prev * eta_prev);
      eta = std::min(eta, 1e-2);
      eta = std::max(eta, std::max(ktol, 0.5 * target / rn));
    }
    eta_prev = eta;
    r_prev = rn;
    if (A.s != 0.0) eta = std::max(eta, 1e-3);  // a pseudo-time step needs no accurate solve
    FV_TRY(bicgstab2<R>(A, b, x.p, eta, o.max_matvec, work.p, info));
    if (info.status != FV_OK && (info.breakdown || info.stalled)) {
      SolveInfo info2;
      FV_TRY(gmres<R>(A, b, x.p, eta, o.gmres_m, o.max_matvec - info.matvecs, basis.p, w.p, info2));
      rep->gmres_fallbacks += 1;
    }
    rep->matvecs += (int)mv;
    if (o.precond) {  // right preconditioning: delta = M^-1 y
      FV_TRY(apply_precond<R>(g, x.p, pre.p, A.s));
      Vec<R> VP{g, n};
      FV_TRY(VP.copy(x.p, pre.p));
    }
    // delta -> FP64, re-projected in FP64 so that q stays divergence free to FP64 accuracy
    if (mixed) {
      FV_TRY(launch_convert(g, n, (const float*)x.p, d64.p));
    } else {
      FV_TRY(V64.copy(d64.p, (const double*)x.p));
    }
    FV_TRY(project_inplace<double>(g, d64.p, 1, 0.0, nullptr, nullptr));
    // backtracking on ||P F||_inf (an inexact correction far from the solution can overshoot): the first
    // of lambda = 1, 1/2, .., 1/16 with sufficient decrease, else the best of them
    double lam = 1.0, best_r = 1e300, best_lam = 1.0;
    for (int bt = 0; bt < 5; ++bt) {
      FV_TRY(V64.lin(qt.p, {{1.0, q}, {lam, d64.p}}));
      double rt;
      const int rs = proj_residual(qt.p, &rt);
      if (rs == FV_OK && rt < best_r) {
        best_r = rt;
        best_lam = lam;
      }
      if (rs == FV_OK && rt <= (1.0 - 1e-4 * lam) * rn) break;
      lam *= 0.5;
    }
    FV_TRY(V64.lin(q, {{1.0, q}, {best_lam, d64.p}}));
    ++steps;
  }
}

}  // namespace fv

extern "C" int newton_steady(fv_grid g, double Gr, double* q_inout, const fv_newton_opts* opts,
                             fv_newton_report* report) {
  if (!g || !q_inout) return invalid("null argument");
  fv_newton_opts o;
  if (opts)
    o = *opts;
  else
    fv_newton_default_opts(&o);
  if (o.precision != FV_FP64 && o.precision != FV_FP32) return invalid("precision must be FV_FP64 or FV_FP32");
  if (o.max_newton < 0 || o.max_matvec < 4 || o.gmres_m < 1 || o.gmres_m > 200 || o.precond < 0 || o.precond > 1 ||
      o.forcing < 0 || o.forcing > 1 || !(o.ptc_dt0 >= 0.0))
    return invalid("bad Newton options");
  fv_newton_report rep;
  std::memset(&rep, 0, sizeof(rep));
  std::vector<double> ladder;
  if (o.gr_start > 0.0 && o.gr_start < Gr) {
    if (!(o.gr_ratio > 1.0)) return invalid("gr_ratio must exceed 1");
    for (double x = o.gr_start; x < Gr; x *= o.gr_ratio) ladder.push_back(x);
  }
  ladder.push_back(Gr);
  int st = FV_OK;
  for (size_t i = 0; i < ladder.size(); ++i) {
    const bool last = (i + 1 == ladder.size());
    fv_newton_report tmp;
    std::memset(&tmp, 0, sizeof(tmp));
    fv_newton_report* r = last ? &rep : &tmp;
    st = (o.precision == FV_FP64) ? newton_at<double>(g, ladder[i], q_inout, o, r, true)
                                  : newton_at<float>(g, ladder[i], q_inout, o, r, true);
    if (!last) {
      rep.matvecs += tmp.matvecs;
      rep.gmres_fallbacks += tmp.gmres_fallbacks;
      if (st != FV_OK) {  // report the Gr point that failed: its residual history and Newton steps
        rep.newton_steps = tmp.newton_steps;
        rep.residual0 = tmp.residual0;
        rep.residual = tmp.residual;
        std::memcpy(rep.history, tmp.history, sizeof(rep.history));
        break;
      }
      rep.continuation_steps += 1;
    }
    if (st != FV_OK) break;
  }
  rep.status = st;
  if (report) *report = rep;
  return st;
}

// ====================================================================== Chebyshev-preconditioned Arnoldi
namespace fv {

static bool ritz_before(const Ritz& a, const Ritz& b) {
  if (a.re != b.re) return a.re > b.re;
  if (std::fabs(a.im) != std::fabs(b.im)) return std::fabs(a.im) > std::fabs(b.im);
  return a.im > b.im;
}

// Statistics of the shifted solves of the implicit-Euler transform.
struct SolveStats {
  int solves = 0, short_ = 0;
  double worst = 0.0;
  void note(bool converged, double rel) {
    ++solves;
    if (!converged) ++short_;
    worst = std::max(worst, rel);
  }
};

// FP64-accurate shifted solve (P J - s) y = x by iterative refinement around FP32 GMRES: the residual
// x - (A - s) y is formed with FP64 products, normalised, solved in FP32 (right-preconditioned GMRES to
// tol32), and the FP32 correction, re-projected in FP64, is added in FP64.  Each round gains the FP32
// solve's digits (~3) at one FP64 product and one FP64 projection; the stiff directions never see FP32
// round-off in y, because every correction passes through M^-1 = P (L - s)^-1 and the FP64 residual.
struct EulerRefine {
  fv_grid_s* g = nullptr;
  double Gr = 0.0, sigma = 0.0, s = 0.0;
  const float* q32 = nullptr;
  const double* q64 = nullptr;
  float *b32 = nullptr, *x32 = nullptr, *pre32 = nullptr, *basis32 = nullptr, *w32 = nullptr;
  double *r64 = nullptr, *t64 = nullptr;
  int inner_m = 50, inner_max = 3000, max_outer = 8;
  double tol32 = 1e-3, tol64 = 1e-9;
  long long* mv64 = nullptr;
  long long mv32 = 0;
  SolveStats* stats = nullptr;

  int solve(const double* in, double* out) {
    const size_t n = 4 * g->N;
    Vec<double> V64{g, n};
    Vec<float> V32{g, n};
    Operator<float> A32{g, Gr, sigma, q32, &mv32};
    A32.pre = pre32;
    A32.s = s;
    Operator<double> A64{g, Gr, sigma, q64, mv64};
    A64.s = s;
    FV_TRY(V64.zero(out));
    FV_TRY(V64.copy(r64, in));
    double xn2;
    FV_TRY(V64.dot(in, in, &xn2));
    const double xn = std::sqrt(xn2);
    double rel = 1.0, rel_prev = 2.0;
    for (int it = 0; it <= max_outer; ++it) {
      double rn2;
      FV_TRY(V64.dot(r64, r64, &rn2));
      const double rn = std::sqrt(rn2);
      rel = xn > 0.0 ? rn / xn : 0.0;
      // converged, or the FP32 corrections no longer halve the FP64 residual (its round-off floor)
      if (rel <= tol64 || it == max_outer || rel > 0.5 * rel_prev) break;
      rel_prev = rel;
      FV_TRY(V64.lin(t64, {{1.0 / rn, r64}}));
      FV_TRY(launch_convert(g, n, t64, b32));
      FV_TRY(V32.zero(x32));
      SolveInfo info;
      FV_TRY(gmres<float>(A32, b32, x32, tol32, inner_m, inner_max, basis32, w32, info, true));
      FV_TRY(apply_precond<float>(g, x32, pre32, s));
      FV_TRY(launch_convert(g, n, pre32, t64));
      FV_TRY(project_inplace<double>(g, t64, 1, 0.0, nullptr, nullptr));
      FV_TRY(V64.lin(out, {{1.0, out}, {rn, t64}}));
      FV_TRY(A64.apply(out, t64));
      FV_TRY(V64.lin(r64, {{1.0, in}, {-1.0, t64}}));
    }
    if (stats) stats->note(rel <= tol64, rel);
    return FV_OK;
  }
};

// Chebyshev polynomial p(z) = T_deg((z - d)/c) / T_deg((lam_ref - d)/c) of one cycle's ellipse.
struct ChebFilter {
  bool on = false;
  double d = 0.0, c2 = 0.0, lam_ref = 0.0;
  int deg = 0;
};

// State one Arnoldi run hands to the next (the FP32 phase of the mixed form to its FP64 phase).
struct ArnoldiCarry {
  double lam_far = 0.0;
  ChebFilter filt;
};

// Advantage per application of p(A) that the degree gives the slowest guard value over the ellipse.
constexpr double kFilterGain = 1e2;

// Chebyshev-preconditioned Arnoldi.  Cycle 0 runs m Arnoldi steps on A itself; every later cycle runs m
// steps on B = p(A) (each application = deg J.v + projection steps of the three-term recurrence), which
// maps the stiff part of the spectrum into the small interior of the ellipse instead of amplifying its
// round-off by ||A|| / |lam| per step.  Eigenvalues of A come from the Rayleigh-Ritz matrix G = V^T A V
// (m more products), the k with the largest real part are tested by their true FP64 residuals, and the
// next cycle starts from p(A) applied to the sum of the normalised wanted Ritz vectors plus a random
// component (relative weight tol / 100) under the next ellipse.
// stall > 0: give up (FV_ENOCONV, Ritz vectors still written) once the largest relative residual has not
// halved over `stall` cycles (the FP32 phase of the mixed form stops at its round-off floor).
// Shift-invert Arnoldi for the implicit-Euler transform, with thick restarts.
//
// B = (A - s I)^-1, s = 1 / euler_dt, on the divergence-free subspace (A = P (J - sigma) + sigma): an
// eigenvalue lam of A is mu = 1 / (lam - s) of B, so the eigenvalues nearest s (the rightmost ones for a
// shift right of the spectrum) have the largest |mu| and the stiff, convection-dominated far spectrum maps
// to |mu| ~ 0.  The Arnoldi process runs on B (each application one GMRES solve of (A - s) y = x,
// right-preconditioned with P (L - s)^-1), and the Ritz pairs are those of B: extremal eigenvalues of B,
// which Rayleigh-Ritz approximates reliably even for this far-from-normal operator (a Rayleigh-Ritz
// extraction with A itself can return values from the field of values of A far right of any eigenvalue).
// The eigenvalue of A reported for a Ritz vector x is its Rayleigh quotient x^H A x / x^H x, and the
// residual ||A x - lam x|| / (|lam| ||x||) is taken with A.
//
// Restart (thick, Krylov-Schur style): B V_m = V_m G + v_m g^T holds for the basis V_m and the projected
// matrix G (not Hessenberg after the first restart).  The Ritz vectors of the p Ritz values of largest
// |mu|, orthonormalised in coefficient space (Y = Q_y R, G Q_y = Q_y (Q_y^T G Q_y) because span Y is
// G-invariant), give the new leading basis V_m Q_y with projected block Q_y^T G Q_y, followed by v_m with
// the row g^T Q_y; the Arnoldi process then expands from v_m.  Inexact solves perturb this relation at
// their tolerance; since the kept block is never recomputed, every solve runs to the same tolerance.
template <typename R>
static int arnoldi_si(fv_grid_s* g, int k, double Gr, const double* q64, const fv_arnoldi_opts& o, double* re,
                      double* im, void* vecs_out, fv_arnoldi_report* rep, const R* start, int stall,
                      EulerRefine* refine) {
  const auto t_start = std::chrono::steady_clock::now();
  const size_t n = 4 * g->N;
  const int m = o.m;
  const bool mixed = !std::is_same<R, double>::value;
  const double sigma = (o.sigma != 0.0) ? o.sigma : g->sigma_default;
  const double s = 1.0 / o.euler_dt;
  const bool refined = refine != nullptr && std::is_same<R, double>::value;
  // Ritz values kept over a restart (largest |mu|) and reported (the k of largest real part among them)
  // (a Ritz value of modest |mu| but large real part, e.g. a pair with a large imaginary part, is reported
  // only if it is kept, hence three times k)
  const int keep_max = std::max(1, std::min(m - 4, std::max(k + o.guard, 3 * k)));
  DevBuf<R> qR, Vb, w, y0, y1, X;
  if (mixed) {
    FV_TRY(qR.alloc(n));
    FV_TRY(launch_convert(g, n, q64, (float*)qR.p));
  }
  const R* q = mixed ? qR.p : (const R*)q64;
  FV_TRY(Vb.alloc((size_t)(m + 1) * n));
  FV_TRY(w.alloc(n));
  FV_TRY(y0.alloc(n));
  FV_TRY(y1.alloc(n));
  FV_TRY(X.alloc((size_t)(keep_max + 2) * n));
  Vec<R> V{g, n};
  long long mv = 0;
  Operator<R> A{g, Gr, sigma, q, &mv};
  DevBuf<R> gbasis, gw, epre;
  if (!refined) {
    FV_TRY(gbasis.alloc((size_t)(o.inner_m + 1) * n));
    FV_TRY(gw.alloc(n));
    FV_TRY(epre.alloc(n));
  }
  Operator<R> Ae{g, Gr, sigma, q, &mv};
  Ae.pre = epre.p;
  Ae.s = s;
  double etol = 1e-3;
  SolveStats sstats;
  if (refined) {
    refine->stats = &sstats;
    refine->mv64 = &mv;  // the refinement's FP64 products count with this run's
  }
  auto apply_B = [&](const R* in, R* out) -> int {
    if constexpr (std::is_same<R, double>::value) {
      if (refined) return refine->solve(in, out);
    }
    FV_TRY(V.zero(out));
    SolveInfo info;
    FV_TRY(gmres<R>(Ae, in, out, etol, o.inner_m, o.inner_max, gbasis.p, gw.p, info, true));
    sstats.note(info.status == FV_OK, info.rel);
    FV_TRY(apply_precond<R>(g, out, epre.p, s));
    return V.copy(out, epre.p);
  };
  // CGS2 of w against Vb[0, j]: coefficients added to column `col` of Gb; returns ||w|| after
  std::vector<double> Gb((size_t)(m + 1) * m, 0.0), h(m + 1);
  auto orthogonalise = [&](R* wv, int j, int col, double* norm) -> int {
    for (int pass = 0; pass < 2; ++pass) {
      FV_TRY(launch_multidot<R>(g, Vb.p, n, j + 1, wv, n, 1));
      FV_TRY(launch_subtract_basis<R>(g, Vb.p, n, j + 1, g->ws.scalars + 1, wv, n));
      FV_TRY(read_scalars(g, 1, j + 1, h.data()));
      for (int i = 0; i <= j; ++i) {
        if (!std::isfinite(h[i])) {
          set_error("non-finite Gram-Schmidt coefficient");
          return FV_ENAN;
        }
        if (col >= 0) Gb[(size_t)i * m + col] += h[i];
      }
    }
    double n2;
    FV_TRY(V.dot(wv, wv, &n2));
    *norm = std::sqrt(n2);
    return FV_OK;
  };
  // start vector: seeded N(0,1) (or the caller's), projected, then one application of B (damps its stiff
  // components, which no later Krylov vector of B could cancel)
  R* x = y0.p;
  if (start) {
    FV_TRY(V.copy(x, start));
  } else {
    FV_TRY(launch_fill_normal<R>(g, o.seed, x));
  }
  FV_TRY(project_inplace<R>(g, x, 1, 0.0, nullptr, nullptr));
  const double etol_floor = o.inner_tol > 0.0 ? o.inner_tol : (mixed ? 1e-3 : std::max(1e-12, 0.01 * o.tol));
  double best = 1e300;
  int best_at = 0, p = 0, status = FV_ENOCONV, nret = 0;
  std::vector<double> Gm, Hg, Qg, hre, him, sh;
  for (int restart = 0; restart <= o.max_restarts; ++restart) {
    // one accuracy for every solve: the projected matrix of the kept vectors is carried over restarts and
    // never recomputed, so a loose early solve would cap the accuracy of every later cycle
    etol = etol_floor;
    if (refined) refine->tol64 = etol;
    if (p == 0) {  // fresh start: v_0 = B x / ||B x||
      std::fill(Gb.begin(), Gb.end(), 0.0);
      FV_TRY(apply_B(x, w.p));
      double xn2;
      FV_TRY(V.dot(w.p, w.p, &xn2));
      const double xn = std::sqrt(xn2);
      if (!(xn > 0.0)) {
        set_error("shift-invert Arnoldi: zero start vector");
        return FV_ENOCONV;
      }
      FV_TRY(V.lin(Vb.p, {{1.0 / xn, w.p}}));
    }
    // ---- expand columns p .. m-1: B v_j = sum_i G[i][j] v_i + G[j+1][j] v_{j+1}
    int mm = m;
    for (int j = p; j < m; ++j) {
      FV_TRY(apply_B(Vb.p + (size_t)j * n, w.p));
      double wn;
      FV_TRY(orthogonalise(w.p, j, j, &wn));
      double colmax = 0.0;
      for (int i = 0; i <= j; ++i) colmax = std::max(colmax, std::fabs(Gb[(size_t)i * m + j]));
      if (wn <= 1e-14 * colmax || wn == 0.0) {
        // the space is invariant under B: continue with a random direction that B does not couple in
        Gb[(size_t)(j + 1) * m + j] = 0.0;
        FV_TRY(launch_fill_normal<R>(g, o.seed + 7919ULL * (unsigned long long)(restart * (m + 1) + j + 1), w.p));
        FV_TRY(project_inplace<R>(g, w.p, 1, 0.0, nullptr, nullptr));
        FV_TRY(orthogonalise(w.p, j, -1, &wn));
        if (!(wn > 0.0)) {
          mm = j + 1;
          break;
        }
      } else {
        Gb[(size_t)(j + 1) * m + j] = wn;
      }
      FV_TRY(V.lin(Vb.p + (size_t)(j + 1) * n, {{1.0 / wn, w.p}}));
    }
    // ---- Ritz values of B: eigenvalues of G (mm x mm)
    Gm.assign((size_t)mm * mm, 0.0);
    for (int i = 0; i < mm; ++i)
      for (int j = 0; j < mm; ++j) Gm[(size_t)i * mm + j] = Gb[(size_t)i * m + j];
    Hg = Gm;
    hessenberg_reduce(mm, Hg, Qg);
    if (!hessenberg_eigvals(mm, Hg.data(), mm, hre, him)) {
      set_error("Hessenberg QR did not converge");
      return FV_ENOCONV;
    }
    struct Mu {
      double re, im;
    };
    std::vector<Mu> mus;
    {
      std::vector<bool> used(mm, false);
      for (int i = 0; i < mm; ++i) {
        if (used[i]) continue;
        used[i] = true;
        if (him[i] == 0.0) {
          mus.push_back({hre[i], 0.0});
          continue;
        }
        int bj = -1;
        double bd = 1e300;
        for (int j2 = 0; j2 < mm; ++j2)
          if (!used[j2] && him[j2] * him[i] < 0.0) {
            const double dd = std::hypot(hre[j2] - hre[i], him[j2] + him[i]);
            if (dd < bd) {
              bd = dd;
              bj = j2;
            }
          }
        if (bj >= 0) {
          used[bj] = true;
          const double r = 0.5 * (hre[i] + hre[bj]), a = 0.5 * (std::fabs(him[i]) + std::fabs(him[bj]));
          mus.push_back({r, a});
        } else {
          mus.push_back({hre[i], std::fabs(him[i])});
        }
      }
    }
    // one entry per real value or conjugate pair (+Im); order by |mu| descending
    std::sort(mus.begin(), mus.end(),
              [](const Mu& a, const Mu& b) { return std::hypot(a.re, a.im) > std::hypot(b.re, b.im); });
    // kept: the largest |mu| filling at most keep_max real slots (a pair takes two)
    std::vector<Mu> kept;
    int slots = 0;
    for (const Mu& u : mus) {
      const int need = u.im != 0.0 ? 2 : 1;
      if (slots + need > keep_max) break;
      kept.push_back(u);
      slots += need;
    }
    if (kept.empty()) kept.push_back(mus[0]);
    // reported: the k (real slots, a pair completed) of largest real part of lam = s + 1/mu among the kept
    auto lam_of = [&](const Mu& u) {
      const std::complex<double> l = s + 1.0 / std::complex<double>(u.re, u.im);
      return l;
    };
    std::vector<int> ord(kept.size());
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return lam_of(kept[a]).real() > lam_of(kept[b]).real(); });
    std::vector<int> rep_idx;
    int rslots = 0;
    for (int i : ord) {
      if (rslots >= k) break;
      rep_idx.push_back(i);
      rslots += kept[i].im != 0.0 ? 2 : 1;
    }
    // ---- eigenvectors of G for the kept values: columns of Y (real, and imaginary part of a pair)
    std::vector<std::vector<double>> Ycols;   // mm each
    std::vector<int> first_col(kept.size());
    for (size_t i = 0; i < kept.size(); ++i) {
      if (!hessenberg_eigvec(mm, Hg.data(), mm, kept[i].re, kept[i].im, sh)) {
        set_error("Ritz vector inverse iteration failed");
        return FV_ENOCONV;
      }
      std::vector<double> yr(mm, 0.0), yi(mm, 0.0);
      for (int r = 0; r < mm; ++r)
        for (int c = 0; c < mm; ++c) {
          yr[r] += Qg[(size_t)r * mm + c] * sh[2 * c];
          yi[r] += Qg[(size_t)r * mm + c] * sh[2 * c + 1];
        }
      first_col[i] = (int)Ycols.size();
      Ycols.push_back(yr);
      if (kept[i].im != 0.0) Ycols.push_back(yi);
    }
    // ---- reported Ritz vectors x = V y into X (slot: Re, then Im of a pair), Rayleigh quotients and
    // true residuals with A
    auto combine = [&](const std::vector<double>& y, R* dst) -> int {
      std::vector<double> c(mm);
      for (int t = 0; t < mm; ++t) c[t] = -y[t];
      FV_CUDA(cudaMemcpyAsync(g->ws.scalars + 1, c.data(), sizeof(double) * mm, cudaMemcpyHostToDevice, g->stream));
      FV_TRY(V.zero(dst));
      FV_TRY(launch_subtract_basis<R>(g, Vb.p, n, mm, g->ws.scalars + 1, dst, n));
      FV_CUDA(cudaStreamSynchronize(g->stream));
      return FV_OK;
    };
    struct Pair {
      double lr, li, res, xn;
      int slot;
    };
    std::vector<Pair> pairs;
    int slot = 0;
    bool all = true;
    double worst = 0.0;
    for (int i : rep_idx) {
      const bool cplx = kept[i].im != 0.0;
      R* xr = X.p + (size_t)slot * n;
      R* xi = cplx ? X.p + (size_t)(slot + 1) * n : nullptr;
      FV_TRY(combine(Ycols[first_col[i]], xr));
      if (cplx) FV_TRY(combine(Ycols[first_col[i] + 1], xi));
      double rr, ii = 0.0, rAr, iAi = 0.0, rAi = 0.0, iAr = 0.0;
      FV_TRY(A.apply(xr, w.p));
      FV_TRY(V.dot(xr, xr, &rr));
      FV_TRY(V.dot(xr, w.p, &rAr));
      if (cplx) {
        FV_TRY(A.apply(xi, y1.p));
        FV_TRY(V.dot(xi, xi, &ii));
        FV_TRY(V.dot(xi, y1.p, &iAi));
        FV_TRY(V.dot(xr, y1.p, &rAi));
        FV_TRY(V.dot(xi, w.p, &iAr));
      }
      // x = xr + i xi: x^H A x = rAr + iAi + i (rAi - iAr)
      const double xn2 = rr + ii;
      double lr = (rAr + iAi) / xn2, li = cplx ? (rAi - iAr) / xn2 : 0.0;
      if (cplx && li < 0.0) {  // the +Im member of the pair is reported first
        li = -li;
        FV_TRY(V.lin(xi, {{-1.0, xi}}));
        FV_TRY(V.lin(y1.p, {{-1.0, y1.p}}));
      }
      double res2, t;
      if (cplx) {  // A xr - (lr xr - li xi), A xi - (lr xi + li xr)
        FV_TRY(V.lin(w.p, {{1.0, w.p}, {-lr, xr}, {li, xi}}));
        FV_TRY(V.dot(w.p, w.p, &res2));
        FV_TRY(V.lin(y1.p, {{1.0, y1.p}, {-lr, xi}, {-li, xr}}));
        FV_TRY(V.dot(y1.p, y1.p, &t));
        res2 += t;
      } else {
        FV_TRY(V.lin(w.p, {{1.0, w.p}, {-lr, xr}}));
        FV_TRY(V.dot(w.p, w.p, &res2));
      }
      const double xn = std::sqrt(xn2), lam = std::hypot(lr, li);
      const double rel = std::sqrt(res2) / (std::max(lam, 1e-300) * std::max(xn, 1e-300));
      pairs.push_back({lr, li, rel, xn, slot});
      if (!(rel <= o.tol)) all = false;
      worst = std::max(worst, rel);
      slot += cplx ? 2 : 1;
    }
    rep->restarts = restart;
    if (worst <= 0.5 * best) {
      best = worst;
      best_at = restart;
    }
    const bool stalled = stall > 0 && restart - best_at >= stall;
    if (all || mm < m || restart == o.max_restarts || stalled) {
      status = all ? FV_OK : FV_ENOCONV;
      // order by real part (then |Im|), +Im first; unit-norm vectors in that order into vecs_out
      std::vector<int> po(pairs.size());
      std::iota(po.begin(), po.end(), 0);
      std::sort(po.begin(), po.end(), [&](int a, int b) {
        if (pairs[a].lr != pairs[b].lr) return pairs[a].lr > pairs[b].lr;
        return pairs[a].li > pairs[b].li;
      });
      int out = 0;
      for (int pi : po) {
        const Pair& pr = pairs[pi];
        const int cnt = pr.li != 0.0 ? 2 : 1;
        for (int c = 0; c < cnt && out < 64; ++c, ++out) {
          re[out] = pr.lr;
          im[out] = c == 0 ? pr.li : -pr.li;
          rep->residual[out] = pr.res;
          if (vecs_out) {
            R* dst = (R*)vecs_out + (size_t)out * n;
            FV_TRY(V.zero(dst));
            FV_TRY(V.lin(dst, {{1.0 / std::max(pr.xn, 1e-300), X.p + (size_t)(pr.slot + c) * n}}));
          }
        }
      }
      nret = out;
      FV_CUDA(cudaStreamSynchronize(g->stream));
      break;
    }
    // ---- thick restart: orthonormalise the kept eigenvector columns Y (coefficient space, MGS twice)
    std::vector<std::vector<double>> Qy;
    for (const auto& y : Ycols) {
      std::vector<double> v = y;
      const double n0 = std::sqrt(std::inner_product(v.begin(), v.end(), v.begin(), 0.0));
      for (int pass = 0; pass < 2; ++pass)
        for (const auto& u : Qy) {
          const double d = std::inner_product(u.begin(), u.end(), v.begin(), 0.0);
          for (int t = 0; t < mm; ++t) v[t] -= d * u[t];
        }
      const double nv = std::sqrt(std::inner_product(v.begin(), v.end(), v.begin(), 0.0));
      if (!(nv > 1e-10 * n0)) continue;
      for (double& e : v) e /= nv;
      Qy.push_back(v);
    }
    const int pn = (int)Qy.size();
    if (pn == 0 || pn >= m) {  // nothing to keep: a fresh start from the leading reported Ritz vector
      FV_TRY(V.copy(y0.p, X.p));
      x = y0.p;
      p = 0;
      continue;
    }
    // new leading vectors V Q_y (into X, free by now, then into Vb), v_m moved to position p
    for (int c = 0; c < pn; ++c) FV_TRY(combine(Qy[c], X.p + (size_t)c * n));
    FV_TRY(V.copy(Vb.p + (size_t)pn * n, Vb.p + (size_t)mm * n));
    for (int c = 0; c < pn; ++c) FV_TRY(V.copy(Vb.p + (size_t)c * n, X.p + (size_t)c * n));
    // projected matrix: Q_y^T G Q_y, and the row g^T Q_y of v_m (g = G[mm][.], nonzero at mm-1 only)
    std::vector<double> GQ((size_t)mm * pn, 0.0);
    for (int r = 0; r < mm; ++r)
      for (int c = 0; c < pn; ++c) {
        double acc = 0.0;
        for (int t = 0; t < mm; ++t) acc += Gm[(size_t)r * mm + t] * Qy[c][t];
        GQ[(size_t)r * pn + c] = acc;
      }
    const double gmm = Gb[(size_t)mm * m + (mm - 1)];
    std::fill(Gb.begin(), Gb.end(), 0.0);
    for (int r = 0; r < pn; ++r)
      for (int c = 0; c < pn; ++c) {
        double acc = 0.0;
        for (int t = 0; t < mm; ++t) acc += Qy[r][t] * GQ[(size_t)t * pn + c];
        Gb[(size_t)r * m + c] = acc;
      }
    for (int c = 0; c < pn; ++c) Gb[(size_t)pn * m + c] = gmm * Qy[c][mm - 1];
    p = pn;
  }
  rep->matvecs = mv + (refined ? refine->mv32 : 0);
  rep->matvecs_fp64 = mixed ? 0 : mv;
  rep->solves = sstats.solves;
  rep->solves_short = sstats.short_;
  rep->solve_worst = sstats.worst;
  rep->nconv = nret;
  rep->status = status;
  for (int i = 0; i < nret && i < 64; ++i) {
    const double sc = Gr > 0.0 ? 1.0 / std::sqrt(Gr) : 0.0;
    rep->lam_scaled_re[i] = re[i] * sc;
    rep->lam_scaled_im[i] = im[i] * sc;
  }
  rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  return status;
}

template <typename R>
static int arnoldi_impl(fv_grid_s* g, int k, double Gr, const double* q64, const fv_arnoldi_opts& o, double* re,
                        double* im, void* vecs_out, fv_arnoldi_report* rep, const R* start = nullptr,
                        ArnoldiCarry* carry = nullptr, int stall = 0, EulerRefine* refine = nullptr) {
  if (o.euler_dt > 0.0) return arnoldi_si<R>(g, k, Gr, q64, o, re, im, vecs_out, rep, start, stall, refine);
  const auto t_start = std::chrono::steady_clock::now();
  const size_t n = 4 * g->N;
  const int m = o.m;
  const bool mixed = !std::is_same<R, double>::value;
  const double sigma = (o.sigma != 0.0) ? o.sigma : g->sigma_default;
  DevBuf<R> qR, Vb, w, y0, y1, X;
  if (mixed) {
    FV_TRY(qR.alloc(n));
    FV_TRY(launch_convert(g, n, q64, (float*)qR.p));
  }
  const R* q = mixed ? qR.p : (const R*)q64;
  FV_TRY(Vb.alloc((size_t)(m + 1) * n));
  FV_TRY(w.alloc(n));
  FV_TRY(y0.alloc(n));
  FV_TRY(y1.alloc(n));
  FV_TRY(X.alloc((size_t)(std::min(k, m) + 2) * n));  // wanted Ritz vectors: real and imaginary parts
  Vec<R> V{g, n};
  long long mv = 0;
  Operator<R> A{g, Gr, sigma, q, &mv};
  // start vector: seeded N(0,1) (or the caller's), projected
  R* x = y0.p;
  if (start) {
    FV_TRY(V.copy(x, start));
  } else {
    FV_TRY(launch_fill_normal<R>(g, o.seed, x));
  }
  FV_TRY(project_inplace<R>(g, x, 1, 0.0, nullptr, nullptr));
  // far end of the spectrum: Rayleigh quotient of a short power iteration (the Krylov spaces of B stop
  // showing it, and the Chebyshev polynomial grows fast outside its ellipse)
  double lam_far = (carry && carry->lam_far != 0.0) ? carry->lam_far : 0.0;
  if (lam_far == 0.0) {
    R* z = y1.p;
    double zn2;
    FV_TRY(V.dot(x, x, &zn2));
    FV_TRY(V.lin(z, {{1.0 / std::sqrt(zn2), x}}));
    for (int it = 0; it < 30; ++it) {
      FV_TRY(A.apply(z, w.p));
      FV_TRY(V.dot(z, w.p, &lam_far));
      double wn2;
      FV_TRY(V.dot(w.p, w.p, &wn2));
      FV_TRY(V.lin(z, {{1.0 / std::sqrt(wn2), w.p}}));
    }
  }
  ChebFilter filt = carry ? carry->filt : ChebFilter{};

  // out = p(A) in by the three-term recurrence
  //   y_1 = tau_1 (A - d) y_0,  y_{j+1} = 2 tau_{j+1} (A - d) y_j - c^2 tau_j tau_{j+1} y_{j-1},
  //   tau_1 = 1 / (lam_ref - d),  tau_{j+1} = 1 / (2 (lam_ref - d) - c^2 tau_j);
  // y0, y1 are scratch, the input is only read.
  auto apply_filter = [&](const R* in, R* out) -> int {
    const double s = filt.lam_ref - filt.d;
    double tau = 1.0 / s;
    FV_TRY(chebyshev_step<R>(g, Gr, sigma, q, in, nullptr, tau, tau * (sigma - filt.d), 0.0, y0.p));
    ++mv;
    const R* yp = in;
    R* yc = y0.p;
    // range check of the recurrence every `chk` steps on the norm its correction pass sums (FP32 data
    // overflows near 3e38: a polynomial that amplifies an outlier strongly can get there within 16 steps)
    const int chk = std::is_same<R, double>::value ? 16 : 4;
    const double big = std::is_same<R, double>::value ? 1e30 : 1e15;
    for (int j = 1; j < filt.deg; ++j) {
      const double tn = 1.0 / (2.0 * s - filt.c2 * tau);
      R* dst = (yp == in) ? y1.p : const_cast<R*>(yp);  // y_{j+1} overwrites y_{j-1} (never the input)
      const bool check = (j % chk == 0);
      FV_TRY(chebyshev_step<R>(g, Gr, sigma, q, yc, yp, 2.0 * tn, 2.0 * tn * (sigma - filt.d), -filt.c2 * tau * tn,
                               dst, check ? 0 : -1));
      ++mv;
      yp = yc;
      yc = dst;
      tau = tn;
      if (check) {  // keep both terms of the recurrence in range (yp is scratch by now)
        double nn;
        FV_TRY(read_scalars(g, 0, 1, &nn));
        if (!std::isfinite(nn)) {
          set_error("non-finite Chebyshev recurrence");
          return FV_ENAN;
        }
        nn = std::sqrt(nn);
        if (nn > big || nn < 1.0 / big) {
          FV_TRY(V.lin(yc, {{1.0 / nn, yc}}));
          FV_TRY(V.lin(const_cast<R*>(yp), {{1.0 / nn, yp}}));
        }
      }
    }
    return V.copy(out, yc);
  };

  std::vector<double> H((size_t)(m + 1) * m), h(m + 1), G, Hg, Qg, hre, him, ycoef, sh;
  std::vector<std::vector<double>> Y;
  std::vector<Ritz> ritz;
  int status = FV_ENOCONV, nret = 0;
  double best = 1e300;
  int best_at = 0;
  for (int restart = 0; restart <= o.max_restarts; ++restart) {
    // ---- m Arnoldi steps (CGS2) on A (first cycle) or on B = p(A) from p(A) x: the restart vector's error
    // in the stiff directions would otherwise sit in v_1 alone, where no later Krylov vector of B (which
    // damps those directions) can cancel it, and every Ritz vector would inherit it
    if (filt.on) {
      FV_TRY(V.copy(Vb.p, x));
      FV_TRY(apply_filter(Vb.p, w.p));
      x = w.p;
    }
    double xn2;
    FV_TRY(V.dot(x, x, &xn2));
    FV_TRY(V.lin(Vb.p, {{1.0 / std::sqrt(xn2), x}}));
    std::fill(H.begin(), H.end(), 0.0);
    int mm = m;
    for (int j = 0; j < m; ++j) {
      const R* vj = Vb.p + (size_t)j * n;
      if (filt.on)
        FV_TRY(apply_filter(vj, w.p));
      else
        FV_TRY(A.apply(vj, w.p));
      for (int pass = 0; pass < 2; ++pass) {
        FV_TRY(launch_multidot<R>(g, Vb.p, n, j + 1, w.p, n, 1));
        FV_TRY(launch_subtract_basis<R>(g, Vb.p, n, j + 1, g->ws.scalars + 1, w.p, n));
        FV_TRY(read_scalars(g, 1, j + 1, h.data()));
        for (int i = 0; i <= j; ++i) {
          if (!std::isfinite(h[i])) {
            set_error("non-finite Gram-Schmidt coefficient");
            return FV_ENAN;
          }
          H[(size_t)i * m + j] += h[i];
        }
      }
      double wn2;
      FV_TRY(V.dot(w.p, w.p, &wn2));
      const double wn = std::sqrt(wn2);
      H[(size_t)(j + 1) * m + j] = wn;
      if (wn <= 1e-14 * std::fabs(H[(size_t)j * m + j]) || wn == 0.0) {
        mm = j + 1;
        break;
      }
      FV_TRY(V.lin(Vb.p + (size_t)(j + 1) * n, {{1.0 / wn, w.p}}));
    }
    // ---- Rayleigh-Ritz matrix G = V^T A V (for a Krylov basis of A it is the Hessenberg matrix itself)
    G.assign((size_t)mm * mm, 0.0);
    if (!filt.on) {
      for (int i = 0; i < mm; ++i)
        for (int j = 0; j < mm; ++j) G[(size_t)i * mm + j] = H[(size_t)i * m + j];
    } else {
      for (int j = 0; j < mm; ++j) {
        FV_TRY(A.apply(Vb.p + (size_t)j * n, w.p));
        FV_TRY(launch_multidot<R>(g, Vb.p, n, mm, w.p, n, 1));
        FV_TRY(read_scalars(g, 1, mm, h.data()));
        for (int i = 0; i < mm; ++i) {
          if (!std::isfinite(h[i])) {
            set_error("non-finite Rayleigh-Ritz entry");
            return FV_ENAN;
          }
          G[(size_t)i * mm + j] = h[i];
        }
      }
    }
    Hg = G;
    hessenberg_reduce(mm, Hg, Qg);
    if (!hessenberg_eigvals(mm, Hg.data(), mm, hre, him)) {
      set_error("Hessenberg QR did not converge");
      return FV_ENOCONV;
    }
    // G is real: pair each +Im value with its nearest -Im partner and make the pair exact mirrors
    // (the complex QR returns them with slightly different real parts), then sort (+Im first)
    ritz.clear();
    {
      std::vector<bool> used(mm, false);
      for (int i = 0; i < mm; ++i) {
        if (used[i]) continue;
        used[i] = true;
        if (him[i] == 0.0) {
          ritz.push_back({hre[i], 0.0});
          continue;
        }
        int bj = -1;
        double bd = 1e300;
        for (int j2 = 0; j2 < mm; ++j2)
          if (!used[j2] && him[j2] * him[i] < 0.0) {
            const double dd = std::hypot(hre[j2] - hre[i], him[j2] + him[i]);
            if (dd < bd) {
              bd = dd;
              bj = j2;
            }
          }
        if (bj >= 0) {
          used[bj] = true;
          const double r = 0.5 * (hre[i] + hre[bj]), a = 0.5 * (std::fabs(him[i]) + std::fabs(him[bj]));
          ritz.push_back({r, a});
          ritz.push_back({r, -a});
        } else {
          ritz.push_back({hre[i], him[i]});
        }
      }
    }
    std::sort(ritz.begin(), ritz.end(), ritz_before);
    int nw = std::min(k, mm);
    if (nw < mm && ritz[nw - 1].im > 0) ++nw;
    // ---- wanted Ritz vectors: eigenvectors s of G (= Qg times those of its Hessenberg form), X = V s;
    // slot i holds Re x (real value or +Im member), slot i + 1 Im x for a conjugate pair
    Y.assign(nw, {});
    for (int i = 0; i < nw; ++i) {
      if (!hessenberg_eigvec(mm, Hg.data(), mm, ritz[i].re, std::fabs(ritz[i].im), sh)) {
        set_error("Ritz vector inverse iteration failed");
        return FV_ENOCONV;
      }
      Y[i].assign(2 * (size_t)mm, 0.0);
      for (int r = 0; r < mm; ++r)
        for (int c = 0; c < mm; ++c) {
          Y[i][2 * r] += Qg[(size_t)r * mm + c] * sh[2 * c];
          Y[i][2 * r + 1] += Qg[(size_t)r * mm + c] * sh[2 * c + 1];
        }
    }
    ycoef.assign(mm, 0.0);
    for (int i = 0; i < nw; ++i) {
      const bool cplx = ritz[i].im != 0.0;
      for (int part = 0; part < (cplx ? 2 : 1); ++part) {
        const int slot = i + part;
        if (slot >= nw) break;
        for (int t = 0; t < mm; ++t) ycoef[t] = -Y[i][2 * t + part];
        FV_CUDA(cudaMemcpyAsync(g->ws.scalars + 1, ycoef.data(), sizeof(double) * mm, cudaMemcpyHostToDevice,
                                g->stream));
        R* xs = X.p + (size_t)slot * n;
        FV_TRY(V.zero(xs));
        FV_TRY(launch_subtract_basis<R>(g, Vb.p, n, mm, g->ws.scalars + 1, xs, n));
        FV_CUDA(cudaStreamSynchronize(g->stream));
      }
      if (cplx) ++i;
    }
    // ---- true residuals ||A x - lam x|| / (|lam| ||x||), FP64 reductions
    bool all = true;
    double worst = 0.0;
    std::vector<double> xnorm(nw, 1.0);
    for (int i = 0; i < nw; ++i) {
      const bool cplx = ritz[i].im != 0.0;
      const double lr = ritz[i].re, li = ritz[i].im;
      R* xr = X.p + (size_t)i * n;
      R* xi = (cplx && i + 1 < nw) ? X.p + (size_t)(i + 1) * n : nullptr;
      double nr2 = 0.0, ni2 = 0.0, res2 = 0.0, t;
      FV_TRY(V.dot(xr, xr, &nr2));
      FV_TRY(A.apply(xr, w.p));  // A xr - (lr xr - li xi)
      if (xi) {
        FV_TRY(V.dot(xi, xi, &ni2));
        FV_TRY(V.lin(w.p, {{1.0, w.p}, {-lr, xr}, {li, xi}}));
      } else {
        FV_TRY(V.lin(w.p, {{1.0, w.p}, {-lr, xr}}));
      }
      FV_TRY(V.dot(w.p, w.p, &t));
      res2 += t;
      if (xi) {
        FV_TRY(A.apply(xi, w.p));  // A xi - (lr xi + li xr)
        FV_TRY(V.lin(w.p, {{1.0, w.p}, {-lr, xi}, {-li, xr}}));
        FV_TRY(V.dot(w.p, w.p, &t));
        res2 += t;
      }
      const double xn = std::sqrt(nr2 + ni2), lam = std::hypot(lr, li);
      const double rel = std::sqrt(res2) / (std::max(lam, 1e-300) * std::max(xn, 1e-300));
      re[i] = lr;
      im[i] = li;
      if (i < 64) rep->residual[i] = rel;
      xnorm[i] = xn;
      if (xi) {
        re[i + 1] = lr;
        im[i + 1] = -li;
        if (i + 1 < 64) rep->residual[i + 1] = rel;
        xnorm[i + 1] = xn;
      }
      if (!(rel <= o.tol)) all = false;
      worst = std::max(worst, rel);
      if (cplx) ++i;
    }
    rep->restarts = restart;
    if (worst <= 0.5 * best) {
      best = worst;
      best_at = restart;
    }
    const bool stalled = stall > 0 && restart - best_at >= stall;
    if (all || mm < m || restart == o.max_restarts || stalled) {
      status = all || mm < m ? FV_OK : FV_ENOCONV;
      nret = nw;
      // unit norm of each (complex) vector
      for (int i = 0; i < nw; ++i) FV_TRY(V.lin(X.p + (size_t)i * n, {{1.0 / std::max(xnorm[i], 1e-300), X.p + (size_t)i * n}}));
      if (vecs_out)
        FV_CUDA(cudaMemcpyAsync(vecs_out, X.p, sizeof(R) * n * nw, cudaMemcpyDeviceToDevice, g->stream));
      FV_CUDA(cudaStreamSynchronize(g->stream));
      break;
    }
    // ---- next ellipse: wanted + guard Ritz values outside, the rest and the far end inside
    int nf = std::min(nw + o.guard, mm - 2);
    if (nf < mm && nf >= 1 && ritz[nf - 1].im > 0) ++nf;
    nf = std::max(nf, nw);
    std::vector<Ritz> wanted(ritz.begin(), ritz.begin() + nf), unwanted(ritz.begin() + nf, ritz.end());
    double left = lam_far;
    for (auto& u : unwanted) left = std::min(left, u.re);
    unwanted.push_back({1.05 * left, 0.0});
    double d = 0, c2 = 0, rate = 0;
    best_ellipse(wanted, unwanted, d, c2, rate);
    int deg = o.max_degree;
    if (rate > 1.0) deg = (int)std::ceil(std::log(kFilterGain) / std::log(rate));
    deg = std::max(o.min_degree, std::min(o.max_degree, deg));
    if (restart < 256) rep->degrees[restart] = deg;
    double lam_ref = -1e300;
    for (auto& wv : wanted) lam_ref = std::max(lam_ref, wv.re);
    filt = ChebFilter{true, d, c2, lam_ref, deg};
    // ---- next start: sum of the normalised wanted Ritz vectors + a divergence-free random component (a mode
    // the start lacked is then present in the Krylov space of B; the noise stays below the tolerance)
    R* z = y0.p;
    FV_TRY(V.zero(z));
    for (int i = 0; i < nw; ++i) {
      double t2;
      FV_TRY(V.dot(X.p + (size_t)i * n, X.p + (size_t)i * n, &t2));
      if (t2 > 0.0) FV_TRY(V.lin(z, {{1.0, z}, {1.0 / std::sqrt(t2), X.p + (size_t)i * n}}));
    }
    {
      double zn2, rn2;
      FV_TRY(launch_fill_normal<R>(g, o.seed + 1000003ULL * (unsigned long long)(restart + 1), w.p));
      FV_TRY(project_inplace<R>(g, w.p, 1, 0.0, nullptr, nullptr));
      FV_TRY(V.dot(z, z, &zn2));
      FV_TRY(V.dot(w.p, w.p, &rn2));
      FV_TRY(V.lin(z, {{1.0, z}, {0.01 * o.tol * std::sqrt(zn2 / std::max(rn2, 1e-300)), w.p}}));
    }
    x = z;
  }
  if (carry) {
    carry->lam_far = lam_far;
    carry->filt = filt;
  }
  rep->matvecs = mv;
  rep->nconv = nret;
  rep->status = status;
  for (int i = 0; i < nret && i < 64; ++i) {
    const double sc = Gr > 0.0 ? 1.0 / std::sqrt(Gr) : 0.0;
    rep->lam_scaled_re[i] = re[i] * sc;
    rep->lam_scaled_im[i] = im[i] * sc;
  }
  rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  return status;
}

}  // namespace fv

namespace fv {

// Mixed precision: FP32 Krylov vectors and J.v + projection until the Ritz residuals reach low_tol or stop
// improving (with FP32 matvecs the residual floor is ~ u_32 ||A|| / |lam|, far above 1e-6 for the small
// leading eigenvalues of this stiff operator), then FP64 cycles started from the sum of the FP32 Ritz
// vectors, under the last FP32 ellipse, refine the same pairs to tol.
static int arnoldi_mixed(fv_grid_s* g, int k, double Gr, const double* q, const fv_arnoldi_opts& o, double* re,
                         double* im, void* vecs_out, fv_arnoldi_report* rep) {
  const auto t0 = std::chrono::steady_clock::now();
  const size_t n = 4 * g->N;
  DevBuf<float> X32;
  DevBuf<double> z64, t64, X64;
  FV_TRY(X32.alloc((size_t)(k + 2) * n));
  fv_arnoldi_opts o1 = o;
  o1.tol = std::max(o.tol, o.low_tol);
  o1.max_restarts = std::max(0, std::min(o.max_restarts, o.low_max_restarts));
  fv_arnoldi_report r1;
  std::memset(&r1, 0, sizeof(r1));
  ArnoldiCarry carry;
  int st1 = arnoldi_impl<float>(g, k, Gr, q, o1, re, im, X32.p, &r1, nullptr, &carry, 3);
  if (st1 != FV_OK && st1 != FV_ENOCONV) return st1;
  FV_TRY(z64.alloc(n));
  FV_TRY(t64.alloc(n));
  Vec<double> V{g, n};
  FV_TRY(V.zero(z64.p));
  for (int i = 0; i < r1.nconv; ++i) {
    FV_TRY(launch_convert(g, n, X32.p + (size_t)i * n, t64.p));
    FV_TRY(project_inplace<double>(g, t64.p, 1, 0.0, nullptr, nullptr));
    double t2;
    FV_TRY(V.dot(t64.p, t64.p, &t2));
    if (t2 > 0.0) FV_TRY(V.lin(z64.p, {{1.0, z64.p}, {1.0 / std::sqrt(t2), t64.p}}));
  }
  fv_arnoldi_report r2;
  std::memset(&r2, 0, sizeof(r2));
  if (vecs_out) FV_TRY(X64.alloc((size_t)(k + 1) * n));
  fv_arnoldi_opts o2 = o;
  o2.precision = FV_FP64;
  // implicit-Euler transform: the FP64 cycles' shifted solves by iterative refinement around FP32 GMRES
  EulerRefine ref;
  DevBuf<float> q32, b32, x32, pre32, basis32, w32;
  DevBuf<double> r64, u64;
  const bool euler = o.euler_dt > 0.0;
  if (euler) {
    FV_TRY(q32.alloc(n));
    FV_TRY(b32.alloc(n));
    FV_TRY(x32.alloc(n));
    FV_TRY(pre32.alloc(n));
    FV_TRY(basis32.alloc((size_t)(o.inner_m + 1) * n));
    FV_TRY(w32.alloc(n));
    FV_TRY(r64.alloc(n));
    FV_TRY(u64.alloc(n));
    FV_TRY(launch_convert(g, n, q, q32.p));
    ref.g = g;
    ref.Gr = Gr;
    ref.sigma = (o.sigma != 0.0) ? o.sigma : g->sigma_default;
    ref.s = 1.0 / o.euler_dt;
    ref.q32 = q32.p;
    ref.q64 = q;
    ref.b32 = b32.p;
    ref.x32 = x32.p;
    ref.pre32 = pre32.p;
    ref.basis32 = basis32.p;
    ref.w32 = w32.p;
    ref.r64 = r64.p;
    ref.t64 = u64.p;
    ref.inner_m = o.inner_m;
    ref.inner_max = o.inner_max;
    ref.tol32 = 1e-3;
    ref.tol64 = o.inner_tol > 0.0 ? o.inner_tol : 1e-9;
  }
  const int st = arnoldi_impl<double>(g, k, Gr, q, o2, re, im, vecs_out ? X64.p : nullptr, &r2, z64.p, &carry, 0,
                                      euler ? &ref : nullptr);
  if (vecs_out && (st == FV_OK || st == FV_ENOCONV)) {
    if (o.vecs_fp64)
      FV_CUDA(cudaMemcpyAsync(vecs_out, X64.p, sizeof(double) * n * r2.nconv, cudaMemcpyDeviceToDevice, g->stream));
    else
      for (int i = 0; i < r2.nconv; ++i)
        FV_TRY(launch_convert(g, n, X64.p + (size_t)i * n, (float*)vecs_out + (size_t)i * n));
  }
  *rep = r2;
  rep->restarts_low = r1.restarts;
  rep->matvecs_low = r1.matvecs;
  rep->restarts = r1.restarts + r2.restarts;
  rep->matvecs = r1.matvecs + r2.matvecs;
  rep->solves = r1.solves + r2.solves;
  rep->solves_short = r1.solves_short + r2.solves_short;
  rep->solve_worst = std::max(r1.solve_worst, r2.solve_worst);
  for (int i = 0; i < 256; ++i) rep->degrees[i] = (i <= r1.restarts) ? r1.degrees[i] : r2.degrees[i - r1.restarts - 1];
  FV_CUDA(cudaStreamSynchronize(g->stream));
  rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return st;
}

}  // namespace fv

extern "C" int arnoldi_leading(fv_grid g, int k, double Gr, const double* q, const fv_arnoldi_opts* opts, double* re,
                               double* im, void* vecs, fv_arnoldi_report* report) {
  if (!g || !q || !re || !im) return invalid("null argument");
  fv_arnoldi_opts o;
  if (opts)
    o = *opts;
  else
    fv_arnoldi_default_opts(&o);
  if (k < 1 || o.m > 200 || k + o.guard + 2 > o.m || o.min_degree < 1 || o.max_degree < o.min_degree ||
      o.max_restarts < 0 || k > 63 || (o.precision == FV_FP32 && !(o.low_tol > 0.0)) || !(o.euler_dt >= 0.0) ||
      (o.euler_dt > 0.0 && (o.inner_m < 1 || o.inner_m > 500 || o.inner_max < 2 || !(o.inner_tol >= 0.0))) ||
      o.vecs_fp64 < 0 || o.vecs_fp64 > 1)
    return invalid("bad Arnoldi options (need 1 <= k <= 63, k + guard + 2 <= m <= 200)");
  if (o.precision != FV_FP64 && o.precision != FV_FP32) return invalid("precision must be FV_FP64 or FV_FP32");
  fv_arnoldi_report rep;
  std::memset(&rep, 0, sizeof(rep));
  int st;
  if (o.precision == FV_FP64) {
    st = arnoldi_impl<double>(g, k, Gr, q, o, re, im, vecs, &rep);
  } else {
    st = arnoldi_mixed(g, k, Gr, q, o, re, im, vecs, &rep);
  }
  rep.status = st;
  if (report) *report = rep;
  return st;
}

// ====================================================================== critical Gr (Section 4.1)
namespace fv {

// The tracked eigenvalue among the returned ones: largest real part overall, among the real values, or
// among the complex pairs (+Im member).  false if the mode has no representative.
static bool pick_mode(int mode, int nconv, const double* re, const double* im, double* lr, double* li) {
  bool found = false;
  for (int i = 0; i < nconv; ++i) {
    const bool cplx = im[i] != 0.0;
    if (mode == FV_MODE_REAL && cplx) continue;
    if (mode == FV_MODE_OSCILLATORY && (!cplx || im[i] < 0.0)) continue;
    if (!found || re[i] > *lr) {
      *lr = re[i];
      *li = std::fabs(im[i]);
      found = true;
    }
  }
  return found;
}

}  // namespace fv

extern "C" void fv_critical_default_opts(fv_critical_opts* o) {
  if (!o) return;
  o->gr_a = 0.0;
  o->gr_b = 0.0;
  o->tol = 1e-7;
  o->max_iter = 16;
  o->mode = FV_MODE_LEADING;
}

namespace fv {

// The root iteration on Re lam(Gr) (Section 4.1): secant steps, each limited to twice the last spacing,
// until a sign change brackets the crossing, then false position with the Illinois halving of an end
// that is retained twice in a row.  eval(gr, &re, &im) returns a status and the tracked eigenvalue; the
// report keeps every successful evaluation and ends at the last one (gr_cr).  Returns the report's status.
template <typename Eval>
static int critical_root(const fv_critical_opts& c, Eval&& eval, fv_critical_report* rep) {
  std::memset(rep, 0, sizeof(*rep));
  rep->status = FV_ENOCONV;
  double x = 0.0, fx = 0.0, ix = 0.0;  // the last successful evaluation
  auto evaluate = [&](double gr, double* lr, double* li) -> int {
    const int st = eval(gr, lr, li);
    if (st != FV_OK) return st;
    if (!std::isfinite(*lr) || !std::isfinite(*li)) {
      set_error("critical Gr: non-finite tracked eigenvalue at Gr = " + std::to_string(gr));
      return FV_ENAN;
    }
    if (rep->evaluations < 40) {
      rep->gr[rep->evaluations] = gr;
      rep->re[rep->evaluations] = *lr;
      rep->im[rep->evaluations] = *li;
    }
    ++rep->evaluations;
    x = gr;
    fx = *lr;
    ix = *li;
    return FV_OK;
  };
  double fa = 0.0, ia = 0.0, fb = 0.0, ib = 0.0;
  double a = c.gr_a, b = c.gr_b;
  int st = evaluate(a, &fa, &ia);
  if (st == FV_OK) st = evaluate(b, &fb, &ib);
  int side = 0;  // Illinois: which end was kept last time (-1: a)
  bool bracketed = st == FV_OK && fa * fb <= 0.0;
  for (int it = 0; st == FV_OK && it < c.max_iter; ++it) {
    if (fb == fa) break;
    double xn = b - fb * (b - a) / (fb - fa);
    if (!bracketed) {  // secant: keep the step within twice the current spacing
      const double lim = 2.0 * std::fabs(b - a);
      xn = std::min(std::max(xn, b - lim), b + lim);
    }
    if (!(xn > 0.0)) xn = 0.5 * std::min(a, b);
    double fn, in;
    st = evaluate(xn, &fn, &in);
    if (st != FV_OK) break;
    const bool done = std::fabs(xn - b) <= c.tol * std::fabs(b) || fn == 0.0;
    // b is always the newest point; once a sign change is seen, a and b keep opposite signs
    if (!bracketed && fn * fa < 0.0 && fn * fb > 0.0) {
      bracketed = true;  // the crossing lies between a and xn: keep a
      b = xn;
      fb = fn;
    } else if (!bracketed && fn * fb < 0.0) {
      bracketed = true;  // between b and xn
      a = b;
      fa = fb;
      b = xn;
      fb = fn;
      side = 0;
    } else if (!bracketed) {  // secant step
      a = b;
      fa = fb;
      b = xn;
      fb = fn;
    } else if (fn * fb < 0.0) {  // false position: the newest end changed sign, the old b becomes a
      a = b;
      fa = fb;
      b = xn;
      fb = fn;
      side = 0;
    } else {  // a is retained again: Illinois halves its value so that it is not retained forever
      if (side == -1) fa *= 0.5;
      side = -1;
      b = xn;
      fb = fn;
    }
    if (done) {
      rep->status = FV_OK;
      break;
    }
  }
  if (rep->evaluations > 0) {
    rep->gr_cr = x;
    rep->lam_re = fx;
    rep->lam_im = ix;
    rep->omega_scaled = ix / std::sqrt(x);
  }
  if (st != FV_OK) rep->status = st;
  return rep->status;
}

static bool critical_opts_ok(const fv_critical_opts& c) {
  return c.gr_a > 0.0 && c.gr_b > 0.0 && c.gr_a != c.gr_b && c.tol > 0.0 && c.max_iter >= 0 && c.max_iter <= 38;
}

}  // namespace fv

extern "C" int fv_critical_gr(fv_grid g, int k, double* q_inout, const fv_newton_opts* nopts,
                              const fv_arnoldi_opts* aopts, const fv_critical_opts* copts, fv_critical_report* report) {
  if (!g || !q_inout || !copts) return invalid("null argument");
  const fv_critical_opts c = *copts;
  if (!critical_opts_ok(c) || c.mode < FV_MODE_LEADING || c.mode > FV_MODE_OSCILLATORY || k < 1 || k > 62)
    return invalid("bad critical-Gr options (need distinct gr_a, gr_b > 0, tol > 0, 0 <= max_iter <= 38)");
  fv_newton_opts no;
  if (nopts)
    no = *nopts;
  else
    fv_newton_default_opts(&no);
  no.gr_start = 0.0;  // every evaluation continues from the nearest state already computed
  fv_arnoldi_opts ao;
  if (aopts)
    ao = *aopts;
  else
    fv_arnoldi_default_opts(&ao);
  const size_t n = 4 * g->N;
  // states of the evaluations so far: a Newton start for the next Gr is the one of the nearest Gr
  std::vector<DevBuf<double>> states(c.max_iter + 2);
  std::vector<double> grs;
  std::vector<double> re(k + 1), im(k + 1);
  Vec<double> V{g, n};
  auto evaluate = [&](double gr, double* lr, double* li) -> int {
    const int idx = (int)grs.size();
    FV_TRY(states[idx].alloc(n));
    if (idx == 0) {
      FV_TRY(V.copy(states[idx].p, q_inout));
    } else {
      int near = 0;
      for (int i = 1; i < idx; ++i)
        if (std::fabs(std::log(grs[i] / gr)) < std::fabs(std::log(grs[near] / gr))) near = i;
      FV_TRY(V.copy(states[idx].p, states[near].p));
    }
    fv_newton_report nr;
    int st = newton_steady(g, gr, states[idx].p, &no, &nr);
    if (st != FV_OK) {
      set_error("critical Gr: Newton did not converge at Gr = " + std::to_string(gr));
      return st == FV_ENOCONV ? FV_ENOCONV : st;
    }
    fv_arnoldi_report ar;
    st = arnoldi_leading(g, k, gr, states[idx].p, &ao, re.data(), im.data(), nullptr, &ar);
    if (st != FV_OK && st != FV_ENOCONV) return st;
    if (!pick_mode(c.mode, ar.nconv, re.data(), im.data(), lr, li)) {
      set_error("critical Gr: no eigenvalue of the tracked kind among the k computed at Gr = " +
                std::to_string(gr) + " (raise k)");
      return FV_ENOCONV;
    }
    grs.push_back(gr);
    return FV_OK;
  };
  fv_critical_report rep;
  critical_root(c, evaluate, &rep);
  if (rep.evaluations > 0) {  // the steady state of the last successful evaluation
    FV_CUDA(cudaMemcpyAsync(q_inout, states[rep.evaluations - 1].p, sizeof(double) * n, cudaMemcpyDeviceToDevice,
                            g->stream));
    FV_CUDA(cudaStreamSynchronize(g->stream));
  }
  if (report) *report = rep;
  return rep.status;
}

extern "C" int fv_critical_root(const fv_critical_opts* copts, fv_tracked_fn f, void* ctx,
                                fv_critical_report* report) {
  if (!copts || !f) return invalid("null argument");
  if (!critical_opts_ok(*copts))
    return invalid("bad critical-Gr options (need distinct gr_a, gr_b > 0, tol > 0, 0 <= max_iter <= 38)");
  fv_critical_report rep;
  critical_root(*copts, [&](double gr, double* lr, double* li) -> int { return f(gr, ctx, lr, li); }, &rep);
  if (report) *report = rep;
  return rep.status;
}

extern "C" int fv_richardson(int n, const double* h2, const double* value, double* limit, double* slope) {
  if (n < 2 || !h2 || !value) return invalid("need n >= 2 points");
  double sx = 0.0, sy = 0.0, sxx = 0.0, sxy = 0.0;
  for (int i = 0; i < n; ++i) {
    sx += h2[i];
    sy += value[i];
    sxx += h2[i] * h2[i];
    sxy += h2[i] * value[i];
  }
  const double det = n * sxx - sx * sx;
  if (!(std::fabs(det) > 1e-300)) return invalid("the grid sizes must differ");
  const double b = (n * sxy - sx * sy) / det;
  const double a = (sy - b * sx) / n;
  if (limit) *limit = a;
  if (slope) *slope = b;
  return FV_OK;
}
