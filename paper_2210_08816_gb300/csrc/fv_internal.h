// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/cube_fv.h"

namespace fv {

constexpr int kMaxN = 1024;

// Device view of the metric arrays of one precision (all pointers into one device buffer).
//   idx[d][c]  = 1 / width of cell c                    (c = 0..n-1)
//   idc[d][f]  = 1 / centre spacing across face f       (f = 1..n-1); idc[d][0] = 2/width[0],
//                idc[d][n] = 2/width[n-1] (half-cell distance from the first centre to the wall)
//   wl[d][f], wr[d][f] = weights of cells f-1 and f in the linear interpolation to face f
template <typename R>
struct Geo {
  int n[3];
  const R* idx[3];
  const R* idc[3];
  const R* wl[3];
  const R* wr[3];
};

// Fast-diagonalisation data of one precision: per axis the forward matrix Finv (mode x cell,
// E^-1 = Y^T W^1/2), the backward matrix E (cell x mode, W^-1/2 Y) and the eigenvalues lam
// (lam[0] = 0 is the constant mode).
template <typename R>
struct FdmDev {
  const R* Einv[3];
  const R* E[3];
  const R* lam[3];
};

struct Workspace {
  // per precision (0 = FP64, 1 = FP32): J.v output (4N), two transform buffers (N each), potential (N)
  void* Y[2] = {nullptr, nullptr};
  void* t0[2] = {nullptr, nullptr};
  void* t1[2] = {nullptr, nullptr};
  int* err = nullptr;              // device error word of bounded device-side waits (0 = none)
  double* partials = nullptr;      // reduction partials
  double* scalars = nullptr;       // device scalars (reduction results)
  double* host_scalars = nullptr;  // pinned host mirror
  // block of vectors (fv_jvp_project_batch), per precision: J.v outputs (cap * 4N), two transform buffers
  // (cap * N each), grown on demand
  void* bY[2] = {nullptr, nullptr};
  void* bt0[2] = {nullptr, nullptr};
  void* bt1[2] = {nullptr, nullptr};
  int bcap[2] = {0, 0};
  unsigned bgen = 0;  // bumped whenever the block buffers are reallocated (captured graphs refer to them)
};
// Launch shapes picked by the autotuner (0 = the built-in default).
struct Tune {
  int pair_zc = 0;        // z-planes marched by one CTA of the two-cell J.v stencil
  int pair_zc_nvec = 0;   // block size the choice was timed on
};

}  // namespace fv

namespace fv {
struct ProfRecord {
  int kind;
  cudaEvent_t start, stop;
};
struct Profiler {
  bool enabled = false;
  std::vector<ProfRecord> records;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
};
// Tensor-core (tcgen05) pressure-solve operands: per axis [fwd_hi, fwd_lo, bwd_hi, bwd_lo] tensor maps.
struct TcState {
  bool ready = false;
  void* buf = nullptr;
  // per axis: [fwd_s_hi, fwd_s_lo, fwd_a_hi, fwd_a_lo, bwd_s_hi, bwd_s_lo, bwd_a_hi, bwd_a_lo]
  CUtensorMap B[3][8];
  const float* lam[3] = {nullptr, nullptr, nullptr};  // eigenvalues in the tensor-core mode order
  // per axis and direction (0 forward, 1 backward): the four B matrices of every K step laid out as the
  // shared-memory stage holds them (64-byte swizzled rows), one contiguous block per step
  const unsigned char* Bsw[3][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};
  int sms = 0;  // multiprocessors of the device (grid of the persistent passes)
};
}  // namespace fv

struct fv_grid_s {
  int nx, ny, nz;
  size_t N;  // nx*ny*nz
  double Pr;
  cudaStream_t stream;
  std::vector<double> xf[3];
  // metrics and FDM data, both precisions
  void* metric_buf[2] = {nullptr, nullptr};
  fv::Geo<double> geo64;
  fv::Geo<float> geo32;
  fv::FdmDev<double> fdm64;
  fv::FdmDev<float> fdm32;
  // Dirichlet diffusion operators (cell-centred, face-centred) of the Newton preconditioner
  fv::FdmDev<double> cd64, fd64;
  fv::FdmDev<float> cd32, fd32;
  fv::Workspace ws;
  long long wait_spins = -1;  // polls of a device-side wait before it gives up; < 0: the default
  double sigma_default;
  double min_width[3];
  mutable fv::Profiler prof;
  fv::TcState tc;
  fv::Tune tune;
  // batched J.v + projection: the captured launch sequence of the last argument set, replayed while the
  // arguments stay the same, and the private stream it is captured on
  cudaStream_t capture_stream = nullptr;
  cudaGraphExec_t batch_exec = nullptr;
  struct BatchKey {
    int prec = -1, nvec = 0;
    double Gr = 0.0, sigma = 0.0;
    const void *q = nullptr, *V = nullptr, *W = nullptr;
    bool operator==(const BatchKey& o) const {
      return prec == o.prec && nvec == o.nvec && Gr == o.Gr && sigma == o.sigma && q == o.q && V == o.V && W == o.W;
    }
  } batch_key;
};

namespace fv {

// Polls of an mbarrier wait in the library's kernels before it records FV_ETIMEOUT and gives up (at least
// seconds on every GPU this library targets, far above any legitimate wait).
constexpr long long kDefaultWaitSpins = 1LL << 22;
inline long long wait_spins(const fv_grid_s* g) { return g->wait_spins < 0 ? kDefaultWaitSpins : g->wait_spins; }

// ------------------------------------------------------------------ error reporting
void set_error(const std::string& msg);
int cuda_status(cudaError_t e, const char* what);
#define FV_CUDA(call)                                  \
  do {                                                 \
    cudaError_t _e = (call);                           \
    if (_e != cudaSuccess) return fv::cuda_status(_e, #call); \
  } while (0)
#define FV_TRY(expr)            \
  do {                          \
    int _s = (expr);            \
    if (_s != FV_OK) return _s; \
  } while (0)

// ------------------------------------------------------------------ measurement
enum {
  PROF_STENCIL = 0,
  PROF_DIVERGENCE = 1,
  PROF_TRANSFORM = 2,
  PROF_CORRECT = 3,
  PROF_REDUCE = 4,
  PROF_VECTOR = 5,
  PROF_TRANSFORM_TC = 6
};
// Records a CUDA event pair around the launches in its scope when profiling is enabled.
struct ProfScope {
  const fv_grid_s* g;
  cudaEvent_t stop = nullptr;
  ProfScope(const fv_grid_s* grid, int kind);
  ~ProfScope();
};

// ------------------------------------------------------------------ kernels (launchers)
// Stencils (kernels_stencil.cu)
template <typename R>
int launch_residual(const fv_grid_s* g, double Gr, const R* q, R* F);
template <typename R>
int launch_jvp(const fv_grid_s* g, double Gr, double sigma, const R* q, const R* v, R* out);
// The one-cell J.v stencil over nvec states stored one after another in v and out (4N each), one launch.
template <typename R>
int launch_jvp_block(const fv_grid_s* g, double Gr, double sigma, const R* q, const R* v, R* out, int nvec);
// nvec > 1: vel holds nvec states (4N each) and rhs nvec fields (N each), one after another.
template <typename R>
int launch_divergence(const fv_grid_s* g, const R* vel, R* rhs, int nvec = 1);
// out = alpha (Y - G phi) + beta v + gamma w   (velocity; T without G phi).  v, w may be null.
// norm_slot >= 0: also ||out||^2 into g->ws.scalars[norm_slot] (fused block partials).
template <typename R>
int launch_correct(const fv_grid_s* g, const R* Y, const R* phi, double alpha, const R* v, double beta,
                   const R* w, double gamma, R* out, int norm_slot = -1);

// out_i = (Y_i - G phi_i) + beta v_i for nvec states one after another (Y, v, out: 4N each; phi: N each);
// v may be null.  No norm.
template <typename R>
int launch_correct_block(const fv_grid_s* g, const R* Y, const R* phi, const R* v, double beta, R* out, int nvec);

// FP32 J.v with two x-adjacent cells per thread (kernels_stencil2.cu): nx a multiple of 64, ny >= 16,
// 16-byte aligned q and v (TMA plane ring).
bool stencil_pair_eligible(const fv_grid_s* g, const float* q, const float* v);
// nvec > 1: v and out hold nvec states one after another (4N elements each), all in one launch.
int launch_stencil_pair(const fv_grid_s* g, double Gr, double sigma, const float* q, const float* v, float* out,
                        int nvec = 1);

// Trilinear transfer of an FP64 state from grid gc to grid gf in physical coordinates, with the wall values
// of Eqs. 4-6 (kernels_prolong.cu); runs on gf's stream.  Not projected.
int launch_prolong(const fv_grid_s* gc, const double* qc, const fv_grid_s* gf, double* qf);

// Diagnostics of Section 4.2.3 (kernels_diag.cu), FP64 state q: E_kin (Eq. 12) and the hot-wall Nusselt
// number (Eq. 13) into g->ws.scalars[slot].
int launch_ekin(const fv_grid_s* g, const double* q, int slot);
int launch_nusselt(const fv_grid_s* g, const double* q, int slot);

// Fast-diagonalisation Poisson solve (kernels_fdm.cu): phi = (DG)^+ rhs; rhs and phi may alias.
template <typename R>
int launch_poisson(const fv_grid_s* g, const R* rhs, R* phi, R* tmp);
// The same solve for nvec fields stored one after another (N elements each) in rhs, phi and tmp.
template <typename R>
int launch_poisson_block(const fv_grid_s* g, const R* rhs, R* phi, R* tmp, int nvec);
// out = L_f^-1 in for one field f (0..2 velocity with no-slip walls, 3 temperature with Eqs. 4-6 homogeneous
// and the 1/Pr factor): the diffusion operator of J, inverted by fast diagonalisation (6 passes).
// s != 0: (L_f - s I)^-1 (the shifted operator of a pseudo-time step 1/s).
template <typename R>
int launch_field_solve(const fv_grid_s* g, int field, const R* in, R* out, R* tmp, double s = 0.0);

// BLAS-1 and reductions (kernels_blas.cu).  Results land in g->ws.scalars[slot...].
template <typename R>
int launch_dot(const fv_grid_s* g, const R* a, const R* b, size_t n, int slot);
template <typename R>
int launch_multidot(const fv_grid_s* g, const R* V, size_t ldv, int m, const R* w, size_t n, int slot);
template <typename R>
int launch_maxabs(const fv_grid_s* g, const R* a, size_t n, int slot);
// out = sum_i c[i] x[i], i < nvec <= 4 (x may alias out)
template <typename R>
int launch_lincomb(const fv_grid_s* g, size_t n, int nvec, const double* c, const R* const* x, R* out);
// w <- w - V h   (V: m vectors with leading dimension ldv; h device FP64)
template <typename R>
int launch_subtract_basis(const fv_grid_s* g, const R* V, size_t ldv, int m, const double* h, R* w, size_t n);
int launch_convert(const fv_grid_s* g, size_t n, const double* src, float* dst);
int launch_convert(const fv_grid_s* g, size_t n, const float* src, double* dst);
template <typename R>
int launch_fill_normal(const fv_grid_s* g, unsigned long long seed, R* out);

constexpr int kReduceBlocks = 1024;
constexpr int kMaxScalars = 512;
constexpr int kPartialSlots = kReduceBlocks * 256;  // capacity of g->ws.partials
// g->ws.scalars[slot] = sum of g->ws.partials[0 .. np) in a fixed order
int launch_sum_partials(const fv_grid_s* g, int np, int slot);

// host scalar readback: copies `count` scalars starting at `slot` and synchronises
int read_scalars(const fv_grid_s* g, int slot, int count, double* out);

// Tiled TMA descriptor of a dense row-major tensor (kernels_tc.cu): rank <= 5, dims innermost first,
// strides in bytes for dims 1..rank-1, zero fill out of bounds.  FV_ECUDA if the driver call fails.
int encode_tensor_map(CUtensorMap* map, CUtensorMapDataType type, int rank, const void* ptr, const uint64_t* dims,
                      const uint64_t* strides, const uint32_t* box, CUtensorMapSwizzle swizzle);

// Tensor-core pressure-solve passes (kernels_tc.cu), FP32 only.
bool tc_eligible(const fv_grid_s* g);
int tc_setup(fv_grid_s* g, const std::vector<double>* idx, const std::vector<double>* idc);
// nvec fields stored one after another are transformed in one launch (persistent form only).
int tc_pass(const fv_grid_s* g, int axis, bool bwd, int na, int nb, const float* in, float* out, bool scale,
            int nvec = 1);

// ------------------------------------------------------------------ host linear algebra (host_linalg.cpp)
// Symmetric tridiagonal eigen-decomposition (implicit QR with Wilkinson shifts).
// d: diagonal (n), e: off-diagonal (n-1); on return d holds eigenvalues, Q (n*n, row-major,
// column j = eigenvector j).  Returns false if it fails to converge.
bool tridiag_eig(int n, std::vector<double>& d, std::vector<double>& e, std::vector<double>& Q);
// Eigenvalues of a real upper Hessenberg matrix (m x m, row-major, leading dimension ld) by complex
// single-shift QR.  Returns false on non-convergence.
bool hessenberg_eigvals(int m, const double* H, int ld, std::vector<double>& re, std::vector<double>& im);
// Eigenvector of H for eigenvalue (re, im) by inverse iteration (complex).  y: 2*m (re, im interleaved).
bool hessenberg_eigvec(int m, const double* H, int ld, double re, double im, std::vector<double>& y);
// Householder reduction of a general m x m matrix (row-major) to upper Hessenberg H, A = Q H Q^T.
void hessenberg_reduce(int m, std::vector<double>& A, std::vector<double>& Q);
// Solve a small dense system A x = b (n x n row-major) with partial pivoting; false if singular.
bool dense_solve(int n, std::vector<double> A, std::vector<double>& b);
// Least squares min || H y - beta e1 || for the (j+1) x j Hessenberg of GMRES (row-major, ld).
void hessenberg_lstsq(int j, const double* H, int ld, double beta, std::vector<double>& y, double* resid);

// ------------------------------------------------------------------ tensor-core operands (host_tc.cpp)
constexpr int kTcSlabCols = 16;  // FP32 K columns per slab of the tensor-core passes (one 64-byte row)
// One float buffer: per axis [fwd_s_hi, fwd_s_lo, fwd_a_hi, fwd_a_lo, bwd_s_hi, bwd_s_lo, bwd_a_hi,
// bwd_a_lo] (h x h each, at moff), the eigenvalues in the tensor-core mode order (n, at loff), and per
// axis and direction the swizzled per-step B blocks of the persistent pass (4 h^2, at soff, 256-byte
// aligned); offsets in floats.
struct TcOperands {
  std::vector<float> buf;
  size_t moff[3][8], loff[3], soff[3][2];
};
// Builds the operands for axes of ns[d] cells (even, ns[d] / 2 a multiple of kTcSlabCols) from the
// metric arrays idx (1 / widths) and idc (1 / centre spacings) of each axis.  FV_EINVAL on failure.
int tc_host_operands(const int ns[3], const std::vector<double>* idx, const std::vector<double>* idc,
                     TcOperands& out);

// ------------------------------------------------------------------ grid axes (host_grid.cpp)
// One axis of the grid, FP64 on the host.  idx[c] = 1 / width of cell c; idc[f] = 1 / centre spacing across
// face f (idc[0] = 2 / width[0], idc[n] = 2 / width[n-1]); wl[f], wr[f] = interpolation weights of cells
// f-1 and f at face f; lam, Einv, E: the Neumann operator L = E diag(lam) Einv (modes by decreasing
// eigenvalue, lam[0] = 0 the constant vector); n x n matrices row-major.
struct AxisHost {
  int n;
  std::vector<double> idx, idc, wl, wr, lam, Einv, E;
  // diffusion operators of the Newton preconditioner: cell-centred with Dirichlet walls half a cell away
  // (transverse velocities, T along x) and face-centred with Dirichlet walls (a velocity along its own
  // axis; mode 0 is a dummy that maps the wall slot 0 to itself)
  std::vector<double> cd_lam, cd_Einv, cd_E, fd_lam, fd_Einv, fd_E;
};
// Faces 0 .. n of the tanh-stretched grid with stretching s (s = 0: uniform), mirrored about 1/2.
std::vector<double> tanh_faces(int n, double s);
// Metrics and 1D decompositions of the axis with faces xf (strictly increasing); FV_EINVAL otherwise.
int build_axis(const std::vector<double>& xf, AxisHost& a);
// True if the faces are their own mirror image about 1/2 (x_f[n-i] = 1 - x_f[i] to 4 units of round-off):
// the tensor-core passes split each 1D eigenproblem into symmetric and antisymmetric halves, which holds
// only on such axes.
bool mirror_symmetric(const std::vector<double>& xf);

// ------------------------------------------------------------------ Chebyshev filter ellipses (host_cheb.cpp)
struct Ritz {
  double re, im;
};
// Level |w| of z = zr + i zi in the confocal family with foci d +- c (c^2 = c2 real, possibly negative;
// c2 = 0: circles about d): z - d = c (w + 1/w) / 2, the branch |w| >= 1.
double ellipse_level(double zr, double zi, double d, double c2);
// Rightmost real point of the ellipse of the given level in that family.
double ellipse_right_end(double d, double c2, double level);
// Scan of real-centred confocal ellipses for the one maximising min over wanted of the level divided by
// max over unwanted of the level, among those whose right end stays left of every wanted real part (the
// best of all if none does); rate_out = that ratio.
void best_ellipse(const std::vector<Ritz>& wanted, const std::vector<Ritz>& unwanted, double& d_out,
                  double& c2_out, double& rate_out);

// ------------------------------------------------------------------ drivers (fv_api.cpp)
template <typename R>
int jvp_project(fv_grid_s* g, double Gr, double sigma, const R* q, const R* v, R* out);
template <typename R>
int chebyshev_step(fv_grid_s* g, double Gr, double sigma, const R* q, const R* y, const R* yprev,
                   double alpha, double beta, double gamma, R* out, int norm_slot = -1);

}  // namespace fv
