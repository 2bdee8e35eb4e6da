// Pressure-correction Poisson solve DG phi = rhs by fast diagonalisation (Lynch, Rice & Thomas 1964).
//
// DG is the Kronecker sum A_x (+) A_y (+) A_z of 1D Neumann operators A = W^-1 S (W = diag(widths),
// S symmetric tridiagonal).  With the generalised eigenvectors E (E^T W E = I) and eigenvalues lam,
//     phi = (E_z x E_y x E_x) diag(1 / (lam_x + lam_y + lam_z)) (E_z x E_y x E_x)^-1 rhs,
// the constant mode (all three lam = 0) set to zero.  Each factor is a dense n x n matrix applied along
// one axis: a batched GEMM with K = n.
//
// Rotating passes.  Every pass contracts the CONTIGUOUS axis of its input and writes the mode index as
// the new slowest axis:  in[a][b][k] (k contiguous)  ->  out[m][a][b] = sum_k M[m][k] in[a][b][k].
// Three passes turn (z, y, x) into (x, z, y), (y, x, z) and back to (z, y, x); the forward three map
// cells to modes (the third one divides by Lambda in its epilogue), the backward three map back.  So
// all six are one GEMM shape, C[p][m] = sum_k A[p][k] B[m][k] with both operands k-contiguous, stored
// transposed (out[m][p]).  Tiles BM (p) x BN (m), slabs of BK; thread (tx, ty) owns p = tx + 16 i and
// m = ty + 16 j, so each store instruction writes 16 consecutive p.
#include "fv_internal.h"

namespace fv {
namespace {

template <typename R>
struct TileCfg;
template <>
struct TileCfg<float> {
  static constexpr int BM = 128, BN = 128, BK = 32, TM = 8, TN = 8;
};
template <>
struct TileCfg<double> {
  static constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
};

struct PassArgs {
  int P, nm, K;          // rows (a*b), modes, contraction length
  int scale;             // third forward pass: multiply by sfac / (lam_z[m] + lam_y[p / nb] + lam_x[p % nb])
  int nb;
  int zero_mode;         // the (0,0,0) mode is the null space (Neumann): set it to zero
  double sfac;
  double shift;          // scaled pass: sfac / (lam_z + lam_y + lam_x - shift)
};

template <typename R>
__global__ void __launch_bounds__(256) k_transform(PassArgs t, const R* __restrict__ in, const R* __restrict__ M,
                                                    R* __restrict__ out, const R* __restrict__ lx,
                                                    const R* __restrict__ ly, const R* __restrict__ lz) {
  using T = TileCfg<R>;
  constexpr int BM = T::BM, BN = T::BN, BK = T::BK, TM = T::TM, TN = T::TN;
  __shared__ R As[BK][BM + 1];
  __shared__ R Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int p0 = blockIdx.x * BM, m0 = blockIdx.y * BN;
  // blockIdx.z: field of a block of fields stored one after another (P x K in, nm x P out)
  in += (size_t)blockIdx.z * t.P * t.K;
  out += (size_t)blockIdx.z * t.nm * t.P;
  R acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = R(0);

  for (int k0 = 0; k0 < t.K; k0 += BK) {
#pragma unroll
    for (int e = tid; e < BM * BK; e += 256) {
      const int kk = e % BK, rr = e / BK;
      const int p = p0 + rr, k = k0 + kk;
      As[kk][rr] = (p < t.P && k < t.K) ? in[(long long)p * t.K + k] : R(0);
    }
#pragma unroll
    for (int e = tid; e < BN * BK; e += 256) {
      const int kk = e % BK, cc = e / BK;
      const int m = m0 + cc, k = k0 + kk;
      Bs[kk][cc] = (m < t.nm && k < t.K) ? M[(long long)m * t.K + k] : R(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      R a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < TN; ++j) {
    const int m = m0 + ty + 16 * j;
    if (m >= t.nm) continue;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int p = p0 + tx + 16 * i;
      if (p >= t.P) continue;
      R val = acc[i][j];
      if (t.scale) {
        const int a = p / t.nb, b = p - a * t.nb;
        val = (t.zero_mode && m == 0 && a == 0 && b == 0) ? R(0) : R(t.sfac) * val / (lz[m] + ly[a] + lx[b] - R(t.shift));
      }
      out[(long long)m * t.P + p] = val;
    }
  }
}

template <typename R>
const FdmDev<R>& fdm_of(const fv_grid_s* g);
template <>
const FdmDev<double>& fdm_of<double>(const fv_grid_s* g) { return g->fdm64; }
template <>
const FdmDev<float>& fdm_of<float>(const fv_grid_s* g) { return g->fdm32; }

// in[a][b][k] -> out[m][a][b] with M (nm x K); a scaled pass divides by the eigenvalue sums of lam[0..2]
template <typename R>
int pass_ops(const fv_grid_s* g, const R* M, int na, int nb, int K, const R* in, R* out, bool scale,
             const R* const lam[3], bool zero_mode, double sfac, int nvec = 1, double shift = 0.0) {
  using T = TileCfg<R>;
  PassArgs t{};
  t.P = na * nb;
  t.nm = K;
  t.K = K;
  t.scale = scale ? 1 : 0;
  t.nb = nb;
  t.zero_mode = zero_mode ? 1 : 0;
  t.sfac = sfac;
  t.shift = shift;
  dim3 grid((t.P + T::BM - 1) / T::BM, (t.nm + T::BN - 1) / T::BN, nvec);
  ProfScope ps(g, PROF_TRANSFORM);
  k_transform<R><<<grid, 256, 0, g->stream>>>(t, in, M, out, lam[0], lam[1], lam[2]);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

template <typename R>
int pass(const fv_grid_s* g, const R* M, int na, int nb, int K, const R* in, R* out, bool scale, int nvec = 1) {
  const FdmDev<R>& f = fdm_of<R>(g);
  return pass_ops<R>(g, M, na, nb, K, in, out, scale, f.lam, true, 1.0, nvec);
}

template <typename R>
const FdmDev<R>& cd_of(const fv_grid_s* g);
template <>
const FdmDev<double>& cd_of<double>(const fv_grid_s* g) { return g->cd64; }
template <>
const FdmDev<float>& cd_of<float>(const fv_grid_s* g) { return g->cd32; }
template <typename R>
const FdmDev<R>& fd_of(const fv_grid_s* g);
template <>
const FdmDev<double>& fd_of<double>(const fv_grid_s* g) { return g->fd64; }
template <>
const FdmDev<float>& fd_of<float>(const fv_grid_s* g) { return g->fd32; }

}  // namespace

template <typename R>
int launch_poisson(const fv_grid_s* g, const R* rhs, R* phi, R* tmp) {
  const FdmDev<R>& f = fdm_of<R>(g);
  const int nx = g->nx, ny = g->ny, nz = g->nz;
  // forward: (z,y,x) -> (mx,z,y) -> (my,mx,z) -> (mz,my,mx) / Lambda
  FV_TRY(pass<R>(g, f.Einv[0], nz, ny, nx, rhs, tmp, false));
  FV_TRY(pass<R>(g, f.Einv[1], nx, nz, ny, tmp, phi, false));
  FV_TRY(pass<R>(g, f.Einv[2], ny, nx, nz, phi, tmp, true));
  // backward: (mz,my,mx) -> (x,mz,my) -> (y,x,mz) -> (z,y,x)
  FV_TRY(pass<R>(g, f.E[0], nz, ny, nx, tmp, phi, false));
  FV_TRY(pass<R>(g, f.E[1], nx, nz, ny, phi, tmp, false));
  FV_TRY(pass<R>(g, f.E[2], ny, nx, nz, tmp, phi, false));
  return FV_OK;
}

template <>
int launch_poisson<float>(const fv_grid_s* g, const float* rhs, float* phi, float* tmp) {
  const int nx = g->nx, ny = g->ny, nz = g->nz;
  if (g->tc.ready) {  // the same six passes on the tensor cores (3 x TF32 split, FP32 accuracy; modes in
                      // the symmetric / antisymmetric order of the mirror-symmetric grid)
    FV_TRY(tc_pass(g, 0, false, nz, ny, rhs, tmp, false));
    FV_TRY(tc_pass(g, 1, false, nx, nz, tmp, phi, false));
    FV_TRY(tc_pass(g, 2, false, ny, nx, phi, tmp, true));
    FV_TRY(tc_pass(g, 0, true, nz, ny, tmp, phi, false));
    FV_TRY(tc_pass(g, 1, true, nx, nz, phi, tmp, false));
    FV_TRY(tc_pass(g, 2, true, ny, nx, tmp, phi, false));
    return FV_OK;
  }
  const FdmDev<float>& f = fdm_of<float>(g);
  FV_TRY(pass<float>(g, f.Einv[0], nz, ny, nx, rhs, tmp, false));
  FV_TRY(pass<float>(g, f.Einv[1], nx, nz, ny, tmp, phi, false));
  FV_TRY(pass<float>(g, f.Einv[2], ny, nx, nz, phi, tmp, true));
  FV_TRY(pass<float>(g, f.E[0], nz, ny, nx, tmp, phi, false));
  FV_TRY(pass<float>(g, f.E[1], nx, nz, ny, phi, tmp, false));
  FV_TRY(pass<float>(g, f.E[2], ny, nx, nz, tmp, phi, false));
  return FV_OK;
}

template <typename R>
int launch_poisson_block(const fv_grid_s* g, const R* rhs, R* phi, R* tmp, int nvec) {
  const int nx = g->nx, ny = g->ny, nz = g->nz;
  if (nvec < 1 || nvec > 65535) {
    set_error("launch_poisson_block: nvec out of range");
    return FV_EINVAL;
  }
  if constexpr (sizeof(R) == 4) {
    if (g->tc.ready && g->tc.sms > 0) {  // the tensor-core passes over the stacked fields, one launch each
      FV_TRY(tc_pass(g, 0, false, nz, ny, rhs, tmp, false, nvec));
      FV_TRY(tc_pass(g, 1, false, nx, nz, tmp, phi, false, nvec));
      FV_TRY(tc_pass(g, 2, false, ny, nx, phi, tmp, true, nvec));
      FV_TRY(tc_pass(g, 0, true, nz, ny, tmp, phi, false, nvec));
      FV_TRY(tc_pass(g, 1, true, nx, nz, phi, tmp, false, nvec));
      FV_TRY(tc_pass(g, 2, true, ny, nx, tmp, phi, false, nvec));
      return FV_OK;
    }
  }
  const FdmDev<R>& f = fdm_of<R>(g);
  FV_TRY(pass<R>(g, f.Einv[0], nz, ny, nx, rhs, tmp, false, nvec));
  FV_TRY(pass<R>(g, f.Einv[1], nx, nz, ny, tmp, phi, false, nvec));
  FV_TRY(pass<R>(g, f.Einv[2], ny, nx, nz, phi, tmp, true, nvec));
  FV_TRY(pass<R>(g, f.E[0], nz, ny, nx, tmp, phi, false, nvec));
  FV_TRY(pass<R>(g, f.E[1], nx, nz, ny, phi, tmp, false, nvec));
  FV_TRY(pass<R>(g, f.E[2], ny, nx, nz, tmp, phi, false, nvec));
  return FV_OK;
}

template int launch_poisson<double>(const fv_grid_s*, const double*, double*, double*);
template int launch_poisson_block<double>(const fv_grid_s*, const double*, double*, double*, int);
template int launch_poisson_block<float>(const fv_grid_s*, const float*, float*, float*, int);

// Diffusion operator of one field, L_f = s_f (L_x (+) L_y (+) L_z), inverted like the pressure operator:
// velocity component c uses the face-centred Dirichlet operator along its own axis and the cell-centred
// Dirichlet operator across (no-slip walls half a cell away); temperature uses cell-centred Dirichlet in
// x (Eq. 4, homogeneous) and the Neumann operator in y and z (Eqs. 5-6), with s_T = 1/Pr.  No zero mode.
// in and out may alias; tmp may not.
// s != 0: (L_f - s I)^-1 instead (the eigenvalues of L_f are (lam_x + lam_y + lam_z) / s_f).
template <typename R>
int launch_field_solve(const fv_grid_s* g, int field, const R* in, R* out, R* tmp, double s) {
  const FdmDev<R>* op[3];
  for (int d = 0; d < 3; ++d) {
    if (field < 3)
      op[d] = (d == field) ? &fd_of<R>(g) : &cd_of<R>(g);
    else
      op[d] = (d == 0) ? &cd_of<R>(g) : &fdm_of<R>(g);
  }
  const R* lam[3] = {op[0]->lam[0], op[1]->lam[1], op[2]->lam[2]};
  const double sfac = (field == 3) ? g->Pr : 1.0;
  const int nx = g->nx, ny = g->ny, nz = g->nz;
  FV_TRY(pass_ops<R>(g, op[0]->Einv[0], nz, ny, nx, in, tmp, false, lam, false, 1.0));
  FV_TRY(pass_ops<R>(g, op[1]->Einv[1], nx, nz, ny, tmp, out, false, lam, false, 1.0));
  FV_TRY(pass_ops<R>(g, op[2]->Einv[2], ny, nx, nz, out, tmp, true, lam, false, sfac, 1, s * sfac));
  FV_TRY(pass_ops<R>(g, op[0]->E[0], nz, ny, nx, tmp, out, false, lam, false, 1.0));
  FV_TRY(pass_ops<R>(g, op[1]->E[1], nx, nz, ny, out, tmp, false, lam, false, 1.0));
  FV_TRY(pass_ops<R>(g, op[2]->E[2], ny, nx, nz, tmp, out, false, lam, false, 1.0));
  return FV_OK;
}

template int launch_field_solve<double>(const fv_grid_s*, int, const double*, double*, double*, double);
template int launch_field_solve<float>(const fv_grid_s*, int, const float*, float*, float*, double);

}  // namespace fv
