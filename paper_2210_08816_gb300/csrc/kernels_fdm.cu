// Pressure-correction Poisson solve DG phi = rhs by fast diagonalisation (Lynch, Rice & Thomas 1964).
//
// DG is the Kronecker sum A_x (+) A_y (+) A_z of 1D Neumann operators A = W^-1 S (W = diag(widths),
// S symmetric tridiagonal).  With the generalised eigenvectors E (E^T W E = I) and eigenvalues lam,
//     phi = (E_z x E_y x E_x) diag(1 / (lam_x + lam_y + lam_z)) (E_z x E_y x E_x)^-1 rhs,
// the constant mode (all three lam = 0) set to zero.  Each factor is a dense n x n matrix applied along
// one axis: a batched GEMM with K = n.  Six passes: x, y, z forward (the z pass scales by 1/Lambda in
// its epilogue), z, y, x backward.
//
// Transform kernel: C[b][r][c] = sum_k A[b][r][k] B[b][k][c] with A k-contiguous in both layouts used:
//   layout X (contract the contiguous x axis): rows = (k, j) lines, cols = modes, A = field, B(k, c) = M[c][k]
//   layout S (contract a strided axis):         rows = modes, cols = contiguous positions, A = M, B = field
// Tiles BM x BN, slabs of BK, 256 threads; thread (tx, ty) owns rows ty + 16 i and cols tx + 16 j so
// that each store instruction writes 16 consecutive elements.
#include "fv_internal.h"

namespace fv {
namespace {

template <typename R>
struct TileCfg;
template <>
struct TileCfg<float> {
  static constexpr int BM = 128, BN = 128, BK = 16, TM = 8, TN = 8;
};
template <>
struct TileCfg<double> {
  static constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
};

struct TransformArgs {
  int rows, cols, K;
  long long lda_r;            // A: k stride is 1
  long long ldb_k, ldb_c;     // B strides
  long long ldc_r;            // C: col stride is 1
  long long batch_a, batch_b, batch_c;
  // scaling epilogue (z-forward): value /= (lz[r] + ly[c / nxm] + lx[c % nxm]); constant mode -> 0
  int scale, nxm;
};

template <typename R, bool B_COLS_CONTIG>
__global__ void __launch_bounds__(256) k_transform(TransformArgs t, const R* __restrict__ A, const R* __restrict__ B,
                                                    R* __restrict__ Cout, const R* __restrict__ lx,
                                                    const R* __restrict__ ly, const R* __restrict__ lz) {
  using T = TileCfg<R>;
  constexpr int BM = T::BM, BN = T::BN, BK = T::BK, TM = T::TM, TN = T::TN;
  __shared__ R As[BK][BM + 1];
  __shared__ R Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int r0 = blockIdx.y * BM, c0 = blockIdx.x * BN;
  const long long bz = blockIdx.z;
  A += bz * t.batch_a;
  B += bz * t.batch_b;
  Cout += bz * t.batch_c;
  R acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = R(0);

  for (int k0 = 0; k0 < t.K; k0 += BK) {
    // A tile: BM x BK, k fastest
#pragma unroll
    for (int e = tid; e < BM * BK; e += 256) {
      const int kk = e % BK, rr = e / BK;
      const int r = r0 + rr, k = k0 + kk;
      As[kk][rr] = (r < t.rows && k < t.K) ? A[(long long)r * t.lda_r + k] : R(0);
    }
    // B tile: BK x BN
    if (B_COLS_CONTIG) {
#pragma unroll
      for (int e = tid; e < BN * BK; e += 256) {
        const int cc = e % BN, kk = e / BN;
        const int c = c0 + cc, k = k0 + kk;
        Bs[kk][cc] = (c < t.cols && k < t.K) ? B[(long long)k * t.ldb_k + c] : R(0);
      }
    } else {
#pragma unroll
      for (int e = tid; e < BN * BK; e += 256) {
        const int kk = e % BK, cc = e / BK;
        const int c = c0 + cc, k = k0 + kk;
        Bs[kk][cc] = (c < t.cols && k < t.K) ? B[(long long)c * t.ldb_c + k] : R(0);
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      R a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int r = r0 + ty + 16 * i;
    if (r >= t.rows) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int c = c0 + tx + 16 * j;
      if (c >= t.cols) continue;
      R val = acc[i][j];
      if (t.scale) {
        const int my = c / t.nxm, mx = c - my * t.nxm;
        const R den = lz[r] + ly[my] + lx[mx];
        val = (r == 0 && my == 0 && mx == 0) ? R(0) : val / den;
      }
      Cout[(long long)r * t.ldc_r + c] = val;
    }
  }
}

template <typename R>
const FdmDev<R>& fdm_of(const fv_grid_s* g);
template <>
const FdmDev<double>& fdm_of<double>(const fv_grid_s* g) { return g->fdm64; }
template <>
const FdmDev<float>& fdm_of<float>(const fv_grid_s* g) { return g->fdm32; }

// contract the x axis: out[(k,j)][m] = sum_i in[(k,j)][i] M[m][i]
template <typename R>
int apply_x(const fv_grid_s* g, const R* M, const R* in, R* out) {
  using T = TileCfg<R>;
  TransformArgs t{};
  t.rows = g->ny * g->nz;
  t.cols = g->nx;
  t.K = g->nx;
  t.lda_r = g->nx;
  t.ldb_k = 1;
  t.ldb_c = g->nx;
  t.ldc_r = g->nx;
  dim3 grid((t.cols + T::BN - 1) / T::BN, (t.rows + T::BM - 1) / T::BM, 1);
  ProfScope ps(g, PROF_TRANSFORM);
  k_transform<R, false><<<grid, 256, 0, g->stream>>>(t, in, M, out, nullptr, nullptr, nullptr);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

// contract the y axis (batched over k-planes): out[k][m][i] = sum_j M[m][j] in[k][j][i]
template <typename R>
int apply_y(const fv_grid_s* g, const R* M, const R* in, R* out) {
  using T = TileCfg<R>;
  TransformArgs t{};
  t.rows = g->ny;
  t.cols = g->nx;
  t.K = g->ny;
  t.lda_r = g->ny;
  t.ldb_k = g->nx;
  t.ldc_r = g->nx;
  t.batch_a = 0;
  t.batch_b = t.batch_c = (long long)g->nx * g->ny;
  dim3 grid((t.cols + T::BN - 1) / T::BN, (t.rows + T::BM - 1) / T::BM, g->nz);
  ProfScope ps(g, PROF_TRANSFORM);
  k_transform<R, true><<<grid, 256, 0, g->stream>>>(t, M, in, out, nullptr, nullptr, nullptr);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

// contract the z axis: out[m][(j,i)] = sum_k M[m][k] in[k][(j,i)], optionally scaled by 1/Lambda
template <typename R>
int apply_z(const fv_grid_s* g, const R* M, const R* in, R* out, bool scale) {
  using T = TileCfg<R>;
  const FdmDev<R>& f = fdm_of<R>(g);
  TransformArgs t{};
  t.rows = g->nz;
  t.cols = g->nx * g->ny;
  t.K = g->nz;
  t.lda_r = g->nz;
  t.ldb_k = (long long)g->nx * g->ny;
  t.ldc_r = (long long)g->nx * g->ny;
  t.scale = scale ? 1 : 0;
  t.nxm = g->nx;
  dim3 grid((t.cols + T::BN - 1) / T::BN, (t.rows + T::BM - 1) / T::BM, 1);
  ProfScope ps(g, PROF_TRANSFORM);
  k_transform<R, true><<<grid, 256, 0, g->stream>>>(t, M, in, out, f.lam[0], f.lam[1], f.lam[2]);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

}  // namespace

template <typename R>
int launch_poisson(const fv_grid_s* g, const R* rhs, R* phi, R* tmp) {
  const FdmDev<R>& f = fdm_of<R>(g);
  // rhs -> tmp -> phi -> tmp (scaled) -> phi -> tmp -> phi
  FV_TRY(apply_x<R>(g, f.Einv[0], rhs, tmp));
  FV_TRY(apply_y<R>(g, f.Einv[1], tmp, phi));
  FV_TRY(apply_z<R>(g, f.Einv[2], phi, tmp, true));
  FV_TRY(apply_z<R>(g, f.E[2], tmp, phi, false));
  FV_TRY(apply_y<R>(g, f.E[1], phi, tmp));
  FV_TRY(apply_x<R>(g, f.E[0], tmp, phi));
  return FV_OK;
}

template int launch_poisson<double>(const fv_grid_s*, const double*, double*, double*);
template int launch_poisson<float>(const fv_grid_s*, const float*, float*, float*);

}  // namespace fv
