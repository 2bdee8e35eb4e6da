// Flow diagnostics of Section 4.2.3: the total kinetic energy (Eq. 12) and the Nusselt number at the hot
// wall (Eq. 13), summed on the device for the time stepper's histories.
//
//   E_kin = 1/2 sum over the interior faces of every velocity component of u_f^2 times the face's control
//           volume: the centre spacing along the component's own axis times the cell widths across it;
//   Nu    = sum over the hot wall's cells (j, k) of (T[k][j][0] - 1) / (dx_0 / 2) dy_j dz_k, Eq. 13 as
//           printed (no sign change: conduction gives -1).
// Both use the metric arrays of the handle (idc[d][f] = 1 / centre spacing, idc[d][0] = 2 / dx_0,
// idx[d][c] = 1 / width) and the library's deterministic two-pass reduction (fixed block partials, then
// their sum in a fixed order).  The wall slot of a face-normal velocity holds 0 and adds nothing.
#include "fv_internal.h"

namespace fv {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (warp == 0) {
    r = (lane < kThreads / 32) ? sh[lane] : 0.0;
    r = warp_sum(r);
  }
  return r;
}

// partial sums of u_f^2 V_f over the three velocity fields (3 N elements), one chunk per block
__global__ void __launch_bounds__(kThreads) k_ekin_partial(Geo<double> g, const double* __restrict__ q,
                                                            double* __restrict__ part) {
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const long long N = (long long)nx * ny * nz, n3 = 3 * N;
  const long long L = (n3 + gridDim.x - 1) / gridDim.x;
  const long long s = (long long)blockIdx.x * L, e = s + L < n3 ? s + L : n3;
  double acc = 0.0;
  for (long long t = s + threadIdx.x; t < e; t += kThreads) {
    const int c = (int)(t / N);
    const long long o = t - (long long)c * N;
    const int i = (int)(o % nx), j = (int)((o / nx) % ny), k = (int)(o / ((long long)nx * ny));
    const int p[3] = {i, j, k};
    // control volume: centre spacing along the own axis (face p), widths across
    double inv = g.idc[c][p[c]];
#pragma unroll
    for (int d = 0; d < 3; ++d)
      if (d != c) inv *= g.idx[d][p[d]];
    const double u = q[t];
    acc += 0.5 * u * u / inv;
  }
  const double r = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = r;
}

// partial sums of the hot-wall flux over the ny * nz wall cells
__global__ void __launch_bounds__(kThreads) k_nusselt_partial(Geo<double> g, const double* __restrict__ q,
                                                               double* __restrict__ part) {
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const long long N = (long long)nx * ny * nz, nw = (long long)ny * nz;
  const long long L = (nw + gridDim.x - 1) / gridDim.x;
  const long long s = (long long)blockIdx.x * L, e = s + L < nw ? s + L : nw;
  const double* T = q + 3 * N;
  double acc = 0.0;
  for (long long t = s + threadIdx.x; t < e; t += kThreads) {
    const int j = (int)(t % ny), k = (int)(t / ny);
    const double grad = (T[((long long)k * ny + j) * nx] - 1.0) * g.idc[0][0];  // over the half cell dx_0 / 2
    acc += grad / (g.idx[1][j] * g.idx[2][k]);
  }
  const double r = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = r;
}

}  // namespace

int launch_ekin(const fv_grid_s* g, const double* q, int slot) {
  ProfScope ps(g, PROF_REDUCE);
  k_ekin_partial<<<kReduceBlocks, kThreads, 0, g->stream>>>(g->geo64, q, g->ws.partials);
  FV_CUDA(cudaGetLastError());
  FV_TRY(launch_sum_partials(g, kReduceBlocks, slot));
  return FV_OK;
}

int launch_nusselt(const fv_grid_s* g, const double* q, int slot) {
  ProfScope ps(g, PROF_REDUCE);
  const long long nw = (long long)g->ny * g->nz;
  const int blocks = (int)std::min<long long>(kReduceBlocks, (nw + kThreads - 1) / kThreads);
  k_nusselt_partial<<<blocks, kThreads, 0, g->stream>>>(g->geo64, q, g->ws.partials);
  FV_CUDA(cudaGetLastError());
  FV_TRY(launch_sum_partials(g, blocks, slot));
  return FV_OK;
}

}  // namespace fv
