// Transfer of a state between two grids of the same cube (grid sequencing: a steady state of a coarse grid
// as the Newton start on a finer one, as the paper refines its grids from 100^3 to 256^3 in Section 4.1).
//
// Every field is interpolated trilinearly in physical coordinates, axis by axis separable.  Along each axis
// the coarse samples of a field are extended by its wall values, so that the interpolant honours the
// boundary conditions of Eqs. 4-6:
//   velocity along its own axis: samples on the faces x_f[0..n], both walls 0 (slot 0 holds the wall);
//   velocity across an axis: samples [0 (wall), centres x_c[0..n-1], 1 (wall)], wall values 0 (no-slip);
//   T along x: samples [0, centres, 1] with the Dirichlet values 1 and 0 of Eq. 4;
//   T along y, z: the centres only, constant beyond the first and last (zero flux, Eqs. 5-6).
// The result is then projected (FP64) so that its velocity is discretely divergence free on the fine grid.
#include <algorithm>
#include <vector>

#include "fv_internal.h"

namespace fv {
namespace {

enum { kOwnAxis = 0, kAcross = 1, kTempX = 2, kTempFlux = 3 };

// Per (field, axis) table for the fine positions: lower extended sample index and weight of the upper one.
struct AxisTable {
  const int* lo;
  const double* w;
  int mode;
  int nc;  // coarse cells along this axis
};
struct ProlongArgs {
  AxisTable t[4][3];
  int nf[3], nc[3];
};

// Value of the extended coarse sample e along one axis: the coarse index (>= 0), or a wall code (< 0):
// -1 the value 0, -2 the value 1.
__device__ __forceinline__ int ext_index(int mode, int e, int nc) {
  switch (mode) {
    case kOwnAxis:
      return e < nc ? e : -1;
    case kAcross:
      return (e >= 1 && e <= nc) ? e - 1 : -1;
    case kTempX:
      return (e >= 1 && e <= nc) ? e - 1 : (e == 0 ? -2 : -1);
    default:
      return e;
  }
}

__global__ void k_prolong(ProlongArgs a, int field, const double* __restrict__ qc, double* __restrict__ qf) {
  const long long Nf = (long long)a.nf[0] * a.nf[1] * a.nf[2];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= Nf) return;
  const int i = (int)(t % a.nf[0]);
  const int j = (int)((t / a.nf[0]) % a.nf[1]);
  const int k = (int)(t / ((long long)a.nf[0] * a.nf[1]));
  const AxisTable& tx = a.t[field][0];
  const AxisTable& ty = a.t[field][1];
  const AxisTable& tz = a.t[field][2];
  const int ex = tx.lo[i], ey = ty.lo[j], ez = tz.lo[k];
  const double wx = tx.w[i], wy = ty.w[j], wz = tz.w[k];
  const long long Nc = (long long)a.nc[0] * a.nc[1] * a.nc[2];
  const double* c = qc + (long long)field * Nc;
  double acc = 0.0;
#pragma unroll
  for (int dz = 0; dz < 2; ++dz) {
    const int kz = ext_index(tz.mode, ez + dz, tz.nc);
    const double fz = dz ? wz : 1.0 - wz;
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
      const int jy = ext_index(ty.mode, ey + dy, ty.nc);
      const double fy = dy ? wy : 1.0 - wy;
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        const int ix = ext_index(tx.mode, ex + dx, tx.nc);
        const double f = fz * fy * (dx ? wx : 1.0 - wx);
        double v;
        if (ix == -2)
          v = 1.0;  // T = 1 on the hot wall (a velocity never has this code)
        else if (ix < 0 || jy < 0 || kz < 0)
          v = 0.0;
        else
          v = c[((long long)kz * a.nc[1] + jy) * a.nc[0] + ix];
        acc += f * v;
      }
    }
  }
  // the face-normal wall slot stays zero
  if ((field == 0 && i == 0) || (field == 1 && j == 0) || (field == 2 && k == 0)) acc = 0.0;
  qf[(long long)field * Nf + t] = acc;
}

// Coarse sample coordinates of (field, axis) and their mode.
std::vector<double> samples(const std::vector<double>& xf, int field, int axis, int* mode) {
  const int n = (int)xf.size() - 1;
  std::vector<double> s;
  if (field < 3 && field == axis) {
    *mode = kOwnAxis;
    s = xf;
    return s;
  }
  *mode = (field < 3) ? kAcross : (axis == 0 ? kTempX : kTempFlux);
  if (*mode != kTempFlux) s.push_back(0.0);
  for (int c = 0; c < n; ++c) s.push_back(0.5 * (xf[c] + xf[c + 1]));
  if (*mode != kTempFlux) s.push_back(1.0);
  return s;
}

// Fine positions of (field, axis): faces for a velocity along its own axis, centres otherwise.
std::vector<double> positions(const std::vector<double>& xf, int field, int axis) {
  const int n = (int)xf.size() - 1;
  std::vector<double> p;
  if (field < 3 && field == axis) {
    for (int f = 0; f < n; ++f) p.push_back(xf[f]);  // slots 0..n-1 (the wall at 1 is not stored)
  } else {
    for (int c = 0; c < n; ++c) p.push_back(0.5 * (xf[c] + xf[c + 1]));
  }
  return p;
}

}  // namespace

int launch_prolong(const fv_grid_s* gc, const double* qc, const fv_grid_s* gf, double* qf) {
  ProlongArgs a;
  const int nc[3] = {gc->nx, gc->ny, gc->nz}, nf[3] = {gf->nx, gf->ny, gf->nz};
  std::vector<int> lo_all;
  std::vector<double> w_all;
  int offs[4][3], modes[4][3];
  for (int f = 0; f < 4; ++f)
    for (int d = 0; d < 3; ++d) {
      int mode;
      const std::vector<double> s = samples(gc->xf[d], f, d, &mode);
      const std::vector<double> p = positions(gf->xf[d], f, d);
      offs[f][d] = (int)lo_all.size();
      modes[f][d] = mode;
      const int ns = (int)s.size();
      for (double x : p) {
        // lower sample: the last s[e] <= x (clamped so that e + 1 is a sample); constant beyond the ends
        int e = (int)(std::upper_bound(s.begin(), s.end(), x) - s.begin()) - 1;
        e = std::max(0, std::min(e, ns - 2));
        double w = (x - s[e]) / (s[e + 1] - s[e]);
        w = std::min(1.0, std::max(0.0, w));
        lo_all.push_back(e);
        w_all.push_back(w);
      }
    }
  int* dlo = nullptr;
  double* dw = nullptr;
  FV_CUDA(cudaMalloc(&dlo, lo_all.size() * sizeof(int)));
  if (cudaMalloc(&dw, w_all.size() * sizeof(double)) != cudaSuccess) {
    cudaFree(dlo);
    set_error("cudaMalloc failed for the interpolation tables");
    return FV_ENOMEM;
  }
  int st = FV_OK;
  cudaError_t e = cudaMemcpyAsync(dlo, lo_all.data(), lo_all.size() * sizeof(int), cudaMemcpyHostToDevice,
                                  gf->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dw, w_all.data(), w_all.size() * sizeof(double), cudaMemcpyHostToDevice, gf->stream);
  if (e != cudaSuccess) st = cuda_status(e, "cudaMemcpyAsync (interpolation tables)");
  if (st == FV_OK) {
    for (int f = 0; f < 4; ++f)
      for (int d = 0; d < 3; ++d) a.t[f][d] = AxisTable{dlo + offs[f][d], dw + offs[f][d], modes[f][d], nc[d]};
    for (int d = 0; d < 3; ++d) {
      a.nf[d] = nf[d];
      a.nc[d] = nc[d];
    }
    const long long Nf = (long long)nf[0] * nf[1] * nf[2];
    const int blocks = (int)((Nf + 255) / 256);
    for (int f = 0; f < 4 && st == FV_OK; ++f) {
      k_prolong<<<blocks, 256, 0, gf->stream>>>(a, f, qc, qf);
      const cudaError_t le = cudaGetLastError();
      if (le != cudaSuccess) st = cuda_status(le, "k_prolong");
    }
  }
  cudaStreamSynchronize(gf->stream);  // the tables are freed below
  cudaFree(dlo);
  cudaFree(dw);
  return st;
}

}  // namespace fv
