// Stencil kernels of the staggered finite-volume discretisation (Section 2, Eqs. 1-6):
//   residual F(q; Gr), Jacobian-vector product J(q) v, divergence D, and the fused
//   gradient correction of the projection.
//
// One thread per cell (i, j, k) produces the four outputs that live in that cell's slots: the
// x-face u at x_f[i], the y-face v at y_f[j], the z-face w at z_f[k] and T at the centre.
// Wall slots (i == 0 for u, ...) are written as zero.  Inputs are read through the read-only
// path; the neighbour re-reads of a block are served by L1/L2, so DRAM sees each field ~once.
#include "fv_internal.h"

namespace fv {
namespace {

// 32-bit offsets: the grid constructor guarantees 4 * nx * ny * nz < 2^31.
template <typename R>
struct Cell {
  int p[3];
  int s[3];
  int o;
};

template <typename R>
__device__ __forceinline__ R ld(const R* __restrict__ a, int o) {
  return __ldg(a + o);
}

// Momentum component C at the C-face slot p[C] (1 <= p[C] <= n[C]-1).
//   conv = S(a, b) = div(a b) + div(b a)  (symmetrised convective bilinear form)
//   lap  = Lap b  (no-slip walls)
// For d == C the fluxes sit at the cell centres p-1 and p bounding the C-control volume:
//   (mean a)(mean b) + (mean b)(mean a) = 2 (mean a)(mean b), differenced over the centre spacing.
// For d != C the fluxes sit on the d-faces p[d] and p[d]+1: the d-velocity interpolated along C to the
// C-face times the C-velocity interpolated along d to the d-face; zero through a wall.
template <typename R, int C>
__device__ __forceinline__ void momentum_terms(const Geo<R>& g, const R* __restrict__ a, const R* __restrict__ b,
                                               int N, const Cell<R>& c, R& conv, R& lap) {
  const R* aC = a + C * N;
  const R* bC = b + C * N;
  const int pc = c.p[C], nc = g.n[C];
  const int o = c.o, sC = c.s[C];
  const R aH = ld(aC, o), bH = ld(bC, o);
  const R aM = (pc >= 2) ? ld(aC, o - sC) : R(0);
  const R bM = (pc >= 2) ? ld(bC, o - sC) : R(0);
  const R aP = (pc + 1 < nc) ? ld(aC, o + sC) : R(0);
  const R bP = (pc + 1 < nc) ? ld(bC, o + sC) : R(0);
  const R idcC = g.idc[C][pc];
  const R aE = R(0.5) * (aH + aP), bE = R(0.5) * (bH + bP);
  const R aW = R(0.5) * (aM + aH), bW = R(0.5) * (bM + bH);
  conv = R(2) * (aE * bE - aW * bW) * idcC;
  lap = ((bP - bH) * g.idx[C][pc] - (bH - bM) * g.idx[C][pc - 1]) * idcC;
  const R wlC = g.wl[C][pc], wrC = g.wr[C][pc];
#pragma unroll
  for (int t = 1; t <= 2; ++t) {
    const int D = (C + t) % 3;
    const R* aD = a + D * N;
    const R* bD = b + D * N;
    const int pd = c.p[D], nd = g.n[D];
    const int sD = c.s[D];
    R fLo = R(0), fHi = R(0), gLo, gHi;
    if (pd >= 1) {  // lower d-face is interior
      const R aDc = wlC * ld(aD, o - sC) + wrC * ld(aD, o);
      const R bDc = wlC * ld(bD, o - sC) + wrC * ld(bD, o);
      const R bCm = ld(bC, o - sD), aCm = ld(aC, o - sD);
      const R aCd = g.wl[D][pd] * aCm + g.wr[D][pd] * aH;
      const R bCd = g.wl[D][pd] * bCm + g.wr[D][pd] * bH;
      fLo = aDc * bCd + bDc * aCd;
      gLo = (bH - bCm) * g.idc[D][pd];
    } else {
      gLo = bH * g.idc[D][0];
    }
    if (pd + 1 <= nd - 1) {  // upper d-face is interior
      const int oU = o + sD;
      const R aDc = wlC * ld(aD, oU - sC) + wrC * ld(aD, oU);
      const R bDc = wlC * ld(bD, oU - sC) + wrC * ld(bD, oU);
      const R bCp = ld(bC, oU), aCp = ld(aC, oU);
      const R aCd = g.wl[D][pd + 1] * aH + g.wr[D][pd + 1] * aCp;
      const R bCd = g.wl[D][pd + 1] * bH + g.wr[D][pd + 1] * bCp;
      fHi = aDc * bCd + bDc * aCd;
      gHi = (bCp - bH) * g.idc[D][pd + 1];
    } else {
      gHi = -bH * g.idc[D][nd];
    }
    const R ixD = g.idx[D][pd];
    conv += (fHi - fLo) * ixD;
    lap += (gHi - gLo) * ixD;
  }
}

// Temperature at the cell: conv = div(a_vel T_b) + div(b_vel T_a); lap = Lap T_b with T = T_hot at
// x = 0 and 0 at x = 1 (Eq. 4), zero flux through the y and z walls (Eqs. 5-6).
template <typename R>
__device__ __forceinline__ void temperature_terms(const Geo<R>& g, const R* __restrict__ a, const R* __restrict__ b,
                                                  int N, const Cell<R>& c, R T_hot, R& conv, R& lap) {
  const R* Ta = a + 3 * N;
  const R* Tb = b + 3 * N;
  const int o = c.o;
  const R TaH = ld(Ta, o), TbH = ld(Tb, o);
  conv = R(0);
  lap = R(0);
#pragma unroll
  for (int D = 0; D < 3; ++D) {
    const R* aD = a + D * N;
    const R* bD = b + D * N;
    const int pd = c.p[D], nd = g.n[D];
    const int sD = c.s[D];
    R fLo = R(0), fHi = R(0), gLo = R(0), gHi = R(0);
    if (pd >= 1) {
      const R Tam = ld(Ta, o - sD), Tbm = ld(Tb, o - sD);
      const R wl = g.wl[D][pd], wr = g.wr[D][pd];
      fLo = ld(aD, o) * (wl * Tbm + wr * TbH) + ld(bD, o) * (wl * Tam + wr * TaH);
      gLo = (TbH - Tbm) * g.idc[D][pd];
    } else if (D == 0) {
      gLo = (TbH - T_hot) * g.idc[0][0];
    }
    if (pd + 1 <= nd - 1) {
      const int oU = o + sD;
      const R Tap = ld(Ta, oU), Tbp = ld(Tb, oU);
      const R wl = g.wl[D][pd + 1], wr = g.wr[D][pd + 1];
      fHi = ld(aD, oU) * (wl * TbH + wr * Tbp) + ld(bD, oU) * (wl * TaH + wr * Tap);
      gHi = (Tbp - TbH) * g.idc[D][pd + 1];
    } else if (D == 0) {
      gHi = -TbH * g.idc[0][nd];
    }
    const R ixD = g.idx[D][pd];
    conv += (fHi - fLo) * ixD;
    lap += (gHi - gLo) * ixD;
  }
}

template <typename R>
__device__ __forceinline__ bool cell_of_thread(const Geo<R>& g, Cell<R>& c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z * blockDim.z + threadIdx.z;
  if (i >= g.n[0] || j >= g.n[1] || k >= g.n[2]) return false;
  c.p[0] = i;
  c.p[1] = j;
  c.p[2] = k;
  c.s[0] = 1;
  c.s[1] = g.n[0];
  c.s[2] = g.n[0] * g.n[1];
  c.o = (k * g.n[1] + j) * g.n[0] + i;
  return true;
}

// mode 0: residual  out = -S(q,q)/2 + Lap q (+ Dirichlet data) + Gr T_q e_z
// mode 1: J.v       out = -S(q,v) + Lap v + Gr T_v e_z - sigma v
template <typename R, int MODE>
__global__ void __launch_bounds__(256) k_stencil(Geo<R> g, int N, R Gr, R invPr, R sigma,
                                                  const R* __restrict__ q, const R* __restrict__ v,
                                                  R* __restrict__ out) {
  Cell<R> c;
  if (!cell_of_thread(g, c)) return;
  const R* b = (MODE == 0) ? q : v;
  const R half = (MODE == 0) ? R(0.5) : R(1);
  R conv, lap;
  // u
  if (c.p[0] >= 1) {
    momentum_terms<R, 0>(g, q, b, N, c, conv, lap);
    R r = lap - half * conv;
    if (MODE == 1) r -= sigma * ld(v, c.o);
    out[c.o] = r;
  } else {
    out[c.o] = R(0);
  }
  // v
  if (c.p[1] >= 1) {
    momentum_terms<R, 1>(g, q, b, N, c, conv, lap);
    R r = lap - half * conv;
    if (MODE == 1) r -= sigma * ld(v, N + c.o);
    out[N + c.o] = r;
  } else {
    out[N + c.o] = R(0);
  }
  // w (+ buoyancy Gr T interpolated to the z-face)
  if (c.p[2] >= 1) {
    momentum_terms<R, 2>(g, q, b, N, c, conv, lap);
    const R* Tb = b + 3 * N;
    const R Tf = g.wl[2][c.p[2]] * ld(Tb, c.o - c.s[2]) + g.wr[2][c.p[2]] * ld(Tb, c.o);
    R r = lap - half * conv + Gr * Tf;
    if (MODE == 1) r -= sigma * ld(v, 2 * N + c.o);
    out[2 * N + c.o] = r;
  } else {
    out[2 * N + c.o] = R(0);
  }
  // T
  temperature_terms<R>(g, q, b, N, c, (MODE == 0) ? R(1) : R(0), conv, lap);
  R r = lap * invPr - half * conv;
  if (MODE == 1) r -= sigma * ld(v, 3 * N + c.o);
  out[3 * N + c.o] = r;
}

// rhs = D vel:  sum_d (vel_d(face p+1) - vel_d(face p)) / width, wall fluxes zero
template <typename R>
__global__ void __launch_bounds__(256) k_divergence(Geo<R> g, int N, const R* __restrict__ vel,
                                                     R* __restrict__ rhs) {
  Cell<R> c;
  if (!cell_of_thread(g, c)) return;
  R acc = R(0);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const R* f = vel + d * N;
    const R lo = (c.p[d] >= 1) ? ld(f, c.o) : R(0);
    const R hi = (c.p[d] + 1 < g.n[d]) ? ld(f, c.o + c.s[d]) : R(0);
    acc += (hi - lo) * g.idx[d][c.p[d]];
  }
  rhs[c.o] = acc;
}

// out = alpha (Y - G phi) + beta v + gamma w, G phi = (phi(cell) - phi(cell - e_d)) / spacing on interior
// faces; T gets no gradient.  Wall slots -> 0.  out may alias Y or w (each element is read, then written,
// by the same thread).
template <typename R>
__global__ void __launch_bounds__(256) k_correct(Geo<R> g, int N, const R* Y, const R* __restrict__ phi,
                                                  R alpha, const R* v, R beta, const R* w, R gamma, R* out) {
  Cell<R> c;
  if (!cell_of_thread(g, c)) return;
  const R ph = ld(phi, c.o);
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    const int o = d * N + c.o;
    R r;
    if (d < 3) {
      if (c.p[d] == 0) {
        out[o] = R(0);
        continue;
      }
      const R G = (ph - ld(phi, c.o - c.s[d])) * g.idc[d][c.p[d]];
      r = alpha * (Y[o] - G);
    } else {
      r = alpha * Y[o];
    }
    if (v) r += beta * v[o];
    if (w) r += gamma * w[o];
    out[o] = r;
  }
}

template <typename R>
const Geo<R>& geo_of(const fv_grid_s* g);
template <>
const Geo<double>& geo_of<double>(const fv_grid_s* g) { return g->geo64; }
template <>
const Geo<float>& geo_of<float>(const fv_grid_s* g) { return g->geo32; }

inline void cell_grid(const fv_grid_s* g, dim3& grid, dim3& block) {
  block = dim3(32, 4, 2);
  grid = dim3((g->nx + block.x - 1) / block.x, (g->ny + block.y - 1) / block.y, (g->nz + block.z - 1) / block.z);
}

}  // namespace

template <typename R>
int launch_residual(const fv_grid_s* g, double Gr, const R* q, R* F) {
  dim3 grid, block;
  cell_grid(g, grid, block);
  ProfScope ps(g, PROF_STENCIL);
  k_stencil<R, 0><<<grid, block, 0, g->stream>>>(geo_of<R>(g), (int)g->N, (R)Gr, (R)(1.0 / g->Pr), R(0), q, q, F);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

template <typename R>
int launch_jvp(const fv_grid_s* g, double Gr, double sigma, const R* q, const R* v, R* out) {
  dim3 grid, block;
  cell_grid(g, grid, block);
  ProfScope ps(g, PROF_STENCIL);
  k_stencil<R, 1><<<grid, block, 0, g->stream>>>(geo_of<R>(g), (int)g->N, (R)Gr, (R)(1.0 / g->Pr), (R)sigma, q, v, out);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

template <typename R>
int launch_divergence(const fv_grid_s* g, const R* vel, R* rhs) {
  dim3 grid, block;
  cell_grid(g, grid, block);
  ProfScope ps(g, PROF_DIVERGENCE);
  k_divergence<R><<<grid, block, 0, g->stream>>>(geo_of<R>(g), (int)g->N, vel, rhs);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

template <typename R>
int launch_correct(const fv_grid_s* g, const R* Y, const R* phi, double alpha, const R* v, double beta,
                   const R* w, double gamma, R* out) {
  dim3 grid, block;
  cell_grid(g, grid, block);
  ProfScope ps(g, PROF_CORRECT);
  k_correct<R><<<grid, block, 0, g->stream>>>(geo_of<R>(g), (int)g->N, Y, phi, (R)alpha, v, (R)beta, w, (R)gamma, out);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

template int launch_residual<double>(const fv_grid_s*, double, const double*, double*);
template int launch_jvp<double>(const fv_grid_s*, double, double, const double*, const double*, double*);
template int launch_jvp<float>(const fv_grid_s*, double, double, const float*, const float*, float*);
template int launch_divergence<double>(const fv_grid_s*, const double*, double*);
template int launch_divergence<float>(const fv_grid_s*, const float*, float*);
template int launch_correct<double>(const fv_grid_s*, const double*, const double*, double, const double*, double,
                                    const double*, double, double*);
template int launch_correct<float>(const fv_grid_s*, const float*, const float*, double, const float*, double,
                                   const float*, double, float*);

}  // namespace fv
