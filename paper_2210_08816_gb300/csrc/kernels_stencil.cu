// Stencil kernels of the staggered finite-volume discretisation (Section 2, Eqs. 1-6):
//   residual F(q; Gr), Jacobian-vector product J(q) v, divergence D, and the fused
//   gradient correction of the projection.
//
// One thread per cell (i, j, k) produces the four outputs that live in that cell's slots: the
// x-face u at x_f[i], the y-face v at y_f[j], the z-face w at z_f[k] and T at the centre.
// Wall slots (i == 0 for u, ...) are written as zero.  Inputs are read through the read-only
// path; the neighbour re-reads of a block are served by L1/L2, so DRAM sees each field ~once.
#include <cstring>

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

// ------------------------------------------------------------------------------------------------
// z-marching variant.  A block owns a 32 x 8 (x, y) tile of cells and marches over a chunk of kZChunk
// planes.  For every input array it keeps the planes k-1, k, k+1 of the tile plus a one-cell x/y halo in
// a 4-slot shared-memory ring (slot = plane mod 4); cp.async copies of plane k+2 fly while plane k is
// computed.  Each input element is read from global memory ~1.3 times (halo) instead of ~7 times
// through L1 as in the one-thread-per-cell kernel.
// Plane tile of one array in shared memory: kHY rows of kPW elements; the cell (tx, ty) sits at row ty + 1,
// column tx + kX0 (columns kX0 - 1 .. kX0 + kTX hold the x halo; the TMA box starts 4 columns left of the
// tile so that its x coordinate stays on a 16-byte boundary).
constexpr int kTX = 32, kTY = 8, kHY = kTY + 2, kPW = 40, kX0 = 4, kPL = kHY * kPW, kZChunk = 32;

template <typename R, int NA>
struct Ring {
  const R* p[3];  // per dz in {-1, 0, +1}: this thread's cell in array 0's slot of that plane
  // array a sits a * kPL further on within a plane slot (a, dx, dy, dz are compile-time constants)
  __device__ __forceinline__ R at(int a, int dx, int dy, int dz) const {
    return p[dz + 1][a * kPL + dy * kPW + dx];
  }
};

__host__ __device__ constexpr int unit(int d, int c) { return d == c ? 1 : 0; }

// The metric values one cell uses along one axis (cell index c): x and y bundles are loaded once per
// thread, the z bundle once per plane.
template <typename R>
struct AxM {
  R ix, ixm;     // 1 / width of cells c and c-1
  R ic, icp;     // 1 / spacing across faces c and c+1 (2 / width at a wall)
  R wl, wr;      // interpolation weights at face c
  R wlp, wrp;    // ... and at face c+1
  R ic0, icn;    // faces 0 and n (walls)
};

template <typename R>
__device__ __forceinline__ AxM<R> load_axm(const Geo<R>& g, int d, int c) {
  AxM<R> m;
  const int n = g.n[d];
  m.ix = g.idx[d][c];
  m.ixm = c >= 1 ? g.idx[d][c - 1] : R(0);
  m.ic = g.idc[d][c];
  m.icp = g.idc[d][c + 1];
  m.wl = g.wl[d][c];
  m.wr = g.wr[d][c];
  m.wlp = c + 1 <= n ? g.wl[d][c + 1] : R(0);
  m.wrp = c + 1 <= n ? g.wr[d][c + 1] : R(0);
  m.ic0 = g.idc[d][0];
  m.icn = g.idc[d][n];
  return m;
}

template <int D, typename R>
__device__ __forceinline__ const AxM<R>& axm(const AxM<R>& x, const AxM<R>& y, const AxM<R>& z) {
  return D == 0 ? x : (D == 1 ? y : z);
}

// Same mathematics as momentum_terms / temperature_terms, reading neighbours from the ring.
// Arrays 0..3 are the advecting state a, arrays AB..AB+3 the advected field b (AB = 0 for F, 4 for J.v).
// GHOST (J.v, homogeneous wall data): the wall cases need no branches, because the general formulas give
// them when they read zeros there: the face-normal wall slot 0 holds zero, everything outside the domain
// arrives zero-filled in the ring, and the metric arrays hold the wall values (idc[0] = 2 / dx_0,
// idc[n] = 2 / dx_{n-1}, wl = wr = 0 on the wall faces).  Only T's zero-flux walls (y, z) keep theirs.
template <typename R, int C, int NA, int AB, bool GHOST>
__device__ __forceinline__ void momentum_ring(const Geo<R>& g, const Ring<R, NA>& S, const int p[3], const AxM<R>& mx,
                                              const AxM<R>& my, const AxM<R>& mz, R& conv, R& lap) {
  constexpr int cx = unit(C, 0), cy = unit(C, 1), cz = unit(C, 2);
  const AxM<R>& MC = axm<C>(mx, my, mz);
  const int pc = p[C], nc = g.n[C];
  const R aH = S.at(C, 0, 0, 0), bH = S.at(AB + C, 0, 0, 0);
  const R aM = (GHOST || pc >= 2) ? S.at(C, -cx, -cy, -cz) : R(0);
  const R bM = (GHOST || pc >= 2) ? S.at(AB + C, -cx, -cy, -cz) : R(0);
  const R aP = (GHOST || pc + 1 < nc) ? S.at(C, cx, cy, cz) : R(0);
  const R bP = (GHOST || pc + 1 < nc) ? S.at(AB + C, cx, cy, cz) : R(0);
  const R aE = R(0.5) * (aH + aP), bE = R(0.5) * (bH + bP);
  const R aW = R(0.5) * (aM + aH), bW = R(0.5) * (bM + bH);
  conv = R(2) * (aE * bE - aW * bW) * MC.ic;
  lap = ((bP - bH) * MC.ix - (bH - bM) * MC.ixm) * MC.ic;
  const R wlC = MC.wl, wrC = MC.wr;
#pragma unroll
  for (int t = 1; t <= 2; ++t) {
    const int D = (C + t) % 3;
    const AxM<R>& MD = (D == 0) ? mx : (D == 1 ? my : mz);
    const int dx = unit(D, 0), dy = unit(D, 1), dz = unit(D, 2);
    const int pd = p[D], nd = g.n[D];
    R fLo = R(0), fHi = R(0), gLo, gHi;
    if (GHOST || pd >= 1) {
      const R aDc = wlC * S.at(D, -cx, -cy, -cz) + wrC * S.at(D, 0, 0, 0);
      const R bDc = wlC * S.at(AB + D, -cx, -cy, -cz) + wrC * S.at(AB + D, 0, 0, 0);
      const R bCm = S.at(AB + C, -dx, -dy, -dz), aCm = S.at(C, -dx, -dy, -dz);
      const R aCd = MD.wl * aCm + MD.wr * aH;
      const R bCd = MD.wl * bCm + MD.wr * bH;
      fLo = aDc * bCd + bDc * aCd;
      gLo = (bH - bCm) * MD.ic;
    } else {
      gLo = bH * MD.ic0;
    }
    if (GHOST || pd + 1 <= nd - 1) {
      const R aDc = wlC * S.at(D, dx - cx, dy - cy, dz - cz) + wrC * S.at(D, dx, dy, dz);
      const R bDc = wlC * S.at(AB + D, dx - cx, dy - cy, dz - cz) + wrC * S.at(AB + D, dx, dy, dz);
      const R bCp = S.at(AB + C, dx, dy, dz), aCp = S.at(C, dx, dy, dz);
      const R aCd = MD.wlp * aH + MD.wrp * aCp;
      const R bCd = MD.wlp * bH + MD.wrp * bCp;
      fHi = aDc * bCd + bDc * aCd;
      gHi = (bCp - bH) * MD.icp;
    } else {
      gHi = -bH * MD.icn;
    }
    conv += (fHi - fLo) * MD.ix;
    lap += (gHi - gLo) * MD.ix;
  }
}

template <typename R, int NA, int AB, bool GHOST>
__device__ __forceinline__ void temperature_ring(const Geo<R>& g, const Ring<R, NA>& S, const int p[3],
                                                 const AxM<R>& mx, const AxM<R>& my, const AxM<R>& mz, R T_hot,
                                                 R& conv, R& lap) {
  const R TaH = S.at(3, 0, 0, 0), TbH = S.at(AB + 3, 0, 0, 0);
  conv = R(0);
  lap = R(0);
#pragma unroll
  for (int D = 0; D < 3; ++D) {
    const AxM<R>& MD = (D == 0) ? mx : (D == 1 ? my : mz);
    const int dx = unit(D, 0), dy = unit(D, 1), dz = unit(D, 2);
    const int pd = p[D], nd = g.n[D];
    R fLo = R(0), fHi = R(0), gLo = R(0), gHi = R(0);
    if constexpr (GHOST) {  // one basic block: x Dirichlet T = 0 by the ghost zero, y / z zero flux by a select
      const R Tam = S.at(3, -dx, -dy, -dz), Tbm = S.at(AB + 3, -dx, -dy, -dz);
      fLo = S.at(D, 0, 0, 0) * (MD.wl * Tbm + MD.wr * TbH) + S.at(AB + D, 0, 0, 0) * (MD.wl * Tam + MD.wr * TaH);
      gLo = (D == 0 || pd >= 1) ? (TbH - Tbm) * MD.ic : R(0);
      const R Tap = S.at(3, dx, dy, dz), Tbp = S.at(AB + 3, dx, dy, dz);
      fHi = S.at(D, dx, dy, dz) * (MD.wlp * TbH + MD.wrp * Tbp) +
            S.at(AB + D, dx, dy, dz) * (MD.wlp * TaH + MD.wrp * Tap);
      gHi = (D == 0 || pd + 1 <= nd - 1) ? (Tbp - TbH) * MD.icp : R(0);
    } else if (pd >= 1) {
      const R Tam = S.at(3, -dx, -dy, -dz), Tbm = S.at(AB + 3, -dx, -dy, -dz);
      fLo = S.at(D, 0, 0, 0) * (MD.wl * Tbm + MD.wr * TbH) + S.at(AB + D, 0, 0, 0) * (MD.wl * Tam + MD.wr * TaH);
      gLo = (TbH - Tbm) * MD.ic;
    } else if (D == 0) {
      gLo = (TbH - T_hot) * MD.ic0;
    }
    if constexpr (!GHOST) {
      if (pd + 1 <= nd - 1) {
        const R Tap = S.at(3, dx, dy, dz), Tbp = S.at(AB + 3, dx, dy, dz);
        fHi = S.at(D, dx, dy, dz) * (MD.wlp * TbH + MD.wrp * Tbp) +
              S.at(AB + D, dx, dy, dz) * (MD.wlp * TaH + MD.wrp * Tap);
        gHi = (Tbp - TbH) * MD.icp;
      } else if (D == 0) {
        gHi = -TbH * MD.icn;
      }
    }
    conv += (fHi - fLo) * MD.ix;
    lap += (gHi - gLo) * MD.ix;
  }
}

// cp.async copy of one element (4 or 8 bytes); src_bytes = 0 fills the destination with zero (halo outside
// the box)
template <int BYTES>
__device__ __forceinline__ void cp_async_elem(void* dst, const void* src, int src_bytes) {
  static_assert(BYTES == 4 || BYTES == 8, "element size");
  if (BYTES == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(src_bytes)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

constexpr int kRing = 4;  // planes k-1, k, k+1 in use, k+2 in flight

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ bool bar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait on an mbarrier phase (at most `spins` polls); on expiry records code 16 in *err
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity, int* err, long long spins) {
  for (long long i = 0; i < spins; ++i)
    if (bar_try(bar, parity)) return true;
  atomicCAS(err, 0, 16);
  return false;
}

// MODE 0: residual (arrays: q), MODE 1: J.v (arrays: q then v).  use_tma: plane tiles arrive by one 4D TMA
// box per state (x, y, z, field) with zero fill outside the domain; otherwise by per-element cp.async.
template <typename R, int MODE>
__global__ void __launch_bounds__(kTX * kTY, sizeof(R) == 4 ? 3 : 2)
    k_stencil_z(const __grid_constant__ CUtensorMap tmq, const __grid_constant__ CUtensorMap tmv, int use_tma,
                int* err, long long spins, Geo<R> g, int N, R Gr, R invPr, R sigma, const R* __restrict__ q, const R* __restrict__ v,
                R* __restrict__ out, int nch) {
  constexpr int NA = (MODE == 0) ? 4 : 8;
  constexpr int AB = (MODE == 0) ? 0 : 4;
  constexpr int NWARP = kTX * kTY / 32;
  constexpr uint32_t kBox = 4u * kPL * sizeof(R);  // one state's box: 4 fields x kHY x kPW
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar[kRing];
  R* sm = reinterpret_cast<R*>(smem_raw);  // [kRing][NA][kPL]
  const int tid = threadIdx.x;
  const int tx = tid % kTX, ty = tid / kTX;
  const int warp = tid / 32, lane = tid % 32;
  // blockIdx.z = z-chunk + nch * vector: vector `vec` of a block of states stored one after another in v and
  // out (4N elements each); its fields are fields 4 vec .. 4 vec + 3 of the tensor map tmv
  const int vec = (int)blockIdx.z / nch;
  const int i0 = blockIdx.x * kTX, j0 = blockIdx.y * kTY, k0 = ((int)blockIdx.z - vec * nch) * kZChunk;
  v += (size_t)vec * 4 * N;
  out += (size_t)vec * 4 * N;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int kend = min(k0 + kZChunk, nz);
  if (use_tma && tid == 0) {
    for (int s = 0; s < kRing; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar[s])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto issue_plane = [&](int kk) {
    R* slot = sm + ((kk + kRing) % kRing) * NA * kPL;
    const bool kin = (kk >= 0 && kk < nz);
    if (use_tma) {
      const uint32_t b = smem_addr(&bar[(kk + kRing) % kRing]);
      if (kin) {
        if (tid == 0) {
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(kBox * (NA / 4))
                       : "memory");
          asm volatile(
              "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, "
              "%5, %6}], [%2];" ::"r"(smem_addr(slot)),
              "l"(reinterpret_cast<uint64_t>(&tmq)), "r"(b), "r"(i0 - kX0), "r"(j0 - 1), "r"(kk), "r"(0)
              : "memory");
          if (NA == 8)
            asm volatile(
                "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
                "%4, %5, %6}], [%2];" ::"r"(smem_addr(slot + 4 * kPL)),
                "l"(reinterpret_cast<uint64_t>(&tmv)), "r"(b), "r"(i0 - kX0), "r"(j0 - 1), "r"(kk), "r"(4 * vec)
                : "memory");
        }
      } else {  // a plane outside the domain: zeros, and a plain arrival completes the barrier phase
        for (int e = tid; e < NA * kPL; e += kTX * kTY) slot[e] = R(0);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (tid == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(b) : "memory");
      }
      return;
    }
    // warp w copies halo rows w, w + NWARP, ...; lane l copies columns l and 32 + l of the (kTX + 2) halo row
    for (int row = warp; row < NA * kHY; row += NWARP) {
      const int arr = row / kHY, hy = row - arr * kHY;
      const int j = j0 + hy - 1;
      const R* base = (arr < 4) ? q + arr * N : v + (arr - 4) * N;
      const bool rin = kin && j >= 0 && j < ny;
      const int roff = (kk * ny + j) * nx + i0 - 1;
      for (int hx = lane; hx < kTX + 2; hx += 32) {
        const int i = i0 + hx - 1;
        const bool in = rin && i >= 0 && i < nx;
        cp_async_elem<sizeof(R)>(slot + arr * kPL + hy * kPW + (kX0 - 1) + hx, in ? base + roff + hx : base,
                                 in ? (int)sizeof(R) : 0);
      }
    }
    cp_async_commit();
  };
  // plane kk lives in slot kk mod kRing; it is that slot's use number (kk - k0 + 1) / kRing
  auto wait_plane = [&](int kk) -> bool {
    if (!use_tma) return true;
    return bar_wait(smem_addr(&bar[(kk + kRing) % kRing]), (uint32_t)(((kk - k0 + 1) / kRing) & 1), err, spins);
  };
  issue_plane(k0 - 1);
  issue_plane(k0);
  issue_plane(k0 + 1);
  int issued = k0 + 1;  // last plane whose copy was started (the same value in every thread)
  if (!use_tma) cp_async_wait_all();
  __syncthreads();
  bool ok = wait_plane(k0 - 1);
  ok = wait_plane(k0) && ok;
  ok = __syncthreads_and(ok);  // one decision for the whole CTA
  const int i = i0 + tx, j = j0 + ty;
  const bool active = (i < nx && j < ny);
  const R half = (MODE == 0) ? R(0.5) : R(1);
  const AxM<R> mx = load_axm(g, 0, active ? i : 0), my = load_axm(g, 1, active ? j : 0);
  for (int k = k0; k < kend && ok; ++k) {
    if (k + 2 <= kend) {  // plane k+2 feeds the output plane k+1
      issue_plane(k + 2);
      issued = k + 2;
    }
    const bool ready = wait_plane(k + 1);
    if (active && ready) {
      const AxM<R> mz = load_axm(g, 2, k);
      Ring<R, NA> S;
#pragma unroll
      for (int dz = -1; dz <= 1; ++dz)
        S.p[dz + 1] = sm + ((k + dz + kRing) % kRing) * NA * kPL + (ty + 1) * kPW + (tx + kX0);
      const int p[3] = {i, j, k};
      const int o = (k * ny + j) * nx + i;
      R conv, lap;
      if constexpr (MODE == 1) {
        // J.v: all four equations in one basic block (the wall outputs by selects), so that the compiler
        // can share the ring loads between them
        momentum_ring<R, 0, NA, AB, true>(g, S, p, mx, my, mz, conv, lap);
        const R r0 = lap - conv - sigma * S.at(AB + 0, 0, 0, 0);
        momentum_ring<R, 1, NA, AB, true>(g, S, p, mx, my, mz, conv, lap);
        const R r1 = lap - conv - sigma * S.at(AB + 1, 0, 0, 0);
        momentum_ring<R, 2, NA, AB, true>(g, S, p, mx, my, mz, conv, lap);
        const R Tf = mz.wl * S.at(AB + 3, 0, 0, -1) + mz.wr * S.at(AB + 3, 0, 0, 0);
        const R r2 = lap - conv + Gr * Tf - sigma * S.at(AB + 2, 0, 0, 0);
        temperature_ring<R, NA, AB, true>(g, S, p, mx, my, mz, R(0), conv, lap);
        const R r3 = lap * invPr - conv - sigma * S.at(AB + 3, 0, 0, 0);
        out[o] = (i >= 1) ? r0 : R(0);
        out[N + o] = (j >= 1) ? r1 : R(0);
        out[2 * N + o] = (k >= 1) ? r2 : R(0);
        out[3 * N + o] = r3;
      } else {
        if (i >= 1) {
          momentum_ring<R, 0, NA, AB, MODE == 1>(g, S, p, mx, my, mz, conv, lap);
          R r = lap - half * conv;
          if (MODE == 1) r -= sigma * S.at(AB + 0, 0, 0, 0);
          out[o] = r;
        } else {
          out[o] = R(0);
        }
        if (j >= 1) {
          momentum_ring<R, 1, NA, AB, MODE == 1>(g, S, p, mx, my, mz, conv, lap);
          R r = lap - half * conv;
          if (MODE == 1) r -= sigma * S.at(AB + 1, 0, 0, 0);
          out[N + o] = r;
        } else {
          out[N + o] = R(0);
        }
        if (k >= 1) {
          momentum_ring<R, 2, NA, AB, MODE == 1>(g, S, p, mx, my, mz, conv, lap);
          const R Tf = mz.wl * S.at(AB + 3, 0, 0, -1) + mz.wr * S.at(AB + 3, 0, 0, 0);
          R r = lap - half * conv + Gr * Tf;
          if (MODE == 1) r -= sigma * S.at(AB + 2, 0, 0, 0);
          out[2 * N + o] = r;
        } else {
          out[2 * N + o] = R(0);
        }
        temperature_ring<R, NA, AB, MODE == 1>(g, S, p, mx, my, mz, (MODE == 0) ? R(1) : R(0), conv, lap);
        R r = lap * invPr - half * conv;
        if (MODE == 1) r -= sigma * S.at(AB + 3, 0, 0, 0);
        out[3 * N + o] = r;
      }
    }
    if (!use_tma) cp_async_wait_all();  // plane k+2 has landed
    ok = __syncthreads_and(ready);      // nobody reads the slot of plane k-1 any more; stop together
  }
  // give-up path: every plane copy still in flight lands (waited for with the full limit) before the CTA
  // exits, so that no bulk copy writes into shared memory the CTA no longer owns
  if (!ok && use_tma && tid == 0)
    for (int kk = max(k0 - 1, issued - kRing + 1); kk <= issued; ++kk)
      bar_wait(smem_addr(&bar[(kk + kRing) % kRing]), (uint32_t)(((kk - k0 + 1) / kRing) & 1), err, 1LL << 22);
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
// by the same thread).  With part != null every block also writes the partial sum of out^2 over its cells
// to part[linear block index] (FP32 data: compensated float pairs up to the warp, FP64 above).
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float x) {
  const float s = hi + x, bb = s - hi;
  lo += (hi - (s - bb)) + (x - bb);
  hi = s;
}

template <typename R>
__global__ void __launch_bounds__(256) k_correct(Geo<R> g, int N, const R* Y, const R* __restrict__ phi,
                                                  R alpha, const R* v, R beta, const R* w, R gamma, R* out,
                                                  double* __restrict__ part) {
  Cell<R> c;
  const bool act = cell_of_thread(g, c);
  float shi = 0.f, slo = 0.f;  // FP32 data
  double sd = 0.0;             // FP64 data
  if (act) {
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
      if (part) {
        if (sizeof(R) == 4) {
          const float rf = (float)r, p2 = rf * rf;
          slo += fmaf(rf, rf, -p2);
          two_sum_add(shi, slo, p2);
        } else {
          sd = fma((double)r, (double)r, sd);
        }
      }
    }
  }
  if (!part) return;
  double wsum;
  if (sizeof(R) == 4) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float h2 = __shfl_down_sync(0xffffffffu, shi, off), l2 = __shfl_down_sync(0xffffffffu, slo, off);
      slo += l2;
      two_sum_add(shi, slo, h2);
    }
    wsum = (double)shi + (double)slo;
  } else {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) sd += __shfl_down_sync(0xffffffffu, sd, off);
    wsum = sd;
  }
  __shared__ double wpart[8];
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  if ((tid & 31) == 0) wpart[tid >> 5] = wsum;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x * blockDim.y * blockDim.z) / 32; ++i) t += wpart[i];
    part[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = t;
  }
}

// FP32 forms of the divergence and the correction for nx % 4 == 0: a thread owns four x-consecutive cells
// (16-byte loads and stores; the x-neighbour across the quad boundary comes from the next or previous lane)
// and marches over kVZ z-planes, carrying the plane below in registers.  Block 32 x 8 (a warp is one
// x-run of 128 cells).  Same arithmetic, element by element, as k_divergence / k_correct.
constexpr int kVZ = 4;

__device__ __forceinline__ float4 ldg4(const float* __restrict__ p, int o) {
  return __ldg(reinterpret_cast<const float4*>(p + o));
}
__device__ __forceinline__ float4 ld4(const float* p, int o) { return *reinterpret_cast<const float4*>(p + o); }
__device__ __forceinline__ float4 zero4() { return make_float4(0.f, 0.f, 0.f, 0.f); }

// blockIdx.z = z-block + nzc * vector (states of 4N, rhs fields of N, one after another)
__global__ void __launch_bounds__(256) k_divergence4(Geo<float> g, int N, const float* __restrict__ vel,
                                                      float* __restrict__ rhs, int nzc) {
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2], pl = nx * ny;
  const int lane = threadIdx.x;
  const int vec = (int)blockIdx.z / nzc;
  vel += (size_t)vec * 4 * N;
  rhs += (size_t)vec * N;
  const int i0 = 4 * (blockIdx.x * 32 + lane);
  const int j = blockIdx.y * 8 + threadIdx.y;
  const int k0 = ((int)blockIdx.z - vec * nzc) * kVZ, k1 = min(k0 + kVZ, nz);
  const bool act = i0 < nx && j < ny;
  const float* U = vel;
  const float* V = vel + N;
  const float* W = vel + 2 * N;
  float4 rx = zero4();
  float ry = 0.f;
  if (act) {
    rx = make_float4(__ldg(g.idx[0] + i0), __ldg(g.idx[0] + i0 + 1), __ldg(g.idx[0] + i0 + 2), __ldg(g.idx[0] + i0 + 3));
    ry = __ldg(g.idx[1] + j);
  }
  const int ob = act ? (k0 * ny + j) * nx + i0 : 0;
  float4 wlo = (act && k0 >= 1) ? ldg4(W, ob) : zero4();
#pragma unroll
  for (int k = k0; k < k1; ++k) {
    const int o = ob + (k - k0) * pl;
    const float4 u = act ? ldg4(U, o) : zero4();
    float un = __shfl_down_sync(0xffffffffu, u.x, 1);  // u on the face i0 + 4
    if (lane == 31 && act && i0 + 4 < nx) un = __ldg(U + o + 4);
    if (i0 + 4 >= nx) un = 0.f;
    const float ux = (i0 == 0) ? 0.f : u.x;
    if (!act) continue;
    const float4 vlo = (j >= 1) ? ldg4(V, o) : zero4();
    const float4 vhi = (j + 1 < ny) ? ldg4(V, o + nx) : zero4();
    const float4 whi = (k + 1 < nz) ? ldg4(W, o + pl) : zero4();
    const float rz = __ldg(g.idx[2] + k);
    float4 r;
    r.x = (u.y - ux) * rx.x + (vhi.x - vlo.x) * ry + (whi.x - wlo.x) * rz;
    r.y = (u.z - u.y) * rx.y + (vhi.y - vlo.y) * ry + (whi.y - wlo.y) * rz;
    r.z = (u.w - u.z) * rx.z + (vhi.z - vlo.z) * ry + (whi.z - wlo.z) * rz;
    r.w = (un - u.w) * rx.w + (vhi.w - vlo.w) * ry + (whi.w - wlo.w) * rz;
    *reinterpret_cast<float4*>(rhs + o) = r;
    wlo = whi;
  }
}

__device__ __forceinline__ void acc_sq(float& hi, float& lo, float r) {
  const float p2 = r * r;
  lo += fmaf(r, r, -p2);
  two_sum_add(hi, lo, p2);
}

// out = alpha (Y - G phi) + beta v + gamma w on four cells; out may alias Y or w (read, then written,
// by the same thread)
__global__ void __launch_bounds__(256) k_correct4(Geo<float> g, int N, const float* Y, const float* __restrict__ phi,
                                                   float alpha, const float* v, float beta, const float* w,
                                                   float gamma, float* out, double* __restrict__ part, int nzc) {
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2], pl = nx * ny;
  const int lane = threadIdx.x;
  // blockIdx.z = z-block + nzc * vector (Y, v, w, out: states of 4N; phi: fields of N, one after another)
  const int vec = (int)blockIdx.z / nzc;
  if (vec > 0) {
    Y += (size_t)vec * 4 * N;
    phi += (size_t)vec * N;
    if (v) v += (size_t)vec * 4 * N;
    if (w) w += (size_t)vec * 4 * N;
    out += (size_t)vec * 4 * N;
  }
  const int i0 = 4 * (blockIdx.x * 32 + lane);
  const int j = blockIdx.y * 8 + threadIdx.y;
  const int k0 = ((int)blockIdx.z - vec * nzc) * kVZ, k1 = min(k0 + kVZ, nz);
  const bool act = i0 < nx && j < ny;
  float4 cx = zero4();
  float cy = 0.f;
  if (act) {
    cx = make_float4(__ldg(g.idc[0] + i0), __ldg(g.idc[0] + i0 + 1), __ldg(g.idc[0] + i0 + 2),
                     __ldg(g.idc[0] + i0 + 3));
    cy = __ldg(g.idc[1] + j);
  }
  const int ob = act ? (k0 * ny + j) * nx + i0 : 0;
  float4 pzm = (act && k0 >= 1) ? ldg4(phi, ob - pl) : zero4();
  float shi = 0.f, slo = 0.f;
  for (int k = k0; k < k1; ++k) {
    const int o = ob + (k - k0) * pl;
    const float4 ph = act ? ldg4(phi, o) : zero4();
    float pxm = __shfl_up_sync(0xffffffffu, ph.w, 1);  // phi in cell i0 - 1
    if (lane == 0 && act && i0 > 0) pxm = __ldg(phi + o - 1);
    if (!act) continue;
    float4 G[3];
    G[0] = make_float4((ph.x - pxm) * cx.x, (ph.y - ph.x) * cx.y, (ph.z - ph.y) * cx.z, (ph.w - ph.z) * cx.w);
    if (j >= 1) {
      const float4 pym = ldg4(phi, o - nx);
      G[1] = make_float4((ph.x - pym.x) * cy, (ph.y - pym.y) * cy, (ph.z - pym.z) * cy, (ph.w - pym.w) * cy);
    } else {
      G[1] = zero4();
    }
    const float cz = __ldg(g.idc[2] + k);
    G[2] = make_float4((ph.x - pzm.x) * cz, (ph.y - pzm.y) * cz, (ph.z - pzm.z) * cz, (ph.w - pzm.w) * cz);
    pzm = ph;
    const bool wall[3] = {false, j == 0, k == 0};
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      const int od = d * N + o;
      float4 r;
      if (d < 3 && wall[d]) {
        r = zero4();
      } else {
        const float4 y = ld4(Y, od);
        const float4 gd = (d < 3) ? G[d] : zero4();
        r = make_float4(alpha * (y.x - gd.x), alpha * (y.y - gd.y), alpha * (y.z - gd.z), alpha * (y.w - gd.w));
        if (v) {
          const float4 a = ld4(v, od);
          r.x += beta * a.x; r.y += beta * a.y; r.z += beta * a.z; r.w += beta * a.w;
        }
        if (w) {
          const float4 a = ld4(w, od);
          r.x += gamma * a.x; r.y += gamma * a.y; r.z += gamma * a.z; r.w += gamma * a.w;
        }
        if (d == 0 && i0 == 0) r.x = 0.f;  // the x = 0 wall slot
      }
      *reinterpret_cast<float4*>(out + od) = r;
      if (part) {
        acc_sq(shi, slo, r.x);
        acc_sq(shi, slo, r.y);
        acc_sq(shi, slo, r.z);
        acc_sq(shi, slo, r.w);
      }
    }
  }
  if (!part) return;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float h2 = __shfl_down_sync(0xffffffffu, shi, off), l2 = __shfl_down_sync(0xffffffffu, slo, off);
    slo += l2;
    two_sum_add(shi, slo, h2);
  }
  __shared__ double wpart[8];
  const int tid = threadIdx.x + 32 * threadIdx.y;
  if ((tid & 31) == 0) wpart[tid >> 5] = (double)shi + (double)slo;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int i = 0; i < 8; ++i) t += wpart[i];
    part[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = t;
  }
}

inline bool quad_ok(const fv_grid_s* g, std::initializer_list<const void*> ptrs) {
  if (g->nx % 4 != 0) return false;
  for (const void* p : ptrs)
    if (p && ((uintptr_t)p % 16) != 0) return false;
  return true;
}

inline dim3 quad_grid(const fv_grid_s* g) {
  return dim3((g->nx / 4 + 31) / 32, (g->ny + 7) / 8, (g->nz + kVZ - 1) / kVZ);
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

// 4D tensor map of one state (x, y, z, field) with boxes of kPW x kHY x 1 x 4 elements
template <typename R>
int state_map(const fv_grid_s* g, const R* ptr, CUtensorMap* m, int nvec = 1) {
  const size_t sz = sizeof(R);
  const uint64_t dims[4] = {(uint64_t)g->nx, (uint64_t)g->ny, (uint64_t)g->nz, 4 * (uint64_t)nvec};
  const uint64_t strides[3] = {g->nx * sz, (uint64_t)g->nx * g->ny * sz, g->N * sz};
  const uint32_t box[4] = {(uint32_t)kPW, (uint32_t)kHY, 1, 4};
  return encode_tensor_map(m, sizeof(R) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                           ptr, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_NONE);
}

template <typename R, int MODE>
int launch_stencil_z(const fv_grid_s* g, double Gr, double sigma, const R* q, const R* v, R* out, int nvec = 1) {
  constexpr int NA = (MODE == 0) ? 4 : 8;
  const size_t smem = (size_t)NA * kRing * kPL * sizeof(R);
  static bool attr_set = false;
  if (!attr_set) {
    FV_CUDA(cudaFuncSetAttribute(k_stencil_z<R, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_set = true;
  }
  // TMA needs 16-byte aligned rows and base addresses; small grids take the cp.async path
  CUtensorMap tq, tv;
  std::memset(&tq, 0, sizeof(tq));
  std::memset(&tv, 0, sizeof(tv));
  int use_tma = ((g->nx * sizeof(R)) % 16 == 0 && g->nx >= 64 && g->ny >= 16 && ((uintptr_t)q % 16) == 0 &&
                 ((uintptr_t)v % 16) == 0) ? 1 : 0;
  if (use_tma && (state_map<R>(g, q, &tq) != FV_OK || state_map<R>(g, v, &tv, nvec) != FV_OK)) use_tma = 0;
  const int nch = (g->nz + kZChunk - 1) / kZChunk;
  if (nvec < 1 || (long long)nch * nvec > 65535) {
    set_error("launch_stencil_z: too many vectors in one block");
    return FV_EINVAL;
  }
  dim3 grid((g->nx + kTX - 1) / kTX, (g->ny + kTY - 1) / kTY, nch * nvec);
  ProfScope ps(g, PROF_STENCIL);
  k_stencil_z<R, MODE><<<grid, kTX * kTY, smem, g->stream>>>(tq, tv, use_tma, g->ws.err, wait_spins(g), geo_of<R>(g), (int)g->N,
                                                             (R)Gr, (R)(1.0 / g->Pr), (R)sigma, q, v, out, nch);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

template <typename R>
int launch_residual(const fv_grid_s* g, double Gr, const R* q, R* F) {
  return launch_stencil_z<R, 0>(g, Gr, 0.0, q, q, F);
}

template <typename R>
int launch_jvp_block(const fv_grid_s* g, double Gr, double sigma, const R* q, const R* v, R* out, int nvec) {
  return launch_stencil_z<R, 1>(g, Gr, sigma, q, v, out, nvec);
}

template <typename R>
int launch_jvp(const fv_grid_s* g, double Gr, double sigma, const R* q, const R* v, R* out) {
  if constexpr (sizeof(R) == 4) {  // two cells per thread (kernels_stencil2.cu) where its tiles fit
    if (stencil_pair_eligible(g, q, v)) return launch_stencil_pair(g, Gr, sigma, q, v, out);
  }
  return launch_stencil_z<R, 1>(g, Gr, sigma, q, v, out);
}

template <typename R>
int launch_divergence(const fv_grid_s* g, const R* vel, R* rhs, int nvec) {
  dim3 grid, block;
  cell_grid(g, grid, block);
  ProfScope ps(g, PROF_DIVERGENCE);
  if constexpr (sizeof(R) == 4) {
    if (quad_ok(g, {vel, rhs})) {
      dim3 qg = quad_grid(g);
      const int nzc = (int)qg.z;
      if ((long long)nzc * nvec > 65535) {
        set_error("launch_divergence: too many vectors in one block");
        return FV_EINVAL;
      }
      qg.z = nzc * nvec;
      k_divergence4<<<qg, dim3(32, 8), 0, g->stream>>>(g->geo32, (int)g->N, vel, rhs, nzc);
      FV_CUDA(cudaGetLastError());
      return FV_OK;
    }
  }
  for (int i = 0; i < nvec; ++i) {
    k_divergence<R><<<grid, block, 0, g->stream>>>(geo_of<R>(g), (int)g->N, vel + (size_t)i * 4 * g->N,
                                                   rhs + (size_t)i * g->N);
    FV_CUDA(cudaGetLastError());
  }
  return FV_OK;
}

template <typename R>
int launch_correct_block(const fv_grid_s* g, const R* Y, const R* phi, const R* v, double beta, R* out, int nvec) {
  bool quad = false;
  if constexpr (sizeof(R) == 4) quad = quad_ok(g, {Y, phi, v, out});
  if (!quad) {
    for (int i = 0; i < nvec; ++i)
      FV_TRY(launch_correct<R>(g, Y + (size_t)i * 4 * g->N, phi + (size_t)i * g->N, 1.0,
                               v ? v + (size_t)i * 4 * g->N : nullptr, beta, nullptr, 0.0,
                               out + (size_t)i * 4 * g->N, -1));
    return FV_OK;
  }
  if constexpr (sizeof(R) == 4) {
    dim3 qg = quad_grid(g);
    const int nzc = (int)qg.z;
    if ((long long)nzc * nvec > 65535) {
      set_error("launch_correct_block: too many vectors in one block");
      return FV_EINVAL;
    }
    qg.z = nzc * nvec;
    ProfScope ps(g, PROF_CORRECT);
    k_correct4<<<qg, dim3(32, 8), 0, g->stream>>>(g->geo32, (int)g->N, Y, phi, 1.0f, v, (float)beta, nullptr, 0.0f,
                                                  out, nullptr, nzc);
    FV_CUDA(cudaGetLastError());
  }
  return FV_OK;
}

template <typename R>
int launch_correct(const fv_grid_s* g, const R* Y, const R* phi, double alpha, const R* v, double beta,
                   const R* w, double gamma, R* out, int norm_slot) {
  dim3 grid, block;
  cell_grid(g, grid, block);
  bool quad = false;
  if constexpr (sizeof(R) == 4) quad = quad_ok(g, {Y, phi, v, w, out});
  if (quad) grid = quad_grid(g);
  const int nblocks = (int)(grid.x * grid.y * grid.z);
  const bool want = norm_slot >= 0 && nblocks <= kPartialSlots - 64;
  {
    ProfScope ps(g, PROF_CORRECT);
    if constexpr (sizeof(R) == 4) {
      if (quad)
        k_correct4<<<grid, dim3(32, 8), 0, g->stream>>>(g->geo32, (int)g->N, Y, phi, (float)alpha, v, (float)beta, w,
                                                        (float)gamma, out, want ? g->ws.partials : nullptr,
                                                        (int)grid.z);
    }
    if (!quad)
      k_correct<R><<<grid, block, 0, g->stream>>>(geo_of<R>(g), (int)g->N, Y, phi, (R)alpha, v, (R)beta, w,
                                                  (R)gamma, out, want ? g->ws.partials : nullptr);
    FV_CUDA(cudaGetLastError());
  }
  if (want) return launch_sum_partials(g, nblocks, norm_slot);
  if (norm_slot >= 0) return launch_dot<R>(g, out, out, 4 * g->N, norm_slot);
  return FV_OK;
}

template int launch_residual<double>(const fv_grid_s*, double, const double*, double*);
template int launch_jvp<double>(const fv_grid_s*, double, double, const double*, const double*, double*);
template int launch_jvp<float>(const fv_grid_s*, double, double, const float*, const float*, float*);
template int launch_jvp_block<double>(const fv_grid_s*, double, double, const double*, const double*, double*, int);
template int launch_jvp_block<float>(const fv_grid_s*, double, double, const float*, const float*, float*, int);
template int launch_divergence<double>(const fv_grid_s*, const double*, double*, int);
template int launch_divergence<float>(const fv_grid_s*, const float*, float*, int);
template int launch_correct_block<double>(const fv_grid_s*, const double*, const double*, const double*, double,
                                          double*, int);
template int launch_correct_block<float>(const fv_grid_s*, const float*, const float*, const float*, double, float*,
                                         int);
template int launch_correct<double>(const fv_grid_s*, const double*, const double*, double, const double*, double,
                                    const double*, double, double*, int);
template int launch_correct<float>(const fv_grid_s*, const float*, const float*, double, const float*, double,
                                   const float*, double, float*, int);

}  // namespace fv
