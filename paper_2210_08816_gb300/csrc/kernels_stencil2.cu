// J.v (FP32) with two x-adjacent cells per thread.
//
// The same discretisation as the z-marching stencil of kernels_stencil.cu (MAC staggering, conservative
// central fluxes, Form A; Eqs. 1-2 linearised about q, homogeneous wall data), the same plane ring in
// shared memory filled by 4D TMA boxes, but a thread computes the cells (x, y) and (x + 1, y), x even.
// The two cells share most of their x-neighbours, so the ring is read with 8-byte loads (pairs at even
// offsets) plus scalars (odd offsets): about half the shared-memory loads per cell, the instruction
// stream that bounded the one-cell form.  Block: 64 x 8 cells (256 threads), z-chunks of 32 planes.
// Wall cases without branches as in the one-cell J.v form: the face-normal wall slot holds zero, the
// halo outside the domain arrives zero-filled, and the metric arrays hold the wall values; only T's
// zero-flux walls (y, z) are selects.
#include <cstring>

#include "fv_internal.h"

namespace fv {
namespace {

constexpr int kPX = 64, kPY = 8, kPHY = kPY + 2;
constexpr int kPW2 = 72;            // ring row: x from i0 - 4 to i0 + 67 (TMA x start on a 16-byte boundary)
constexpr int kPX0 = 4;             // column of the tile's first cell
constexpr int kPL2 = kPHY * kPW2;   // one array's plane tile
constexpr int kPZChunk = 32, kPRing = 4, kPNA = 8;  // default z-chunk (planes marched by one CTA)
constexpr long long kPWaitLimit = 1LL << 22;

// ---------------------------------------------------------------- pair arithmetic
// Blackwell's packed FP32 instructions (PTX add / sub / mul / fma .rn.f32x2): one instruction per pair,
// the same IEEE round-to-nearest results as the two scalar operations.
__device__ __forceinline__ unsigned long long pk(float2 a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ float2 upk(unsigned long long r) {
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
__device__ __forceinline__ float2 operator+(float2 a, float2 b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk(a)), "l"(pk(b)));
  return upk(r);
}
__device__ __forceinline__ float2 operator-(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk(a)), "l"(pk(b)));
  return upk(r);
}
__device__ __forceinline__ float2 operator*(float2 a, float2 b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk(a)), "l"(pk(b)));
  return upk(r);
}
// a * b + c, one rounding
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(pk(a)), "l"(pk(b)), "l"(pk(c)));
  return upk(r);
}
__device__ __forceinline__ float2 bc(float s) { return make_float2(s, s); }

// Metric values of one axis as the stencil uses them (cell index c): per pair (float2, x) or per thread
// (float, y and z).
template <typename T>
struct Bundle {
  T ix, ixm, ic, icp, wl, wr, wlp, wrp;
};

__device__ __forceinline__ Bundle<float> load_bundle(const Geo<float>& g, int d, int c) {
  Bundle<float> m;
  const int n = g.n[d];
  m.ix = __ldg(g.idx[d] + c);
  m.ixm = c >= 1 ? __ldg(g.idx[d] + c - 1) : 0.f;
  m.ic = __ldg(g.idc[d] + c);
  m.icp = __ldg(g.idc[d] + c + 1);
  m.wl = __ldg(g.wl[d] + c);
  m.wr = __ldg(g.wr[d] + c);
  m.wlp = c + 1 <= n ? __ldg(g.wl[d] + c + 1) : 0.f;
  m.wrp = c + 1 <= n ? __ldg(g.wr[d] + c + 1) : 0.f;
  return m;
}

__device__ __forceinline__ Bundle<float2> broadcast(const Bundle<float>& a) {
  Bundle<float2> m;
  m.ix = bc(a.ix);
  m.ixm = bc(a.ixm);
  m.ic = bc(a.ic);
  m.icp = bc(a.icp);
  m.wl = bc(a.wl);
  m.wr = bc(a.wr);
  m.wlp = bc(a.wlp);
  m.wrp = bc(a.wrp);
  return m;
}

__device__ __forceinline__ Bundle<float2> load_bundle_pair(const Geo<float>& g, int c) {
  const Bundle<float> a = load_bundle(g, 0, c), b = load_bundle(g, 0, c + 1);
  Bundle<float2> m;
  m.ix = make_float2(a.ix, b.ix);
  m.ixm = make_float2(a.ixm, b.ixm);
  m.ic = make_float2(a.ic, b.ic);
  m.icp = make_float2(a.icp, b.icp);
  m.wl = make_float2(a.wl, b.wl);
  m.wr = make_float2(a.wr, b.wr);
  m.wlp = make_float2(a.wlp, b.wlp);
  m.wrp = make_float2(a.wrp, b.wrp);
  return m;
}

template <int D>
__device__ __forceinline__ decltype(auto) pick(const Bundle<float2>& x, const Bundle<float2>& y, const Bundle<float2>& z) {
  if constexpr (D == 0)
    return (x);
  else if constexpr (D == 1)
    return (y);
  else
    return (z);
}

__host__ __device__ constexpr int unit_(int d, int c) { return d == c ? 1 : 0; }

// The ring seen from one pair: p[dz + 1] points at the pair's first cell in array 0 of plane k + dz.
struct Ring2 {
  const float* p[3];
  template <int A, int DX, int DY, int DZ>
  __device__ __forceinline__ float2 ld() const {
    const float* s = p[DZ + 1] + A * kPL2 + DY * kPW2 + DX;
    if constexpr ((DX & 1) == 0)
      return *reinterpret_cast<const float2*>(s);  // 8-byte aligned: the pair's column is even
    else
      return make_float2(s[0], s[1]);
  }
};


// Transverse (D != C) fluxes of momentum component C through the D-faces of its control volume:
// the D-velocity interpolated along C to the C-face times the C-velocity interpolated along D.
template <int C, int D, typename BC, typename BD>
__device__ __forceinline__ void transverse(const Ring2& S, const BC& MC, const BD& MD, float2 aH, float2 bH,
                                           float2& conv, float2& lap) {
  constexpr int cx = unit_(C, 0), cy = unit_(C, 1), cz = unit_(C, 2);
  constexpr int dx = unit_(D, 0), dy = unit_(D, 1), dz = unit_(D, 2);
  constexpr int AB = 4;
  // low face
  const float2 aDcL = fma2(MC.wl, S.ld<D, -cx, -cy, -cz>(), MC.wr * S.ld<D, 0, 0, 0>());
  const float2 bDcL = fma2(MC.wl, S.ld<AB + D, -cx, -cy, -cz>(), MC.wr * S.ld<AB + D, 0, 0, 0>());
  const float2 bCm = S.ld<AB + C, -dx, -dy, -dz>(), aCm = S.ld<C, -dx, -dy, -dz>();
  const float2 aCdL = fma2(MD.wl, aCm, MD.wr * aH);
  const float2 bCdL = fma2(MD.wl, bCm, MD.wr * bH);
  const float2 fLo = fma2(aDcL, bCdL, bDcL * aCdL);
  const float2 gLo = (bH - bCm) * MD.ic;
  // high face
  const float2 aDcH = fma2(MC.wl, S.ld<D, dx - cx, dy - cy, dz - cz>(), MC.wr * S.ld<D, dx, dy, dz>());
  const float2 bDcH = fma2(MC.wl, S.ld<AB + D, dx - cx, dy - cy, dz - cz>(), MC.wr * S.ld<AB + D, dx, dy, dz>());
  const float2 bCp = S.ld<AB + C, dx, dy, dz>(), aCp = S.ld<C, dx, dy, dz>();
  const float2 aCdH = fma2(MD.wlp, aH, MD.wrp * aCp);
  const float2 bCdH = fma2(MD.wlp, bH, MD.wrp * bCp);
  const float2 fHi = fma2(aDcH, bCdH, bDcH * aCdH);
  const float2 gHi = (bCp - bH) * MD.icp;
  conv = fma2(fHi - fLo, MD.ix, conv);
  lap = fma2(gHi - gLo, MD.ix, lap);
}

// Momentum component C: conv = S(q, v) (symmetrised convective form), lap = Lap v
template <int C>
__device__ __forceinline__ void momentum_pair(const Ring2& S, const Bundle<float2>& mx, const Bundle<float2>& my,
                                              const Bundle<float2>& mz, float2& conv, float2& lap) {
  constexpr int cx = unit_(C, 0), cy = unit_(C, 1), cz = unit_(C, 2);
  constexpr int AB = 4;
  const auto& MC = pick<C>(mx, my, mz);
  const float2 aH = S.ld<C, 0, 0, 0>(), bH = S.ld<AB + C, 0, 0, 0>();
  const float2 aM = S.ld<C, -cx, -cy, -cz>(), bM = S.ld<AB + C, -cx, -cy, -cz>();
  const float2 aP = S.ld<C, cx, cy, cz>(), bP = S.ld<AB + C, cx, cy, cz>();
  const float2 half = bc(0.5f), two = bc(2.f);
  const float2 aE = half * (aH + aP), bE = half * (bH + bP);
  const float2 aW = half * (aM + aH), bW = half * (bM + bH);
  conv = two * (aE * bE - aW * bW) * MC.ic;
  lap = ((bP - bH) * MC.ix - (bH - bM) * MC.ixm) * MC.ic;
  constexpr int D1 = (C + 1) % 3, D2 = (C + 2) % 3;
  transverse<C, D1>(S, MC, pick<D1>(mx, my, mz), aH, bH, conv, lap);
  transverse<C, D2>(S, MC, pick<D2>(mx, my, mz), aH, bH, conv, lap);
}

// Temperature fluxes through the D-faces of the cell; y, z walls: zero flux (select), x: Dirichlet 0
template <int D, typename BD>
__device__ __forceinline__ void temperature_dir(const Ring2& S, const BD& MD, float2 TaH, float2 TbH, bool lo_in,
                                                bool hi_in, float2& conv, float2& lap) {
  constexpr int dx = unit_(D, 0), dy = unit_(D, 1), dz = unit_(D, 2);
  constexpr int AB = 4;
  const float2 Tam = S.ld<3, -dx, -dy, -dz>(), Tbm = S.ld<AB + 3, -dx, -dy, -dz>();
  const float2 fLo = fma2(S.ld<D, 0, 0, 0>(), fma2(MD.wl, Tbm, MD.wr * TbH),
                          S.ld<AB + D, 0, 0, 0>() * fma2(MD.wl, Tam, MD.wr * TaH));
  float2 gLo = (TbH - Tbm) * MD.ic;
  const float2 Tap = S.ld<3, dx, dy, dz>(), Tbp = S.ld<AB + 3, dx, dy, dz>();
  const float2 fHi = fma2(S.ld<D, dx, dy, dz>(), fma2(MD.wlp, TbH, MD.wrp * Tbp),
                          S.ld<AB + D, dx, dy, dz>() * fma2(MD.wlp, TaH, MD.wrp * Tap));
  float2 gHi = (Tbp - TbH) * MD.icp;
  if (!lo_in) gLo = make_float2(0.f, 0.f);
  if (!hi_in) gHi = make_float2(0.f, 0.f);
  conv = fma2(fHi - fLo, MD.ix, conv);
  lap = fma2(gHi - gLo, MD.ix, lap);
}

__device__ __forceinline__ void temperature_pair(const Ring2& S, const Bundle<float2>& mx, const Bundle<float2>& my,
                                                 const Bundle<float2>& mz, int j, int ny, int k, int nz, float2& conv,
                                                 float2& lap) {
  const float2 TaH = S.ld<3, 0, 0, 0>(), TbH = S.ld<4 + 3, 0, 0, 0>();
  conv = make_float2(0.f, 0.f);
  lap = make_float2(0.f, 0.f);
  temperature_dir<0>(S, mx, TaH, TbH, true, true, conv, lap);
  temperature_dir<1>(S, my, TaH, TbH, j >= 1, j + 1 <= ny - 1, conv, lap);
  temperature_dir<2>(S, mz, TaH, TbH, k >= 1, k + 1 <= nz - 1, conv, lap);
}

__device__ __forceinline__ uint32_t smem_addr2(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ bool bar_try2(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait on an mbarrier phase (at most `spins` polls); on expiry records code 17 in *err
__device__ __forceinline__ bool bar_wait2(uint32_t bar, uint32_t parity, int* err, long long spins) {
  for (long long i = 0; i < spins; ++i)
    if (bar_try2(bar, parity)) return true;
  atomicCAS(err, 0, 17);
  return false;
}


// J.v, FP32, two cells per thread; ring planes arrive as one 4D TMA box per state (x, y, z, field)
template <bool BLOCK>
__global__ void __launch_bounds__(kPX / 2 * kPY, 2)
    k_stencil_pair(const __grid_constant__ CUtensorMap tmq, const __grid_constant__ CUtensorMap tmv, int* err,
                   long long spins, Geo<float> g, int N, float Gr, float invPr, float sigma, float* __restrict__ out, int zc,
                   int nch) {
  constexpr uint32_t kBox = 4u * kPL2 * sizeof(float);  // one state's box: 4 fields x kPHY x kPW2
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar[kPRing];
  float* sm = reinterpret_cast<float*>(smem_raw);  // [kPRing][kPNA][kPL2]
  const int tid = threadIdx.x;
  const int tx = tid % (kPX / 2), ty = tid / (kPX / 2);
  // BLOCK: blockIdx.z = z-chunk + nch * vector, vector `vec` of the block is fields 4 vec .. 4 vec + 3 of
  // tmv; otherwise one vector in chunks of kPZChunk planes
  if (!BLOCK) zc = kPZChunk, nch = gridDim.z;
  const int vec = BLOCK ? (int)blockIdx.z / nch : 0;
  const int i0 = blockIdx.x * kPX, j0 = blockIdx.y * kPY, k0 = ((int)blockIdx.z - vec * nch) * zc;
  if (BLOCK) out += (size_t)vec * 4 * N;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int kend = min(k0 + zc, nz);
  if (tid == 0) {
    for (int s2 = 0; s2 < kPRing; ++s2)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr2(&bar[s2])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto issue_plane = [&](int kk) {
    float* slot = sm + ((kk + kPRing) % kPRing) * kPNA * kPL2;
    const uint32_t b = smem_addr2(&bar[(kk + kPRing) % kPRing]);
    if (kk >= 0 && kk < nz) {
      if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(2u * kBox) : "memory");
        asm volatile(
            "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, "
            "%5, %6}], [%2];" ::"r"(smem_addr2(slot)),
            "l"(reinterpret_cast<uint64_t>(&tmq)), "r"(b), "r"(i0 - kPX0), "r"(j0 - 1), "r"(kk), "r"(0)
            : "memory");
        asm volatile(
            "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, "
            "%5, %6}], [%2];" ::"r"(smem_addr2(slot + 4 * kPL2)),
            "l"(reinterpret_cast<uint64_t>(&tmv)), "r"(b), "r"(i0 - kPX0), "r"(j0 - 1), "r"(kk), "r"(4 * vec)
            : "memory");
      }
    } else {  // a plane outside the domain: zeros, and a plain arrival completes the barrier phase
      for (int e = tid; e < kPNA * kPL2; e += kPX / 2 * kPY) slot[e] = 0.f;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      if (tid == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(b) : "memory");
    }
  };
  // plane kk lives in slot kk mod kPRing; it is that slot's use number (kk - k0 + 1) / kPRing
  auto wait_plane = [&](int kk) -> bool {
    return bar_wait2(smem_addr2(&bar[(kk + kPRing) % kPRing]), (uint32_t)(((kk - k0 + 1) / kPRing) & 1), err,
                     spins);
  };
  issue_plane(k0 - 1);
  issue_plane(k0);
  issue_plane(k0 + 1);
  int issued = k0 + 1;  // last plane whose copy was started (the same value in every thread)
  __syncthreads();
  bool ok = wait_plane(k0 - 1);
  ok = wait_plane(k0) && ok;
  ok = __syncthreads_and(ok);  // one decision for the whole CTA
  const int x = i0 + 2 * tx, j = j0 + ty;
  const bool active = (x < nx && j < ny);  // nx is a multiple of kPX: both cells are in the domain
  const Bundle<float2> mx = load_bundle_pair(g, active ? x : 0);
  const Bundle<float2> my = broadcast(load_bundle(g, 1, active ? j : 0));
  for (int k = k0; k < kend && ok; ++k) {
    if (k + 2 <= kend) {  // plane k+2 feeds the output plane k+1
      issue_plane(k + 2);
      issued = k + 2;
    }
    const bool ready = wait_plane(k + 1);
    if (active && ready) {
      const Bundle<float2> mz = broadcast(load_bundle(g, 2, k));
      Ring2 S;
#pragma unroll
      for (int dz = -1; dz <= 1; ++dz)
        S.p[dz + 1] = sm + ((k + dz + kPRing) % kPRing) * kPNA * kPL2 + (ty + 1) * kPW2 + (2 * tx + kPX0);
      float2 conv, lap;
      momentum_pair<0>(S, mx, my, mz, conv, lap);
      const float2 msig = bc(-sigma);
      float2 r0 = fma2(msig, S.ld<4, 0, 0, 0>(), lap - conv);
      momentum_pair<1>(S, mx, my, mz, conv, lap);
      const float2 r1 = fma2(msig, S.ld<5, 0, 0, 0>(), lap - conv);
      momentum_pair<2>(S, mx, my, mz, conv, lap);
      const float2 Tf = fma2(mz.wl, S.ld<7, 0, 0, -1>(), mz.wr * S.ld<7, 0, 0, 0>());
      const float2 r2 = fma2(msig, S.ld<6, 0, 0, 0>(), fma2(bc(Gr), Tf, lap - conv));
      temperature_pair(S, mx, my, mz, j, ny, k, nz, conv, lap);
      const float2 r3 = fma2(msig, S.ld<7, 0, 0, 0>(), lap * bc(invPr) - conv);
      const int o = (k * ny + j) * nx + x;
      if (x == 0) r0.x = 0.f;  // the x = 0 wall slot of u
      const float2 zero = make_float2(0.f, 0.f);
      *reinterpret_cast<float2*>(out + o) = r0;
      *reinterpret_cast<float2*>(out + N + o) = (j >= 1) ? r1 : zero;
      *reinterpret_cast<float2*>(out + 2 * N + o) = (k >= 1) ? r2 : zero;
      *reinterpret_cast<float2*>(out + 3 * N + o) = r3;
    }
    ok = __syncthreads_and(ready);  // nobody reads the slot of plane k-1 any more; stop together on a give-up
  }
  // give-up path: every plane copy still in flight lands (waited for with the full limit) before the CTA
  // exits, so that no bulk copy writes into shared memory the CTA no longer owns
  if (!ok && tid == 0)
    for (int kk = max(k0 - 1, issued - kPRing + 1); kk <= issued; ++kk)
      bar_wait2(smem_addr2(&bar[(kk + kPRing) % kPRing]), (uint32_t)(((kk - k0 + 1) / kPRing) & 1), err,
                kPWaitLimit);
}

// 4D tensor map of nvec FP32 states stored one after another (x, y, z, field; 4 nvec fields) with boxes
// of kPW2 x kPHY x 1 x 4 elements
int pair_map(const fv_grid_s* g, const float* ptr, CUtensorMap* m, int nvec = 1) {
  const uint64_t dims[4] = {(uint64_t)g->nx, (uint64_t)g->ny, (uint64_t)g->nz, 4 * (uint64_t)nvec};
  const uint64_t strides[3] = {g->nx * sizeof(float), (uint64_t)g->nx * g->ny * sizeof(float), g->N * sizeof(float)};
  const uint32_t box[4] = {(uint32_t)kPW2, (uint32_t)kPHY, 1, 4};
  return encode_tensor_map(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ptr, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_NONE);
}

}  // namespace

bool stencil_pair_eligible(const fv_grid_s* g, const float* q, const float* v) {
  return g->nx % kPX == 0 && g->ny >= 16 && ((uintptr_t)q % 16) == 0 && ((uintptr_t)v % 16) == 0;
}

int launch_stencil_pair(const fv_grid_s* g, double Gr, double sigma, const float* q, const float* v, float* out,
                        int nvec) {
  const size_t smem = (size_t)kPRing * kPNA * kPL2 * sizeof(float);
  static bool attr_set = false;
  if (!attr_set) {
    FV_CUDA(cudaFuncSetAttribute(k_stencil_pair<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FV_CUDA(cudaFuncSetAttribute(k_stencil_pair<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_set = true;
  }
  // blocks of vectors march the z-chunk the autotuner picked (if it ran); single vectors the default
  const int zc = (nvec > 1 && g->tune.pair_zc > 0) ? g->tune.pair_zc : kPZChunk;
  const int nch = (g->nz + zc - 1) / zc;
  if (nvec < 1 || (long long)nch * nvec > 65535) {
    set_error("launch_stencil_pair: too many vectors in one block for this z-chunk");
    return FV_EINVAL;
  }
  CUtensorMap tq, tv;
  std::memset(&tq, 0, sizeof(tq));
  std::memset(&tv, 0, sizeof(tv));
  FV_TRY(pair_map(g, q, &tq));
  FV_TRY(pair_map(g, v, &tv, nvec));
  dim3 grid(g->nx / kPX, (g->ny + kPY - 1) / kPY, nch * nvec);
  ProfScope ps(g, PROF_STENCIL);
  if (nvec > 1)
    k_stencil_pair<true><<<grid, kPX / 2 * kPY, smem, g->stream>>>(tq, tv, g->ws.err, wait_spins(g), g->geo32, (int)g->N, (float)Gr,
                                                                 (float)(1.0 / g->Pr), (float)sigma, out, zc, nch);
  else
    k_stencil_pair<false><<<grid, kPX / 2 * kPY, smem, g->stream>>>(tq, tv, g->ws.err, wait_spins(g), g->geo32, (int)g->N, (float)Gr,
                                                                  (float)(1.0 / g->Pr), (float)sigma, out, zc, nch);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

}  // namespace fv
