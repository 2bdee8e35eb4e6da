// Tensor-core (tcgen05) version of the fast-diagonalisation passes for FP32 fields.
//
// A pass is the GEMM  C[p][m] = sum_k A[p][k] B[m][k]  (A = field rows, k contiguous; B = a 1D eigenvector
// matrix), stored transposed as out[m][p] (see kernels_fdm.cu).
//
// Mirror symmetry.  The grid is symmetric about 1/2, so the 1D operators are centro-symmetric and every
// eigenvector is either symmetric or antisymmetric.  With the modes ordered [symmetric | antisymmetric]
// (the "tensor-core order"):
//   forward  (cells -> modes):  phi_s = sum_{k<n/2} F_s[s][k] (r[k] + r[n-1-k]),
//                               phi_a = sum_{k<n/2} F_a[a][k] (r[k] - r[n-1-k]);
//   backward (modes -> cells):  S[i] = sum_s E_s[i][s] phi_s,  A[i] = sum_a E_a[i][a] phi_a  (i < n/2),
//                               out[i] = S + A,  out[n-1-i] = S - A.
// Each pass is then two GEMMs with K = n/2 and N = n/2: half the tensor work and half the B traffic of the
// dense transform.  The forward sum / difference is formed in shared memory by the converter warps; the
// backward S +- A in the epilogue.
//
// FP32 accuracy on TF32 tensor cores by the three-product split: A = A_hi + A_lo, B = B_hi + B_lo with
// A_hi, B_hi exactly representable in TF32, and  A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi  (the dropped
// A_lo B_lo and the TF32 rounding of the lo parts are ~2^-22 relative).  B_hi / B_lo are prepared on the
// host; A is split in shared memory by the converter warps.
//
// One CTA = one 128-row tile of p and all n (<= 256) outputs; per stage two 16-wide K slabs of A (slab j
// and its mirror n/16-1-j forward, slab j and j + n/32 backward) and the matching 16-wide slabs of the two
// half-size B matrices, in a 3-stage ring:
//   warp 0      TMA producer
//   warp 1      TMEM allocation; one elected thread issues tcgen05.mma (M = 128, N = n/2, K = 8): per
//               stage 2 k-steps x 3 products x 2 halves into two accumulators (TMEM columns 0 and n/2)
//   warps 2..5  converters (sum / difference, hi / lo split), then the epilogue: tcgen05.ld -> out[m][p]
// Every mbarrier wait is bounded; on expiry the kernel records an error code and drains.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "fv_internal.h"

namespace fv {
namespace {

constexpr int kTcBM = 128;                 // rows per tile
constexpr int kTcBK = 16;                  // fp32 elements per K slab (64 bytes: one 64-byte swizzle row)
constexpr int kTcRowBytes = kTcBK * 4;
constexpr int kTcABytes = kTcBM * kTcRowBytes;  // one A slab tile (8 KB)
constexpr int kTcStages = 3;
constexpr int kTcThreads = 192;
constexpr long long kWaitLimit = 1LL << 22;  // bounded spin on every mbarrier (seconds at most)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait (at most `spins` polls); on expiry records `code` in *err and returns false
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err, int code,
                                          long long spins = kWaitLimit) {
  for (long long i = 0; i < spins; ++i)
    if (mbar_try(bar, parity)) return true;
  atomicCAS(err, 0, code);
  return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
          "r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
      : "memory");
}

// Plain bulk copy global -> shared (contiguous bytes, 16-byte aligned ends), completing on an mbarrier.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
               : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 64-byte swizzle, 8-row groups 512 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);        // start address
  d |= (uint64_t)1 << 16;                         // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)((8 * kTcRowBytes) >> 4) << 32;  // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                         // descriptor version (sm_100 family)
  d |= (uint64_t)4 << 61;                         // 64-byte swizzle
  return d;
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Converter helpers.  A 64-byte swizzled row r keeps its 16-byte chunk c at physical chunk c ^ ((r >> 1) & 3).
__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return __uint_as_float(u);
}
// approximate reciprocal (PTX rcp.approx, relative error about 2^-23): far below the 3 x TF32 error
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void split4(const float4 x, float4& h, float4& l) {
  h.x = tf32_hi(x.x);
  h.y = tf32_hi(x.y);
  h.z = tf32_hi(x.z);
  h.w = tf32_hi(x.w);
  l.x = x.x - h.x;
  l.y = x.y - h.y;
  l.z = x.z - h.z;
  l.w = x.w - h.w;
}

template <bool SCALE, bool BWD>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_transform_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB1hi,
                   const __grid_constant__ CUtensorMap tmB1lo, const __grid_constant__ CUtensorMap tmB2hi,
                   const __grid_constant__ CUtensorMap tmB2lo, float* __restrict__ out, int P, int n,
                   const float* __restrict__ lx, const float* __restrict__ ly, const float* __restrict__ lz, int nb,
                   int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar_full[kTcStages], bar_conv[kTcStages], bar_empty[kTcStages], bar_acc;
  __shared__ uint32_t tmem_slot;
  __shared__ float lz_s[256];  // eigenvalues of the contracted axis (scaled pass only)
  const int h = n / 2;         // outputs per half, K per half
  // 1024-byte aligned ring; per stage tiles T0..T7: A1, A2 (loaded), A1_lo, A2_lo (converted),
  // B1_hi, B1_lo, B2_hi, B2_lo (loaded, h rows x 64 B each)
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t b_bytes = (uint32_t)h * kTcRowBytes;
  const uint32_t stage_bytes = 4u * kTcABytes + 4u * b_bytes;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int nst = n / (2 * kTcBK);  // stages per tile: pairs of slabs
  const int p0 = blockIdx.x * kTcBM;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(smem_u32(&bar_full[s]), 1);
      mbar_init(smem_u32(&bar_conv[s]), 128);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    mbar_init(smem_u32(&bar_acc), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (SCALE)
    for (int m = threadIdx.x; m < n; m += kTcThreads) lz_s[m] = lz[m];
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(256)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      for (int j = 0; j < nst; ++j) {
        const int st = j % kTcStages;
        if (j >= kTcStages && !mbar_wait(smem_u32(&bar_empty[st]), ((j / kTcStages) - 1) & 1, err, 1)) break;
        const uint32_t sb = base + st * stage_bytes;
        const uint32_t fb = smem_u32(&bar_full[st]);
        const int k1 = j * kTcBK;
        const int k2 = BWD ? h + j * kTcBK : n - kTcBK - j * kTcBK;
        mbar_expect_tx(fb, 2u * kTcABytes + 4u * b_bytes);
        tma_load_2d(sb, &tmA, fb, k1, p0);
        tma_load_2d(sb + kTcABytes, &tmA, fb, k2, p0);
        tma_load_2d(sb + 4u * kTcABytes, &tmB1hi, fb, j * kTcBK, 0);
        tma_load_2d(sb + 4u * kTcABytes + b_bytes, &tmB1lo, fb, j * kTcBK, 0);
        tma_load_2d(sb + 4u * kTcABytes + 2u * b_bytes, &tmB2hi, fb, j * kTcBK, 0);
        tma_load_2d(sb + 4u * kTcABytes + 3u * b_bytes, &tmB2lo, fb, j * kTcBK, 0);
        ++issued;
      }
      // drain: every issued copy has landed before the block may exit
      for (int j = (issued > kTcStages ? issued - kTcStages : 0); j < issued; ++j)
        mbar_wait(smem_u32(&bar_full[j % kTcStages]), (j / kTcStages) & 1, err, 2);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc =
          (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(h >> 3) << 17) | ((uint32_t)(kTcBM >> 4) << 24);
      bool ok = true;
      for (int j = 0; j < nst && ok; ++j) {
        const int st = j % kTcStages;
        ok = mbar_wait(smem_u32(&bar_conv[st]), (j / kTcStages) & 1, err, 3);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t sb = base + st * stage_bytes;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          const uint32_t a_hi = sb + half * kTcABytes, a_lo = sb + (2 + half) * kTcABytes;
          const uint32_t b_hi = sb + 4u * kTcABytes + (2 * half) * b_bytes, b_lo = b_hi + b_bytes;
          const uint32_t d = tmem + (uint32_t)(half * h);
#pragma unroll
          for (int kk = 0; kk < kTcBK / 8; ++kk) {
            const uint64_t ahi = smem_desc(a_hi + kk * 32), alo = smem_desc(a_lo + kk * 32);
            const uint64_t bhi = smem_desc(b_hi + kk * 32), blo = smem_desc(b_lo + kk * 32);
            mma_tf32(d, ahi, bhi, idesc, (j > 0 || kk > 0) ? 1u : 0u);
            mma_tf32(d, ahi, blo, idesc, 1u);
            mma_tf32(d, alo, bhi, idesc, 1u);
          }
        }
        mma_commit(smem_u32(&bar_empty[st]));
      }
      mma_commit(smem_u32(&bar_acc));  // arrives once every MMA issued above has completed
    }
  } else {
    // converters: thread t owns row t of the stage's A tiles
    const int t = threadIdx.x - 64;
    const int x = (t >> 1) & 3;  // swizzle pattern of this row
    bool ok = true;
    for (int j = 0; j < nst; ++j) {
      const int st = j % kTcStages;
      ok = mbar_wait(smem_u32(&bar_full[st]), (j / kTcStages) & 1, err, 4);
      if (!ok) break;
      unsigned char* sp = smem_raw + ((base + st * stage_bytes) - smem_u32(smem_raw)) + t * kTcRowBytes;
      float4* a1 = reinterpret_cast<float4*>(sp);
      float4* a2 = reinterpret_cast<float4*>(sp + kTcABytes);
      float4* l1 = reinterpret_cast<float4*>(sp + 2 * kTcABytes);
      float4* l2 = reinterpret_cast<float4*>(sp + 3 * kTcABytes);
      if (BWD) {  // plain hi / lo split of both slabs, chunks visited in the swizzled order (no bank conflicts)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int pc = c ^ x;
          float4 hh, ll;
          split4(a1[pc], hh, ll);
          a1[pc] = hh;
          l1[pc] = ll;
          split4(a2[pc], hh, ll);
          a2[pc] = hh;
          l2[pc] = ll;
        }
      } else {  // r[k] +- r[n-1-k]: logical chunk c of slab j pairs with logical chunk 3-c of the mirror slab,
                // element e with element 3-e
        float4 av[4], mv[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          av[c] = a1[c ^ x];
          mv[c] = a2[(3 - c) ^ x];
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float4 a = av[c], m = mv[c];
          const float4 sum = make_float4(a.x + m.w, a.y + m.z, a.z + m.y, a.w + m.x);
          const float4 dif = make_float4(a.x - m.w, a.y - m.z, a.z - m.y, a.w - m.x);
          float4 hh, ll;
          split4(sum, hh, ll);
          a1[c ^ x] = hh;
          l1[c ^ x] = ll;
          split4(dif, hh, ll);
          a2[c ^ x] = hh;
          l2[c ^ x] = ll;
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(smem_u32(&bar_conv[st]));
    }
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31, one row of the tile per thread; the
    // tcgen05.ld below is warp-collective, so the go/no-go decision is made per warp
    if (ok) ok = mbar_wait(smem_u32(&bar_acc), 0, err, 5);
    if (__all_sync(0xffffffffu, ok)) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int q = warp % 4;
      const int row = q * 32 + lane;
      const int p = p0 + row;
      float sa = 0.f, sb2 = 0.f;
      int pa = 0, pb = 0;
      if (SCALE && p < P) {
        pa = p / nb;
        pb = p - pa * nb;
        sa = ly[pa];
        sb2 = lx[pb];
      }
      const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
      for (int c0 = 0; c0 < h; c0 += 16) {
        uint32_t r1[16], r2[16];
        tmem_ld16(lane_base + (uint32_t)c0, r1);
        tmem_ld16(lane_base + (uint32_t)(h + c0), r2);
        if (p < P) {
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            const int m = c0 + jj;
            const float v1 = __uint_as_float(r1[jj]), v2 = __uint_as_float(r2[jj]);
            if (BWD) {  // cells m and n-1-m
              out[(long long)m * P + p] = v1 + v2;
              out[(long long)(n - 1 - m) * P + p] = v1 - v2;
            } else if (SCALE) {  // symmetric mode m, antisymmetric mode h + m
              const float s1 = (m == 0 && pa == 0 && pb == 0) ? 0.f : v1 * rcp_approx(lz_s[m] + sa + sb2);
              out[(long long)m * P + p] = s1;
              out[(long long)(h + m) * P + p] = v2 * rcp_approx(lz_s[h + m] + sa + sb2);
            } else {
              out[(long long)m * P + p] = v1;
              out[(long long)(h + m) * P + p] = v2;
            }
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    // if anything timed out, wait (bounded) for the MMAs issued so far before freeing their accumulator
    if (*err != 0 && lane == 0) mbar_wait(smem_u32(&bar_acc), 0, err, 6);
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256) : "memory");
  }
}

// Persistent form of the same pass: one CTA per SM walks the tiles blockIdx.x, +gridDim.x, ...; the
// shared-memory ring's phases run on across tiles (global stage counter), and two TMEM accumulators
// (columns 0 and 256) let a separate epilogue warpgroup drain tile t while the MMAs of tile t + 1 run.
// Warps: 0 TMA producer, 1 MMA issuer, 2-5 converters (row t of the A tiles), 6-9 epilogue.
// Barriers per step gi: full (TMA landed) -> conv (hi in place, lo in slot gi % 2) -> MMAs, whose commits
// free the TMA stage (empty) and the remainder slot (lofree) for step gi + 4 and gi + 2.
constexpr int kTcpThreads = 320;
// Ring depths of the persistent pass: the TMA ring (A slabs by tensor copies, the step's B slabs by one
// bulk copy of their pre-swizzled image) runs four stages deep; the converters' TF32 remainders of A live
// in a separate two-slot ring, so the bytes in flight from DRAM per SM grow by a third within the same
// shared memory.
constexpr int kTcpStages = 4;
constexpr int kTcpLoSlots = 2;
constexpr bool kTcPersistent = true;  // the one-tile-per-CTA kernel above stays as the reference form

template <bool SCALE, bool BWD>
__global__ void __launch_bounds__(kTcpThreads, 1)
    k_transform_tcp(const __grid_constant__ CUtensorMap tmA, const unsigned char* __restrict__ bsw,
                    float* __restrict__ out, int P, int Ptot, int n, const float* __restrict__ lx,
                    const float* __restrict__ ly, const float* __restrict__ lz, int nb, int* err, long long spins) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar_full[kTcpStages], bar_conv[kTcpStages], bar_empty[kTcpStages];
  __shared__ __align__(8) uint64_t bar_lofree[kTcpLoSlots], bar_accf[2], bar_acce[2], bar_drain;
  __shared__ uint32_t tmem_slot;
  __shared__ float lz_s[256];
  const int h = n / 2;
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t b_bytes = (uint32_t)h * kTcRowBytes;
  const uint32_t stage_bytes = 2u * kTcABytes + 4u * b_bytes;  // [A1 | A2 | B1hi | B1lo | B2hi | B2lo]
  const uint32_t lo_base = base + kTcpStages * stage_bytes;  // slot s: [L1 | L2] at lo_base + s * 2 A slabs
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int nst = n / (2 * kTcBK);
  const int ntiles = (Ptot + kTcBM - 1) / kTcBM;
  const int my_tiles = (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcpStages; ++s) {
      mbar_init(smem_u32(&bar_full[s]), 1);
      mbar_init(smem_u32(&bar_conv[s]), 128);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    for (int s = 0; s < kTcpLoSlots; ++s) mbar_init(smem_u32(&bar_lofree[s]), 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&bar_accf[b]), 1);
      mbar_init(smem_u32(&bar_acce[b]), 4);  // one arrival per epilogue warp
    }
    mbar_init(smem_u32(&bar_drain), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (SCALE)
    for (int m = threadIdx.x; m < n; m += kTcpThreads) lz_s[m] = lz[m];
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      bool ok = true;
      for (int ti = 0; ti < my_tiles && ok; ++ti) {
        const int p0 = ((int)blockIdx.x + ti * (int)gridDim.x) * kTcBM;
        for (int j = 0; j < nst; ++j) {
          const int gi = ti * nst + j, st = gi % kTcpStages;
          if (gi >= kTcpStages && !mbar_wait(smem_u32(&bar_empty[st]), ((gi / kTcpStages) - 1) & 1, err, 11, spins)) {
            ok = false;
            break;
          }
          const uint32_t sb = base + st * stage_bytes;
          const uint32_t fb = smem_u32(&bar_full[st]);
          const int k1 = j * kTcBK;
          const int k2 = BWD ? h + j * kTcBK : n - kTcBK - j * kTcBK;
          mbar_expect_tx(fb, 2u * kTcABytes + 4u * b_bytes);
          tma_load_2d(sb, &tmA, fb, k1, p0);
          tma_load_2d(sb + kTcABytes, &tmA, fb, k2, p0);
          // the four B slabs of step j, already in the stage's swizzled layout: one contiguous copy
          bulk_load(sb + 2u * kTcABytes, bsw + (size_t)j * 4u * b_bytes, 4u * b_bytes, fb);
          ++issued;
        }
      }
      // drain: every issued copy has landed before the block may exit
      for (int gi = (issued > kTcpStages ? issued - kTcpStages : 0); gi < issued; ++gi)
        mbar_wait(smem_u32(&bar_full[gi % kTcpStages]), (gi / kTcpStages) & 1, err, 12, kWaitLimit);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc =
          (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(h >> 3) << 17) | ((uint32_t)(kTcBM >> 4) << 24);
      bool ok = true;
      int last = -1;  // last tile whose accumulator commit was issued
      for (int ti = 0; ti < my_tiles && ok; ++ti) {
        const int b = ti & 1;
        if (ti >= 2 && !mbar_wait(smem_u32(&bar_acce[b]), ((ti / 2) - 1) & 1, err, 13, spins)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dacc = tmem + (uint32_t)(b * 256);
        for (int j = 0; j < nst; ++j) {
          const int gi = ti * nst + j, st = gi % kTcpStages;
          if (!mbar_wait(smem_u32(&bar_conv[st]), (gi / kTcpStages) & 1, err, 14, spins)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t sb = base + st * stage_bytes;
          const uint32_t lb = lo_base + (uint32_t)(gi % kTcpLoSlots) * (2u * kTcABytes);
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            const uint32_t a_hi = sb + half * kTcABytes, a_lo = lb + half * kTcABytes;
            const uint32_t b_hi = sb + 2u * kTcABytes + (2 * half) * b_bytes, b_lo = b_hi + b_bytes;
            const uint32_t d = dacc + (uint32_t)(half * h);
#pragma unroll
            for (int kk = 0; kk < kTcBK / 8; ++kk) {
              const uint64_t ahi = smem_desc(a_hi + kk * 32), alo = smem_desc(a_lo + kk * 32);
              const uint64_t bhi = smem_desc(b_hi + kk * 32), blo = smem_desc(b_lo + kk * 32);
              mma_tf32(d, ahi, bhi, idesc, (j > 0 || kk > 0) ? 1u : 0u);
              mma_tf32(d, ahi, blo, idesc, 1u);
              mma_tf32(d, alo, bhi, idesc, 1u);
            }
          }
          mma_commit(smem_u32(&bar_empty[st]));
          mma_commit(smem_u32(&bar_lofree[gi % kTcpLoSlots]));  // the remainder slot is free again
        }
        mma_commit(smem_u32(&bar_accf[b]));  // arrives once every MMA issued so far has completed
        last = ti;
      }
      // give-up path: a commit after every MMA issued so far (including those of a tile left half done)
      // arrives once they have all completed; wait for it (full limit) before the accumulators are freed
      (void)last;
      if (!ok) {
        mma_commit(smem_u32(&bar_drain));
        mbar_wait(smem_u32(&bar_drain), 0, err, 16, kWaitLimit);
      }
    }
  } else if (warp < 6) {
    // converters: thread t owns row t of every stage's A tiles and of every remainder slot
    const int t = threadIdx.x - 64;
    const int x = (t >> 1) & 3;  // swizzle pattern of this row
    bool ok = true;
    for (int ti = 0; ti < my_tiles && ok; ++ti) {
      for (int j = 0; j < nst; ++j) {
        const int gi = ti * nst + j, st = gi % kTcpStages, ls = gi % kTcpLoSlots;
        if (!mbar_wait(smem_u32(&bar_full[st]), (gi / kTcpStages) & 1, err, 17, spins)) {
          ok = false;
          break;
        }
        // the remainder slot was last read by the MMAs of step gi - kTcpLoSlots
        if (gi >= kTcpLoSlots &&
            !mbar_wait(smem_u32(&bar_lofree[ls]), ((gi / kTcpLoSlots) - 1) & 1, err, 19, spins)) {
          ok = false;
          break;
        }
        unsigned char* sp = smem_raw + ((base + st * stage_bytes) - smem_u32(smem_raw)) + t * kTcRowBytes;
        unsigned char* lp =
            smem_raw + ((lo_base + ls * 2u * kTcABytes) - smem_u32(smem_raw)) + t * kTcRowBytes;
        float4* a1 = reinterpret_cast<float4*>(sp);
        float4* a2 = reinterpret_cast<float4*>(sp + kTcABytes);
        float4* l1 = reinterpret_cast<float4*>(lp);
        float4* l2 = reinterpret_cast<float4*>(lp + kTcABytes);
        if (BWD) {  // chunks in the swizzled order: no bank conflicts
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int pc = c ^ x;
            float4 hh, ll;
            split4(a1[pc], hh, ll);
            a1[pc] = hh;
            l1[pc] = ll;
            split4(a2[pc], hh, ll);
            a2[pc] = hh;
            l2[pc] = ll;
          }
        } else {
          float4 av[4], mv[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            av[c] = a1[c ^ x];
            mv[c] = a2[(3 - c) ^ x];
          }
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const float4 a = av[c], m = mv[c];
            const float4 sum = make_float4(a.x + m.w, a.y + m.z, a.z + m.y, a.w + m.x);
            const float4 dif = make_float4(a.x - m.w, a.y - m.z, a.z - m.y, a.w - m.x);
            float4 hh, ll;
            split4(sum, hh, ll);
            a1[c ^ x] = hh;
            l1[c ^ x] = ll;
            split4(dif, hh, ll);
            a2[c ^ x] = hh;
            l2[c ^ x] = ll;
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(smem_u32(&bar_conv[st]));
      }
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31, one row of the tile per thread
    const int q = warp % 4;
    const int row = q * 32 + lane;
    for (int ti = 0; ti < my_tiles; ++ti) {
      const int b = ti & 1;
      const bool ok = mbar_wait(smem_u32(&bar_accf[b]), (ti / 2) & 1, err, 18, spins);
      if (!__all_sync(0xffffffffu, ok)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // row pg of the stacked block: row p of field vec (fields of P x n, one after another)
      const int pg = ((int)blockIdx.x + ti * (int)gridDim.x) * kTcBM + row;
      const int vec = pg / P, p = pg - vec * P;
      const bool live = pg < Ptot;
      float* __restrict__ o = out + (long long)vec * P * n;
      float sa = 0.f, sb2 = 0.f;
      int pa = 0, pb = 0;
      if (SCALE && live) {
        pa = p / nb;
        pb = p - pa * nb;
        sa = ly[pa];
        sb2 = lx[pb];
      }
      const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * 256);
      for (int c0 = 0; c0 < h; c0 += 16) {
        uint32_t r1[16], r2[16];
        tmem_ld16(lane_base + (uint32_t)c0, r1);
        tmem_ld16(lane_base + (uint32_t)(h + c0), r2);
        if (live) {
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            const int m = c0 + jj;
            const float v1 = __uint_as_float(r1[jj]), v2 = __uint_as_float(r2[jj]);
            if (BWD) {  // cells m and n-1-m
              o[(long long)m * P + p] = v1 + v2;
              o[(long long)(n - 1 - m) * P + p] = v1 - v2;
            } else if (SCALE) {  // symmetric mode m, antisymmetric mode h + m
              const float s1 = (m == 0 && pa == 0 && pb == 0) ? 0.f : v1 * rcp_approx(lz_s[m] + sa + sb2);
              o[(long long)m * P + p] = s1;
              o[(long long)(h + m) * P + p] = v2 * rcp_approx(lz_s[h + m] + sa + sb2);
            } else {
              o[(long long)m * P + p] = v1;
              o[(long long)(h + m) * P + p] = v2;
            }
          }
        }
      }
      // the accumulator's values are in registers (tcgen05.wait::ld): the MMAs may reuse it
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bar_acce[b]));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encoder() {
  static EncodeFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
  }
  return fn;
}

// rows x cols fp32 row-major matrix (cols contiguous), boxes of 16 columns x box_rows rows, 64-byte swizzle
int encode(CUtensorMap* m, const float* ptr, long long rows, int cols, int box_rows) {
  const uint64_t dims[2] = {(uint64_t)cols, (uint64_t)rows};
  const uint64_t strides[1] = {(uint64_t)cols * 4};
  const uint32_t box[2] = {(uint32_t)kTcBK, (uint32_t)box_rows};
  return encode_tensor_map(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, ptr, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_64B);
}

}  // namespace

int encode_tensor_map(CUtensorMap* map, CUtensorMapDataType type, int rank, const void* ptr, const uint64_t* dims,
                      const uint64_t* strides, const uint32_t* box, CUtensorMapSwizzle swizzle) {
  EncodeFn fn = encoder();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled unavailable");
    return FV_ECUDA;
  }
  cuuint64_t d[5], st[4];
  cuuint32_t b[5], e[5];
  for (int i = 0; i < rank; ++i) {
    d[i] = dims[i];
    b[i] = box[i];
    e[i] = 1;
    if (i + 1 < rank) st[i] = strides[i];
  }
  const CUresult r = fn(map, type, (cuuint32_t)rank, const_cast<void*>(ptr), d, st, b, e, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed");
    return FV_ECUDA;
  }
  return FV_OK;
}

namespace {

size_t tc_smem_bytes(int n) { return (size_t)kTcStages * (4 * kTcABytes + 4 * (size_t)(n / 2) * kTcRowBytes) + 1024; }
size_t tcp_smem_bytes(int n) {
  return (size_t)kTcpStages * (2 * kTcABytes + 4 * (size_t)(n / 2) * kTcRowBytes) +
         (size_t)kTcpLoSlots * 2 * kTcABytes + 1024;
}

}  // namespace

bool tc_eligible(const fv_grid_s* g) {
  const int ns[3] = {g->nx, g->ny, g->nz};
  for (int d = 0; d < 3; ++d) {
    if (ns[d] < 32 || ns[d] > 256 || ns[d] % 32 != 0) return false;
    if (!mirror_symmetric(g->xf[d])) return false;  // the half-size eigenproblems need a symmetric axis
  }
  return encoder() != nullptr;
}

// Builds the passes' operands on the host (tc_host_operands), uploads them into one device buffer,
// encodes the tensor maps of the B matrices and sets the kernels' shared-memory limits.
int tc_setup(fv_grid_s* g, const std::vector<double>* idx, const std::vector<double>* idc) {
  static_assert(kTcBK == kTcSlabCols, "the host operand layout and the kernels share the K slab width");
  const int ns[3] = {g->nx, g->ny, g->nz};
  TcOperands op;
  FV_TRY(tc_host_operands(ns, idx, idc, op));
  const size_t total = op.buf.size();
  const std::vector<float>& hbuf = op.buf;
  const auto& moff = op.moff;
  const auto& loff = op.loff;
  const auto& soff = op.soff;
  void* buf = nullptr;
  if (cudaMalloc(&buf, total * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    set_error("tensor-core operand allocation failed");
    return FV_ENOMEM;
  }
  g->tc.buf = buf;
  FV_CUDA(cudaMemcpy(buf, hbuf.data(), total * sizeof(float), cudaMemcpyHostToDevice));
  for (int d = 0; d < 3; ++d) {
    const int h = ns[d] / 2;
    for (int j = 0; j < 8; ++j) FV_TRY(encode(&g->tc.B[d][j], (const float*)buf + moff[d][j], h, h, h));
    g->tc.lam[d] = (const float*)buf + loff[d];
    for (int dir = 0; dir < 2; ++dir) g->tc.Bsw[d][dir] = (const unsigned char*)((const float*)buf + soff[d][dir]);
  }
  const int smem_max = (int)tc_smem_bytes(256);
  FV_CUDA(cudaFuncSetAttribute(k_transform_tc<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max));
  FV_CUDA(cudaFuncSetAttribute(k_transform_tc<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max));
  FV_CUDA(cudaFuncSetAttribute(k_transform_tc<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max));
  const int smemp_max = (int)tcp_smem_bytes(256);
  FV_CUDA(cudaFuncSetAttribute(k_transform_tcp<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smemp_max));
  FV_CUDA(cudaFuncSetAttribute(k_transform_tcp<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smemp_max));
  FV_CUDA(cudaFuncSetAttribute(k_transform_tcp<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smemp_max));
  {
    int dev = 0, sms = 0;
    FV_CUDA(cudaGetDevice(&dev));
    FV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    g->tc.sms = sms;
  }
  g->tc.ready = true;
  return FV_OK;
}

// one pass: in[a][b][k] (na*nb rows of n) -> out[m][a][b] with the matrices of `axis`; bwd selects the
// backward (modes -> cells) matrices.  Mode indices are in the tensor-core order throughout.  nvec > 1:
// that many fields of na*nb*n elements one after another in `in` and in `out`, each transformed alone,
// all in one persistent launch.
int tc_pass(const fv_grid_s* g, int axis, bool bwd, int na, int nb, const float* in, float* out, bool scale,
            int nvec) {
  const int n = (axis == 0) ? g->nx : (axis == 1) ? g->ny : g->nz;
  const long long P = (long long)na * nb;
  if (nvec < 1 || (nvec > 1 && !(kTcPersistent && g->tc.sms > 0)) || P * nvec > (1LL << 30)) {
    set_error("tc_pass: batch of fields not supported here");
    return FV_EINVAL;
  }
  const long long Ptot = P * nvec;
  CUtensorMap tmA;
  FV_TRY(encode(&tmA, in, Ptot, n, kTcBM));
  const long long ntiles = (Ptot + kTcBM - 1) / kTcBM;
  const dim3 grid((unsigned)ntiles);
  const size_t smem = tc_smem_bytes(n);
  const CUtensorMap* B = g->tc.B[axis] + (bwd ? 4 : 0);
  ProfScope ps(g, PROF_TRANSFORM_TC);
  if (kTcPersistent && g->tc.sms > 0) {
    const size_t smemp = tcp_smem_bytes(n);
    const unsigned char* bsw = g->tc.Bsw[axis][bwd ? 1 : 0];
    const dim3 pgrid((unsigned)std::min<long long>(ntiles, g->tc.sms));
    if (bwd)
      k_transform_tcp<false, true><<<pgrid, kTcpThreads, smemp, g->stream>>>(
          tmA, bsw, out, (int)P, (int)Ptot, n, nullptr, nullptr, nullptr, nb, g->ws.err, wait_spins(g));
    else if (scale)
      k_transform_tcp<true, false><<<pgrid, kTcpThreads, smemp, g->stream>>>(
          tmA, bsw, out, (int)P, (int)Ptot, n, g->tc.lam[0], g->tc.lam[1], g->tc.lam[2], nb, g->ws.err,
          wait_spins(g));
    else
      k_transform_tcp<false, false><<<pgrid, kTcpThreads, smemp, g->stream>>>(
          tmA, bsw, out, (int)P, (int)Ptot, n, nullptr, nullptr, nullptr, nb, g->ws.err, wait_spins(g));
    FV_CUDA(cudaGetLastError());
    return FV_OK;
  }
  if (bwd)
    k_transform_tc<false, true><<<grid, kTcThreads, smem, g->stream>>>(tmA, B[0], B[1], B[2], B[3], out, (int)P, n,
                                                                       nullptr, nullptr, nullptr, nb, g->ws.err);
  else if (scale)
    k_transform_tc<true, false><<<grid, kTcThreads, smem, g->stream>>>(
        tmA, B[0], B[1], B[2], B[3], out, (int)P, n, g->tc.lam[0], g->tc.lam[1], g->tc.lam[2], nb, g->ws.err);
  else
    k_transform_tc<false, false><<<grid, kTcThreads, smem, g->stream>>>(tmA, B[0], B[1], B[2], B[3], out, (int)P, n,
                                                                        nullptr, nullptr, nullptr, nb, g->ws.err);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

}  // namespace fv
