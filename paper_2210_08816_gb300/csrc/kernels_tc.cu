// Tensor-core (tcgen05) version of one fast-diagonalisation pass for FP32 fields.
//
// The pass is the GEMM  C[p][m] = sum_k A[p][k] B[m][k]  (A = field rows, k contiguous; B = the n x n
// 1D eigenvector matrix, k contiguous), stored transposed as out[m][p] (see kernels_fdm.cu).  FP32
// accuracy on TF32 tensor cores by the three-product split: A = A_hi + A_lo, B = B_hi + B_lo with
// A_hi, B_hi exactly representable in TF32, and  A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi  (the dropped
// A_lo B_lo and the TF32 rounding of the lo parts are ~2^-22 relative).  B_hi / B_lo are prepared on the
// host; A is split in shared memory by the converter warps.
//
// One CTA = one 128-row tile of p and all n (<= 256) modes, K in slabs of 16 (one 64-byte swizzle row):
//   warp 0      TMA producer: A slab (128 x 16) and B_hi, B_lo slabs (n x 16) into a 4-stage ring
//   warp 1      TMEM allocation; one elected thread issues tcgen05.mma (M = 128, N = n, K = 8) x 3 x 2
//   warps 2..5  split A into hi/lo in place, then the epilogue: tcgen05.ld rows -> out[m][p]
// Every mbarrier wait is bounded; on expiry the kernel records an error code and drains.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "fv_internal.h"

namespace fv {
namespace {

constexpr int kTcBM = 128;                 // rows per tile
constexpr int kTcBK = 16;                  // fp32 elements per K slab (64 bytes: one 64-byte swizzle row)
constexpr int kTcRowBytes = kTcBK * 4;
constexpr int kTcABytes = kTcBM * kTcRowBytes;  // one A (or A_lo) slab
constexpr int kTcStages = 4;
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

// bounded wait; on expiry records `code` in *err and returns false
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err, int code) {
  for (long long i = 0; i < kWaitLimit; ++i)
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

template <bool SCALE>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_transform_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmBhi,
                   const __grid_constant__ CUtensorMap tmBlo, float* __restrict__ out, int P, int n,
                   const float* __restrict__ lx, const float* __restrict__ ly, const float* __restrict__ lz, int nb,
                   int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar_full[kTcStages], bar_conv[kTcStages], bar_empty[kTcStages], bar_acc;
  __shared__ uint32_t tmem_slot;
  __shared__ float lz_s[256];  // eigenvalues of the contracted axis (scaled pass only)
  // 1024-byte aligned ring: per stage A (8 KB), A_lo (8 KB), B_hi (n x 64 B), B_lo (n x 64 B)
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t b_bytes = (uint32_t)n * kTcRowBytes;
  const uint32_t stage_bytes = 2u * kTcABytes + 2u * b_bytes;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int nk = n / kTcBK;
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
      for (int s = 0; s < nk; ++s) {
        const int st = s % kTcStages;
        if (s >= kTcStages && !mbar_wait(smem_u32(&bar_empty[st]), ((s / kTcStages) - 1) & 1, err, 1)) break;
        const uint32_t sb = base + st * stage_bytes;
        const uint32_t fb = smem_u32(&bar_full[st]);
        mbar_expect_tx(fb, kTcABytes + 2u * b_bytes);
        tma_load_2d(sb, &tmA, fb, s * kTcBK, p0);
        tma_load_2d(sb + 2u * kTcABytes, &tmBhi, fb, s * kTcBK, 0);
        tma_load_2d(sb + 2u * kTcABytes + b_bytes, &tmBlo, fb, s * kTcBK, 0);
        ++issued;
      }
      // drain: every issued copy has landed before the block may exit
      for (int s = (issued > kTcStages ? issued - kTcStages : 0); s < issued; ++s)
        mbar_wait(smem_u32(&bar_full[s % kTcStages]), (s / kTcStages) & 1, err, 2);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTcBM >> 4) << 24);
      bool ok = true;
      for (int s = 0; s < nk && ok; ++s) {
        const int st = s % kTcStages;
        ok = mbar_wait(smem_u32(&bar_conv[st]), (s / kTcStages) & 1, err, 3);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t sb = base + st * stage_bytes;
#pragma unroll
        for (int kk = 0; kk < kTcBK / 8; ++kk) {
          const uint64_t ahi = smem_desc(sb + kk * 32), alo = smem_desc(sb + kTcABytes + kk * 32);
          const uint64_t bhi = smem_desc(sb + 2u * kTcABytes + kk * 32);
          const uint64_t blo = smem_desc(sb + 2u * kTcABytes + b_bytes + kk * 32);
          mma_tf32(tmem, ahi, bhi, idesc, (s > 0 || kk > 0) ? 1u : 0u);
          mma_tf32(tmem, ahi, blo, idesc, 1u);
          mma_tf32(tmem, alo, bhi, idesc, 1u);
        }
        mma_commit(smem_u32(&bar_empty[st]));
      }
      mma_commit(smem_u32(&bar_acc));  // arrives once every MMA issued above has completed
    }
  } else {
    // converters: thread t splits row t of the A slab (64 bytes, whatever its swizzled position)
    const int t = threadIdx.x - 64;
    bool ok = true;
    for (int s = 0; s < nk; ++s) {
      const int st = s % kTcStages;
      ok = mbar_wait(smem_u32(&bar_full[st]), (s / kTcStages) & 1, err, 4);
      if (!ok) break;
      const uint32_t sb = base + st * stage_bytes;
      float4* a = reinterpret_cast<float4*>(smem_raw + (sb - smem_u32(smem_raw)) + t * kTcRowBytes);
      float4* alo = reinterpret_cast<float4*>(smem_raw + (sb - smem_u32(smem_raw)) + kTcABytes + t * kTcRowBytes);
#pragma unroll
      for (int c = 0; c < kTcRowBytes / 16; ++c) {
        float4 x = a[c], h, l;
        uint32_t u;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x.x));
        h.x = __uint_as_float(u);
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x.y));
        h.y = __uint_as_float(u);
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x.z));
        h.z = __uint_as_float(u);
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x.w));
        h.w = __uint_as_float(u);
        l.x = x.x - h.x;
        l.y = x.y - h.y;
        l.z = x.z - h.z;
        l.w = x.w - h.w;
        a[c] = h;
        alo[c] = l;
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
      for (int c0 = 0; c0 < n; c0 += 16) {
        uint32_t r[16];
        tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, r);
        if (p < P) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int m = c0 + j;
            float v = __uint_as_float(r[j]);
            if (SCALE) v = (m == 0 && pa == 0 && pb == 0) ? 0.f : v * __frcp_rn(lz_s[m] + sa + sb2);
            out[(long long)m * P + p] = v;
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

size_t tc_smem_bytes(int n) { return (size_t)kTcStages * (2 * kTcABytes + 2 * (size_t)n * kTcRowBytes) + 1024; }

}  // namespace

bool tc_eligible(const fv_grid_s* g) {
  const int ns[3] = {g->nx, g->ny, g->nz};
  for (int d = 0; d < 3; ++d)
    if (ns[d] < 32 || ns[d] > 256 || ns[d] % 32 != 0) return false;
  return encoder() != nullptr;
}

// B operands: per axis the forward (E^-1) and backward (E) matrices split into TF32-exact hi and the
// FP32 remainder lo, in one device buffer: [axis][fwd_hi, fwd_lo, bwd_hi, bwd_lo][n x n].
int tc_setup(fv_grid_s* g, const std::vector<double>* Einv, const std::vector<double>* E) {
  size_t total = 0;
  const int ns[3] = {g->nx, g->ny, g->nz};
  for (int d = 0; d < 3; ++d) total += 4 * (size_t)ns[d] * ns[d];
  std::vector<float> h(total);
  size_t o = 0;
  size_t off[3][4];
  auto split = [&](const std::vector<double>& M, size_t n2) {
    const size_t ohi = o, olo = o + n2;
    for (size_t i = 0; i < n2; ++i) {
      const float f = (float)M[i];
      uint32_t u;
      std::memcpy(&u, &f, 4);
      // round to nearest TF32 (10 explicit mantissa bits): add half of the dropped range, clear it
      u = (u + 0x1000u) & 0xFFFFE000u;
      float hi;
      std::memcpy(&hi, &u, 4);
      h[ohi + i] = hi;
      h[olo + i] = (float)(M[i] - (double)hi);
    }
    o += 2 * n2;
    return std::make_pair(ohi, olo);
  };
  for (int d = 0; d < 3; ++d) {
    const size_t n2 = (size_t)ns[d] * ns[d];
    auto f = split(Einv[d], n2);
    auto b = split(E[d], n2);
    off[d][0] = f.first;
    off[d][1] = f.second;
    off[d][2] = b.first;
    off[d][3] = b.second;
  }
  void* buf = nullptr;
  if (cudaMalloc(&buf, total * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    set_error("tensor-core operand allocation failed");
    return FV_ENOMEM;
  }
  g->tc.buf = buf;
  FV_CUDA(cudaMemcpy(buf, h.data(), total * sizeof(float), cudaMemcpyHostToDevice));
  for (int d = 0; d < 3; ++d)
    for (int j = 0; j < 4; ++j) {
      const float* p = (const float*)buf + off[d][j];
      FV_TRY(encode(&g->tc.B[d][j], p, ns[d], ns[d], ns[d]));
    }
  const int smem_max = (int)tc_smem_bytes(256);
  FV_CUDA(cudaFuncSetAttribute(k_transform_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max));
  FV_CUDA(cudaFuncSetAttribute(k_transform_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max));
  g->tc.ready = true;
  return FV_OK;
}

// one pass: in[a][b][k] (na*nb rows of n) -> out[m][a][b], with the matrix of `axis` (which = 0 forward, 2 backward)
int tc_pass(const fv_grid_s* g, int axis, int which, int na, int nb, const float* in, float* out, bool scale) {
  const int n = (axis == 0) ? g->nx : (axis == 1) ? g->ny : g->nz;
  const long long P = (long long)na * nb;
  CUtensorMap tmA;
  FV_TRY(encode(&tmA, in, P, n, kTcBM));
  const FdmDev<float>& f = g->fdm32;
  const dim3 grid((unsigned)((P + kTcBM - 1) / kTcBM));
  const size_t smem = tc_smem_bytes(n);
  ProfScope ps(g, PROF_TRANSFORM_TC);
  if (scale)
    k_transform_tc<true><<<grid, kTcThreads, smem, g->stream>>>(tmA, g->tc.B[axis][which], g->tc.B[axis][which + 1],
                                                                out, (int)P, n, f.lam[0], f.lam[1], f.lam[2], nb,
                                                                g->ws.err);
  else
    k_transform_tc<false><<<grid, kTcThreads, smem, g->stream>>>(tmA, g->tc.B[axis][which], g->tc.B[axis][which + 1],
                                                                 out, (int)P, n, f.lam[0], f.lam[1], f.lam[2], nb,
                                                                 g->ws.err);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

}  // namespace fv
