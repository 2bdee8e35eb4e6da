// Inner products, norms, linear combinations and conversions of Krylov vectors (the dot products and
// axpys of BiCGstab(2), GMRES and the Chebyshev-preconditioned Arnoldi iteration, Section 1).
//
// Reductions are two-pass and deterministic: a fixed grid of kReduceBlocks blocks, each summing a fixed
// contiguous chunk in a fixed order (warp-shuffle tree in FP64), then one block summing the partials in a
// fixed order.  Reruns are bit-identical.
//
// Accumulation precision.  FP64 vectors accumulate in FP64.  For FP32 vectors each thread keeps a
// compensated pair (hi, lo) of floats: the product a*b is split exactly into p + e with an FMA and added
// by Knuth's TwoSum, so a thread's partial carries ~44 significant bits before it is converted to FP64.
// This keeps the inner products at FP64-like accuracy on GB300, whose FP64 pipe is ~1/64 of FP32.
#include <string>

#include "fv_internal.h"

namespace fv {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double nanmax(double a, double b) {
  if (a != a || b != b) return __longlong_as_double(0x7ff8000000000000ULL);
  return a > b ? a : b;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = nanmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// block-wide reduction of NV values per thread; thread 0 receives the results in out[]
template <int NV, bool MAX>
__device__ __forceinline__ void block_reduce(double (&v)[NV], double* out) {
  __shared__ double sh[NV][kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double x = MAX ? warp_max(v[i]) : warp_sum(v[i]);
    if (lane == 0) sh[i][warp] = x;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double x = (lane < kThreads / 32) ? sh[i][lane] : (MAX ? 0.0 : 0.0);
      x = MAX ? warp_max(x) : warp_sum(x);
      if (lane == 0) out[i] = x;
    }
  }
}

__device__ __forceinline__ void chunk_of(size_t n, size_t& b, size_t& e) {
  const size_t L = (n + gridDim.x - 1) / gridDim.x;
  b = (size_t)blockIdx.x * L;
  e = b + L < n ? b + L : n;
}

// compensated float accumulator: value = hi + lo
struct F2 {
  float hi = 0.0f, lo = 0.0f;
  __device__ __forceinline__ void add_product(float a, float b) {
    const float p = a * b;
    const float pe = fmaf(a, b, -p);  // a*b = p + pe exactly
    const float s = hi + p;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (p - bb);  // hi + p = s + err exactly
    hi = s;
    lo += err + pe;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

template <typename R>
__device__ __forceinline__ double dot_chunk(const R* __restrict__ a, const R* __restrict__ b, size_t s, size_t e) {
  double acc = 0.0;
  for (size_t t = s + threadIdx.x; t < e; t += kThreads) acc = fma((double)a[t], (double)b[t], acc);
  return acc;
}
template <>
__device__ __forceinline__ double dot_chunk<float>(const float* __restrict__ a, const float* __restrict__ b, size_t s,
                                                   size_t e) {
  F2 acc;
  for (size_t t = s + threadIdx.x; t < e; t += kThreads) acc.add_product(a[t], b[t]);
  return acc.value();
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_dot_partial(const R* __restrict__ a, const R* __restrict__ b, size_t n,
                                                           double* __restrict__ part) {
  size_t s, e;
  chunk_of(n, s, e);
  double acc[1] = {dot_chunk<R>(a, b, s, e)};
  double r[1];
  block_reduce<1, false>(acc, r);
  if (threadIdx.x == 0) part[blockIdx.x] = r[0];
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_maxabs_partial(const R* __restrict__ a, size_t n, double* __restrict__ part) {
  size_t s, e;
  chunk_of(n, s, e);
  R m = R(0);
  bool nan = false;
  for (size_t t = s + threadIdx.x; t < e; t += kThreads) {
    const R x = a[t];
    nan |= (x != x);
    const R ax = x < R(0) ? -x : x;
    m = ax > m ? ax : m;
  }
  double acc[1] = {nan ? __longlong_as_double(0x7ff8000000000000ULL) : (double)m};
  double r[1];
  block_reduce<1, true>(acc, r);
  if (threadIdx.x == 0) part[blockIdx.x] = r[0];
}

// partial inner products of up to 8 basis vectors V[i] (leading dimension ldv) with w
template <typename R>
__global__ void __launch_bounds__(kThreads) k_multidot_partial(const R* __restrict__ V, size_t ldv, int m,
                                                                const R* __restrict__ w, size_t n,
                                                                double* __restrict__ part) {
  size_t s, e;
  chunk_of(n, s, e);
  const int i0 = blockIdx.y * 8;
  const int nv = min(8, m - i0);
  double acc[8];
  if (sizeof(R) == 4) {
    F2 f[8];
    for (size_t t = s + threadIdx.x; t < e; t += kThreads) {
      const float wt = (float)w[t];
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (i < nv) f[i].add_product((float)V[(size_t)(i0 + i) * ldv + t], wt);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = f[i].value();
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = 0.0;
    for (size_t t = s + threadIdx.x; t < e; t += kThreads) {
      const double wt = (double)w[t];
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (i < nv) acc[i] = fma((double)V[(size_t)(i0 + i) * ldv + t], wt, acc[i]);
    }
  }
  double r[8];
  block_reduce<8, false>(acc, r);
  if (threadIdx.x == 0)
    for (int i = 0; i < nv; ++i) part[(size_t)(i0 + i) * gridDim.x + blockIdx.x] = r[i];
}

// final pass: out[slot + blockIdx.x] = reduce(part[blockIdx.x * np .. + np])
template <bool MAX>
__global__ void __launch_bounds__(1024) k_finish(const double* __restrict__ part, int np, double* __restrict__ out) {
  __shared__ double sh[32];
  const double* p = part + (size_t)blockIdx.x * np;
  double v = 0.0;
  for (int t = threadIdx.x; t < np; t += 1024) v = MAX ? nanmax(v, p[t]) : v + p[t];
  v = MAX ? warp_max(v) : warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = sh[lane];
    v = MAX ? warp_max(v) : warp_sum(v);
    if (lane == 0) out[blockIdx.x] = v;
  }
}

// Vector updates run in the vectors' own precision (coefficients rounded to it once).
// out[b] = sum of part[b * chunk .. min(np, (b + 1) * chunk)) in a fixed order
__global__ void __launch_bounds__(1024) k_finish_chunks(const double* __restrict__ part, int np, int chunk,
                                                         double* __restrict__ out) {
  __shared__ double sh[32];
  const int s = blockIdx.x * chunk, e = min(np, s + chunk);
  double v = 0.0;
  for (int t = s + threadIdx.x; t < e; t += 1024) v += part[t];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = warp_sum(sh[lane]);
    if (lane == 0) out[blockIdx.x] = v;
  }
}

template <typename R>
__global__ void k_lincomb(size_t n, int nvec, R c0, R c1, R c2, R c3, const R* x0, const R* x1, const R* x2,
                          const R* x3, R* out) {
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    R r = c0 * x0[t];
    if (nvec > 1) r = fma(c1, x1[t], r);
    if (nvec > 2) r = fma(c2, x2[t], r);
    if (nvec > 3) r = fma(c3, x3[t], r);
    out[t] = r;
  }
}

template <typename R>
__global__ void k_subtract_basis(const R* __restrict__ V, size_t ldv, int m, const double* __restrict__ h, R* w,
                                 size_t n) {
  __shared__ R hs[256];
  for (int i = threadIdx.x; i < m; i += blockDim.x) hs[i] = (R)h[i];
  __syncthreads();
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    R r = w[t];
    for (int i = 0; i < m; ++i) r = fma(-hs[i], V[(size_t)i * ldv + t], r);
    w[t] = r;
  }
}

template <typename S, typename D>
__global__ void k_convert(size_t n, const S* __restrict__ src, D* __restrict__ dst) {
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    dst[t] = (D)src[t];
}

// SplitMix64 (Steele, Lea & Flood 2014) keyed by (seed, stream) as counter-based uniforms, then
// Box-Muller on consecutive pairs: the same stream definition as the Python-side input generator.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ULL;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBULL;
  z ^= z >> 31;
  return z;
}
__device__ __forceinline__ double uniform_at(unsigned long long base, unsigned long long t) {
  const unsigned long long z = mix64(base + (t + 1ULL) * 0x9E3779B97F4A7C15ULL);
  return ((double)(z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

template <typename R>
__global__ void k_fill_normal(int nx, int ny, int nz, unsigned long long seed, R* out) {
  const size_t N = (size_t)nx * ny * nz;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < 4 * N; t += (size_t)gridDim.x * blockDim.x) {
    const int f = (int)(t / N);
    const size_t e = t - (size_t)f * N;
    const int i = (int)(e % nx), j = (int)((e / nx) % ny), k = (int)(e / ((size_t)nx * ny));
    if ((f == 0 && i == 0) || (f == 1 && j == 0) || (f == 2 && k == 0)) {
      out[t] = R(0);
      continue;
    }
    const unsigned long long base = mix64(((seed & 0xffffffffULL) << 20) | (unsigned long long)(f & 0xfffff));
    const size_t pr = e >> 1;
    const double u1 = uniform_at(base, 2 * pr), u2 = uniform_at(base, 2 * pr + 1);
    const double r = sqrt(-2.0 * log(u1));
    const double th = 6.283185307179586 * u2;
    out[t] = (R)((e & 1) ? r * sin(th) : r * cos(th));
  }
}

inline int stream_grid(size_t n) {
  size_t b = (n + 255) / 256;
  return (int)(b < 152 * 16 ? (b ? b : 1) : 152 * 16);
}

}  // namespace

template <typename R>
int launch_dot(const fv_grid_s* g, const R* a, const R* b, size_t n, int slot) {
  ProfScope ps(g, PROF_REDUCE);
  k_dot_partial<R><<<kReduceBlocks, kThreads, 0, g->stream>>>(a, b, n, g->ws.partials);
  FV_CUDA(cudaGetLastError());
  k_finish<false><<<1, 1024, 0, g->stream>>>(g->ws.partials, kReduceBlocks, g->ws.scalars + slot);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

template <typename R>
int launch_maxabs(const fv_grid_s* g, const R* a, size_t n, int slot) {
  ProfScope ps(g, PROF_REDUCE);
  k_maxabs_partial<R><<<kReduceBlocks, kThreads, 0, g->stream>>>(a, n, g->ws.partials);
  FV_CUDA(cudaGetLastError());
  k_finish<true><<<1, 1024, 0, g->stream>>>(g->ws.partials, kReduceBlocks, g->ws.scalars + slot);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

template <typename R>
int launch_multidot(const fv_grid_s* g, const R* V, size_t ldv, int m, const R* w, size_t n, int slot) {
  if (m <= 0) return FV_OK;
  dim3 grid(kReduceBlocks, (m + 7) / 8);
  ProfScope ps(g, PROF_REDUCE);
  k_multidot_partial<R><<<grid, kThreads, 0, g->stream>>>(V, ldv, m, w, n, g->ws.partials);
  FV_CUDA(cudaGetLastError());
  k_finish<false><<<m, 1024, 0, g->stream>>>(g->ws.partials, kReduceBlocks, g->ws.scalars + slot);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

template <typename R>
int launch_lincomb(const fv_grid_s* g, size_t n, int nvec, const double* c, const R* const* x, R* out) {
  ProfScope ps(g, PROF_VECTOR);
  k_lincomb<R><<<stream_grid(n), 256, 0, g->stream>>>(n, nvec, (R)c[0], (R)(nvec > 1 ? c[1] : 0.0),
                                                       (R)(nvec > 2 ? c[2] : 0.0), (R)(nvec > 3 ? c[3] : 0.0),
                                                       x[0], nvec > 1 ? x[1] : x[0],
                                                       nvec > 2 ? x[2] : x[0], nvec > 3 ? x[3] : x[0], out);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

template <typename R>
int launch_subtract_basis(const fv_grid_s* g, const R* V, size_t ldv, int m, const double* h, R* w, size_t n) {
  if (m <= 0) return FV_OK;
  if (m > 256) return FV_EINVAL;
  ProfScope ps(g, PROF_VECTOR);
  k_subtract_basis<R><<<stream_grid(n), 256, 0, g->stream>>>(V, ldv, m, h, w, n);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

int launch_convert(const fv_grid_s* g, size_t n, const double* src, float* dst) {
  ProfScope ps(g, PROF_VECTOR);
  k_convert<double, float><<<stream_grid(n), 256, 0, g->stream>>>(n, src, dst);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}
int launch_convert(const fv_grid_s* g, size_t n, const float* src, double* dst) {
  ProfScope ps(g, PROF_VECTOR);
  k_convert<float, double><<<stream_grid(n), 256, 0, g->stream>>>(n, src, dst);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

template <typename R>
int launch_fill_normal(const fv_grid_s* g, unsigned long long seed, R* out) {
  ProfScope ps(g, PROF_VECTOR);
  k_fill_normal<R><<<stream_grid(4 * g->N), 256, 0, g->stream>>>(g->nx, g->ny, g->nz, seed, out);
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

int launch_sum_partials(const fv_grid_s* g, int np, int slot) {
  ProfScope ps(g, PROF_REDUCE);
  if (np > 4096) {  // two levels: 64 fixed chunks, then their sums (deterministic order)
    const int chunk = (np + 63) / 64;
    k_finish_chunks<<<64, 1024, 0, g->stream>>>(g->ws.partials, np, chunk, g->ws.partials + kPartialSlots - 64);
    FV_CUDA(cudaGetLastError());
    k_finish<false><<<1, 1024, 0, g->stream>>>(g->ws.partials + kPartialSlots - 64, 64, g->ws.scalars + slot);
  } else {
    k_finish<false><<<1, 1024, 0, g->stream>>>(g->ws.partials, np, g->ws.scalars + slot);
  }
  FV_CUDA(cudaGetLastError());
  return FV_OK;
}

int read_scalars(const fv_grid_s* g, int slot, int count, double* out) {
  FV_CUDA(cudaMemcpyAsync(g->ws.host_scalars, g->ws.scalars + slot, sizeof(double) * count, cudaMemcpyDeviceToHost,
                          g->stream));
  int dev_err = 0;
  if (g->ws.err) FV_CUDA(cudaMemcpyAsync(&dev_err, g->ws.err, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
  FV_CUDA(cudaStreamSynchronize(g->stream));
  if (dev_err != 0) {
    cudaMemsetAsync(g->ws.err, 0, sizeof(int), g->stream);
    set_error("a bounded device-side wait expired (code " + std::to_string(dev_err) + ")");
    return FV_ETIMEOUT;
  }
  for (int i = 0; i < count; ++i) out[i] = g->ws.host_scalars[i];
  return FV_OK;
}

#define FV_INST(R)                                                                                  \
  template int launch_dot<R>(const fv_grid_s*, const R*, const R*, size_t, int);                    \
  template int launch_maxabs<R>(const fv_grid_s*, const R*, size_t, int);                           \
  template int launch_multidot<R>(const fv_grid_s*, const R*, size_t, int, const R*, size_t, int);  \
  template int launch_lincomb<R>(const fv_grid_s*, size_t, int, const double*, const R* const*, R*); \
  template int launch_subtract_basis<R>(const fv_grid_s*, const R*, size_t, int, const double*, R*, size_t); \
  template int launch_fill_normal<R>(const fv_grid_s*, unsigned long long, R*);
FV_INST(double)
FV_INST(float)
#undef FV_INST

}  // namespace fv
