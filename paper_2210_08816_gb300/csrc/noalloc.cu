// fv_dot_noalloc: the Krylov inner product for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: real-time or safety-critical loops that forbid any allocation
// after start-up (an allocation can block or fail at an unpredictable moment), applications whose
// device memory is carved out once by a memory pool or a framework they do not own, and host programs
// that embed this library with a fixed memory budget and hand it only pre-allocated buffers.  fv_dot
// needs an fv_grid handle, whose creation allocates workspace.  This entry point needs no handle: the per-block partial
// sums go to the file-scope device array below, which every GPU that loads the library holds until the
// process exits (kNoAllocSlots doubles = 32 KiB).  The caller passes the two input vectors and a
// device double for the result; nothing is allocated or freed here.
//
// Set-up: the first call on a device looks up the array's device address with cudaGetSymbolAddress
// (with that device current) and caches it; make that first call before any stream capture.
// Every call shares the array and overwrites the slots it uses; calls that overlap on the GPU (for
// example on two streams) race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/cube_fv.h"

namespace {

constexpr int kNoAllocSlots = 4096;                 // partial sums held in the static scratch
constexpr long long kNoAllocChunk = 1LL << 18;      // elements summed by one block
constexpr long long kNoAllocMaxN = kNoAllocSlots * kNoAllocChunk;
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocSlots];

struct ScratchAddr {
  bool ready = false;
  double* ptr = nullptr;
};
ScratchAddr g_addr[kMaxDevices];
std::mutex g_addr_mu;

// A pointer the kernels on device `dev` may dereference: device memory of that device, or managed memory.
// Host memory and another device's memory are refused: the kernels launch on the current device.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free error of a failed query
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

// Device address of the scratch array on the current device (host code must not use its name).
int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FV_ECUDA;
  std::lock_guard<std::mutex> lk(g_addr_mu);
  if (!g_addr[dev].ready) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return FV_ECUDA;
    g_addr[dev].ptr = static_cast<double*>(p);
    g_addr[dev].ready = true;
  }
  *out = g_addr[dev].ptr;
  return FV_OK;
}

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

// FP64 inputs: FP64 fused multiply-add accumulation.
__device__ __forceinline__ double chunk_dot(const double* a, const double* b, long long s, long long e) {
  double acc = 0.0;
  for (long long t = s + threadIdx.x; t < e; t += kThreads) acc = fma(a[t], b[t], acc);
  return acc;
}

// FP32 inputs: exact products split by an FMA, summed as a compensated float pair (TwoSum).
__device__ __forceinline__ double chunk_dot(const float* a, const float* b, long long s, long long e) {
  float hi = 0.0f, lo = 0.0f;
  for (long long t = s + threadIdx.x; t < e; t += kThreads) {
    const float x = a[t], y = b[t];
    const float p = x * y;
    const float pe = fmaf(x, y, -p);
    const float sum = hi + p;
    const float bb = sum - hi;
    lo += ((hi - (sum - bb)) + (p - bb)) + pe;
    hi = sum;
  }
  return (double)hi + (double)lo;
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_dot_partial_static(const R* __restrict__ a, const R* __restrict__ b,
                                                                  long long n, double* __restrict__ scratch) {
  const long long s = (long long)blockIdx.x * kNoAllocChunk;
  const long long e = (s + kNoAllocChunk < n) ? s + kNoAllocChunk : n;
  const double r = block_sum(chunk_dot(a, b, s, e));
  if (threadIdx.x == 0) scratch[blockIdx.x] = r;
}

__global__ void __launch_bounds__(1024) k_dot_finish_static(const double* __restrict__ scratch, int np,
                                                             double* __restrict__ result) {
  __shared__ double sh[32];
  double v = 0.0;
  for (int t = threadIdx.x; t < np; t += 1024) v += scratch[t];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = warp_sum(sh[lane]);
    if (lane == 0) *result = v;
  }
}

}  // namespace

extern "C" int fv_dot_noalloc(int prec, long long n, const void* a, const void* b, double* result, void* stream) {
  if (!a || !b || !result) return FV_EINVAL;
  if (prec != FV_FP64 && prec != FV_FP32) return FV_EINVAL;
  if (n < 1 || n > kNoAllocMaxN) return FV_EINVAL;  // beyond the static scratch: 4096 blocks of 2^18 elements
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FV_ECUDA;
  // a, b and result must live on the current device, where the kernels run
  if (!on_device(a, dev) || !on_device(b, dev) || !on_device(result, dev)) return FV_EINVAL;
  double* scratch = nullptr;
  const int st = scratch_address(&scratch);
  if (st != FV_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int blocks = (int)((n + kNoAllocChunk - 1) / kNoAllocChunk);
  if (prec == FV_FP64)
    k_dot_partial_static<double><<<blocks, kThreads, 0, s>>>(static_cast<const double*>(a),
                                                             static_cast<const double*>(b), n, scratch);
  else
    k_dot_partial_static<float><<<blocks, kThreads, 0, s>>>(static_cast<const float*>(a), static_cast<const float*>(b),
                                                            n, scratch);
  if (cudaGetLastError() != cudaSuccess) return FV_ECUDA;
  k_dot_finish_static<<<1, 1024, 0, s>>>(scratch, blocks, result);
  if (cudaGetLastError() != cudaSuccess) return FV_ECUDA;
  return FV_OK;
}
