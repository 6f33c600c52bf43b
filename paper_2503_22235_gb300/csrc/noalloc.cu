// Allocation-free variant of the FP64 error reduction (wm_rel_l2_noalloc).
//
// wm_rel_l2 obtains its two-double accumulator with cudaMalloc and releases
// it with cudaFree on every call. Some callers cannot allow that: code that
// runs while a framework's caching allocator owns all free device memory,
// serving loops that must not take the driver's allocation path (cudaFree
// synchronises the whole device and stalls every other stream), and
// monitoring hooks that run between launches of someone else's work. This
// variant keeps its scratch in a fixed device array compiled into the
// library instead, and allocates nothing.
//
// The reduction is also deterministic: block i sums elements
// [i * kChunk, (i + 1) * kChunk) in a fixed order into partial i, and one
// block then adds the partials in a fixed order.
#include "wm_internal.cuh"

namespace {

constexpr int kChunk = 65536;         // elements reduced by one block
constexpr int kMaxPartials = 4096;    // blocks per call, so n <= kChunk * kMaxPartials
constexpr int kThreads = 256;
constexpr size_t kMaxElements = (size_t)kChunk * kMaxPartials;   // 268,435,456 floats (1 GiB per operand)

// [2 * kMaxPartials] per-block partial sums, then the 2 final sums. 64 KiB,
// held on every device that loads the library until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[2 * kMaxPartials + 2];

__device__ __forceinline__ void block_sum2(double& x, double& y) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    x += __shfl_xor_sync(0xffffffffu, x, o);
    y += __shfl_xor_sync(0xffffffffu, y, o);
  }
  __shared__ double red[2][kThreads / 32];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    red[0][w] = x;
    red[1][w] = y;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sx = 0.0, sy = 0.0;
    for (int i = 0; i < kThreads / 32; ++i) {
      sx += red[0][i];
      sy += red[1][i];
    }
    x = sx;
    y = sy;
  }
}

__global__ void __launch_bounds__(kThreads) noalloc_partial_kernel(const float* __restrict__ a,
                                                                   const float* __restrict__ b, size_t n,
                                                                   double* __restrict__ scratch) {
  const size_t lo = (size_t)blockIdx.x * kChunk;
  const size_t hi = lo + kChunk < n ? lo + kChunk : n;
  double sd = 0.0, sb = 0.0;
  for (size_t i = lo + threadIdx.x; i < hi; i += kThreads) {
    const double x = a[i], y = b[i];
    sd += (x - y) * (x - y);
    sb += y * y;
  }
  block_sum2(sd, sb);
  if (threadIdx.x == 0) {
    scratch[2 * blockIdx.x] = sd;
    scratch[2 * blockIdx.x + 1] = sb;
  }
}

__global__ void __launch_bounds__(kThreads) noalloc_finish_kernel(double* __restrict__ scratch, int nparts) {
  double sd = 0.0, sb = 0.0;
  for (int i = threadIdx.x; i < nparts; i += kThreads) {
    sd += scratch[2 * i];
    sb += scratch[2 * i + 1];
  }
  block_sum2(sd, sb);
  if (threadIdx.x == 0) {
    scratch[2 * kMaxPartials] = sd;
    scratch[2 * kMaxPartials + 1] = sb;
  }
}

// Device address of the scratch array on the current device. Host code only
// sees a stand-in for the array, so the address is looked up on every call:
// the lookup allocates nothing and costs no launch, and a cached address would
// go stale if the module were reloaded (for example after cudaDeviceReset).
wm_status scratch_address(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return wm::cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
  *out = static_cast<double*>(p);
  return WM_OK;
}

}  // namespace

extern "C" wm_status wm_rel_l2_noalloc(const float* a, const float* b, size_t n, double* out, void* stream) {
  if (!a || !b || !out) return wm::fail(WM_ERR_INVALID_ARG, "NULL argument");
  if (n > kMaxElements)
    return wm::fail(WM_ERR_INVALID_ARG, "wm_rel_l2_noalloc takes at most 268435456 elements (its fixed scratch "
                                        "holds 4096 partial sums of 65536 elements each); got " +
                                            std::to_string(n));
  double* scratch = nullptr;
  wm_status st = scratch_address(&scratch);
  if (st != WM_OK) return st;
  if (n == 0) {
    out[0] = out[1] = 0.0;
    return WM_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int nparts = (int)((n + kChunk - 1) / kChunk);
  noalloc_partial_kernel<<<nparts, kThreads, 0, s>>>(a, b, n, scratch);
  WM_CUDA(cudaGetLastError());
  noalloc_finish_kernel<<<1, kThreads, 0, s>>>(scratch, nparts);
  WM_CUDA(cudaGetLastError());
  WM_CUDA(cudaMemcpyAsync(out, scratch + 2 * kMaxPartials, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  WM_CUDA(cudaStreamSynchronize(s));
  return WM_OK;
}
