// Small kernels: precision casts, the FP64 error reduction, the device status
// word and the bounded-wait self test.
#include <algorithm>
#include <mutex>

#include <cuda_fp8.h>

#include "wm_internal.cuh"

namespace wm {

// ---------------------------------------------------------------- errors ----
static thread_local std::string t_last_error;

void set_error(const std::string& msg) { t_last_error = msg; }

wm_status fail(wm_status st, const std::string& msg) {
  t_last_error = msg;
  return st;
}

wm_status cuda_fail(cudaError_t e, const char* what) {
  t_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return WM_ERR_CUDA;
}

const char* last_error_cstr() { return t_last_error.c_str(); }

// --------------------------------------------------------- device status ----
static std::mutex g_status_mu;
static int* g_status_words[64] = {};

int* device_status_word() {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_status_mu);
  if (!g_status_words[dev]) {
    int* p = nullptr;
    if (cudaMalloc(&p, sizeof(int)) != cudaSuccess) return nullptr;
    cudaMemset(p, 0, sizeof(int));
    g_status_words[dev] = p;
  }
  return g_status_words[dev];
}

int num_sms() {
  static int cached[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && cached[dev]) return cached[dev];
  int n = 0;
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  if (n <= 0) n = 1;
  if (dev >= 0 && dev < 64) cached[dev] = n;
  return n;
}

wm_status prepare_na_f32();

wm_status prepare_kernels() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  if (dev >= 0 && dev < 64 && done[dev]) return WM_OK;
  wm_status st = prepare_gemm_tc();
  if (st == WM_OK) st = prepare_na_bf16();
  if (st == WM_OK) st = prepare_na_tc();
  if (st == WM_OK) st = prepare_na_f32();
  if (st == WM_OK && !device_status_word()) st = fail(WM_ERR_OOM, "device status word allocation failed");
  if (st == WM_OK && dev >= 0 && dev < 64) done[dev] = true;
  return st;
}

// ---------------------------------------------------------------- casts ----
__global__ void f32_to_bf16_kernel(const float* __restrict__ in, __nv_bfloat16* __restrict__ out, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = __float2bfloat16_rn(in[i]);
}

wm_status launch_f32_to_bf16(const float* in, __nv_bfloat16* out, size_t n, cudaStream_t s) {
  if (!n) return WM_OK;
  const int blocks = (int)std::min<size_t>((n + 255) / 256, (size_t)num_sms() * 8);
  f32_to_bf16_kernel<<<blocks, 256, 0, s>>>(in, out, n);
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

__global__ void f32_to_e4m3_kernel(const float* __restrict__ in, uint8_t* __restrict__ out, size_t n,
                                   float inv_scale) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (uint8_t)(__nv_cvt_float2_to_fp8x2(make_float2(in[i] * inv_scale, 0.f), __NV_SATFINITE, __NV_E4M3) & 0xFF);
}

wm_status launch_f32_to_e4m3(const float* in, uint8_t* out, size_t n, float inv_scale, cudaStream_t s) {
  if (!n) return WM_OK;
  const int blocks = (int)std::min<size_t>((n + 255) / 256, (size_t)num_sms() * 8);
  f32_to_e4m3_kernel<<<blocks, 256, 0, s>>>(in, out, n, inv_scale);
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

// ------------------------------------------------- FP64 error reduction ----
// acc2[0] += sum (a - b)^2, acc2[1] += sum b^2, in double precision.
__global__ void sqdiff_kernel(const float* __restrict__ a, const float* __restrict__ b, size_t n,
                              double* __restrict__ acc2) {
  double sd = 0.0, sb = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double x = a[i], y = b[i];
    sd += (x - y) * (x - y);
    sb += y * y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sd += __shfl_xor_sync(0xffffffffu, sd, o);
    sb += __shfl_xor_sync(0xffffffffu, sb, o);
  }
  __shared__ double red[2][32];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    red[0][w] = sd;
    red[1][w] = sb;
  }
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    sd = l < nw ? red[0][l] : 0.0;
    sb = l < nw ? red[1][l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sd += __shfl_xor_sync(0xffffffffu, sd, o);
      sb += __shfl_xor_sync(0xffffffffu, sb, o);
    }
    if (l == 0) {
      atomicAdd(acc2, sd);
      atomicAdd(acc2 + 1, sb);
    }
  }
}

wm_status launch_sqdiff(const float* a, const float* b, size_t n, double* acc2, cudaStream_t s) {
  if (!n) return WM_OK;
  const int blocks = (int)std::min<size_t>((n + 255) / 256, (size_t)num_sms() * 4);
  sqdiff_kernel<<<blocks, 256, 0, s>>>(a, b, n, acc2);
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

// NaN / infinity scan: *count += the non-finite elements of x.
__global__ void count_nonfinite_kernel(const float* __restrict__ x, size_t n, unsigned long long* __restrict__ count) {
  unsigned int c = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    c += isfinite(x[i]) ? 0u : 1u;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, (unsigned long long)c);
}

wm_status launch_count_nonfinite(const float* x, size_t n, unsigned long long* count, cudaStream_t s) {
  if (!n) return WM_OK;
  const int blocks = (int)std::min<size_t>((n + 255) / 256, (size_t)num_sms() * 4);
  count_nonfinite_kernel<<<blocks, 256, 0, s>>>(x, n, count);
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

// ------------------------------------------------- bounded-wait self test ----
// Waits for *flag to become non-zero -- nothing ever sets it -- for at most
// limit_ns, then records WM_ERR_TIMEOUT in the status word and returns.
__global__ void wait_selftest_kernel(volatile int* flag, unsigned long long limit_ns, int* status) {
  if (threadIdx.x != 0) return;
  unsigned long long t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  while (*flag == 0) {
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > limit_ns) {
      atomicExch(status, (int)WM_ERR_TIMEOUT);
      return;
    }
    __nanosleep(1000);
  }
}

wm_status launch_wait_selftest(int timeout_us, cudaStream_t s) {
  int* flag = nullptr;
  WM_CUDA(cudaMalloc(&flag, sizeof(int)));
  cudaMemsetAsync(flag, 0, sizeof(int), s);
  wait_selftest_kernel<<<1, 32, 0, s>>>(flag, (unsigned long long)timeout_us * 1000ull, device_status_word());
  cudaError_t e = cudaGetLastError();
  cudaStreamSynchronize(s);
  cudaFree(flag);
  if (e != cudaSuccess) return cuda_fail(e, "wait_selftest_kernel");
  return WM_OK;
}

}  // namespace wm
