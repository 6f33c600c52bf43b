// Plain FP32 path: LayerNorm, FP32-FMA GEMM with fused epilogues, and 3D
// neighborhood attention on CUDA cores. Strict FP32 FMA everywhere (no TF32),
// so that a block matches the float64 oracle to ~1e-6 relative L2.
#include <cuda_fp8.h>

#include <algorithm>

#include "wm_internal.cuh"

namespace wm {

// ------------------------------------------------------------ LayerNorm ----
// One warp per row. Mean and biased variance over C in FP32 (two passes over
// the row held in registers when C is a multiple of 128 and <= 1024).

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename OutT>
__device__ __forceinline__ void store_val(OutT* p, float v);
template <>
__device__ __forceinline__ void store_val<float>(float* p, float v) { *p = v; }
template <>
__device__ __forceinline__ void store_val<__nv_bfloat16>(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

template <typename OutT, int V4>  // V4 float4 per lane, C = 128 * V4
__global__ void ln_rows_reg(const float* __restrict__ x, const float* __restrict__ g, const float* __restrict__ b,
                            OutT* __restrict__ out, int M, float eps) {
  const int C = 128 * V4;
  const int lane = threadIdx.x & 31;
  const long row = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= M) return;
  const float4* xr = reinterpret_cast<const float4*>(x + row * C);
  float4 v[V4];
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < V4; ++i) {
    v[i] = xr[lane + 32 * i];
    s += (v[i].x + v[i].y) + (v[i].z + v[i].w);
  }
  const float mean = warp_sum(s) / C;
  float q = 0.f;
#pragma unroll
  for (int i = 0; i < V4; ++i) {
    float a = v[i].x - mean, bb = v[i].y - mean, c = v[i].z - mean, d = v[i].w - mean;
    q += (a * a + bb * bb) + (c * c + d * d);
  }
  const float rstd = rsqrtf(warp_sum(q) / C + eps);
  const float4* g4 = reinterpret_cast<const float4*>(g);
  const float4* b4 = reinterpret_cast<const float4*>(b);
  OutT* orow = out + row * C;
#pragma unroll
  for (int i = 0; i < V4; ++i) {
    const int c = 4 * (lane + 32 * i);
    float4 gg = g4[lane + 32 * i], bb = b4[lane + 32 * i];
    float r0 = (v[i].x - mean) * rstd * gg.x + bb.x;
    float r1 = (v[i].y - mean) * rstd * gg.y + bb.y;
    float r2 = (v[i].z - mean) * rstd * gg.z + bb.z;
    float r3 = (v[i].w - mean) * rstd * gg.w + bb.w;
    if constexpr (sizeof(OutT) == 4) {
      *reinterpret_cast<float4*>(reinterpret_cast<float*>(orow) + c) = make_float4(r0, r1, r2, r3);
    } else {
      __nv_bfloat162 p0 = __floats2bfloat162_rn(r0, r1), p1 = __floats2bfloat162_rn(r2, r3);
      uint2 u;
      u.x = *reinterpret_cast<uint32_t*>(&p0);
      u.y = *reinterpret_cast<uint32_t*>(&p1);
      *reinterpret_cast<uint2*>(reinterpret_cast<__nv_bfloat16*>(orow) + c) = u;
    }
  }
}

template <typename OutT>
__global__ void ln_rows_generic(const float* __restrict__ x, const float* __restrict__ g,
                                const float* __restrict__ b, OutT* __restrict__ out, int M, int C, float eps) {
  const int lane = threadIdx.x & 31;
  const long row = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= M) return;
  const float* xr = x + row * C;
  float s = 0.f;
  for (int c = lane; c < C; c += 32) s += xr[c];
  const float mean = warp_sum(s) / C;
  float q = 0.f;
  for (int c = lane; c < C; c += 32) {
    float d = xr[c] - mean;
    q += d * d;
  }
  const float rstd = rsqrtf(warp_sum(q) / C + eps);
  for (int c = lane; c < C; c += 32) store_val(out + row * C + c, (xr[c] - mean) * rstd * g[c] + b[c]);
}

// Row statistics: one warp per row, (mean, M2) in FP32 from the row held in
// registers, plus the bf16 copy of the row.
template <int V4>
__global__ void row_stats_kernel(const float* __restrict__ x, __nv_bfloat16* __restrict__ xb, float* __restrict__ st,
                                 int M) {
  const int C = 128 * V4;
  const int lane = threadIdx.x & 31;
  const long row = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  pdl_wait();
  pdl_trigger();
  if (row >= M) return;
  const float4* xr = reinterpret_cast<const float4*>(x + row * C);
  float4 v[V4];
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < V4; ++i) {
    v[i] = xr[lane + 32 * i];
    s += (v[i].x + v[i].y) + (v[i].z + v[i].w);
  }
  const float mean = warp_sum(s) / C;
  float q = 0.f;
#pragma unroll
  for (int i = 0; i < V4; ++i) {
    float a = v[i].x - mean, bb = v[i].y - mean, c = v[i].z - mean, d = v[i].w - mean;
    q += (a * a + bb * bb) + (c * c + d * d);
    __nv_bfloat162 p0 = __floats2bfloat162_rn(v[i].x, v[i].y), p1 = __floats2bfloat162_rn(v[i].z, v[i].w);
    uint2 u;
    u.x = *reinterpret_cast<uint32_t*>(&p0);
    u.y = *reinterpret_cast<uint32_t*>(&p1);
    *reinterpret_cast<uint2*>(xb + row * C + 4 * (lane + 32 * i)) = u;
  }
  const float m2 = warp_sum(q);
  if (lane == 0) {
    st[2 * row] = mean;
    st[2 * row + 1] = m2;
  }
}

wm_status launch_row_stats(const float* x, __nv_bfloat16* xb, float* stats, int M, int C, cudaStream_t s,
                           bool pdl) {
  if (M <= 0) return WM_OK;
  const int warps = 8;
  dim3 grid((M + warps - 1) / warps), block(32 * warps);
  switch (C) {
    case 128: WM_CUDA(launch_pdl(row_stats_kernel<1>, grid, block, 0, s, pdl, x, xb, stats, M)); break;
    case 256: WM_CUDA(launch_pdl(row_stats_kernel<2>, grid, block, 0, s, pdl, x, xb, stats, M)); break;
    case 384: WM_CUDA(launch_pdl(row_stats_kernel<3>, grid, block, 0, s, pdl, x, xb, stats, M)); break;
    case 512: WM_CUDA(launch_pdl(row_stats_kernel<4>, grid, block, 0, s, pdl, x, xb, stats, M)); break;
    case 768: WM_CUDA(launch_pdl(row_stats_kernel<6>, grid, block, 0, s, pdl, x, xb, stats, M)); break;
    case 1024: WM_CUDA(launch_pdl(row_stats_kernel<8>, grid, block, 0, s, pdl, x, xb, stats, M)); break;
    default: return fail(WM_ERR_INVALID_ARG, "row statistics need C in {128, 256, 384, 512, 768, 1024}");
  }
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

// LayerNorm rows to e4m3: one warp per row, FP32 statistics as above, output
// e4m3(LN(x) * inv_scale) with round-to-nearest-even and saturation.
template <int V4>
__global__ void ln_rows_e4m3(const float* __restrict__ x, const float* __restrict__ g, const float* __restrict__ b,
                             uint8_t* __restrict__ out, int M, float eps, float inv_scale) {
  const int C = 128 * V4;
  const int lane = threadIdx.x & 31;
  const long row = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  pdl_wait();
  pdl_trigger();
  if (row >= M) return;
  const float4* xr = reinterpret_cast<const float4*>(x + row * C);
  float4 v[V4];
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < V4; ++i) {
    v[i] = xr[lane + 32 * i];
    s += (v[i].x + v[i].y) + (v[i].z + v[i].w);
  }
  const float mean = warp_sum(s) / C;
  float q = 0.f;
#pragma unroll
  for (int i = 0; i < V4; ++i) {
    float a = v[i].x - mean, bb = v[i].y - mean, c = v[i].z - mean, d = v[i].w - mean;
    q += (a * a + bb * bb) + (c * c + d * d);
  }
  const float rstd = rsqrtf(warp_sum(q) / C + eps);
  const float4* g4 = reinterpret_cast<const float4*>(g);
  const float4* b4 = reinterpret_cast<const float4*>(b);
#pragma unroll
  for (int i = 0; i < V4; ++i) {
    const int c = 4 * (lane + 32 * i);
    float4 gg = g4[lane + 32 * i], bb = b4[lane + 32 * i];
    const float r0 = ((v[i].x - mean) * rstd * gg.x + bb.x) * inv_scale;
    const float r1 = ((v[i].y - mean) * rstd * gg.y + bb.y) * inv_scale;
    const float r2 = ((v[i].z - mean) * rstd * gg.z + bb.z) * inv_scale;
    const float r3 = ((v[i].w - mean) * rstd * gg.w + bb.w) * inv_scale;
    const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(r0, r1), __NV_SATFINITE, __NV_E4M3);
    const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(r2, r3), __NV_SATFINITE, __NV_E4M3);
    *reinterpret_cast<uint32_t*>(out + row * C + c) = lo | (hi << 16);
  }
}

wm_status launch_layernorm_e4m3(const float* x, const float* g, const float* b, uint8_t* out, int M, int C,
                                float eps, float inv_scale, cudaStream_t s, bool pdl) {
  if (M <= 0) return WM_OK;
  const int warps = 8;
  dim3 grid((M + warps - 1) / warps), block(32 * warps);
  switch (C) {
    case 128: WM_CUDA(launch_pdl(ln_rows_e4m3<1>, grid, block, 0, s, pdl, x, g, b, out, M, eps, inv_scale)); break;
    case 256: WM_CUDA(launch_pdl(ln_rows_e4m3<2>, grid, block, 0, s, pdl, x, g, b, out, M, eps, inv_scale)); break;
    case 384: WM_CUDA(launch_pdl(ln_rows_e4m3<3>, grid, block, 0, s, pdl, x, g, b, out, M, eps, inv_scale)); break;
    case 512: WM_CUDA(launch_pdl(ln_rows_e4m3<4>, grid, block, 0, s, pdl, x, g, b, out, M, eps, inv_scale)); break;
    case 768: WM_CUDA(launch_pdl(ln_rows_e4m3<6>, grid, block, 0, s, pdl, x, g, b, out, M, eps, inv_scale)); break;
    case 1024: WM_CUDA(launch_pdl(ln_rows_e4m3<8>, grid, block, 0, s, pdl, x, g, b, out, M, eps, inv_scale)); break;
    default: return fail(WM_ERR_INVALID_ARG, "e4m3 LayerNorm needs C in {128, 256, 384, 512, 768, 1024}");
  }
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

wm_status launch_layernorm(const float* x, const float* g, const float* b, void* out, bool out_bf16, int M, int C,
                           float eps, cudaStream_t s) {
  if (M <= 0) return WM_OK;
  const int warps = 8;
  dim3 grid((M + warps - 1) / warps), block(32 * warps);
  const bool aligned = ((uintptr_t)x % 16 == 0) && ((uintptr_t)g % 16 == 0) && ((uintptr_t)b % 16 == 0) &&
                       ((uintptr_t)out % 16 == 0);
  const int v4 = (C % 128 == 0 && aligned) ? C / 128 : 0;
#define WM_LN_CASE(N)                                                                                          \
  case N:                                                                                                     \
    if (out_bf16)                                                                                             \
      ln_rows_reg<__nv_bfloat16, N><<<grid, block, 0, s>>>(x, g, b, (__nv_bfloat16*)out, M, eps);             \
    else                                                                                                      \
      ln_rows_reg<float, N><<<grid, block, 0, s>>>(x, g, b, (float*)out, M, eps);                             \
    break;
  switch (v4) {
    WM_LN_CASE(1)
    WM_LN_CASE(2)
    WM_LN_CASE(3)
    WM_LN_CASE(4)
    WM_LN_CASE(6)
    WM_LN_CASE(8)
    default:
      if (out_bf16)
        ln_rows_generic<__nv_bfloat16><<<grid, block, 0, s>>>(x, g, b, (__nv_bfloat16*)out, M, C, eps);
      else
        ln_rows_generic<float><<<grid, block, 0, s>>>(x, g, b, (float*)out, M, C, eps);
  }
#undef WM_LN_CASE
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

// ----------------------------------------------------------------- SGEMM ----
// out[M, N] (epilogue) A[M, K] . W[N, K]^T + bias. 128 x 128 tile, k-step 16,
// 256 threads, 8 x 8 outputs per thread, double-buffered shared memory.

__device__ __forceinline__ float gelu_erf(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }

template <bool VEC>
__global__ void __launch_bounds__(256) sgemm_kernel(const float* __restrict__ A, const float* __restrict__ W,
                                                    const float* __restrict__ bias, float* __restrict__ out, int M,
                                                    int N, int K, int epi) {
  constexpr int BM = 128, BN = 128, BK = 16;
  __shared__ __align__(16) float As[2][BK][BM + 4];
  __shared__ __align__(16) float Bs[2][BK][BN + 4];
  const int tid = threadIdx.x;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int tx = tid % 16, ty = tid / 16;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  // each thread loads 2 float4 of A and of W per k-step: rows (tid/4) + 64*r, k (tid%4)*4
  float4 ra[2], rb[2];
  auto load_tiles = [&](int k0) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int row = tid / 4 + 64 * r, kk = k0 + (tid % 4) * 4;
      const int am = m0 + row, bn = n0 + row;
      if (VEC) {
        ra[r] = (am < M && kk < K) ? *reinterpret_cast<const float4*>(A + (size_t)am * K + kk) : make_float4(0, 0, 0, 0);
        rb[r] = (bn < N && kk < K) ? *reinterpret_cast<const float4*>(W + (size_t)bn * K + kk) : make_float4(0, 0, 0, 0);
      } else {
        float t[4], u[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          t[e] = (am < M && kk + e < K) ? A[(size_t)am * K + kk + e] : 0.f;
          u[e] = (bn < N && kk + e < K) ? W[(size_t)bn * K + kk + e] : 0.f;
        }
        ra[r] = make_float4(t[0], t[1], t[2], t[3]);
        rb[r] = make_float4(u[0], u[1], u[2], u[3]);
      }
    }
  };
  auto store_tiles = [&](int buf) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int row = tid / 4 + 64 * r, kk = (tid % 4) * 4;
      As[buf][kk + 0][row] = ra[r].x;
      As[buf][kk + 1][row] = ra[r].y;
      As[buf][kk + 2][row] = ra[r].z;
      As[buf][kk + 3][row] = ra[r].w;
      Bs[buf][kk + 0][row] = rb[r].x;
      Bs[buf][kk + 1][row] = rb[r].y;
      Bs[buf][kk + 2][row] = rb[r].z;
      Bs[buf][kk + 3][row] = rb[r].w;
    }
  };

  const int nk = (K + BK - 1) / BK;
  load_tiles(0);
  store_tiles(0);
  __syncthreads();
  for (int kt = 0; kt < nk; ++kt) {
    const int cur = kt & 1;
    if (kt + 1 < nk) load_tiles((kt + 1) * BK);
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      float a[8], b[8];
      const float4 a0 = *reinterpret_cast<const float4*>(&As[cur][k][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[cur][k][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[cur][k][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[cur][k][64 + tx * 4]);
      a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w; a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
      b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w; b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (kt + 1 < nk) store_tiles(cur ^ 1);
    __syncthreads();
  }

#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int n = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
      if (n >= N) continue;
      float v = acc[i][j] + (bias ? bias[n] : 0.f);
      float* o = out + (size_t)m * N + n;
      if (epi == EPI_GELU)
        *o = gelu_erf(v);
      else if (epi == EPI_RESID_F32)
        *o = *o + v;
      else
        *o = v;
    }
  }
}

wm_status launch_sgemm(const float* A, const float* W, const float* bias, float* out, int M, int N, int K, int epi,
                       cudaStream_t s) {
  if (M <= 0 || N <= 0) return WM_OK;
  dim3 grid((N + 127) / 128, (M + 127) / 128), block(256);
  const bool vec = (K % 4 == 0) && ((uintptr_t)A % 16 == 0) && ((uintptr_t)W % 16 == 0);
  if (vec)
    sgemm_kernel<true><<<grid, block, 0, s>>>(A, W, bias, out, M, N, K, epi);
  else
    sgemm_kernel<false><<<grid, block, 0, s>>>(A, W, bias, out, M, N, K, epi);
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

// ------------------------------------------------------- rotary embedding ----
// One thread per (token, rotation pair) of q and of k in an fp32 qkv [M, 3C].
__global__ void rope_f32_kernel(float* __restrict__ qkv, long M, const RopeArgs* __restrict__ R) {
  const int P = R->C / 2;
  const long total = M * 2 * P;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const long m = i / (2 * P);
    const int r = (int)(i % (2 * P));   // pair index over q (r < P) then k
    const int col = 2 * (r % P) + (r >= P ? R->C : 0);
    const int p = (col % R->C) % R->dh / 2;
    const int tok = (int)(m % ((long)R->D * R->H * R->W));
    const int pos[3] = {tok / (R->H * R->W), (tok / R->W) % R->H, tok % R->W};
    const int ax = p < R->n[0] ? 0 : (p < R->n[0] + R->n[1] ? 1 : 2);
    const int pm = p - (ax > 0 ? R->n[0] : 0) - (ax > 1 ? R->n[1] : 0);
    const float2 cs = R->tab[ax][pos[ax] * R->n[ax] + pm];
    float* v = qkv + m * 3L * R->C + col;
    const float a0 = v[0], a1 = v[1];
    v[0] = a0 * cs.x - a1 * cs.y;
    v[1] = a0 * cs.y + a1 * cs.x;
  }
}

wm_status launch_rope_f32(float* qkv, long M, const RopeArgs* rope_dev, const RopeArgs& rope_host, cudaStream_t s) {
  if (M <= 0) return WM_OK;
  const long total = M * rope_host.C;
  const int blocks = (int)std::min<long>((total + 255) / 256, (long)num_sms() * 16);
  rope_f32_kernel<<<blocks, 256, 0, s>>>(qkv, M, rope_dev);
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

// ------------------------------------------------- neighborhood attention ----
// One warp per (token, head). Scores for the kd*kh*kw neighbours go to shared
// memory, the softmax max and sum are warp-shuffle reductions in FP32, and the
// output channels are split across lanes.

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__global__ void na_f32_kernel(const float* __restrict__ qkv, float* __restrict__ out, int B, int D, int H, int W,
                              int C, int heads, int kd, int kh, int kw, int periodic) {
  extern __shared__ float smem[];
  const int warps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int dh = C / heads, K = kd * kh * kw;
  float* qs = smem + warp * (K + dh);
  float* sc = qs + dh;
  const long N = (long)D * H * W;
  const long gw = (long)blockIdx.x * warps + warp;
  if (gw >= (long)B * N * heads) return;  // whole warp leaves together
  const int head = (int)(gw % heads);
  const long bt = gw / heads;
  const long t = bt % N, b = bt / N;
  const int l = (int)(t / ((long)H * W)), i = (int)((t / W) % H), j = (int)(t % W);
  const int sl = clampi(l - kd / 2, 0, D - kd), si = clampi(i - kh / 2, 0, H - kh);
  const int sj = periodic ? j - kw / 2 : clampi(j - kw / 2, 0, W - kw);
  const long C3 = 3L * C;
  const float scale = rsqrtf((float)dh);
  const float* qrow = qkv + (b * N + t) * C3 + head * dh;
  for (int c = lane; c < dh; c += 32) qs[c] = qrow[c];
  __syncwarp();

  auto key_token = [&](int kk) -> long {
    const int a = kk / (kh * kw), bb = (kk / kw) % kh, cc = kk % kw;
    int jj = sj + cc;
    if (periodic) jj = ((jj % W) + W) % W;
    return ((long)(sl + a) * H + (si + bb)) * W + jj;
  };

  float mx = -INFINITY;
  for (int kk = lane; kk < K; kk += 32) {
    const float* krow = qkv + (b * N + key_token(kk)) * C3 + C + head * dh;
    float d = 0.f;
    for (int c = 0; c < dh; ++c) d = fmaf(qs[c], krow[c], d);
    d *= scale;
    sc[kk] = d;
    mx = fmaxf(mx, d);
  }
  mx = warp_max(mx);
  float sum = 0.f;
  for (int kk = lane; kk < K; kk += 32) {
    const float e = expf(sc[kk] - mx);
    sc[kk] = e;
    sum += e;
  }
  sum = warp_sum(sum);
  __syncwarp();
  const float inv = 1.f / sum;
  float* orow = out + (b * N + t) * C + head * dh;
  for (int c = lane; c < dh; c += 32) {
    float acc = 0.f;
    for (int kk = 0; kk < K; ++kk) acc = fmaf(sc[kk], qkv[(b * N + key_token(kk)) * C3 + 2 * C + head * dh + c], acc);
    orow[c] = acc * inv;
  }
}

// Tiled FP32 attention: CTA = batch element, head, query level and an 8 x 8
// block of queries; four threads per query, each owning a quarter of the
// head's channels (a score is the quarters' dot products added with two
// shuffles).
// For every key level the CTA stages the tile's K and V halo slabs (rows of
// dh + 4 floats: 128-bit loads of consecutive keys hit distinct banks) in
// shared memory; each query walks its own window row by row with an online
// softmax (running max and sum in FP32, O rescaled once per window row).
// Strict FP32 FMA and expf throughout.
template <int DH>
__global__ void __launch_bounds__(256, 2) na_f32_tile_kernel(const float* __restrict__ qkv, float* __restrict__ out,
                                                          int B, int D, int H, int W, int C, int heads, int kd, int kh,
                                                          int kw, int periodic, int tiles_h, int tiles_w,
                                                          int* __restrict__ dstatus) {
  constexpr int TH = 8, TW = 8, TPQ = 4, HD = DH / TPQ, KS = DH + 4;   // KS: key row stride in shared memory (floats)
  constexpr int KW_MAX = 9;
  extern __shared__ __align__(16) float sm[];
  const int HR = min(TH + kh - 1, H);
  const int WC = periodic ? TW + kw - 1 : min(TW + kw - 1, W);
  float* Ks = sm;
  float* Vs = sm + HR * WC * KS;
  int t = blockIdx.x;
  const int tw = t % tiles_w;
  t /= tiles_w;
  const int th = t % tiles_h;
  t /= tiles_h;
  const int d = t % D;
  t /= D;
  const int head = t % heads, b = t / heads;
  const int h0 = th * TH, w0 = tw * TW, rh = kh / 2, rw = kw / 2;
  const int hs0 = clampi(h0 - rh, 0, H - HR);
  const int ws0 = periodic ? w0 - rw : clampi(w0 - rw, 0, W - WC);
  const int ld0 = clampi(d - kd / 2, 0, D - kd);
  const int pair = threadIdx.x / TPQ, half = threadIdx.x % TPQ;   // query of the tile, channel quarter
  const int hq = h0 + pair / TW, wq = w0 + pair % TW;
  bool valid = hq < H && wq < W;
  const int hc = min(hq, H - 1), wc = min(wq, W - 1);
  int ra = clampi(hc - rh, 0, H - kh) - hs0;                                   // window rows in the slab
  int cb = (periodic ? wc - rw : clampi(wc - rw, 0, W - kw)) - ws0;            // window columns
  // debug builds: the window lies inside the staged slab; on a failure it is
  // clamped into the slab and the query is not written
  if (!WM_DCHECK(ra >= 0 && ra + kh <= HR && cb >= 0 && cb + kw <= WC && ld0 >= 0 && ld0 + kd <= D, dstatus)) {
    ra = clampi(ra, 0, HR - kh);
    cb = clampi(cb, 0, WC - kw);
    valid = false;
  }
  const long N = (long)D * H * W, C3 = 3L * C;
  const float scale = rsqrtf((float)DH);
  float q[HD], o[HD];
  {
    const float4* qs = reinterpret_cast<const float4*>(qkv + ((long)b * N + ((long)d * H + hc) * W + wc) * C3 +
                                                       head * DH + half * HD);
#pragma unroll
    for (int i = 0; i < HD / 4; ++i) {
      const float4 v = qs[i];
      q[4 * i] = v.x; q[4 * i + 1] = v.y; q[4 * i + 2] = v.z; q[4 * i + 3] = v.w;
    }
  }
#pragma unroll
  for (int i = 0; i < HD; ++i) o[i] = 0.f;
  float m = -INFINITY, l = 0.f;
  const int slab_keys = HR * WC;
  for (int li = 0; li < kd; ++li) {
    __syncthreads();   // the previous level's slabs are no longer read
    const long lev = (long)b * D + ld0 + li;
    for (int idx = threadIdx.x; idx < 2 * slab_keys * (DH / 4); idx += blockDim.x) {
      const int kv = idx / (slab_keys * (DH / 4));
      const int rem = idx - kv * slab_keys * (DH / 4);
      const int key = rem / (DH / 4), c4 = rem - key * (DH / 4);
      const int r = key / WC, c = key - r * WC;
      int lon = ws0 + c;
      if (periodic) lon = ((lon % W) + W) % W;
      const float4 v = *reinterpret_cast<const float4*>(qkv + ((lev * H + hs0 + r) * W + lon) * C3 + (1 + kv) * C +
                                                        head * DH + 4 * c4);
      *reinterpret_cast<float4*>((kv ? Vs : Ks) + key * KS + 4 * c4) = v;
    }
    __syncthreads();
    for (int a = 0; a < kh; ++a) {
      const int row = (ra + a) * WC + cb;
      float sc[KW_MAX];
      float rmax = -INFINITY;
#pragma unroll
      for (int j = 0; j < KW_MAX; ++j) {
        if (j < kw) {
          const float4* kr = reinterpret_cast<const float4*>(Ks + (row + j) * KS + half * HD);
          float acc = 0.f;
#pragma unroll
          for (int i = 0; i < HD / 4; ++i) {
            const float4 k4 = kr[i];
            acc = fmaf(q[4 * i], k4.x, acc);
            acc = fmaf(q[4 * i + 1], k4.y, acc);
            acc = fmaf(q[4 * i + 2], k4.z, acc);
            acc = fmaf(q[4 * i + 3], k4.w, acc);
          }
          acc += __shfl_xor_sync(0xffffffffu, acc, 1);   // the other channel quarters
          acc += __shfl_xor_sync(0xffffffffu, acc, 2);
          sc[j] = acc * scale;
          rmax = fmaxf(rmax, sc[j]);
        }
      }
      if (rmax > m) {
        const float alpha = expf(m - rmax);   // 0 while m = -inf: O and l are still zero
        l *= alpha;
#pragma unroll
        for (int i = 0; i < HD; ++i) o[i] *= alpha;
        m = rmax;
      }
#pragma unroll
      for (int j = 0; j < KW_MAX; ++j) {
        if (j < kw) {
          const float p = expf(sc[j] - m);
          l += p;
          const float4* vr = reinterpret_cast<const float4*>(Vs + (row + j) * KS + half * HD);
#pragma unroll
          for (int i = 0; i < HD / 4; ++i) {
            const float4 v4 = vr[i];
            o[4 * i] = fmaf(p, v4.x, o[4 * i]);
            o[4 * i + 1] = fmaf(p, v4.y, o[4 * i + 1]);
            o[4 * i + 2] = fmaf(p, v4.z, o[4 * i + 2]);
            o[4 * i + 3] = fmaf(p, v4.w, o[4 * i + 3]);
          }
        }
      }
    }
  }
  if (!valid) return;
  const float inv = 1.f / l;
  float4* orow = reinterpret_cast<float4*>(out + ((long)b * N + ((long)d * H + hq) * W + wq) * C + head * DH +
                                           half * HD);
#pragma unroll
  for (int i = 0; i < HD / 4; ++i)
    orow[i] = make_float4(o[4 * i] * inv, o[4 * i + 1] * inv, o[4 * i + 2] * inv, o[4 * i + 3] * inv);
}

// Shared memory of the tiled FP32 attention (K and V slabs), or 0 if the
// shape does not fit it.
static size_t na_f32_tile_smem(int H, int W, int dh, int kh, int kw, bool periodic) {
  if (kw > 9 || (dh != 16 && dh != 32 && dh != 48 && dh != 64)) return 0;   // dh / 4 channels per thread in float4
  const int HR = std::min(8 + kh - 1, H), WC = periodic ? 8 + kw - 1 : std::min(8 + kw - 1, W);
  const size_t bytes = (size_t)2 * HR * WC * (dh + 4) * sizeof(float);
  return bytes <= 227 * 1024 ? bytes : 0;
}

wm_status prepare_na_f32() {
  WM_CUDA(cudaFuncSetAttribute(na_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  WM_CUDA(cudaFuncSetAttribute(na_f32_tile_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  WM_CUDA(cudaFuncSetAttribute(na_f32_tile_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  WM_CUDA(cudaFuncSetAttribute(na_f32_tile_kernel<48>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  WM_CUDA(cudaFuncSetAttribute(na_f32_tile_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  return WM_OK;
}

wm_status launch_na_f32(const float* qkv, float* out, int B, int D, int H, int W, int C, int heads, int kd, int kh,
                        int kw, bool periodic, cudaStream_t s) {
  const long total = (long)B * D * H * W * heads;
  if (total <= 0) return WM_OK;
  const int dh0 = C / heads;
  const size_t tsm = na_f32_tile_smem(H, W, dh0, kh, kw, periodic);
  if (tsm && (C % 4) == 0 && (reinterpret_cast<uintptr_t>(qkv) & 15) == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0) {
    const int tiles_h = (H + 7) / 8, tiles_w = (W + 7) / 8;
    const long ctas = (long)tiles_h * tiles_w * D * heads * B;
    if (ctas > (1L << 31) - 1) return fail(WM_ERR_INVALID_ARG, "too many attention tiles");
    const dim3 grid((unsigned)ctas), block(256);
    const int per = periodic ? 1 : 0;
    switch (dh0) {
      case 16: na_f32_tile_kernel<16><<<grid, block, tsm, s>>>(qkv, out, B, D, H, W, C, heads, kd, kh, kw, per, tiles_h, tiles_w, device_status_word()); break;
      case 32: na_f32_tile_kernel<32><<<grid, block, tsm, s>>>(qkv, out, B, D, H, W, C, heads, kd, kh, kw, per, tiles_h, tiles_w, device_status_word()); break;
      case 48: na_f32_tile_kernel<48><<<grid, block, tsm, s>>>(qkv, out, B, D, H, W, C, heads, kd, kh, kw, per, tiles_h, tiles_w, device_status_word()); break;
      default: na_f32_tile_kernel<64><<<grid, block, tsm, s>>>(qkv, out, B, D, H, W, C, heads, kd, kh, kw, per, tiles_h, tiles_w, device_status_word()); break;
    }
    WM_CUDA(cudaGetLastError());
    return WM_OK;
  }
  // other shapes: one warp per (query, head)
  const int warps = 8;
  const int K = kd * kh * kw, dh = C / heads;
  const size_t smem = (size_t)warps * (K + dh) * sizeof(float);
  if (smem > 227 * 1024) return fail(WM_ERR_INVALID_ARG, "neighborhood window too large for the FP32 attention kernel");
  dim3 grid((unsigned)((total + warps - 1) / warps)), block(32 * warps);
  na_f32_kernel<<<grid, block, smem, s>>>(qkv, out, B, D, H, W, C, heads, kd, kh, kw, periodic ? 1 : 0);
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

}  // namespace wm
