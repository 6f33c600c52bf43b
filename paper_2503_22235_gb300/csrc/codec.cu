// Encoder and decoder around the latent (Section 2.1, Appendix A.2; the
// readings are listed with wm_codec_config in wm.h).
//
// Encoder: the patch embeddings are GEMMs over a patch matrix that one
// gather kernel writes (bf16 for the tensor-core path, fp32 for the plain
// path; rows = latent tokens, columns = (level, row, column, channel) of the
// token's input patch); the NA blocks are a wm_ctx of width Ce whose six-hour
// stack holds the encoder's blocks; the output map is one more GEMM. The
// decoder runs the one-hour stack of the same wm_ctx and scatters the
// transposed convolutions' outputs (one GEMM per part) back to the grid.
#include <cstring>
#include <vector>

#include "wm_internal.cuh"

using wm::fail;
using bf16 = __nv_bfloat16;

#define WM_TRY(expr)                 \
  do {                               \
    wm_status st_ = (expr);          \
    if (st_ != WM_OK) return st_;    \
  } while (0)

namespace {

enum CodecTensor {
  T_EMBED_ATM_W, T_EMBED_ATM_B, T_EMBED_SFC_W, T_EMBED_SFC_B, T_ENC_OUT_W, T_ENC_OUT_B,
  T_DEC_IN_W, T_DEC_IN_B, T_UNEMBED_ATM_W, T_UNEMBED_ATM_B, T_UNEMBED_SFC_W, T_UNEMBED_SFC_B, T_COUNT
};

struct Dims {
  int D, H, W;
  long ntok;      // latent tokens
  long m_atm;     // atmospheric tokens ((D - 1) H W)
  long m_sfc;     // surface tokens (H W)
  int k_atm;      // pd p p v_atm
  int k_sfc;      // p p (v_sfc_in + n_const)
  int n_sfc_out;  // p p v_sfc_out
};

Dims dims_of(const wm_codec_config& c) {
  Dims d;
  d.D = c.level_pad / c.pd + 1;
  d.H = c.H0 / c.p;
  d.W = c.W0 / c.p;
  d.m_sfc = (long)d.H * d.W;
  d.m_atm = (long)(d.D - 1) * d.m_sfc;
  d.ntok = d.m_atm + d.m_sfc;
  d.k_atm = c.pd * c.p * c.p * c.v_atm;
  d.k_sfc = c.p * c.p * (c.v_sfc_in + c.n_const);
  d.n_sfc_out = c.p * c.p * c.v_sfc_out;
  return d;
}

void tensor_sizes(const wm_codec_config& c, const Dims& d, size_t* n) {
  n[T_EMBED_ATM_W] = (size_t)c.Ce * d.k_atm;      n[T_EMBED_ATM_B] = c.Ce;
  n[T_EMBED_SFC_W] = (size_t)c.Ce * d.k_sfc;      n[T_EMBED_SFC_B] = c.Ce;
  n[T_ENC_OUT_W] = (size_t)c.C * c.Ce;            n[T_ENC_OUT_B] = c.C;
  n[T_DEC_IN_W] = (size_t)c.Ce * c.C;             n[T_DEC_IN_B] = c.Ce;
  n[T_UNEMBED_ATM_W] = (size_t)d.k_atm * c.Ce;    n[T_UNEMBED_ATM_B] = d.k_atm;
  n[T_UNEMBED_SFC_W] = (size_t)d.n_sfc_out * c.Ce; n[T_UNEMBED_SFC_B] = d.n_sfc_out;
}

// ---------------------------------------------------------------- kernels --
// One thread per patch-matrix element; consecutive threads walk a token's
// columns, so each (level, row) stretch of p * v consecutive input floats is
// read by consecutive threads.

template <typename T>
__device__ __forceinline__ T from_f32(float v);
template <>
__device__ __forceinline__ float from_f32<float>(float v) { return v; }
template <>
__device__ __forceinline__ bf16 from_f32<bf16>(float v) { return __float2bfloat16_rn(v); }

template <typename T>
__global__ void patch_atm_kernel(const float* __restrict__ atm, T* __restrict__ out, long total, int H, int W,
                                 int H0, int W0, int pd, int p, int v, int top) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int K = pd * p * p * v;
  const long tok = e / K;
  int col = (int)(e - tok * K);
  const int vv = col % v; col /= v;
  const int dx = col % p; col /= p;
  const int dy = col % p;
  const int dl = col / p;
  const int w = (int)(tok % W), h = (int)((tok / W) % H), l = (int)(tok / ((long)W * H));
  const int lev = l * pd + dl - top;          // zero levels above the first input level
  float val = 0.f;
  if (lev >= 0) val = atm[(((long)lev * H0 + (long)h * p + dy) * W0 + (long)w * p + dx) * v + vv];
  out[e] = from_f32<T>(val);
}

template <typename T>
__global__ void patch_sfc_kernel(const float* __restrict__ sfc, const float* __restrict__ cst, T* __restrict__ out,
                                 long total, int W, int W0, int p, int vs, int nc) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int cin = vs + nc;
  const int K = p * p * cin;
  const long tok = e / K;
  int col = (int)(e - tok * K);
  const int c = col % cin; col /= cin;
  const int dx = col % p;
  const int dy = col / p;
  const long w = tok % W, h = tok / W;
  const long pix = (h * p + dy) * W0 + w * p + dx;
  const float val = c < vs ? sfc[pix * vs + c] : cst[pix * nc + (c - vs)];
  out[e] = from_f32<T>(val);
}

// Transposed convolutions: output pixel (level, y, x, var) reads column
// ((level % pd) p + y % p) p + x % p) v + var of token (level / pd, y / p, x / p).
__global__ void unpatch_atm_kernel(const float* __restrict__ y, float* __restrict__ atm, long total, int H, int W,
                                   int H0, int W0, int pd, int p, int v, int top) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  long r = e;
  const int vv = (int)(r % v); r /= v;
  const int x = (int)(r % W0); r /= W0;
  const int yy = (int)(r % H0);
  const int lev = (int)(r / H0) + top;
  const long tok = ((long)(lev / pd) * H + yy / p) * W + x / p;
  const int col = (((lev % pd) * p + yy % p) * p + x % p) * v + vv;
  atm[e] = y[tok * (long)(pd * p * p * v) + col];
}

__global__ void unpatch_sfc_kernel(const float* __restrict__ y, float* __restrict__ sfc, long total, int W, int W0,
                                   int p, int v) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  long r = e;
  const int vv = (int)(r % v); r /= v;
  const int x = (int)(r % W0);
  const int yy = (int)(r / W0);
  const long tok = (long)(yy / p) * W + x / p;
  const int col = ((yy % p) * p + x % p) * v + vv;
  sfc[e] = y[tok * (long)(p * p * v) + col];
}

unsigned blocks_for(long total) { return (unsigned)((total + 255) / 256); }

}  // namespace

struct wm_codec {
  wm_codec_config cfg;
  Dims d;
  wm_ctx* inner = nullptr;           // the NA blocks (width Ce): encoder = six-hour stack, decoder = one-hour stack
  float* w32[T_COUNT] = {};          // fp32 tensors (biases; matrices of the plain path)
  bf16* w16[T_COUNT] = {};           // bf16 matrices (tensor-core path)
  void* patches = nullptr;           // [m_atm, k_atm] bf16 or fp32; also the surface patches
  float* xe = nullptr;               // [ntok, Ce] fp32: the encoder's / decoder's residual stream
  bf16* xh = nullptr;                // [ntok, max(Ce, C)] bf16 copy for the tensor-core GEMMs
  float* outp = nullptr;             // [m_atm, max(k_atm, n_sfc_out)] fp32: transposed-convolution outputs
  std::vector<void*> allocs;
};

namespace {

wm_status codec_alloc(wm_codec* cd, void** p, size_t bytes) {
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? WM_ERR_OOM : WM_ERR_CUDA, "codec allocation failed");
  }
  cd->allocs.push_back(*p);
  return WM_OK;
}

bool odd_pos(int k) { return k >= 1 && k % 2 == 1; }

wm_status validate(const wm_codec_config* c) {
  if (!c) return fail(WM_ERR_INVALID_ARG, "NULL codec config");
  if (c->p < 1 || c->pd < 1 || c->H0 < c->p || c->W0 < c->p || c->H0 % c->p || c->W0 % c->p)
    return fail(WM_ERR_INVALID_ARG, "the grid must be a positive multiple of the patch size p");
  if (c->levels < 1 || c->level_pad < c->levels || c->level_pad % c->pd)
    return fail(WM_ERR_INVALID_ARG, "need 1 <= levels <= level_pad and level_pad % pd == 0");
  if (c->v_atm < 1 || c->v_sfc_in < 0 || c->n_const < 0 || c->v_sfc_in + c->n_const < 1 || c->v_sfc_out < 1)
    return fail(WM_ERR_INVALID_ARG, "bad variable counts");
  if (c->C < 1 || c->Ce < 1 || c->heads < 1 || c->Ce % c->heads || c->blocks < 1)
    return fail(WM_ERR_INVALID_ARG, "bad widths or head count");
  if (!odd_pos(c->kd) || !odd_pos(c->kh) || !odd_pos(c->kw)) return fail(WM_ERR_INVALID_ARG, "window sizes must be odd");
  if (c->precision != WM_PREC_FP32 && c->precision != WM_PREC_BF16)
    return fail(WM_ERR_INVALID_ARG, "codec precision must be FP32 or BF16");
  if (c->precision == WM_PREC_BF16) {
    const int k_atm = c->pd * c->p * c->p * c->v_atm, k_sfc = c->p * c->p * (c->v_sfc_in + c->n_const);
    const int n_sfc = c->p * c->p * c->v_sfc_out;
    if (c->Ce % 8 || c->C % 8 || k_atm % 8 || k_sfc % 8 || n_sfc % 8)
      return fail(WM_ERR_INVALID_ARG, "the BF16 codec needs Ce, C and every patch width to be multiples of 8");
  }
  return WM_OK;
}

wm_status linear(const wm_codec* cd, const void* A, int t_w, int t_b, float* out, long M, int N, int K,
                 cudaStream_t s) {
  if (M == 0) return WM_OK;
  const bool bf = cd->cfg.precision == WM_PREC_BF16;
  return wm_op_linear(A, bf ? (const void*)cd->w16[t_w] : (const void*)cd->w32[t_w], cd->w32[t_b], out, (int)M, N, K,
                      cd->cfg.precision, wm::EPI_STORE_F32, s);
}

// fp32 [rows, n] -> the GEMM operand: a bf16 copy (tensor-core path) or the array itself
wm_status operand(const wm_codec* cd, const float* x, long n, const void** A, cudaStream_t s) {
  if (cd->cfg.precision == WM_PREC_FP32) {
    *A = x;
    return WM_OK;
  }
  WM_TRY(wm::launch_f32_to_bf16(x, cd->xh, (size_t)n, s));
  *A = cd->xh;
  return WM_OK;
}

}  // namespace

extern "C" {

wm_status wm_codec_create(const wm_codec_config* cfg, const float* host_weights, size_t n_floats, wm_codec** out) {
  if (!out || !host_weights) return fail(WM_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  WM_TRY(validate(cfg));
  const wm_codec_config c = *cfg;
  const Dims d = dims_of(c);
  size_t sizes[T_COUNT];
  tensor_sizes(c, d, sizes);
  size_t own = 0;
  for (size_t n : sizes) own += n;
  const size_t per_block = 12ull * c.Ce * c.Ce + 13ull * c.Ce;
  if (n_floats != own + 2ull * c.blocks * per_block)
    return fail(WM_ERR_INVALID_ARG, "codec weight blob has the wrong length for this config");
  WM_TRY(wm::prepare_kernels());
  wm_codec* cd = new wm_codec();
  cd->cfg = c;
  cd->d = d;
  auto cleanup = [&](wm_status st) {
    wm_codec_destroy(cd);
    return st;
  };
  // the NA blocks, as a context of width Ce
  wm_config ic{};
  ic.D = d.D; ic.H = d.H; ic.W = d.W; ic.C = c.Ce; ic.heads = c.heads;
  ic.kd = c.kd; ic.kh = c.kh; ic.kw = c.kw;
  ic.blocks_p6 = c.blocks; ic.blocks_p1 = c.blocks;
  ic.lon_periodic = c.lon_periodic; ic.ln_eps = c.ln_eps; ic.precision = c.precision; ic.max_batch = 1; ic.rope = 0;
  wm_status st = wm_create_from_host(&ic, host_weights + own, n_floats - own, &cd->inner);
  if (st != WM_OK) return cleanup(st);
  // own tensors
  size_t off = 0;
  for (int t = 0; t < T_COUNT; ++t) {
    void* p = nullptr;
    if ((st = codec_alloc(cd, &p, sizes[t] * 4)) != WM_OK) return cleanup(st);
    cd->w32[t] = (float*)p;
    if (cudaMemcpy(p, host_weights + off, sizes[t] * 4, cudaMemcpyHostToDevice) != cudaSuccess)
      return cleanup(fail(WM_ERR_CUDA, "codec weight upload failed"));
    const bool matrix = (t % 2) == 0;
    if (matrix && c.precision == WM_PREC_BF16) {
      if ((st = codec_alloc(cd, &p, sizes[t] * 2)) != WM_OK) return cleanup(st);
      cd->w16[t] = (bf16*)p;
      if ((st = wm::launch_f32_to_bf16(cd->w32[t], cd->w16[t], sizes[t], 0)) != WM_OK) return cleanup(st);
    }
    off += sizes[t];
  }
  // workspace
  const size_t el = c.precision == WM_PREC_BF16 ? 2 : 4;
  const size_t pcols = (size_t)std::max(d.k_atm, d.k_sfc);
  void* p = nullptr;
  if ((st = codec_alloc(cd, &cd->patches, (size_t)std::max(d.m_atm, 1L) * pcols * el)) != WM_OK) return cleanup(st);
  if ((st = codec_alloc(cd, &p, (size_t)d.ntok * c.Ce * 4)) != WM_OK) return cleanup(st);
  cd->xe = (float*)p;
  if (c.precision == WM_PREC_BF16) {
    if ((st = codec_alloc(cd, &p, (size_t)d.ntok * std::max(c.Ce, c.C) * 2)) != WM_OK) return cleanup(st);
    cd->xh = (bf16*)p;
  }
  if ((st = codec_alloc(cd, &p, (size_t)std::max(d.m_atm, d.m_sfc) * std::max(d.k_atm, d.n_sfc_out) * 4)) != WM_OK)
    return cleanup(st);
  cd->outp = (float*)p;
  if (cudaDeviceSynchronize() != cudaSuccess) return cleanup(fail(WM_ERR_CUDA, "codec setup failed"));
  *out = cd;
  return WM_OK;
}

wm_status wm_codec_destroy(wm_codec* cd) {
  if (!cd) return WM_OK;
  if (cd->inner) wm_destroy(cd->inner);
  for (void* p : cd->allocs) cudaFree(p);
  delete cd;
  return WM_OK;
}

wm_status wm_encode(wm_codec* cd, const float* atm, const float* sfc, const float* consts, float* latent,
                    void* stream) {
  if (!cd || !atm || !latent) return fail(WM_ERR_INVALID_ARG, "NULL argument");
  const wm_codec_config& c = cd->cfg;
  const Dims& d = cd->d;
  if ((c.v_sfc_in > 0 && !sfc) || (c.n_const > 0 && !consts)) return fail(WM_ERR_INVALID_ARG, "NULL surface input");
  cudaStream_t s = (cudaStream_t)stream;
  const bool bf = c.precision == WM_PREC_BF16;
  const int top = c.level_pad - c.levels;
  // atmosphere: patch matrix, embedding GEMM into latent levels 0 .. D-2
  long total = d.m_atm * d.k_atm;
  if (bf) patch_atm_kernel<bf16><<<blocks_for(total), 256, 0, s>>>(atm, (bf16*)cd->patches, total, d.H, d.W, c.H0,
                                                                    c.W0, c.pd, c.p, c.v_atm, top);
  else patch_atm_kernel<float><<<blocks_for(total), 256, 0, s>>>(atm, (float*)cd->patches, total, d.H, d.W, c.H0,
                                                                  c.W0, c.pd, c.p, c.v_atm, top);
  WM_CUDA(cudaGetLastError());
  WM_TRY(linear(cd, cd->patches, T_EMBED_ATM_W, T_EMBED_ATM_B, cd->xe, d.m_atm, c.Ce, d.k_atm, s));
  // surface + constants: the last latent level
  total = d.m_sfc * d.k_sfc;
  if (bf) patch_sfc_kernel<bf16><<<blocks_for(total), 256, 0, s>>>(sfc, consts, (bf16*)cd->patches, total, d.W,
                                                                    c.W0, c.p, c.v_sfc_in, c.n_const);
  else patch_sfc_kernel<float><<<blocks_for(total), 256, 0, s>>>(sfc, consts, (float*)cd->patches, total, d.W, c.W0,
                                                                  c.p, c.v_sfc_in, c.n_const);
  WM_CUDA(cudaGetLastError());
  WM_TRY(linear(cd, cd->patches, T_EMBED_SFC_W, T_EMBED_SFC_B, cd->xe + d.m_atm * c.Ce, d.m_sfc, c.Ce, d.k_sfc, s));
  // NA blocks, then the map to the processor's width
  WM_TRY(wm_processor_step(cd->inner, cd->xe, 1, WM_P6, stream));
  const void* A = nullptr;
  WM_TRY(operand(cd, cd->xe, d.ntok * c.Ce, &A, s));
  return linear(cd, A, T_ENC_OUT_W, T_ENC_OUT_B, latent, d.ntok, c.C, c.Ce, s);
}

wm_status wm_decode(wm_codec* cd, const float* latent, float* atm_out, float* sfc_out, void* stream) {
  if (!cd || !latent || !atm_out || !sfc_out) return fail(WM_ERR_INVALID_ARG, "NULL argument");
  const wm_codec_config& c = cd->cfg;
  const Dims& d = cd->d;
  cudaStream_t s = (cudaStream_t)stream;
  const void* A = nullptr;
  WM_TRY(operand(cd, latent, d.ntok * c.C, &A, s));
  WM_TRY(linear(cd, A, T_DEC_IN_W, T_DEC_IN_B, cd->xe, d.ntok, c.Ce, c.C, s));
  WM_TRY(wm_processor_step(cd->inner, cd->xe, 1, WM_P1, stream));
  WM_TRY(operand(cd, cd->xe, d.ntok * c.Ce, &A, s));
  const size_t el = c.precision == WM_PREC_BF16 ? 2 : 4;
  const int top = c.level_pad - c.levels;
  // atmosphere: one GEMM over levels 0 .. D-2, then the scatter to the grid
  WM_TRY(linear(cd, A, T_UNEMBED_ATM_W, T_UNEMBED_ATM_B, cd->outp, d.m_atm, d.k_atm, c.Ce, s));
  long total = (long)c.levels * c.H0 * c.W0 * c.v_atm;
  unpatch_atm_kernel<<<blocks_for(total), 256, 0, s>>>(cd->outp, atm_out, total, d.H, d.W, c.H0, c.W0, c.pd, c.p,
                                                        c.v_atm, top);
  WM_CUDA(cudaGetLastError());
  // surface: the last latent level
  const void* As = (const char*)A + (size_t)d.m_atm * c.Ce * el;
  WM_TRY(linear(cd, As, T_UNEMBED_SFC_W, T_UNEMBED_SFC_B, cd->outp, d.m_sfc, d.n_sfc_out, c.Ce, s));
  total = (long)c.H0 * c.W0 * c.v_sfc_out;
  unpatch_sfc_kernel<<<blocks_for(total), 256, 0, s>>>(cd->outp, sfc_out, total, d.W, c.W0, c.p, c.v_sfc_out);
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

wm_status wm_forecast_fields(wm_ctx* ctx, wm_codec* cd, const float* atm, const float* sfc, const float* consts,
                             int lead_hours, float* latent_ws, float* atm_out, float* sfc_out, void* stream) {
  if (!ctx || !cd || !latent_ws) return fail(WM_ERR_INVALID_ARG, "NULL argument");
  if (lead_hours < 0) return fail(WM_ERR_INVALID_ARG, "lead time must be >= 0");
  const wm_config* pc = wm::ctx_config(ctx);
  const Dims& d = cd->d;
  if (pc->D != d.D || pc->H != d.H || pc->W != d.W || pc->C != cd->cfg.C)
    return fail(WM_ERR_INVALID_ARG, "the processor's latent shape differs from the codec's");
  WM_TRY(wm_encode(cd, atm, sfc, consts, latent_ws, stream));
  WM_TRY(wm_latent_rollout(ctx, latent_ws, 1, lead_hours, stream));
  return wm_decode(cd, latent_ws, atm_out, sfc_out, stream);
}

}  // extern "C"
