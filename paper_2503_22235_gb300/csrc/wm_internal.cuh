// Internal declarations shared by the libwm translation units.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <utility>

#include "../../include/wm.h"

namespace wm {

// The configuration a context was created with.
const wm_config* ctx_config(const wm_ctx* ctx);
// One processor step on `batch` contiguous latents, replayed from a CUDA graph
// captured per (latent buffer, batch, processor, precision).
wm_status processor_step_graphed(wm_ctx* ctx, float* x, int batch, int which, cudaStream_t s);
// The same for n latents at arbitrary device addresses, in place, when the
// whole-rollout kernel takes the step (processor_step_inplace_ok).
bool processor_step_inplace_ok(wm_ctx* ctx, int n);
wm_status processor_step_inplace(wm_ctx* ctx, float* const* xs, int n, int which, cudaStream_t s);

// ------------------------------------------------------------ errors ----
void set_error(const std::string& msg);
wm_status fail(wm_status st, const std::string& msg);
wm_status cuda_fail(cudaError_t e, const char* what);

#define WM_CUDA(call)                                      \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return wm::cuda_fail(e_, #call); \
  } while (0)

// NVTX range for the lifetime of a scope (host side): profilers show one range
// per processor step, block and kernel launch. Without a profiler attached the
// push and pop are no-ops.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Device status word written by bounded device-side waits (one per device).
int* device_status_word();

// Debug builds (WM_DEBUG_CHECKS=1, libwm_debug.so): WM_DCHECK(cond, status)
// is a device-side index check; when cond is false it records
// WM_ERR_BOUNDS in the status word (first failure wins) and yields false so
// that the caller skips the access. Release builds compile it to true.
#ifndef WM_DEBUG_CHECKS
#define WM_DEBUG_CHECKS 0
#endif
#if WM_DEBUG_CHECKS
__device__ __forceinline__ bool dcheck_fail(int* status) {
  if (status) atomicCAS(status, 0, (int)WM_ERR_BOUNDS);
  return false;
}
#define WM_DCHECK(cond, status) ((cond) ? true : ::wm::dcheck_fail(status))
#else
#define WM_DCHECK(cond, status) true
#endif

// Upper bound on any single device-side spin-wait (nanoseconds).
constexpr unsigned long long kWaitLimitNs = 4000000000ull;

// Programmatic dependent launch. Kernels of the block chain are launched
// with launch_pdl: such a kernel may start while its predecessor in the
// stream is still running, so it runs only its prologue (barrier init, TMEM
// allocation, descriptor prefetch: nothing that touches global memory) before
// pdl_wait(), which returns once every earlier grid in the stream has
// completed and its writes are visible. pdl_trigger() lets the next grid be
// scheduled as soon as every CTA of this one has issued it (or exited). Both
// are no-ops for a kernel launched without the attribute. The attribute pays
// where launch latency and prologues are a visible share of a kernel (small
// problems); on large batches it was measured slightly slower, so callers
// enable it only up to kPdlMaxTokens tokens.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

constexpr long kPdlMaxTokens = 65536;

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              bool enable, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = enable ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// launch_pdl for a grid of two-CTA clusters (consecutive blockIdx.x pairs).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl_pairs(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                    bool enable, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = enable ? 2 : 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Paired FP32 arithmetic (f32x2 instructions: one instruction, two lanes,
// each rounded exactly as the scalar instruction) and a three-input max.
__device__ __forceinline__ uint64_t pack_f2(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
// (d0, d1) = (a0, a1) * b2 + c2
__device__ __forceinline__ void fma_f2(float& d0, float& d1, float a0, float a1, uint64_t b2, uint64_t c2) {
  asm("{\n .reg .b64 ra, rd;\n mov.b64 ra, {%2, %3};\n fma.rn.f32x2 rd, ra, %4, %5;\n mov.b64 {%0, %1}, rd;\n}"
      : "=f"(d0), "=f"(d1)
      : "f"(a0), "f"(a1), "l"(b2), "l"(c2));
}
// (d0, d1) = (a0, a1) - b2
__device__ __forceinline__ void sub_f2(float& d0, float& d1, float a0, float a1, uint64_t b2) {
  asm("{\n .reg .b64 ra, rd;\n mov.b64 ra, {%2, %3};\n sub.rn.f32x2 rd, ra, %4;\n mov.b64 {%0, %1}, rd;\n}"
      : "=f"(d0), "=f"(d1)
      : "f"(a0), "f"(a1), "l"(b2));
}
// (d0, d1) = (a0, a1) + (b0, b1)
__device__ __forceinline__ void add_f2(float& d0, float& d1, float a0, float a1, float b0, float b1) {
  asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n add.rn.f32x2 rd, ra, rb;\n"
      " mov.b64 {%0, %1}, rd;\n}"
      : "=f"(d0), "=f"(d1)
      : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}
// (x0, x1) *= b2
__device__ __forceinline__ void mul_f2(float& x0, float& x1, uint64_t b2) {
  asm("{\n .reg .b64 ra, rd;\n mov.b64 ra, {%2, %3};\n mul.rn.f32x2 rd, ra, %4;\n mov.b64 {%0, %1}, rd;\n}"
      : "=f"(x0), "=f"(x1)
      : "f"(x0), "f"(x1), "l"(b2));
}
__device__ __forceinline__ float max3(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

enum Epilogue : int {
  EPI_STORE = 0,       // out = acc + bias (fp32 path: float; bf16 path: bfloat16)
  EPI_GELU = 1,        // out = GELU(acc + bias)
  EPI_RESID_F32 = 2,   // out(float) += acc + bias
  EPI_STORE_F32 = 3,   // out(float) = acc + bias
  EPI_GELU_F8 = 4,     // out(e4m3) = GELU(alpha * acc + bias) * out_scale, RNE, saturating
  EPI_RESID_LN = 5,    // x(float) += acc + bias; also writes bf16(x) (tmC2) and per-row partial
                       // (mean, M2) over each half tile into stats [M][2 * N/BN][2]
  EPI_LNF_STORE = 6,   // LayerNorm folded: out(bf16) = rstd (acc - mean colsum) + bias, where mean
                       // and rstd come from the np partials per row in stats
  EPI_LNF_GELU = 7,    // as EPI_LNF_STORE, then GELU
};

struct RopeArgs;
struct EpiArgs {
  const float* bias;
  const float* colsum;  // LayerNorm-folded epilogues: per-column sum of the folded bf16 weights
  float* x;             // EPI_RESID_LN: the fp32 residual (read, then rewritten through tmC)
  float* stats;         // EPI_RESID_LN writes, EPI_LNF_* read
  int np;               // EPI_LNF_*: partials per row
  float eps;            // EPI_LNF_*: LayerNorm epsilon
  float alpha, out_scale;
  const struct RopeArgs* rope;   // EPI_LNF_STORE: rotate q and k (columns < 2C) when non-null
};

// 3D rotary position embedding tables (device): for each axis, cos/sin of
// pos * w_m as float2, [positions][pairs of that axis].
struct RopeArgs {
  const float2* tab[3];  // level, latitude, longitude
  int n[3];              // pairs per axis (n_lev, n_lat, n_lon)
  int D, H, W, C, dh;
};

int num_sms();

// Sets kernel attributes (dynamic shared memory limits) once per device, so
// that no attribute call happens later inside a stream capture.
wm_status prepare_kernels();
wm_status prepare_gemm_tc();
wm_status prepare_na_bf16();

// ------------------------------------------------------- fp32 plain path ----
wm_status launch_layernorm(const float* x, const float* g, const float* b, void* out, bool out_bf16, int M,
                           int C, float eps, cudaStream_t s);
// LayerNorm with e4m3 output: out = e4m3(LN(x) * inv_scale), RNE, saturating.
// Row statistics for the first LayerNorm-folded GEMM of a processor call:
// xb = bf16(x) and stats[m] = (mean, M2) of row m (one partial per row).
wm_status launch_row_stats(const float* x, __nv_bfloat16* xb, float* stats, int M, int C, cudaStream_t s,
                           bool pdl = false);
wm_status launch_layernorm_e4m3(const float* x, const float* g, const float* b, uint8_t* out, int M, int C,
                                float eps, float inv_scale, cudaStream_t s, bool pdl = false);
wm_status launch_sgemm(const float* A, const float* W, const float* bias, float* out, int M, int N, int K,
                       int epi, cudaStream_t s);
wm_status launch_na_f32(const float* qkv, float* out, int B, int D, int H, int W, int C, int heads, int kd,
                        int kh, int kw, bool periodic, cudaStream_t s);

// ------------------------------------------------------------ bf16 path ----
// 4D map over a qkv buffer [DB = batch * levels][H][W][C3] (bf16) whose box
// is (box_c channels, box_w longitudes, box_h latitudes, 1 level): one
// attention key slab. Out-of-range elements read as zero.
bool make_tmap_qkv_slab(CUtensorMap* map, const void* qkv, uint64_t C3, uint64_t W, uint64_t H, uint64_t DB,
                        uint32_t box_c, uint32_t box_w, uint32_t box_h);
// TMA descriptor of a row-major bf16 matrix [rows, cols] (cols contiguous),
// box = box_rows x 64 columns, 128-byte swizzle.
bool make_tmap_bf16(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, uint32_t box_rows);
// bf16 q, k, v viewed as [levels][H][W][C3]: box of 32 channels x box_w
// longitudes x box_h latitudes x 1 level, 64-byte swizzle (16-byte unit u of
// a 64-byte row at shared offset o lands at u ^ ((o >> 7) & 3)); rows past H
// read as zeros.
bool make_tmap_kv_slab(CUtensorMap* map, const void* qkv, uint64_t C3, uint64_t W, uint64_t H, uint64_t levels,
                       uint32_t box_w, uint32_t box_h);

// TMA descriptor of the GEMM output [rows, cols] (bf16 or fp32, row major),
// box 32 x 32, 64-byte (bf16) / 128-byte (fp32) swizzle.
bool make_tmap_out(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, bool f32);

// TMA descriptors for e4m3 (byte) matrices: operand [rows, cols] with box
// box_rows x 128 columns and the 128-byte swizzle; output with box 32 x 32 and
// the 32-byte swizzle.
bool make_tmap_e4m3(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, uint32_t box_rows);
bool make_tmap_out_e4m3(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols);

struct GemmArgs {
  CUtensorMap tmA;     // A [M, K], box 128 rows x 128 bytes
  CUtensorMap tmB;     // W [N, K], box BN rows x 128 bytes
  CUtensorMap tmC;     // output [M, N]: bf16 (EPI_STORE / EPI_GELU / EPI_LNF_*), e4m3 (EPI_GELU_F8), fp32 otherwise
  CUtensorMap tmC2;    // EPI_RESID_LN: bf16 copy of the new residual [M, N] (make_tmap_out, bf16)
  int M, N, K;
  const float* bias;
  const float* colsum = nullptr;
  float* x = nullptr;
  float* stats = nullptr;
  int np = 0;
  float eps = 0.f;
  int epi;
  int bn;              // 64, 128 or 256 (tmB box rows must match)
  bool f8 = false;     // A and W are e4m3 (kind::f8f6f4); otherwise bf16 (kind::f16)
  float alpha = 1.f;   // e4m3 only: accumulator scale (product of the operand scales)
  float out_scale = 1.f;  // EPI_GELU_F8: 1 / output scale
  const RopeArgs* rope = nullptr;  // device pointer; EPI_LNF_STORE rotates q and k
  bool pdl = false;    // launch as a programmatic dependent of the previous kernel
  int dual = -1;       // EPI_RESID_LN: second staging tile (1) or not (0); -1: by K (K <= 1024)
  bool pair = false;   // BN = 256 only: 256 x 256 tiles on CTA pairs (cta_group::2); tmB box of 128 rows
};
// Rotate q and k in an fp32 qkv [M, 3C] (the FP32 plain path).
wm_status launch_rope_f32(float* qkv, long M, const RopeArgs* rope_dev, const RopeArgs& rope_host, cudaStream_t s);
wm_status launch_gemm_tc(const GemmArgs& a, cudaStream_t s);

// The small latent's MLP (C = 128, hidden 512) fused into one kernel: FC1 with
// LayerNorm 2 folded (stats_in: the output projection's np_in partials per
// row, colsum1 / bias1: the folded W1's column sums and bias), GELU, FC2,
// x += (.) + bias2, the bf16 copy xb and LayerNorm-1 partials of the new x
// (np_out per row: 2 or 4, as FC2 on 128- or 64-column tiles writes them).
// Bit-identical to FC1 and FC2 as two GEMMs.
struct MlpArgs {
  CUtensorMap tmA;    // bf16 x [M, C] (make_tmap_bf16, box 128 rows)
  CUtensorMap tmW1;   // folded bf16 W1 [4C, C] (box 128 rows)
  CUtensorMap tmW2;   // bf16 W2 [C, 4C] (box 128 rows)
  int M = 0;
  const float* colsum1 = nullptr;
  const float* bias1 = nullptr;
  const float* bias2 = nullptr;
  const float* stats_in = nullptr;
  float* stats_out = nullptr;
  float* x = nullptr;
  __nv_bfloat16* xb = nullptr;
  int np_in = 0;
  int np_out = 2;
  float eps = 0.f;
  bool pdl = false;
};
wm_status launch_mlp_small(const MlpArgs& a, cudaStream_t s);

// Whole-rollout kernel for latents with C = 128 and 4 heads (k_rollout_small.cu):
// one cooperative launch runs every block of every latent's greedy schedule.
constexpr int kRolloutSmallMaxLatents = 8;
constexpr size_t kRolloutBlockBytes = 12 * 32768 + 1664 * 4;   // one RolloutBlock's weights and vectors
struct RolloutBlock {
  const __nv_bfloat16* w;   // 12 chunks of 128 x 128 bf16 in the 128B-swizzled K-major
                            // layout (Wqkv rows 0-127, 128-255, 256-383; Wo; W1 rows
                            // 0-127 .. 384-511; W2 columns 0-127 .. 384-511), then the
                            // block's vectors as fp32: bqkv[384] bo ln1_g ln1_b ln2_g
                            // ln2_b [128 each] b1[512] b2[128]
};
struct RolloutSmallArgs {
  CUtensorMap tm_kv[3];      // make_tmap_kv_slab over qkv ([2 G D][H][W][384]): 20, 18, 2 longitudes x 12 latitudes
  const RolloutBlock* blk;   // device array: the six-hour blocks, then the one-hour blocks
  int L6, L1;                // blocks per processor
  int G, T;                  // latents; CTAs (8 x 16-token patches) per latent
  int D, H, W, kd, kh, kw;   // H % 8 == 0, W % 16 == 0, W >= 32, kh <= 5, kw <= 5, periodic longitude
  float* x[kRolloutSmallMaxLatents];     // fp32 latents [D*H*W, 128], updated in place
  int n6[kRolloutSmallMaxLatents];       // six-hour steps per latent (then n1 one-hour steps)
  int n1[kRolloutSmallMaxLatents];
  __nv_bfloat16* qkv;        // workspace [2][G][D*H*W][384]
  unsigned int* bar;         // [G] counters, zero at launch
  int* status;               // device status word
  float eps, scale_log2;     // LayerNorm epsilon; log2(e) / sqrt(32)
};
// CTAs the device can hold at once for the rollout kernel (0 when unknown).
int rollout_small_capacity();
wm_status launch_rollout_small(const RolloutSmallArgs& a, cudaStream_t s);
// W[n][k] (row stride ld floats), n, k < 128, to one bf16 chunk of the layout above.
wm_status launch_swizzle_chunk(const float* W, int ld, __nv_bfloat16* out, cudaStream_t s);

// variant: WM_NA_* of wm.h (0 = tuned plan / the shape's fixed family).
wm_status launch_na_bf16(const __nv_bfloat16* qkv, __nv_bfloat16* out, int B, int D, int H, int W, int C,
                         int heads, int kd, int kh, int kw, bool periodic, cudaStream_t s, int variant = 0,
                         bool pdl = false);
// The tcgen05 attention kernel (k_na_tc.cu): whether it supports a shape, and
// its launch (same inputs and outputs as launch_na_bf16).
bool na_tc_supported(int H, int W, int C, int heads, int kh, int kw, bool periodic);
wm_status prepare_na_tc();
wm_status launch_na_tc(const __nv_bfloat16* qkv, __nv_bfloat16* out, int B, int D, int H, int W, int C, int heads,
                       int kd, int kh, int kw, bool periodic, cudaStream_t s, bool pdl = false);
// One line per autotuned attention shape: the plan chosen and its time.
std::string describe_na_plans();
// Times the candidate CTA plans of the attention kernel for this exact shape
// and keeps the fastest for later launch_na_bf16 calls (writes `out`).
wm_status autotune_na_bf16(const __nv_bfloat16* qkv, __nv_bfloat16* out, int B, int D, int H, int W, int C,
                           int heads, int kd, int kh, int kw, bool periodic, cudaStream_t s, double* best_ms);

// ---------------------------------------------------------------- misc ----
wm_status launch_f32_to_bf16(const float* in, __nv_bfloat16* out, size_t n, cudaStream_t s);
wm_status launch_f32_to_e4m3(const float* in, uint8_t* out, size_t n, float inv_scale, cudaStream_t s);
wm_status launch_sqdiff(const float* a, const float* b, size_t n, double* acc2, cudaStream_t s);
// *count += number of NaN or infinite elements of x[0, n).
wm_status launch_count_nonfinite(const float* x, size_t n, unsigned long long* count, cudaStream_t s);
wm_status launch_wait_selftest(int timeout_us, cudaStream_t s);

}  // namespace wm
