// libwm C ABI: context, weights, workspace, the block / processor / rollout
// orchestration, CUDA-graph capture of rollouts, batched uneven rollouts and
// the op-level entry points.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <array>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "wm_internal.cuh"

namespace wm {
const char* last_error_cstr();
}

using wm::fail;
using bf16 = __nv_bfloat16;

#define WM_TRY(expr)                 \
  do {                               \
    wm_status st_ = (expr);          \
    if (st_ != WM_OK) return st_;    \
  } while (0)

namespace {

struct BlockW {
  const float *ln1_g, *ln1_b, *wqkv, *bqkv, *wo, *bo, *ln2_g, *ln2_b, *w1, *b1, *w2, *b2;
  bf16 *ho, *h2;       // bf16 Wo and W2 (Wqkv and W1 are used LayerNorm-folded, below)
  CUtensorMap tm_o[3], tm_2[3];  // [0]: box 128 rows, [1]: box 256 rows, [2]: box 64 rows
  // LayerNorm folded into QKV and FC1: bf16 W diag(gamma), its column sums,
  // and the folded bias b + W beta
  bf16 *fqkv, *f1;
  const float *cs_qkv, *bb_qkv, *cs_1, *bb_1;
  CUtensorMap tm_fqkv[3], tm_f1[3];
  // FP8 MLP: e4m3 copies of W1, W2 and the static per-tensor scales
  uint8_t *q1, *q2;
  CUtensorMap tm_q1[3], tm_q2[3];
  float s_u, s_w1, s_h, s_w2;   // LN2 output, W1, GELU output, W2
};

}  // namespace

struct wm_ctx {
  wm_config cfg{};
  int device = 0;
  long N = 0;
  float* d_w32 = nullptr;
  bf16* d_wh = nullptr;
  uint8_t* d_wq = nullptr;   // e4m3 W1, W2 per block
  bf16* d_wf = nullptr;      // LayerNorm-folded bf16 Wqkv, W1 per block
  float2* d_rope_tab = nullptr;       // rotary embedding cos/sin tables (level, latitude, longitude)
  wm::RopeArgs* d_rope = nullptr;     // device copy of rope_host (pointers into d_rope_tab)
  wm::RopeArgs rope_host{};
  float* d_vf = nullptr;     // their column sums and folded biases
  std::vector<BlockW> blk[2];
  // workspace for cap32 (FP32 path) / cap16 (BF16 path) latents
  int cap32 = 0, cap16 = 0;
  float *f_u = nullptr, *f_qkv = nullptr, *f_o = nullptr, *f_h = nullptr;
  bf16 *h_u = nullptr, *h_qkv = nullptr, *h_o = nullptr, *h_h = nullptr;
  uint8_t *q_u = nullptr, *q_h = nullptr;   // e4m3 MLP operands (FP8 MLP precision)
  CUtensorMap tm_qu{}, tm_qh{}, tmc_qh{};
  bf16* xb = nullptr;        // bf16 copy of the residual, A operand of the folded GEMMs
  float* stats = nullptr;    // per-row (mean, M2) partials feeding the folded GEMMs
  CUtensorMap tm_xb{}, tmc_xb{};
  int np_next = 0;           // partials per row the last residual GEMM left in `stats`
  CUtensorMap tm_u{}, tm_o{}, tm_h{};
  CUtensorMap tmc_qkv{}, tmc_h{};   // GEMM outputs (TMA store descriptors)
  // staging
  float* d_stage = nullptr;
  size_t stage_cap = 0;  // floats
  float* d_io = nullptr;
  size_t io_cap = 0;     // floats
  float* d_ring[3] = {};                    // wm_forecast_host_many's ring of device latents
  size_t ring_cap[3] = {};
  cudaStream_t up_stream = nullptr, down_stream = nullptr;   // its copy streams
  cudaEvent_t io_ev[9] = {};                // uploaded[3], computed[3], downloaded[3]
  // graphs
  std::map<std::vector<uintptr_t>, cudaGraphExec_t> graphs;
  // optional per-launch timing (CUDA events around each hot-path kernel)
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, int>> ev_marks;  // (kernel kind, index of the start event)
  cudaStream_t cap_stream = nullptr;
  // whole-rollout kernel for narrow latents (k_rollout_small.cu)
  bf16* d_rs_w = nullptr;                 // per block: 12 swizzled bf16 weight chunks and the fp32 vectors
  wm::RolloutBlock* d_rs_blk = nullptr;   // per-block table: six-hour blocks, then one-hour blocks
  float* d_rs_qkv = nullptr;              // its double-buffered bf16 q, k, v (capacity in floats)
  size_t rs_qkv_cap = 0;
  unsigned int* d_rs_bar = nullptr;       // one barrier counter per latent
  std::recursive_mutex mu;
};

namespace {

constexpr int kMaxGraphs = 64;

bool is_odd_pos(int k) { return k >= 1 && (k % 2) == 1; }

wm_status validate(const wm_config* c) {
  if (!c) return fail(WM_ERR_INVALID_ARG, "config is NULL");
  if (c->D <= 0 || c->H <= 0 || c->W <= 0 || c->C <= 0 || c->heads <= 0)
    return fail(WM_ERR_INVALID_ARG, "D, H, W, C and heads must be positive");
  if (c->C % c->heads != 0) return fail(WM_ERR_INVALID_ARG, "C must be a multiple of heads");
  if (!is_odd_pos(c->kd) || !is_odd_pos(c->kh) || !is_odd_pos(c->kw))
    return fail(WM_ERR_INVALID_ARG, "window sizes must be odd and positive");
  if (c->kd > c->D || c->kh > c->H || c->kw > c->W)
    return fail(WM_ERR_INVALID_ARG, "a window is larger than its axis");
  if (c->blocks_p6 < 1 || c->blocks_p1 < 1) return fail(WM_ERR_INVALID_ARG, "each processor needs >= 1 block");
  if (c->rope != 0 && c->rope != 1) return fail(WM_ERR_INVALID_ARG, "rope must be 0 or 1");
  if (c->rope && ((c->C / c->heads) % 2 != 0 || c->C / c->heads < 6))
    return fail(WM_ERR_INVALID_ARG, "rotary embedding needs an even head dimension >= 6");
  if (c->precision < WM_PREC_FP32 || c->precision > WM_PREC_BF16_FP8MLP)
    return fail(WM_ERR_INVALID_ARG, "unknown precision");
  if (!(c->ln_eps >= 0.f)) return fail(WM_ERR_INVALID_ARG, "ln_eps must be >= 0");
  return WM_OK;
}

wm_status check_bf16_shape(const wm_config& c) {
  const int dh = c.C / c.heads;
  if (c.C % 64 != 0) return fail(WM_ERR_INVALID_ARG, "BF16 path needs C % 64 == 0");
  if (dh != 16 && dh != 32 && dh != 48 && dh != 64)
    return fail(WM_ERR_INVALID_ARG, "BF16 path needs head dim 16, 32, 48 or 64");
  return WM_OK;
}

size_t block_floats(int C) { return 12ull * C * C + 13ull * C; }

void destroy_graphs(wm_ctx* ctx) {
  for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
  ctx->graphs.clear();
}

void free_workspace(wm_ctx* ctx) {
  cudaFree(ctx->f_u); cudaFree(ctx->f_qkv); cudaFree(ctx->f_o); cudaFree(ctx->f_h);
  cudaFree(ctx->h_u); cudaFree(ctx->h_qkv); cudaFree(ctx->h_o); cudaFree(ctx->h_h);
  cudaFree(ctx->q_u); cudaFree(ctx->q_h);
  ctx->q_u = ctx->q_h = nullptr;
  cudaFree(ctx->xb); cudaFree(ctx->stats);
  ctx->xb = nullptr;
  ctx->stats = nullptr;
  ctx->f_u = ctx->f_qkv = ctx->f_o = ctx->f_h = nullptr;
  ctx->h_u = ctx->h_qkv = ctx->h_o = ctx->h_h = nullptr;
  ctx->cap32 = ctx->cap16 = 0;
}

wm_status tune_block_gemms(wm_ctx* ctx, int batch);

// Grow the workspace of one precision family to hold `batch` latents. Never
// called during capture; growing invalidates captured graphs (they hold
// workspace addresses).
wm_status ensure_workspace(wm_ctx* ctx, int batch, bool fp32) {
  int& cap = fp32 ? ctx->cap32 : ctx->cap16;
  if (batch <= cap) return WM_OK;
  destroy_graphs(ctx);
  const size_t M = (size_t)batch * ctx->N, C = ctx->cfg.C;
  const size_t el = fp32 ? 4 : 2;
  void** bufs[4];
  if (fp32) {
    bufs[0] = (void**)&ctx->f_u; bufs[1] = (void**)&ctx->f_qkv; bufs[2] = (void**)&ctx->f_o; bufs[3] = (void**)&ctx->f_h;
  } else {
    bufs[0] = (void**)&ctx->h_u; bufs[1] = (void**)&ctx->h_qkv; bufs[2] = (void**)&ctx->h_o; bufs[3] = (void**)&ctx->h_h;
  }
  const size_t widths[4] = {C, 3 * C, C, 4 * C};
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 4; ++i) {
    cudaFree(*bufs[i]);
    *bufs[i] = nullptr;
  }
  cap = 0;
  for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaMalloc(bufs[i], M * widths[i] * el);
  if (e != cudaSuccess) {
    for (int i = 0; i < 4; ++i) {
      cudaFree(*bufs[i]);
      *bufs[i] = nullptr;
    }
    cudaGetLastError();
    return fail(WM_ERR_OOM, "workspace allocation failed for batch " + std::to_string(batch));
  }
  if (!fp32) {
    cudaFree(ctx->q_u);
    cudaFree(ctx->q_h);
    cudaFree(ctx->xb);
    cudaFree(ctx->stats);
    ctx->q_u = ctx->q_h = nullptr;
    ctx->xb = nullptr;
    ctx->stats = nullptr;
    const size_t np_max = 2 * ((C + 63) / 64);   // LayerNorm partials: two per 64-column tile at most
    if (cudaMalloc(&ctx->xb, M * C * 2) != cudaSuccess || cudaMalloc(&ctx->stats, M * np_max * 2 * 4) != cudaSuccess) {
      cudaGetLastError();
      return fail(WM_ERR_OOM, "LayerNorm statistics workspace allocation failed");
    }
    if (C % 8 == 0 && (!wm::make_tmap_bf16(&ctx->tm_xb, ctx->xb, M, C, 128) ||
                       !wm::make_tmap_out(&ctx->tmc_xb, ctx->xb, M, C, false)))
      return fail(WM_ERR_CUDA, "cuTensorMapEncodeTiled failed for the residual copy");
    if (cudaMalloc(&ctx->q_u, M * C) != cudaSuccess || cudaMalloc(&ctx->q_h, M * 4 * C) != cudaSuccess) {
      cudaGetLastError();
      return fail(WM_ERR_OOM, "e4m3 workspace allocation failed");
    }
    if (C % 16 == 0 && (!wm::make_tmap_e4m3(&ctx->tm_qu, ctx->q_u, M, C, 128) ||
                        !wm::make_tmap_e4m3(&ctx->tm_qh, ctx->q_h, M, 4 * C, 128) ||
                        !wm::make_tmap_out_e4m3(&ctx->tmc_qh, ctx->q_h, M, 4 * C)))
      return fail(WM_ERR_CUDA, "cuTensorMapEncodeTiled failed for the e4m3 workspace");
  }
  cap = batch;
  if (!fp32 && check_bf16_shape(ctx->cfg) == WM_OK) {
    // pick the attention kernel's CTA plan for this batch by timing the candidates
    const wm_config& c = ctx->cfg;
    WM_CUDA(cudaMemset(ctx->h_qkv, 0, M * 3 * C * 2));
    WM_TRY(wm::autotune_na_bf16(ctx->h_qkv, ctx->h_o, batch, c.D, c.H, c.W, c.C, c.heads, c.kd, c.kh, c.kw,
                                c.lon_periodic != 0, 0, nullptr));
    WM_CUDA(cudaDeviceSynchronize());
  }
  if (!fp32 && ctx->cfg.C % 8 == 0) {
    if (!wm::make_tmap_bf16(&ctx->tm_u, ctx->h_u, M, C, 128) || !wm::make_tmap_bf16(&ctx->tm_o, ctx->h_o, M, C, 128) ||
        !wm::make_tmap_bf16(&ctx->tm_h, ctx->h_h, M, 4 * C, 128) ||
        !wm::make_tmap_out(&ctx->tmc_qkv, ctx->h_qkv, M, 3 * C, false) ||
        !wm::make_tmap_out(&ctx->tmc_h, ctx->h_h, M, 4 * C, false))
      return fail(WM_ERR_CUDA, "cuTensorMapEncodeTiled failed for the workspace");
    if (check_bf16_shape(ctx->cfg) == WM_OK) WM_TRY(tune_block_gemms(ctx, batch));
  }
  return WM_OK;
}

wm_status ensure_workspace(wm_ctx* ctx, int batch) {
  return ensure_workspace(ctx, batch, ctx->cfg.precision == WM_PREC_FP32);
}

wm_status ensure_buffer(float** p, size_t* cap, size_t floats) {
  if (floats <= *cap) return WM_OK;
  cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  if (cudaMalloc(p, floats * 4) != cudaSuccess) {
    cudaGetLastError();
    return fail(WM_ERR_OOM, "staging allocation failed");
  }
  *cap = floats;
  return WM_OK;
}

int pick_bn(long M, int N) {
  // wide tiles only when they still fill every SM at least once
  if (N % 256 == 0 && ((M + 127) / 128) * (N / 256) >= wm::num_sms()) return 256;
  return 128;
}

// ---- GEMM tile autotuner
// Tile width BN (64, 128 or 256 output columns; 256 also as 256 x 256 tiles on
// CTA pairs) and, for the residual epilogue, one or two staging tiles,
// chosen per GEMM of the block by timing every candidate when a context's
// BF16 workspace is allocated. BN changes no
// output of the LayerNorm-folded and GELU epilogues (every element's K sum
// runs in the same order), so those are tuned per row count. The residual
// epilogue writes one LayerNorm partial per half tile, so its BN fixes how a
// row's statistics are split and merged: it is tuned once per (N, K,
// operand type) and kept for every batch size, so that batched results stay
// identical to single-latent results. Untuned shapes take pick_bn.
struct GemmPick {
  int bn = 0, dual = -1;
  bool pair = false;
  double ms = 0.0;
};
// Test hook (wm_gemm_tile_override): 0 = tuned plans, 1 = BN 128, 2 = BN 256, 3 = BN 256 on CTA pairs,
// 4 = BN 64.
std::atomic<int> g_gemm_override{0};
// wm_set_fused_mlp: 1 runs the C = 128 MLP as the fused kernel, 0 (default) as two GEMMs.
std::atomic<int> g_mlp_fused{0};
// 1: rollouts of eligible narrow latents run as one whole-rollout launch
// (k_rollout_small.cu); 0: one launch per GEMM / attention as for any shape.
std::atomic<int> g_fused_rollout{1};
using GemmKey = std::array<long, 5>;   // rows (-1 for the residual epilogue), N, K, epilogue, e4m3
std::mutex g_gemm_mu;
std::map<GemmKey, GemmPick> g_gemm_picks;
std::string g_gemm_log;

GemmKey gemm_key(long M, int N, int K, int epi, bool f8) {
  return GemmKey{epi == wm::EPI_RESID_LN ? -1L : M, (long)N, (long)K, (long)epi, f8 ? 1L : 0L};
}

GemmPick pick_gemm(long M, int N, int K, int epi, bool f8) {
  const int ov = g_gemm_override.load();
  if (ov != 0) {
    GemmPick g;
    g.bn = ov == 4 ? (N % 64 == 0 ? 64 : 128) : (ov == 1 || N % 256 != 0) ? 128 : 256;
    // the pair kernel carries the block's epilogues (not the FP8-MLP path's plain residual add)
    g.pair = ov == 3 && g.bn == 256 && epi != wm::EPI_RESID_F32;
    return g;
  }
  {
    std::lock_guard<std::mutex> lk(g_gemm_mu);
    auto it = g_gemm_picks.find(gemm_key(M, N, K, epi, f8));
    if (it != g_gemm_picks.end()) return it->second;
  }
  GemmPick g;
  g.bn = pick_bn(M, N);
  return g;
}

// Times the candidates of one GEMM (a: every field but bn / dual / tmB set;
// tmB[0], tmB[1]: the W map for BN = 128 and 256) and records the fastest.
wm_status tune_gemm(wm::GemmArgs a, const CUtensorMap (&tmB)[3], const char* name, cudaStream_t s) {
  const GemmKey key = gemm_key(a.M, a.N, a.K, a.epi, a.f8);
  {
    std::lock_guard<std::mutex> lk(g_gemm_mu);
    if (g_gemm_picks.count(key)) return WM_OK;   // residual epilogue: fixed at its first tuning
  }
  cudaEvent_t e0, e1;
  WM_CUDA(cudaEventCreate(&e0));
  WM_CUDA(cudaEventCreate(&e1));
  GemmPick best;
  best.ms = 1e30;
  wm_status st = WM_OK;
  for (int cand : {64, 128, 256, 512}) {   // 512: BN = 256 on CTA pairs
    const int bn = cand == 512 ? 256 : cand;
    const bool pair = cand == 512;
    if (a.epi == wm::EPI_RESID_LN && a.N % bn != 0) continue;
    if (pair && a.N % 256 != 0) continue;
    for (int dual : {0, 1}) {
      if (a.epi != wm::EPI_RESID_LN && dual == 1) continue;
      a.bn = bn;
      a.pair = pair;
      a.dual = a.epi == wm::EPI_RESID_LN ? dual : -1;
      a.tmB = tmB[bn == 64 ? 2 : (bn == 256 && !pair ? 1 : 0)];
      st = wm::launch_gemm_tc(a, s);
      if (st != WM_OK) break;
      cudaEventRecord(e0, s);
      for (int r = 0; r < 3 && st == WM_OK; ++r) st = wm::launch_gemm_tc(a, s);
      cudaEventRecord(e1, s);
      if (st != WM_OK) break;
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        st = fail(WM_ERR_CUDA, "GEMM autotune synchronisation failed");
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      char line[200];
      std::snprintf(line, sizeof line, "  candidate %s M=%d N=%d K=%d BN=%d%s staging=%s: %.4f ms\n", name, a.M, a.N,
                    a.K, bn, pair ? " pair" : "", a.epi == wm::EPI_RESID_LN ? (dual ? "two" : "one") : "-", ms / 3.0);
      {
        std::lock_guard<std::mutex> lk(g_gemm_mu);
        g_gemm_log += line;
      }
      if (ms / 3.0 < best.ms) {
        best.ms = ms / 3.0;
        best.bn = bn;
        best.pair = pair;
        best.dual = a.dual;
      }
    }
    if (st != WM_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != WM_OK) return st;
  if (best.bn) {
    std::lock_guard<std::mutex> lk(g_gemm_mu);
    g_gemm_picks[key] = best;
  }
  return WM_OK;
}

std::string describe_gemm_plans() {
  std::lock_guard<std::mutex> lk(g_gemm_mu);
  static const char* const names[] = {"store", "gelu", "resid", "store_f32", "gelu_e4m3", "resid_ln", "ln_store",
                                      "ln_gelu"};
  std::string out;
  for (const auto& kv : g_gemm_picks) {
    const GemmKey& k = kv.first;
    char line[200];
    std::snprintf(line, sizeof line, "gemm rows=%s N=%ld K=%ld epilogue=%s%s -> BN=%d%s staging=%s %.4f ms\n",
                  k[0] < 0 ? "any" : std::to_string(k[0]).c_str(), k[1], k[2], names[k[3]], k[4] ? " e4m3" : "",
                  kv.second.bn, kv.second.pair ? " pair" : "", kv.second.dual < 0 ? "-" : (kv.second.dual ? "two" : "one"),
                  kv.second.ms);
    out += line;
  }
  return out + g_gemm_log;
}

// Time the tile candidates of the block's GEMMs (QKV, output projection,
// FC1, FC2 and the e4m3 FC1 / FC2) at `batch` latents with the first
// six-hour block's weights, on the workspace and a scratch residual; the
// outputs are discarded.
wm_status tune_block_gemms(wm_ctx* ctx, int batch) {
  const wm_config& c = ctx->cfg;
  const BlockW& w = ctx->blk[0][0];
  const long M = (long)batch * ctx->N;
  const int C = c.C;
  float* xt = nullptr;
  if (cudaMalloc(&xt, (size_t)M * C * 4) != cudaSuccess) {
    cudaGetLastError();
    return fail(WM_ERR_OOM, "GEMM autotune scratch allocation failed");
  }
  wm_status st = WM_OK;
  auto chk = [&](wm_status x) { if (st == WM_OK) st = x; };
  const size_t np_max = 2 * ((C + 63) / 64);
  if (cudaMemset(xt, 0, (size_t)M * C * 4) != cudaSuccess ||
      cudaMemset(ctx->stats, 0, (size_t)M * np_max * 2 * 4) != cudaSuccess)
    st = fail(WM_ERR_CUDA, "GEMM autotune scratch clear failed");
  CUtensorMap tm_x;
  if (st == WM_OK && !wm::make_tmap_out(&tm_x, xt, (uint64_t)M, (uint64_t)C, true))
    st = fail(WM_ERR_CUDA, "cuTensorMapEncodeTiled failed for the autotune scratch");
  if (st == WM_OK) {
    wm::GemmArgs a;
    a.M = (int)M; a.K = C; a.N = 3 * C;
    a.tmA = ctx->tm_xb; a.tmC = ctx->tmc_qkv;
    a.bias = w.bb_qkv; a.colsum = w.cs_qkv; a.stats = ctx->stats; a.np = 1; a.eps = c.ln_eps;
    a.epi = wm::EPI_LNF_STORE;
    chk(tune_gemm(a, w.tm_fqkv, "qkv", 0));
    a = wm::GemmArgs();
    a.M = (int)M; a.K = C; a.N = C;
    a.tmA = ctx->tm_o; a.tmC = tm_x; a.tmC2 = ctx->tmc_xb;
    a.bias = w.bo; a.x = xt; a.stats = ctx->stats;
    a.epi = wm::EPI_RESID_LN;
    chk(tune_gemm(a, w.tm_o, "proj", 0));
    a = wm::GemmArgs();
    a.M = (int)M; a.K = C; a.N = 4 * C;
    a.tmA = ctx->tm_xb; a.tmC = ctx->tmc_h;
    a.bias = w.bb_1; a.colsum = w.cs_1; a.stats = ctx->stats; a.np = 1; a.eps = c.ln_eps;
    a.epi = wm::EPI_LNF_GELU;
    chk(tune_gemm(a, w.tm_f1, "fc1", 0));
    a = wm::GemmArgs();
    a.M = (int)M; a.K = 4 * C; a.N = C;
    a.tmA = ctx->tm_h; a.tmC = tm_x; a.tmC2 = ctx->tmc_xb;
    a.bias = w.b2; a.x = xt; a.stats = ctx->stats;
    a.epi = wm::EPI_RESID_LN;
    chk(tune_gemm(a, w.tm_2, "fc2", 0));
    if (C == 128 || C == 256 || C == 384 || C == 512 || C == 768 || C == 1024) {
      a = wm::GemmArgs();
      a.f8 = true;
      a.M = (int)M; a.K = C; a.N = 4 * C;
      a.tmA = ctx->tm_qu; a.tmC = ctx->tmc_qh;
      a.bias = w.b1; a.epi = wm::EPI_GELU_F8; a.alpha = w.s_u * w.s_w1; a.out_scale = 1.f / w.s_h;
      chk(tune_gemm(a, w.tm_q1, "fc1_e4m3", 0));
      a = wm::GemmArgs();
      a.f8 = true;
      a.M = (int)M; a.K = 4 * C; a.N = C;
      a.tmA = ctx->tm_qh; a.tmC = tm_x; a.tmC2 = ctx->tmc_xb;
      a.bias = w.b2; a.epi = wm::EPI_RESID_LN; a.alpha = w.s_h * w.s_w2; a.x = xt; a.stats = ctx->stats;
      chk(tune_gemm(a, w.tm_q2, "fc2_e4m3", 0));
    }
  }
  const cudaError_t e = cudaDeviceSynchronize();
  if (st == WM_OK && e != cudaSuccess) st = wm::cuda_fail(e, "GEMM autotune");
  cudaFree(xt);
  return st;
}

void set_tile(wm::GemmArgs& a, long M, int epi, bool f8) {
  const GemmPick g = pick_gemm(M, a.N, a.K, epi, f8);
  a.bn = g.bn;
  a.pair = g.pair;
  a.dual = g.dual;
}

// Which of a weight's W maps the tile reads: boxes of 256 rows for single-CTA
// BN = 256 tiles, of 128 rows for BN = 128 and for each CTA of a pair, of 64
// rows for BN = 64.
int wmap(const wm::GemmArgs& a) { return a.bn == 64 ? 2 : (a.bn == 256 && !a.pair ? 1 : 0); }

// ---- optional per-launch timing: an event pair around each hot-path kernel
const char* const kKernelNames[WM_KERNEL_KINDS] = {"ln1", "qkv", "attention", "proj", "ln2", "fc1", "fc2"};

// Also an NVTX range named for the kernel kind.
struct TimedLaunch {
  wm_ctx* ctx;
  cudaStream_t s;
  int idx = -1;
  wm::NvtxRange range;
  TimedLaunch(wm_ctx* c, int kind, cudaStream_t st) : ctx(c), s(st), range(kKernelNames[kind]) {
    if (!ctx->timing) return;
    const size_t i = ctx->ev_marks.size() * 2;
    if (i + 2 > ctx->ev_pool.size()) return;
    if (cudaEventRecord(ctx->ev_pool[i], s) != cudaSuccess) return;
    idx = (int)i;
    ctx->ev_marks.push_back({kind, idx});
  }
  ~TimedLaunch() {
    if (idx >= 0) cudaEventRecord(ctx->ev_pool[idx + 1], s);
  }
};

wm_status block_forward(wm_ctx* ctx, float* x, int batch, int which, int b, bool first, cudaStream_t s) {
  char range_name[32];
  std::snprintf(range_name, sizeof range_name, "%s block %d", which == WM_P6 ? "P6" : "P1", b);
  wm::NvtxRange range(range_name);
  const wm_config& c = ctx->cfg;
  const BlockW& w = ctx->blk[which][b];
  const long M = (long)batch * ctx->N;
  const int C = c.C;
  const bool per = c.lon_periodic != 0;
  if (c.precision == WM_PREC_FP32) {
    { TimedLaunch t(ctx, WM_K_LN1, s);
      WM_TRY(wm::launch_layernorm(x, w.ln1_g, w.ln1_b, ctx->f_u, false, (int)M, C, c.ln_eps, s)); }
    { TimedLaunch t(ctx, WM_K_QKV, s);
      WM_TRY(wm::launch_sgemm(ctx->f_u, w.wqkv, w.bqkv, ctx->f_qkv, (int)M, 3 * C, C, wm::EPI_STORE_F32, s));
      if (c.rope) WM_TRY(wm::launch_rope_f32(ctx->f_qkv, M, ctx->d_rope, ctx->rope_host, s)); }
    { TimedLaunch t(ctx, WM_K_ATTN, s);
      WM_TRY(wm::launch_na_f32(ctx->f_qkv, ctx->f_o, batch, c.D, c.H, c.W, C, c.heads, c.kd, c.kh, c.kw, per, s)); }
    { TimedLaunch t(ctx, WM_K_PROJ, s);
      WM_TRY(wm::launch_sgemm(ctx->f_o, w.wo, w.bo, x, (int)M, C, C, wm::EPI_RESID_F32, s)); }
    { TimedLaunch t(ctx, WM_K_LN2, s);
      WM_TRY(wm::launch_layernorm(x, w.ln2_g, w.ln2_b, ctx->f_u, false, (int)M, C, c.ln_eps, s)); }
    { TimedLaunch t(ctx, WM_K_FC1, s);
      WM_TRY(wm::launch_sgemm(ctx->f_u, w.w1, w.b1, ctx->f_h, (int)M, 4 * C, C, wm::EPI_GELU, s)); }
    { TimedLaunch t(ctx, WM_K_FC2, s);
      WM_TRY(wm::launch_sgemm(ctx->f_h, w.w2, w.b2, x, (int)M, C, 4 * C, wm::EPI_RESID_F32, s)); }
    return WM_OK;
  }
  CUtensorMap tm_x;   // the caller's latent as the residual target
  if (!wm::make_tmap_out(&tm_x, x, (uint64_t)M, (uint64_t)C, true))
    return fail(WM_ERR_INVALID_ARG, "latent pointer must be 16-byte aligned for the BF16 path");
  const bool fp8 = c.precision == WM_PREC_BF16_FP8MLP;
  // small problems: let each kernel's prologue overlap its predecessor's tail
  const bool pdl = M <= wm::kPdlMaxTokens;
  // LayerNorm 1, folded into the QKV GEMM. Its row statistics come from the
  // previous block's FC2 epilogue, or from one statistics pass for the first
  // block of a processor call.
  if (first) {
    TimedLaunch t(ctx, WM_K_LN1, s);
    WM_TRY(wm::launch_row_stats(x, ctx->xb, ctx->stats, (int)M, C, s, pdl));
    ctx->np_next = 1;
  }
  wm::GemmArgs a;
  a.M = (int)M;
  a.K = C;
  a.N = 3 * C;
  set_tile(a, M, wm::EPI_LNF_STORE, false);
  a.tmA = ctx->tm_xb; a.tmB = w.tm_fqkv[wmap(a)]; a.tmC = ctx->tmc_qkv;
  a.bias = w.bb_qkv; a.colsum = w.cs_qkv; a.stats = ctx->stats; a.np = ctx->np_next; a.eps = c.ln_eps;
  a.epi = wm::EPI_LNF_STORE;
  a.rope = c.rope ? ctx->d_rope : nullptr;
  { TimedLaunch t(ctx, WM_K_QKV, s); a.pdl = pdl; WM_TRY(wm::launch_gemm_tc(a, s)); }
  { TimedLaunch t(ctx, WM_K_ATTN, s);
    WM_TRY(wm::launch_na_bf16(ctx->h_qkv, ctx->h_o, batch, c.D, c.H, c.W, C, c.heads, c.kd, c.kh, c.kw, per, s,
                              0, pdl)); }
  // output projection + residual; in BF16 it also leaves LayerNorm 2's statistics
  a = wm::GemmArgs();
  a.M = (int)M; a.K = C; a.N = C;
  set_tile(a, M, fp8 ? wm::EPI_RESID_F32 : wm::EPI_RESID_LN, false);
  a.tmA = ctx->tm_o; a.tmB = w.tm_o[wmap(a)]; a.tmC = tm_x;
  a.bias = w.bo;
  if (fp8) {
    a.epi = wm::EPI_RESID_F32;
  } else {
    a.epi = wm::EPI_RESID_LN; a.tmC2 = ctx->tmc_xb; a.x = x; a.stats = ctx->stats;
  }
  { TimedLaunch t(ctx, WM_K_PROJ, s); a.pdl = pdl; WM_TRY(wm::launch_gemm_tc(a, s)); }
  const int np2 = 2 * ((C + a.bn - 1) / a.bn);
  if (fp8) {
    // MLP in e4m3 with static per-tensor scales: u2 / s_u and W1 / s_w1 into
    // FC1 (alpha = s_u s_w1), GELU output / s_h and W2 / s_w2 into FC2
    { TimedLaunch t(ctx, WM_K_LN2, s);
      WM_TRY(wm::launch_layernorm_e4m3(x, w.ln2_g, w.ln2_b, ctx->q_u, (int)M, C, c.ln_eps, 1.f / w.s_u, s,
                                       pdl)); }
    a = wm::GemmArgs();
    a.f8 = true;
    a.M = (int)M; a.K = C; a.N = 4 * C;
    set_tile(a, M, wm::EPI_GELU_F8, true);
    a.tmA = ctx->tm_qu; a.tmB = w.tm_q1[wmap(a)]; a.tmC = ctx->tmc_qh;
    a.bias = w.b1; a.epi = wm::EPI_GELU_F8; a.alpha = w.s_u * w.s_w1; a.out_scale = 1.f / w.s_h;
    { TimedLaunch t(ctx, WM_K_FC1, s); a.pdl = pdl; WM_TRY(wm::launch_gemm_tc(a, s)); }
    a = wm::GemmArgs();
    a.f8 = true;
    a.M = (int)M; a.K = 4 * C; a.N = C;
    set_tile(a, M, wm::EPI_RESID_LN, true);
    a.tmA = ctx->tm_qh; a.tmB = w.tm_q2[wmap(a)]; a.tmC = tm_x; a.tmC2 = ctx->tmc_xb;
    a.bias = w.b2; a.epi = wm::EPI_RESID_LN; a.alpha = w.s_h * w.s_w2; a.x = x; a.stats = ctx->stats;
    { TimedLaunch t(ctx, WM_K_FC2, s); a.pdl = pdl; WM_TRY(wm::launch_gemm_tc(a, s)); }
    ctx->np_next = 2 * ((C + a.bn - 1) / a.bn);
    return WM_OK;
  }
  if (C == 128 && g_mlp_fused.load() == 1) {
    // the small latent's MLP as one kernel (bit-identical to the two GEMMs below)
    wm::MlpArgs m;
    m.tmA = ctx->tm_xb; m.tmW1 = w.tm_f1[0]; m.tmW2 = w.tm_2[0];
    m.M = (int)M;
    m.colsum1 = w.cs_1; m.bias1 = w.bb_1; m.bias2 = w.b2;
    // the same LayerNorm partials as FC2 on the tiles the tuner keeps for it
    const int bn2 = pick_gemm(M, C, 4 * C, wm::EPI_RESID_LN, false).bn;
    m.stats_in = ctx->stats; m.stats_out = ctx->stats; m.np_in = np2; m.np_out = 2 * C / bn2; m.eps = c.ln_eps;
    m.x = x; m.xb = ctx->xb; m.pdl = pdl;
    { TimedLaunch t(ctx, WM_K_FC1, s); WM_TRY(wm::launch_mlp_small(m, s)); }
    ctx->np_next = m.np_out;
    return WM_OK;
  }
  // LayerNorm 2 folded into FC1 (+ GELU)
  a = wm::GemmArgs();
  a.M = (int)M; a.K = C; a.N = 4 * C;
  set_tile(a, M, wm::EPI_LNF_GELU, false);
  a.tmA = ctx->tm_xb; a.tmB = w.tm_f1[wmap(a)]; a.tmC = ctx->tmc_h;
  a.bias = w.bb_1; a.colsum = w.cs_1; a.stats = ctx->stats; a.np = np2; a.eps = c.ln_eps;
  a.epi = wm::EPI_LNF_GELU;
  { TimedLaunch t(ctx, WM_K_FC1, s); a.pdl = pdl; WM_TRY(wm::launch_gemm_tc(a, s)); }
  // FC2 + residual, leaving the next block's LayerNorm-1 statistics
  a = wm::GemmArgs();
  a.M = (int)M; a.K = 4 * C; a.N = C;
  set_tile(a, M, wm::EPI_RESID_LN, false);
  a.tmA = ctx->tm_h; a.tmB = w.tm_2[wmap(a)]; a.tmC = tm_x; a.tmC2 = ctx->tmc_xb;
  a.bias = w.b2; a.epi = wm::EPI_RESID_LN; a.x = x; a.stats = ctx->stats;
  { TimedLaunch t(ctx, WM_K_FC2, s); a.pdl = pdl; WM_TRY(wm::launch_gemm_tc(a, s)); }
  ctx->np_next = 2 * ((C + a.bn - 1) / a.bn);
  return WM_OK;
}

int rollout_small_group(const wm_ctx* ctx, int batch);
wm_status rollout_small(wm_ctx* ctx, float* const* x, const int* n6, const int* n1, int G, cudaStream_t s);

wm_status processor_step(wm_ctx* ctx, float* x, int batch, int which, cudaStream_t s) {
  wm::NvtxRange range(which == WM_P6 ? "six-hour step" : "one-hour step");
  const int G = rollout_small_group(ctx, batch);
  if (G > 0) {
    // narrow latent: the step's blocks as one whole-rollout launch per G latents
    const size_t lat = (size_t)ctx->N * ctx->cfg.C;
    for (int i0 = 0; i0 < batch; i0 += G) {
      const int g = std::min(G, batch - i0);
      std::vector<float*> xs(g);
      std::vector<int> a6(g, which == WM_P6 ? 1 : 0), a1(g, which == WM_P1 ? 1 : 0);
      for (int i = 0; i < g; ++i) xs[i] = x + (i0 + i) * lat;
      WM_TRY(rollout_small(ctx, xs.data(), a6.data(), a1.data(), g, s));
    }
    return WM_OK;
  }
  const int L = which == WM_P6 ? ctx->cfg.blocks_p6 : ctx->cfg.blocks_p1;
  for (int b = 0; b < L; ++b) WM_TRY(block_forward(ctx, x, batch, which, b, b == 0, s));
  return WM_OK;
}

wm_status check_compute(wm_ctx* ctx, const void* latent, int batch) {
  if (!ctx) return fail(WM_ERR_INVALID_ARG, "context is NULL");
  if (!latent) return fail(WM_ERR_INVALID_ARG, "latent is NULL");
  if (batch <= 0) return fail(WM_ERR_INVALID_ARG, "batch must be >= 1");
  if (ctx->cfg.precision != WM_PREC_FP32) WM_TRY(check_bf16_shape(ctx->cfg));
  if (ctx->cfg.precision == WM_PREC_BF16_FP8MLP) {
    const int C = ctx->cfg.C;
    if (C != 128 && C != 256 && C != 384 && C != 512 && C != 768 && C != 1024)
      return fail(WM_ERR_INVALID_ARG, "FP8 MLP precision needs C in {128, 256, 384, 512, 768, 1024}");
  }
  return WM_OK;
}

// Capture `body` on the context's capture stream once per key, then replay the
// cached graph on `stream`.
template <typename F>
wm_status run_graph(wm_ctx* ctx, const std::vector<uintptr_t>& key, cudaStream_t stream, F body) {
  if (ctx->timing) return body(stream);  // per-launch events need eager launches
  auto it = ctx->graphs.find(key);
  if (it == ctx->graphs.end()) {
    if ((int)ctx->graphs.size() >= kMaxGraphs) destroy_graphs(ctx);
    WM_CUDA(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    wm_status st = body(ctx->cap_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &g);
    if (st != WM_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return wm::cuda_fail(e, "cudaStreamEndCapture");
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return wm::cuda_fail(e, "cudaGraphInstantiate");
    it = ctx->graphs.emplace(key, ex).first;
  }
  WM_CUDA(cudaGraphLaunch(it->second, stream));
  return WM_OK;
}

// ---- whole-rollout kernel for narrow latents

// Patches of 8 x 16 tokens tile every level; the latitude halo of every patch
// row spans 8 to 12 rows (a warp's 8-row key rectangle fits in it).
bool rollout_small_shape(const wm_config& c) {
  if (c.precision != WM_PREC_BF16 || c.C != 128 || c.heads != 4 || !c.lon_periodic || c.rope) return false;
  if (c.H % 8 || c.W % 16 || c.W < 32 || c.kh > 5 || c.kw > 5 || c.kd > c.D) return false;
  const int rh = c.kh / 2;
  auto start = [&](int h) { return std::min(std::max(h - rh, 0), c.H - c.kh); };
  for (int h0 = 0; h0 < c.H; h0 += 8) {
    const int rows = start(h0 + 7) + c.kh - start(h0);
    if (rows < 8 || rows > 12) return false;
  }
  return true;
}

// G latents of this context in one launch: the shape above, room on the
// device for all their patches at once, and no per-launch timing requested.
bool rollout_small_fits(const wm_ctx* ctx, int G) {
  if (g_fused_rollout.load() == 0 || ctx->timing || !rollout_small_shape(ctx->cfg)) return false;
  if (G < 1 || G > wm::kRolloutSmallMaxLatents) return false;
  const int T = ctx->cfg.D * (ctx->cfg.H / 8) * (ctx->cfg.W / 16);
  return G * T <= wm::rollout_small_capacity();
}

// Latents per whole-rollout launch for `batch` latents of this context: the
// most that fit on the device at once (at most `batch`), 0 when the kernel
// does not apply.
int rollout_small_group(const wm_ctx* ctx, int batch) {
  if (batch < 1 || !rollout_small_fits(ctx, 1)) return 0;
  const int T = ctx->cfg.D * (ctx->cfg.H / 8) * (ctx->cfg.W / 16);
  return std::min({batch, wm::kRolloutSmallMaxLatents, wm::rollout_small_capacity() / T});
}

// Once per context: every block's weights as 12 swizzled bf16 chunks and the
// per-block table the kernel reads.
wm_status prepare_rollout_small(wm_ctx* ctx) {
  if (ctx->d_rs_blk) return WM_OK;
  const size_t C = 128, chunk = 128 * 128;
  const size_t nb = ctx->blk[0].size() + ctx->blk[1].size();
  const size_t per = wm::kRolloutBlockBytes / sizeof(bf16);
  WM_CUDA(cudaMalloc(&ctx->d_rs_w, nb * wm::kRolloutBlockBytes));
  std::vector<wm::RolloutBlock> tab;
  for (int which = 0; which < 2; ++which)
    for (const BlockW& w : ctx->blk[which]) {
      bf16* out = ctx->d_rs_w + tab.size() * per;
      for (size_t c = 0; c < 3; ++c) WM_TRY(wm::launch_swizzle_chunk(w.wqkv + 128 * c * C, (int)C, out + c * chunk, 0));
      WM_TRY(wm::launch_swizzle_chunk(w.wo, (int)C, out + 3 * chunk, 0));
      for (size_t j = 0; j < 4; ++j) WM_TRY(wm::launch_swizzle_chunk(w.w1 + 128 * j * C, (int)C, out + (4 + j) * chunk, 0));
      for (size_t j = 0; j < 4; ++j) WM_TRY(wm::launch_swizzle_chunk(w.w2 + 128 * j, (int)(4 * C), out + (8 + j) * chunk, 0));
      // the vectors, fp32, after the chunks
      float* vec = reinterpret_cast<float*>(out + 12 * chunk);
      const std::pair<const float*, size_t> parts[8] = {{w.bqkv, 3 * C}, {w.bo, C},     {w.ln1_g, C}, {w.ln1_b, C},
                                                        {w.ln2_g, C},    {w.ln2_b, C}, {w.b1, 4 * C}, {w.b2, C}};
      for (const auto& pv : parts) {
        WM_CUDA(cudaMemcpy(vec, pv.first, pv.second * sizeof(float), cudaMemcpyDeviceToDevice));
        vec += pv.second;
      }
      tab.push_back({out});
    }
  WM_CUDA(cudaMalloc(&ctx->d_rs_blk, tab.size() * sizeof(wm::RolloutBlock)));
  WM_CUDA(cudaMemcpy(ctx->d_rs_blk, tab.data(), tab.size() * sizeof(wm::RolloutBlock), cudaMemcpyHostToDevice));
  WM_CUDA(cudaMalloc(&ctx->d_rs_bar, wm::kRolloutSmallMaxLatents * sizeof(unsigned int)));
  WM_CUDA(cudaDeviceSynchronize());
  return WM_OK;
}

// Weights and workspace for launches of up to the group size of `batch`
// latents, before a graph capture that may contain such launches.
wm_status rollout_small_reserve(wm_ctx* ctx, int batch) {
  const int G = rollout_small_group(ctx, batch);
  if (G == 0) return WM_OK;
  WM_TRY(prepare_rollout_small(ctx));
  return ensure_buffer(&ctx->d_rs_qkv, &ctx->rs_qkv_cap, (size_t)G * ctx->N * 384);
}

// Latents x[0..G) advance n6[i] six-hour then n1[i] one-hour steps (each at
// least one block) in one launch; rollout_small_fits(ctx, G) must hold.
wm_status rollout_small(wm_ctx* ctx, float* const* x, const int* n6, const int* n1, int G, cudaStream_t s) {
  const wm_config& c = ctx->cfg;
  const size_t qkv_floats = (size_t)G * ctx->N * 384;   // 2 x G x N x 384 bf16
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  WM_CUDA(cudaStreamIsCapturing(s, &cap));
  if (cap != cudaStreamCaptureStatusNone) {
    // inside a graph capture nothing may be allocated: rollout_small_reserve ran before
    if (!ctx->d_rs_blk || qkv_floats > ctx->rs_qkv_cap)
      return fail(WM_ERR_INVALID_ARG, "whole-rollout kernel captured without its workspace reserved");
  } else {
    WM_TRY(prepare_rollout_small(ctx));
    WM_TRY(ensure_buffer(&ctx->d_rs_qkv, &ctx->rs_qkv_cap, qkv_floats));
  }
  wm::RolloutSmallArgs a{};
  a.blk = ctx->d_rs_blk;
  a.L6 = c.blocks_p6;
  a.L1 = c.blocks_p1;
  a.G = G;
  a.T = c.D * (c.H / 8) * (c.W / 16);
  a.D = c.D; a.H = c.H; a.W = c.W; a.kd = c.kd; a.kh = c.kh; a.kw = c.kw;
  for (int i = 0; i < G; ++i) {
    a.x[i] = x[i];
    a.n6[i] = n6[i];
    a.n1[i] = n1[i];
  }
  a.qkv = reinterpret_cast<bf16*>(ctx->d_rs_qkv);
  const uint32_t box_w[3] = {20, 18, 2};
  for (int k = 0; k < 3; ++k)
    if (!wm::make_tmap_kv_slab(&a.tm_kv[k], a.qkv, 384, (uint64_t)c.W, (uint64_t)c.H, 2ull * G * c.D, box_w[k], 12))
      return fail(WM_ERR_CUDA, "cuTensorMapEncodeTiled failed for the whole-rollout K/V rows");
  a.bar = ctx->d_rs_bar;
  a.status = wm::device_status_word();
  a.eps = c.ln_eps;
  a.scale_log2 = (float)(1.4426950408889634 / std::sqrt(32.0));
  WM_CUDA(cudaMemsetAsync(ctx->d_rs_bar, 0, G * sizeof(unsigned int), s));
  wm::NvtxRange range("whole rollout (narrow latent)");
  return wm::launch_rollout_small(a, s);
}

}  // namespace

namespace wm {
bool processor_step_inplace_ok(wm_ctx* ctx, int n) {
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  return n >= 1 && rollout_small_group(ctx, n) >= 1;
}

// One processor step on n latents at arbitrary device addresses (the
// server's slots), read and written in place by whole-rollout launches of as
// many latents as the device holds at once.
wm_status processor_step_inplace(wm_ctx* ctx, float* const* xs, int n, int which, cudaStream_t s) {
  if (which != WM_P6 && which != WM_P1) return fail(WM_ERR_INVALID_ARG, "which must be WM_P6 or WM_P1");
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  const int G = rollout_small_group(ctx, n);
  if (G < 1) return fail(WM_ERR_INVALID_ARG, "the whole-rollout kernel does not take this step");
  for (int i0 = 0; i0 < n; i0 += G) {
    const int g = std::min(G, n - i0);
    std::vector<int> a6(g, which == WM_P6 ? 1 : 0), a1(g, which == WM_P1 ? 1 : 0);
    WM_TRY(rollout_small(ctx, xs + i0, a6.data(), a1.data(), g, s));
  }
  return WM_OK;
}

// One processor step on `batch` contiguous latents, replayed from a CUDA
// graph captured once per (latent buffer, batch, processor, precision): the
// server's ticks launch one graph instead of every kernel of the step.
wm_status processor_step_graphed(wm_ctx* ctx, float* x, int batch, int which, cudaStream_t s) {
  WM_TRY(check_compute(ctx, x, batch));
  if (which != WM_P6 && which != WM_P1) return fail(WM_ERR_INVALID_ARG, "which must be WM_P6 or WM_P1");
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  WM_TRY(ensure_workspace(ctx, batch));
  WM_TRY(rollout_small_reserve(ctx, batch));
  const std::vector<uintptr_t> key = {4, (uintptr_t)x, (uintptr_t)batch, (uintptr_t)which,
                                      (uintptr_t)ctx->cfg.precision};
  return run_graph(ctx, key, s, [&](cudaStream_t st) -> wm_status { return processor_step(ctx, x, batch, which, st); });
}
}  // namespace wm

namespace {

// Rotary embedding tables: pair m of an axis at position pos has angle
// pos * w_m (w_m = 10000^(-m/n) for level and latitude, 2 pi (m + 1) / W for
// longitude); stored as (cos, sin) computed in double.
wm_status build_rope(wm_ctx* ctx) {
  const wm_config& c = ctx->cfg;
  const int dh = c.C / c.heads, P = dh / 2;
  const int n_lon = (P + 2) / 3;
  const int n_lat = (P - n_lon + 1) / 2;
  const int n_lev = P - n_lon - n_lat;
  const int npos[3] = {c.D, c.H, c.W};
  const int npair[3] = {n_lev, n_lat, n_lon};
  std::vector<float2> tab;
  size_t off[3];
  for (int ax = 0; ax < 3; ++ax) {
    off[ax] = tab.size();
    for (int pos = 0; pos < npos[ax]; ++pos)
      for (int m = 0; m < npair[ax]; ++m) {
        const double w = ax < 2 ? std::pow(10000.0, -(double)m / npair[ax]) : 2.0 * M_PI * (m + 1) / c.W;
        const double a = pos * w;
        tab.push_back(make_float2((float)std::cos(a), (float)std::sin(a)));
      }
  }
  WM_CUDA(cudaMalloc(&ctx->d_rope_tab, tab.size() * sizeof(float2)));
  WM_CUDA(cudaMemcpy(ctx->d_rope_tab, tab.data(), tab.size() * sizeof(float2), cudaMemcpyHostToDevice));
  wm::RopeArgs& R = ctx->rope_host;
  for (int ax = 0; ax < 3; ++ax) {
    R.tab[ax] = ctx->d_rope_tab + off[ax];
    R.n[ax] = npair[ax];
  }
  R.D = c.D; R.H = c.H; R.W = c.W; R.C = c.C; R.dh = dh;
  WM_CUDA(cudaMalloc(&ctx->d_rope, sizeof(wm::RopeArgs)));
  WM_CUDA(cudaMemcpy(ctx->d_rope, &R, sizeof(wm::RopeArgs), cudaMemcpyHostToDevice));
  return WM_OK;
}

// IEEE round-to-nearest-even of a float to bfloat16 (bit pattern).
uint16_t bf16_bits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((u >> 16) | 0x40u);
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
float bf16_value(uint16_t b) {
  const uint32_t u = (uint32_t)b << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

// LayerNorm folded into a linear layer W [N, C] with bias b:
//   LN(x) W^T + b = rstd (x W'^T - mean colsum(W')) + (b + W beta),  W' = W diag(gamma).
// Writes bf16(W') and, from those rounded values, colsum; and b + W beta.
void fold_layernorm(const float* W, const float* b, const float* gamma, const float* beta, size_t N, size_t C,
                    uint16_t* wf, float* colsum, float* bias) {
  for (size_t n = 0; n < N; ++n) {
    double cs = 0.0, bb = b[n];
    for (size_t k = 0; k < C; ++k) {
      const uint16_t q = bf16_bits(W[n * C + k] * gamma[k]);
      wf[n * C + k] = q;
      cs += bf16_value(q);
      bb += (double)W[n * C + k] * beta[k];
    }
    colsum[n] = (float)cs;
    bias[n] = (float)bb;
  }
}

wm_status upload_weights(wm_ctx* ctx, const float* host, size_t n) {
  const wm_config& c = ctx->cfg;
  const int nb = c.blocks_p6 + c.blocks_p1;
  const size_t per = block_floats(c.C);
  if (n != per * nb)
    return fail(WM_ERR_INVALID_ARG, "weight count " + std::to_string(n) + " != expected " + std::to_string(per * nb));
  WM_CUDA(cudaMalloc(&ctx->d_w32, n * 4));
  WM_CUDA(cudaMemcpy(ctx->d_w32, host, n * 4, cudaMemcpyHostToDevice));
  const size_t C = c.C;
  const size_t mats = 5 * C * C;   // bf16 wo + w2 per block
  WM_CUDA(cudaMalloc(&ctx->d_wh, mats * nb * 2));
  WM_CUDA(cudaMalloc(&ctx->d_wq, 8 * C * C * nb));
  WM_CUDA(cudaMalloc(&ctx->d_wf, 7 * C * C * nb * 2));
  WM_CUDA(cudaMalloc(&ctx->d_vf, 14 * C * nb * 4));
  std::vector<uint16_t> hf(7 * C * C);
  std::vector<float> hv(14 * C);
  for (int i = 0; i < nb; ++i) {
    const int which = i < c.blocks_p6 ? 0 : 1;
    const float* p = ctx->d_w32 + per * i;
    BlockW w{};
    w.ln1_g = p; p += C;
    w.ln1_b = p; p += C;
    w.wqkv = p; p += 3 * C * C;
    w.bqkv = p; p += 3 * C;
    w.wo = p; p += C * C;
    w.bo = p; p += C;
    w.ln2_g = p; p += C;
    w.ln2_b = p; p += C;
    w.w1 = p; p += 4 * C * C;
    w.b1 = p; p += 4 * C;
    w.w2 = p; p += 4 * C * C;
    w.b2 = p; p += C;
    bf16* h = ctx->d_wh + mats * i;
    w.ho = h; h += C * C;
    w.h2 = h;
    WM_TRY(wm::launch_f32_to_bf16(w.wo, w.ho, C * C, 0));
    WM_TRY(wm::launch_f32_to_bf16(w.w2, w.h2, 4 * C * C, 0));
    // ---- FP8 MLP: static per-tensor scales from bounds that hold for every input
    {
      const float* hp = host + per * i;
      const float* g2 = hp + 6 * C + 4 * C * C;   // ln1_g ln1_b wqkv bqkv wo bo precede ln2_g
      const float* b2v = g2 + C;
      const float* hw1 = b2v + C;
      const float* hb1 = hw1 + 4 * C * C;
      const float* hw2 = hb1 + 4 * C;
      // |LN2(x)_c| <= |gamma_c| sqrt(C - 1) + |beta_c|  (|x_c - mean| <= sqrt(C-1) * biased std)
      std::vector<double> bu(C);
      double bu_max = 0.0;
      for (size_t c2 = 0; c2 < C; ++c2) {
        bu[c2] = std::fabs((double)g2[c2]) * std::sqrt((double)C - 1.0) + std::fabs((double)b2v[c2]);
        bu_max = std::max(bu_max, bu[c2]);
      }
      double aw1 = 0.0, aw2 = 0.0, bz = 0.0;
      for (size_t j = 0; j < 4 * C; ++j) {
        double z = std::fabs((double)hb1[j]);
        for (size_t c2 = 0; c2 < C; ++c2) {
          const double a = std::fabs((double)hw1[j * C + c2]);
          aw1 = std::max(aw1, a);
          z += a * bu[c2];
        }
        bz = std::max(bz, z);
      }
      for (size_t j = 0; j < 4 * C * C; ++j) aw2 = std::max(aw2, std::fabs((double)hw2[j]));
      // |GELU(z)| <= max(|z|, 0.17): the GELU minimum is -0.16997 at z = -0.7518
      const double bh = std::max(bz, 0.17);
      w.s_u = (float)(std::max(bu_max, 1e-30) / 448.0);
      w.s_w1 = (float)(std::max(aw1, 1e-30) / 448.0);
      w.s_h = (float)(bh / 448.0);
      w.s_w2 = (float)(std::max(aw2, 1e-30) / 448.0);
    }
    {
      const float* hp = host + per * i;
      const float* g1 = hp;
      const float* be1 = hp + C;
      const float* hqkv = hp + 2 * C;
      const float* hbqkv = hqkv + 3 * C * C;
      const float* g2 = hp + 6 * C + 4 * C * C;
      const float* be2 = g2 + C;
      const float* hw1 = be2 + C;
      const float* hb1 = hw1 + 4 * C * C;
      fold_layernorm(hqkv, hbqkv, g1, be1, 3 * C, C, hf.data(), hv.data(), hv.data() + 3 * C);
      fold_layernorm(hw1, hb1, g2, be2, 4 * C, C, hf.data() + 3 * C * C, hv.data() + 6 * C, hv.data() + 10 * C);
      w.fqkv = ctx->d_wf + 7 * C * C * i;
      w.f1 = w.fqkv + 3 * C * C;
      float* v = ctx->d_vf + 14 * C * i;
      w.cs_qkv = v;
      w.bb_qkv = v + 3 * C;
      w.cs_1 = v + 6 * C;
      w.bb_1 = v + 10 * C;
      WM_CUDA(cudaMemcpy(w.fqkv, hf.data(), 7 * C * C * 2, cudaMemcpyHostToDevice));
      WM_CUDA(cudaMemcpy(v, hv.data(), 14 * C * 4, cudaMemcpyHostToDevice));
      if (C % 8 == 0) {
        bool ok = true;
        for (int k = 0; k < 3; ++k) {
          const uint32_t box = k == 0 ? 128 : (k == 1 ? 256 : 64);
          ok = ok && wm::make_tmap_bf16(&w.tm_fqkv[k], w.fqkv, 3 * C, C, box);
          ok = ok && wm::make_tmap_bf16(&w.tm_f1[k], w.f1, 4 * C, C, box);
        }
        if (!ok) return fail(WM_ERR_CUDA, "cuTensorMapEncodeTiled failed for the folded weights");
      }
    }
    w.q1 = ctx->d_wq + 8 * C * C * i;
    w.q2 = w.q1 + 4 * C * C;
    WM_TRY(wm::launch_f32_to_e4m3(w.w1, w.q1, 4 * C * C, 1.f / w.s_w1, 0));
    WM_TRY(wm::launch_f32_to_e4m3(w.w2, w.q2, 4 * C * C, 1.f / w.s_w2, 0));
    if (C % 16 == 0) {
      bool ok = true;
      for (int k = 0; k < 3; ++k) {
        const uint32_t box = k == 0 ? 128 : (k == 1 ? 256 : 64);
        ok = ok && wm::make_tmap_e4m3(&w.tm_q1[k], w.q1, 4 * C, C, box);
        ok = ok && wm::make_tmap_e4m3(&w.tm_q2[k], w.q2, C, 4 * C, box);
      }
      if (!ok) return fail(WM_ERR_CUDA, "cuTensorMapEncodeTiled failed for the e4m3 weights");
    }
    if (C % 8 == 0) {
      bool ok = true;
      for (int k = 0; k < 3; ++k) {
        const uint32_t box = k == 0 ? 128 : (k == 1 ? 256 : 64);
        ok = ok && wm::make_tmap_bf16(&w.tm_o[k], w.ho, C, C, box);
        ok = ok && wm::make_tmap_bf16(&w.tm_2[k], w.h2, C, 4 * C, box);
      }
      if (!ok) return fail(WM_ERR_CUDA, "cuTensorMapEncodeTiled failed for the weights");
    }
    ctx->blk[which].push_back(w);
  }
  WM_CUDA(cudaDeviceSynchronize());
  return WM_OK;
}

}  // namespace

namespace wm {
const wm_config* ctx_config(const wm_ctx* ctx) { return &ctx->cfg; }
}  // namespace wm

// =================================================================== C ABI ===
extern "C" {

const char* wm_last_error(void) { return wm::last_error_cstr(); }

wm_status wm_schedule(int lead_hours, int* n6, int* n1) {
  if (lead_hours < 0) return fail(WM_ERR_INVALID_ARG, "lead time must be >= 0");
  if (!n6 || !n1) return fail(WM_ERR_INVALID_ARG, "output pointers are NULL");
  *n6 = lead_hours / 6;
  *n1 = lead_hours % 6;
  return WM_OK;
}

wm_status wm_create_from_host(const wm_config* cfg, const float* weights, size_t n_floats, wm_ctx** out) {
  if (!out) return fail(WM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  WM_TRY(validate(cfg));
  if (!weights) return fail(WM_ERR_INVALID_ARG, "weights are NULL");
  WM_TRY(wm::prepare_kernels());
  wm_ctx* ctx = new wm_ctx();
  ctx->cfg = *cfg;
  if (ctx->cfg.max_batch < 1) ctx->cfg.max_batch = 1;
  cudaGetDevice(&ctx->device);
  ctx->N = (long)cfg->D * cfg->H * cfg->W;
  wm_status st = upload_weights(ctx, weights, n_floats);
  if (st == WM_OK && cfg->rope) st = build_rope(ctx);
  if (st == WM_OK) st = ensure_workspace(ctx, ctx->cfg.max_batch);
  if (st == WM_OK && cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    st = fail(WM_ERR_CUDA, "cudaStreamCreate failed");
  if (st == WM_OK && !wm::device_status_word()) st = fail(WM_ERR_OOM, "device status word allocation failed");
  if (st != WM_OK) {
    wm_destroy(ctx);
    return st;
  }
  *out = ctx;
  return WM_OK;
}

wm_status wm_create(const wm_config* cfg, const char* weights_path, wm_ctx** out) {
  if (!out) return fail(WM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  WM_TRY(validate(cfg));
  if (!weights_path) return fail(WM_ERR_INVALID_ARG, "weights_path is NULL");
  FILE* f = std::fopen(weights_path, "rb");
  if (!f) return fail(WM_ERR_IO, std::string("cannot open ") + weights_path);
  char magic[8];
  int32_t hdr[4];
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "WM3WGT1\0", 8) == 0 &&
            std::fread(hdr, 4, 4, f) == 4;
  if (!ok || hdr[0] != cfg->C || hdr[1] != cfg->blocks_p6 || hdr[2] != cfg->blocks_p1) {
    std::fclose(f);
    return fail(WM_ERR_IO, "weight file header does not match the config");
  }
  const size_t n = block_floats(cfg->C) * (cfg->blocks_p6 + cfg->blocks_p1);
  std::vector<float> buf(n);
  const size_t got = std::fread(buf.data(), 4, n, f);
  std::fclose(f);
  if (got != n) return fail(WM_ERR_IO, "weight file is short");
  return wm_create_from_host(cfg, buf.data(), n, out);
}

wm_status wm_destroy(wm_ctx* ctx) {
  if (!ctx) return WM_OK;
  cudaDeviceSynchronize();
  destroy_graphs(ctx);
  free_workspace(ctx);
  cudaFree(ctx->d_w32);
  cudaFree(ctx->d_wh);
  cudaFree(ctx->d_wq);
  cudaFree(ctx->d_wf);
  cudaFree(ctx->d_vf);
  cudaFree(ctx->d_rope_tab);
  cudaFree(ctx->d_rope);
  cudaFree(ctx->d_rs_w);
  cudaFree(ctx->d_rs_blk);
  cudaFree(ctx->d_rs_qkv);
  cudaFree(ctx->d_rs_bar);
  cudaFree(ctx->d_stage);
  cudaFree(ctx->d_io);
  for (float* p : ctx->d_ring) cudaFree(p);
  if (ctx->up_stream) cudaStreamDestroy(ctx->up_stream);
  if (ctx->down_stream) cudaStreamDestroy(ctx->down_stream);
  for (cudaEvent_t e : ctx->io_ev)
    if (e) cudaEventDestroy(e);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  delete ctx;
  return WM_OK;
}

wm_status wm_set_precision(wm_ctx* ctx, int precision) {
  if (!ctx) return fail(WM_ERR_INVALID_ARG, "context is NULL");
  if (precision < WM_PREC_FP32 || precision > WM_PREC_BF16_FP8MLP) return fail(WM_ERR_INVALID_ARG, "unknown precision");
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  ctx->cfg.precision = precision;
  return WM_OK;
}

wm_status wm_block_forward(wm_ctx* ctx, float* latent, int batch, int which, int block, void* stream) {
  WM_TRY(check_compute(ctx, latent, batch));
  if (which != WM_P6 && which != WM_P1) return fail(WM_ERR_INVALID_ARG, "which must be WM_P6 or WM_P1");
  if (block < 0 || block >= (int)ctx->blk[which].size()) return fail(WM_ERR_INVALID_ARG, "block index out of range");
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  WM_TRY(ensure_workspace(ctx, batch));
  return block_forward(ctx, latent, batch, which, block, true, (cudaStream_t)stream);
}

wm_status wm_processor_step(wm_ctx* ctx, float* latent, int batch, int which, void* stream) {
  WM_TRY(check_compute(ctx, latent, batch));
  if (which != WM_P6 && which != WM_P1) return fail(WM_ERR_INVALID_ARG, "which must be WM_P6 or WM_P1");
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  WM_TRY(ensure_workspace(ctx, batch));
  return processor_step(ctx, latent, batch, which, (cudaStream_t)stream);
}

wm_status wm_latent_rollout(wm_ctx* ctx, float* latent, int batch, int lead_hours, void* stream) {
  if (lead_hours < 0) return fail(WM_ERR_INVALID_ARG, "lead time must be >= 0");
  WM_TRY(check_compute(ctx, latent, batch));
  if (lead_hours == 0) return WM_OK;
  int n6 = 0, n1 = 0;
  wm_schedule(lead_hours, &n6, &n1);
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  const int G = rollout_small_group(ctx, batch);
  if (G > 0) {
    // narrow latent: whole rollouts in launches of G latents each
    const size_t lat = (size_t)ctx->N * ctx->cfg.C;
    for (int i0 = 0; i0 < batch; i0 += G) {
      const int g = std::min(G, batch - i0);
      std::vector<float*> xs(g);
      std::vector<int> a6(g, n6), a1(g, n1);
      for (int i = 0; i < g; ++i) xs[i] = latent + (i0 + i) * lat;
      WM_TRY(rollout_small(ctx, xs.data(), a6.data(), a1.data(), g, (cudaStream_t)stream));
    }
    return WM_OK;
  }
  WM_TRY(ensure_workspace(ctx, batch));
  std::vector<uintptr_t> key = {1, (uintptr_t)latent, (uintptr_t)batch, (uintptr_t)n6, (uintptr_t)n1,
                                (uintptr_t)ctx->cfg.precision};
  return run_graph(ctx, key, (cudaStream_t)stream, [&](cudaStream_t s) -> wm_status {
    for (int i = 0; i < n6; ++i) WM_TRY(processor_step(ctx, latent, batch, WM_P6, s));
    for (int i = 0; i < n1; ++i) WM_TRY(processor_step(ctx, latent, batch, WM_P1, s));
    return WM_OK;
  });
}

wm_status wm_forecast_host(wm_ctx* ctx, const float* host_in, float* host_out, int batch, int lead_hours,
                           void* stream) {
  if (!ctx || !host_in || !host_out) return fail(WM_ERR_INVALID_ARG, "NULL argument");
  if (batch <= 0) return fail(WM_ERR_INVALID_ARG, "batch must be >= 1");
  if (lead_hours < 0) return fail(WM_ERR_INVALID_ARG, "lead time must be >= 0");
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  const size_t floats = (size_t)batch * ctx->N * ctx->cfg.C;
  WM_TRY(ensure_buffer(&ctx->d_io, &ctx->io_cap, floats));
  cudaStream_t s = (cudaStream_t)stream;
  auto enqueue = [&]() -> wm_status {
    WM_CUDA(cudaMemcpyAsync(ctx->d_io, host_in, floats * 4, cudaMemcpyHostToDevice, s));
    WM_TRY(wm_latent_rollout(ctx, ctx->d_io, batch, lead_hours, stream));
    WM_CUDA(cudaMemcpyAsync(host_out, ctx->d_io, floats * 4, cudaMemcpyDeviceToHost, s));
    return WM_OK;
  };
  const wm_status st = enqueue();
  const cudaError_t e = cudaStreamSynchronize(s);   // the copies are done with the host buffers
  if (st != WM_OK) return st;
  if (e != cudaSuccess) return fail(WM_ERR_CUDA, cudaGetErrorString(e));
  return WM_OK;
}

wm_status wm_forecast_host_many(wm_ctx* ctx, const float* const* host_in, float* const* host_out, int n, int batch,
                                int lead_hours, void* stream) {
  if (!ctx || !host_in || !host_out || n < 0) return fail(WM_ERR_INVALID_ARG, "bad arguments");
  if (batch <= 0) return fail(WM_ERR_INVALID_ARG, "batch must be >= 1");
  if (lead_hours < 0) return fail(WM_ERR_INVALID_ARG, "lead time must be >= 0");
  for (int i = 0; i < n; ++i)
    if (!host_in[i] || !host_out[i]) return fail(WM_ERR_INVALID_ARG, "a host pointer is NULL");
  if (n == 0) return WM_OK;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  constexpr int R = 3;
  const size_t floats = (size_t)batch * ctx->N * ctx->cfg.C;
  for (int r = 0; r < R; ++r) WM_TRY(ensure_buffer(&ctx->d_ring[r], &ctx->ring_cap[r], floats));
  if (!ctx->up_stream) WM_CUDA(cudaStreamCreateWithFlags(&ctx->up_stream, cudaStreamNonBlocking));
  if (!ctx->down_stream) WM_CUDA(cudaStreamCreateWithFlags(&ctx->down_stream, cudaStreamNonBlocking));
  for (cudaEvent_t& e : ctx->io_ev)
    if (!e) WM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t* up = ctx->io_ev;          // forecast's input is on the device
  cudaEvent_t* comp = ctx->io_ev + R;    // forecast's rollout is done
  cudaEvent_t* down = ctx->io_ev + 2 * R;  // forecast's result has left its latent
  // nothing queued earlier on `stream` may still be using the ring
  WM_CUDA(cudaEventRecord(comp[0], s));
  WM_CUDA(cudaStreamWaitEvent(ctx->up_stream, comp[0], 0));
  // Forecast i uses latent i mod 3: its upload overlaps forecast i - 1's
  // rollout and needs only forecast i - 3's download to be done, so an upload
  // and a download may each take up to a whole rollout.
  auto upload = [&](int i) -> wm_status {
    const int b = i % R;
    if (i >= R) WM_CUDA(cudaStreamWaitEvent(ctx->up_stream, down[b], 0));
    WM_CUDA(cudaMemcpyAsync(ctx->d_ring[b], host_in[i], floats * 4, cudaMemcpyHostToDevice, ctx->up_stream));
    WM_CUDA(cudaEventRecord(up[b], ctx->up_stream));
    return WM_OK;
  };
  auto enqueue = [&]() -> wm_status {
    WM_TRY(upload(0));
    for (int i = 0; i < n; ++i) {
      const int b = i % R;
      if (i + 1 < n) WM_TRY(upload(i + 1));
      WM_CUDA(cudaStreamWaitEvent(s, up[b], 0));
      WM_TRY(wm_latent_rollout(ctx, ctx->d_ring[b], batch, lead_hours, stream));
      WM_CUDA(cudaEventRecord(comp[b], s));
      WM_CUDA(cudaStreamWaitEvent(ctx->down_stream, comp[b], 0));
      WM_CUDA(cudaMemcpyAsync(host_out[i], ctx->d_ring[b], floats * 4, cudaMemcpyDeviceToHost, ctx->down_stream));
      WM_CUDA(cudaEventRecord(down[b], ctx->down_stream));
    }
    return WM_OK;
  };
  const wm_status st = enqueue();
  // every copy has finished with the caller's host buffers before returning,
  // on the error path too
  const cudaError_t e1 = cudaStreamSynchronize(ctx->down_stream);
  const cudaError_t e2 = cudaStreamSynchronize(ctx->up_stream);
  const cudaError_t e3 = cudaStreamSynchronize(s);
  if (st != WM_OK) return st;
  for (cudaError_t e : {e1, e2, e3})
    if (e != cudaSuccess) return fail(WM_ERR_CUDA, cudaGetErrorString(e));
  return WM_OK;
}

wm_status wm_rollout_batch(wm_ctx* ctx, float* const* latents, const int* lead_hours, int n, void* stream) {
  if (!ctx || !latents || !lead_hours || n < 1) return fail(WM_ERR_INVALID_ARG, "bad batch arguments");
  for (int i = 0; i < n; ++i) {
    if (!latents[i]) return fail(WM_ERR_INVALID_ARG, "a latent pointer is NULL");
    if (lead_hours[i] < 0) return fail(WM_ERR_INVALID_ARG, "lead time must be >= 0");
  }
  WM_TRY(check_compute(ctx, latents[0], 1));
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  std::vector<int> n6(n), n1(n);
  int ticks = 0;
  for (int i = 0; i < n; ++i) {
    wm_schedule(lead_hours[i], &n6[i], &n1[i]);
    ticks = std::max(ticks, n6[i] + n1[i]);
  }
  if (ticks == 0) return WM_OK;
  const int G = rollout_small_group(ctx, n);
  if (G > 0) {
    // narrow latent: launches of up to G latents with their own schedules,
    // longest rollouts together, read and written in place (no gather)
    std::vector<int> order;
    for (int i = 0; i < n; ++i)
      if (n6[i] + n1[i] > 0) order.push_back(i);
    const int L6 = ctx->cfg.blocks_p6, L1 = ctx->cfg.blocks_p1;
    std::stable_sort(order.begin(), order.end(),
                     [&](int p, int q) { return n6[p] * L6 + n1[p] * L1 > n6[q] * L6 + n1[q] * L1; });
    for (size_t i0 = 0; i0 < order.size(); i0 += G) {
      const int g = (int)std::min(order.size() - i0, (size_t)G);
      std::vector<float*> xs(g);
      std::vector<int> a6(g), a1(g);
      for (int i = 0; i < g; ++i) {
        xs[i] = latents[order[i0 + i]];
        a6[i] = n6[order[i0 + i]];
        a1[i] = n1[order[i0 + i]];
      }
      WM_TRY(rollout_small(ctx, xs.data(), a6.data(), a1.data(), g, (cudaStream_t)stream));
    }
    return WM_OK;
  }
  WM_TRY(ensure_workspace(ctx, n));
  const size_t lat = (size_t)ctx->N * ctx->cfg.C;
  WM_TRY(ensure_buffer(&ctx->d_stage, &ctx->stage_cap, lat * n));
  std::vector<uintptr_t> key = {2, (uintptr_t)n, (uintptr_t)ctx->cfg.precision};
  for (int i = 0; i < n; ++i) {
    key.push_back((uintptr_t)latents[i]);
    key.push_back((uintptr_t)lead_hours[i]);
  }
  return run_graph(ctx, key, (cudaStream_t)stream, [&](cudaStream_t s) -> wm_status {
    std::vector<int> grp;
    for (int k = 0; k < ticks; ++k) {
      for (int which = 0; which < 2; ++which) {
        grp.clear();
        for (int i = 0; i < n; ++i) {
          const bool due = which == WM_P6 ? (k < n6[i]) : (k >= n6[i] && k < n6[i] + n1[i]);
          if (due) grp.push_back(i);
        }
        if (grp.empty()) continue;
        if (grp.size() == 1) {
          WM_TRY(processor_step(ctx, latents[grp[0]], 1, which, s));
          continue;
        }
        // gather the due latents into one contiguous batch, step, scatter back
        for (size_t j = 0; j < grp.size(); ++j)
          WM_CUDA(cudaMemcpyAsync(ctx->d_stage + j * lat, latents[grp[j]], lat * 4, cudaMemcpyDeviceToDevice, s));
        WM_TRY(processor_step(ctx, ctx->d_stage, (int)grp.size(), which, s));
        for (size_t j = 0; j < grp.size(); ++j)
          WM_CUDA(cudaMemcpyAsync(latents[grp[j]], ctx->d_stage + j * lat, lat * 4, cudaMemcpyDeviceToDevice, s));
      }
    }
    return WM_OK;
  });
}

wm_status wm_ctx_sizes(wm_ctx* ctx, int batch, size_t* latent_floats, size_t* workspace_bytes) {
  if (!ctx || batch < 1 || !latent_floats || !workspace_bytes) return fail(WM_ERR_INVALID_ARG, "bad size query");
  const size_t C = ctx->cfg.C, M = (size_t)batch * ctx->N;
  *latent_floats = (size_t)ctx->N * C;
  *workspace_bytes = M * C * 9 * (ctx->cfg.precision == WM_PREC_FP32 ? 4 : 2);
  return WM_OK;
}

wm_status wm_autotune_report(char* buf, size_t len) {
  if (!buf || len == 0) return fail(WM_ERR_INVALID_ARG, "bad report buffer");
  const std::string r = wm::describe_na_plans() + describe_gemm_plans();
  const size_t n = std::min(len - 1, r.size());
  std::memcpy(buf, r.data(), n);
  buf[n] = 0;
  return WM_OK;
}

wm_status wm_ctx_reserve(wm_ctx* ctx, int batch) {
  if (!ctx || batch < 1) return fail(WM_ERR_INVALID_ARG, "bad reserve arguments");
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  return ensure_workspace(ctx, batch);
}

wm_status wm_timing_begin(wm_ctx* ctx, int max_launches) {
  if (!ctx || max_launches < 1) return fail(WM_ERR_INVALID_ARG, "bad timing arguments");
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  const size_t want = 2 * (size_t)max_launches;
  while (ctx->ev_pool.size() < want) {
    cudaEvent_t e;
    WM_CUDA(cudaEventCreate(&e));
    ctx->ev_pool.push_back(e);
  }
  ctx->ev_marks.clear();
  ctx->timing = true;
  return WM_OK;
}

wm_status wm_timing_end(wm_ctx* ctx, double* ms_by_kind, int* launches_by_kind) {
  if (!ctx || !ms_by_kind || !launches_by_kind) return fail(WM_ERR_INVALID_ARG, "bad timing arguments");
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  ctx->timing = false;
  for (int k = 0; k < WM_KERNEL_KINDS; ++k) {
    ms_by_kind[k] = 0.0;
    launches_by_kind[k] = 0;
  }
  WM_CUDA(cudaDeviceSynchronize());
  for (const auto& m : ctx->ev_marks) {
    float ms = 0.f;
    WM_CUDA(cudaEventElapsedTime(&ms, ctx->ev_pool[m.second], ctx->ev_pool[m.second + 1]));
    ms_by_kind[m.first] += ms;
    launches_by_kind[m.first] += 1;
  }
  ctx->ev_marks.clear();
  return WM_OK;
}

wm_status wm_rollout_hourly(wm_ctx* ctx, const float* x, int max_lead, float* out, int max_batch, void* stream) {
  if (!ctx || !x || !out || max_lead < 0 || max_batch < 1) return fail(WM_ERR_INVALID_ARG, "bad hourly arguments");
  WM_TRY(check_compute(ctx, x, 1));
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  const size_t lat = (size_t)ctx->N * ctx->cfg.C;
  const int K = max_lead / 6;
  WM_TRY(ensure_workspace(ctx, std::max(1, std::min(max_batch, K + 1))));
  WM_TRY(ensure_buffer(&ctx->d_stage, &ctx->stage_cap, lat * std::min(max_batch, K + 1)));
  WM_TRY(rollout_small_reserve(ctx, std::max(1, std::min(max_batch, K + 1))));
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<uintptr_t> key = {3, (uintptr_t)x, (uintptr_t)out, (uintptr_t)max_lead, (uintptr_t)max_batch,
                                (uintptr_t)ctx->cfg.precision};
  return run_graph(ctx, key, s, [&](cudaStream_t st) -> wm_status {
    if (out != x) WM_CUDA(cudaMemcpyAsync(out, x, lat * 4, cudaMemcpyDeviceToDevice, st));
    // the six-hour anchors: out[6k] = P6(out[6(k-1)])
    for (int k = 1; k <= K; ++k) {
      WM_CUDA(cudaMemcpyAsync(out + (size_t)6 * k * lat, out + (size_t)6 * (k - 1) * lat, lat * 4,
                              cudaMemcpyDeviceToDevice, st));
      WM_TRY(processor_step(ctx, out + (size_t)6 * k * lat, 1, WM_P6, st));
    }
    // the one-hour branches of every anchor advance together: out[6k + r] = P1(out[6k + r - 1])
    std::vector<int> ks;
    for (int r = 1; r <= 5; ++r) {
      ks.clear();
      for (int k = 0; k <= K; ++k)
        if (6 * k + r <= max_lead) ks.push_back(k);
      for (size_t b0 = 0; b0 < ks.size(); b0 += max_batch) {
        const int g = (int)std::min<size_t>(max_batch, ks.size() - b0);
        for (int j = 0; j < g; ++j)
          WM_CUDA(cudaMemcpyAsync(ctx->d_stage + (size_t)j * lat, out + (size_t)(6 * ks[b0 + j] + r - 1) * lat,
                                  lat * 4, cudaMemcpyDeviceToDevice, st));
        WM_TRY(processor_step(ctx, ctx->d_stage, g, WM_P1, st));
        for (int j = 0; j < g; ++j)
          WM_CUDA(cudaMemcpyAsync(out + (size_t)(6 * ks[b0 + j] + r) * lat, ctx->d_stage + (size_t)j * lat,
                                  lat * 4, cudaMemcpyDeviceToDevice, st));
      }
    }
    return WM_OK;
  });
}

wm_status wm_rel_l2(const float* a, const float* b, size_t n, double* out, void* stream) {
  if (!a || !b || !out) return fail(WM_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  double* acc = nullptr;
  WM_CUDA(cudaMalloc(&acc, 2 * sizeof(double)));
  wm_status st = WM_OK;
  const cudaError_t ez = cudaMemsetAsync(acc, 0, 2 * sizeof(double), s);
  if (ez != cudaSuccess) st = wm::cuda_fail(ez, "wm_rel_l2 accumulator clear");
  if (st == WM_OK) st = wm::launch_sqdiff(a, b, n, acc, s);
  if (st == WM_OK) {
    cudaError_t e = cudaMemcpyAsync(out, acc, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = wm::cuda_fail(e, "wm_rel_l2 readback");
  }
  cudaFree(acc);
  return st;
}

wm_status wm_count_nonfinite(const float* x, size_t n, unsigned long long* count, void* stream) {
  if (!count) return fail(WM_ERR_INVALID_ARG, "NULL count");
  *count = 0;
  if (n == 0) return WM_OK;   // nothing to read: x may be NULL
  if (!x) return fail(WM_ERR_INVALID_ARG, "NULL x");
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* acc = nullptr;
  WM_CUDA(cudaMalloc(&acc, sizeof(unsigned long long)));
  wm_status st = WM_OK;
  const cudaError_t ez = cudaMemsetAsync(acc, 0, sizeof(unsigned long long), s);
  if (ez != cudaSuccess) st = wm::cuda_fail(ez, "wm_count_nonfinite counter clear");
  if (st == WM_OK) st = wm::launch_count_nonfinite(x, n, acc, s);
  if (st == WM_OK) {
    cudaError_t e = cudaMemcpyAsync(count, acc, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = wm::cuda_fail(e, "wm_count_nonfinite readback");
  }
  cudaFree(acc);
  return st;
}

wm_status wm_device_status(void) {
  int* w = wm::device_status_word();
  if (!w) return fail(WM_ERR_OOM, "no device status word");
  WM_CUDA(cudaDeviceSynchronize());
  int v = 0;
  WM_CUDA(cudaMemcpy(&v, w, sizeof(int), cudaMemcpyDeviceToHost));
  WM_CUDA(cudaMemset(w, 0, sizeof(int)));
  if (v == WM_ERR_TIMEOUT) return fail(WM_ERR_TIMEOUT, "a bounded device-side wait timed out");
  if (v != 0) return fail((wm_status)v, "device reported status " + std::to_string(v));
  return WM_OK;
}

wm_status wm_selftest_wait_timeout(int timeout_us) {
  if (timeout_us <= 0 || timeout_us > 10000000) return fail(WM_ERR_INVALID_ARG, "timeout must be in (0, 10 s]");
  WM_TRY(wm::prepare_kernels());
  WM_TRY(wm::launch_wait_selftest(timeout_us, 0));
  return wm_device_status();
}

// ----------------------------------------------------------------- ops ----
wm_status wm_op_layernorm(const float* x, const float* gamma, const float* beta, void* out, int out_bf16, int M,
                          int C, float eps, void* stream) {
  if (!x || !gamma || !beta || !out || M < 0 || C <= 0) return fail(WM_ERR_INVALID_ARG, "bad layernorm arguments");
  WM_TRY(wm::prepare_kernels());
  return wm::launch_layernorm(x, gamma, beta, out, out_bf16 != 0, M, C, eps, (cudaStream_t)stream);
}

wm_status wm_op_linear(const void* A, const void* W, const float* bias, void* out, int M, int N, int K,
                       int precision, int epilogue, void* stream) {
  if (!A || !W || !out || M < 0 || N <= 0 || K <= 0) return fail(WM_ERR_INVALID_ARG, "bad linear arguments");
  if (epilogue < 0 || epilogue > 3) return fail(WM_ERR_INVALID_ARG, "unknown epilogue");
  WM_TRY(wm::prepare_kernels());
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == WM_PREC_FP32)
    return wm::launch_sgemm((const float*)A, (const float*)W, bias, (float*)out, M, N, K, epilogue, s);
  if (precision != WM_PREC_BF16) return fail(WM_ERR_INVALID_ARG, "linear precision must be FP32 or BF16");
  if (M == 0) return WM_OK;
  if (K % 8 != 0 || N % 8 != 0) return fail(WM_ERR_INVALID_ARG, "BF16 linear needs K % 8 == 0 and N % 8 == 0");
  wm::GemmArgs a;
  const int ov = g_gemm_override.load();
  a.bn = ov == 1 ? 128 : ov == 4 ? 64 : (ov >= 2 && N % 256 == 0) ? 256 : pick_bn(M, N);
  a.pair = ov == 3 && a.bn == 256 && epilogue == wm::EPI_STORE;
  const bool out_f32 = epilogue == wm::EPI_RESID_F32 || epilogue == wm::EPI_STORE_F32;
  if (!wm::make_tmap_bf16(&a.tmA, A, (uint64_t)M, (uint64_t)K, 128) ||
      !wm::make_tmap_bf16(&a.tmB, W, (uint64_t)N, (uint64_t)K, (uint32_t)(a.pair ? 128 : a.bn)) ||
      !wm::make_tmap_out(&a.tmC, out, (uint64_t)M, (uint64_t)N, out_f32))
    return fail(WM_ERR_INVALID_ARG, "cannot build TMA descriptors (pointer alignment or sizes)");
  a.M = M; a.N = N; a.K = K;
  a.bias = bias; a.epi = epilogue;
  return wm::launch_gemm_tc(a, s);
}

wm_status wm_set_fused_rollout(int enable) {
  if (enable < 0 || enable > 1) return fail(WM_ERR_INVALID_ARG, "fused rollout switch must be 0 or 1");
  g_fused_rollout.store(enable);
  return WM_OK;
}

wm_status wm_set_fused_mlp(int enable) {
  if (enable < 0 || enable > 1) return fail(WM_ERR_INVALID_ARG, "fused MLP switch must be 0 or 1");
  g_mlp_fused.store(enable);
  return WM_OK;
}

wm_status wm_gemm_tile_override(int mode) {
  if (mode < 0 || mode > 4) return fail(WM_ERR_INVALID_ARG, "GEMM tile override must be 0..4");
  g_gemm_override.store(mode);
  return WM_OK;
}

wm_status wm_fp8_scales(wm_ctx* ctx, int which, int block, float* out) {
  if (!ctx || !out || (which != WM_P6 && which != WM_P1)) return fail(WM_ERR_INVALID_ARG, "bad arguments");
  if (block < 0 || block >= (int)ctx->blk[which].size()) return fail(WM_ERR_INVALID_ARG, "block index out of range");
  const BlockW& w = ctx->blk[which][block];
  out[0] = w.s_u;
  out[1] = w.s_w1;
  out[2] = w.s_h;
  out[3] = w.s_w2;
  return WM_OK;
}

wm_status wm_op_layernorm_e4m3(const float* x, const float* gamma, const float* beta, void* out, int M, int C,
                               float eps, float inv_scale, void* stream) {
  if (!x || !gamma || !beta || !out || M < 0 || C <= 0) return fail(WM_ERR_INVALID_ARG, "bad layernorm arguments");
  WM_TRY(wm::prepare_kernels());
  return wm::launch_layernorm_e4m3(x, gamma, beta, (uint8_t*)out, M, C, eps, inv_scale, (cudaStream_t)stream);
}

wm_status wm_op_linear_e4m3(const void* A, const void* W, float alpha, const float* bias, void* out, float out_scale,
                            int M, int N, int K, int epilogue, void* stream) {
  if (!A || !W || !out || M < 0 || N <= 0 || K <= 0) return fail(WM_ERR_INVALID_ARG, "bad linear arguments");
  if (epilogue != wm::EPI_STORE_F32 && epilogue != wm::EPI_RESID_F32 && epilogue != wm::EPI_GELU_F8)
    return fail(WM_ERR_INVALID_ARG, "e4m3 linear epilogue must be 2, 3 or 4");
  if (K % 16 != 0 || N % 16 != 0) return fail(WM_ERR_INVALID_ARG, "e4m3 linear needs K % 16 == 0 and N % 16 == 0");
  WM_TRY(wm::prepare_kernels());
  if (M == 0) return WM_OK;
  wm::GemmArgs a;
  a.f8 = true;
  a.bn = pick_bn(M, N);
  const bool okc = epilogue == wm::EPI_GELU_F8 ? wm::make_tmap_out_e4m3(&a.tmC, out, (uint64_t)M, (uint64_t)N)
                                               : wm::make_tmap_out(&a.tmC, out, (uint64_t)M, (uint64_t)N, true);
  if (!okc || !wm::make_tmap_e4m3(&a.tmA, A, (uint64_t)M, (uint64_t)K, 128) ||
      !wm::make_tmap_e4m3(&a.tmB, W, (uint64_t)N, (uint64_t)K, (uint32_t)a.bn))
    return fail(WM_ERR_INVALID_ARG, "cannot build TMA descriptors (pointer alignment or sizes)");
  a.M = M; a.N = N; a.K = K;
  a.bias = bias; a.epi = epilogue; a.alpha = alpha; a.out_scale = out_scale;
  return wm::launch_gemm_tc(a, (cudaStream_t)stream);
}

wm_status wm_op_neighborhood_attention(const void* qkv, void* out, int batch, int D, int H, int W, int C, int heads,
                                       int kd, int kh, int kw, int lon_periodic, int precision, int variant,
                                       void* stream) {
  wm_config c{};
  c.D = D; c.H = H; c.W = W; c.C = C; c.heads = heads; c.kd = kd; c.kh = kh; c.kw = kw;
  c.blocks_p6 = c.blocks_p1 = 1;
  c.precision = precision;
  WM_TRY(validate(&c));
  if (!qkv || !out || batch < 0) return fail(WM_ERR_INVALID_ARG, "bad attention arguments");
  WM_TRY(wm::prepare_kernels());
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == WM_PREC_FP32) {
    if (variant != WM_NA_AUTO) return fail(WM_ERR_INVALID_ARG, "the FP32 attention has one variant (WM_NA_AUTO)");
    return wm::launch_na_f32((const float*)qkv, (float*)out, batch, D, H, W, C, heads, kd, kh, kw, lon_periodic != 0, s);
  }
  if (precision != WM_PREC_BF16) return fail(WM_ERR_INVALID_ARG, "attention precision must be FP32 or BF16");
  if (C % 8 != 0) return fail(WM_ERR_INVALID_ARG, "BF16 attention needs C % 8 == 0");
  if (variant != WM_NA_TCGEN05 &&
      (variant < 0 || variant > 15 || (variant & 12) == 12 || (variant != 0 && (variant & 3) == 0)))
    return fail(WM_ERR_INVALID_ARG, "bad attention variant");
  return wm::launch_na_bf16((const bf16*)qkv, (bf16*)out, batch, D, H, W, C, heads, kd, kh, kw, lon_periodic != 0, s,
                            variant);
}

}  // extern "C"
