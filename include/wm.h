/*
 * wm.h -- C ABI of libwm, the GB300 (sm_103a) latent-rollout library for the
 * WeatherMesh-3 processor (arXiv 2503.22235).
 *
 * What the library computes (paper Section 2.1 and Appendix A.2):
 *   A forecast to an integer lead time T is a latent rollout: the six-hour
 *   processor is applied floor(T/6) times, then the one-hour processor T mod 6
 *   times (the "simple greedy schedule" of Section 2.1). Each processor is a
 *   stack of neighborhood-attention transformer blocks. One block on a latent
 *   x [B, D, H, W, C] (channel last; token n = (level*H + lat)*W + lon) is
 *       u  = LN1(x);  q,k,v = u Wqkv^T + bqkv
 *       o  = 3D neighborhood attention of q,k,v (per head, window kd x kh x kw,
 *            clamped -- "bump" -- along level and latitude, periodic along
 *            longitude -- "circular padding", Appendix A.2), softmax scale 1/sqrt(dh)
 *       x1 = x + o Wo^T + bo
 *       x2 = x1 + GELU(LN2(x1) W1^T + b1) W2^T + b2     (exact erf GELU)
 *   LayerNorm: biased variance, eps from the config, affine.
 *
 * Conventions for every call:
 *   - Status codes are returned, never aborts. On failure wm_last_error()
 *     gives a message for the calling thread.
 *   - "device" pointers are CUDA global memory of the current device, owned by
 *     the caller unless stated otherwise; "host" pointers are CPU memory.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream). Calls taking a
 *     stream are asynchronous on it unless stated otherwise.
 *   - Latents at the boundary are always float32 [batch, D, H, W, C],
 *     contiguous, whatever the internal precision.
 *   - The library owns weights, workspace, CUDA graphs and server slots.
 *   - Concurrency: a context's compute calls share its workspace. Host calls
 *     from several threads are serialised by the context, but their GPU work
 *     must not overlap: issue one context's calls on one stream (or order
 *     the streams), or use one context per concurrent stream.
 */
#ifndef WM_H
#define WM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  WM_OK = 0,
  WM_ERR_INVALID_ARG = 1,  /* bad shape, window, lead time, pointer or enum */
  WM_ERR_OOM = 2,          /* a device or host allocation failed */
  WM_ERR_CUDA = 3,         /* a CUDA runtime call failed (message has the CUDA error) */
  WM_ERR_TIMEOUT = 4,      /* a bounded device-side wait ran out; the context stays usable */
  WM_ERR_BUSY = 5,         /* server admission: the HBM budget or slot table is full */
  WM_ERR_IO = 6,           /* weight file missing, short or malformed */
  WM_ERR_NOT_FOUND = 7,    /* unknown request id */
  WM_ERR_BOUNDS = 8        /* debug build (libwm_debug.so) only: a device-side index check failed
                              (attention window or slab geometry, tail tile); the access was skipped */
} wm_status;

typedef enum { WM_P6 = 0 /* six-hour processor */, WM_P1 = 1 /* one-hour processor */ } wm_processor;

typedef enum {
  WM_PREC_FP32 = 0,        /* plain path: FP32 FMA everywhere (no TF32), CUDA cores */
  WM_PREC_BF16 = 1,        /* BF16 tcgen05 GEMMs + BF16 tensor-core attention, FP32 accumulate,
                              FP32 residual stream, FP32 LayerNorm statistics and softmax normalisers */
  WM_PREC_BF16_FP8MLP = 2  /* as BF16, with the MLP GEMMs in FP8 E4M3 (per-tensor scales) */
} wm_precision;

typedef struct {
  int D, H, W, C;          /* latent levels, latitudes, longitudes, channels */
  int heads;               /* attention heads; C % heads == 0 */
  int kd, kh, kw;          /* odd window sizes; kd <= D, kh <= H, kw <= W */
  int blocks_p6;           /* blocks in the six-hour processor (>= 1) */
  int blocks_p1;           /* blocks in the one-hour processor (>= 1) */
  int lon_periodic;        /* 1: periodic longitude windows; 0: clamped like the other axes */
  float ln_eps;            /* LayerNorm epsilon (the processor uses 1e-5) */
  int precision;           /* wm_precision used by the compute calls */
  int max_batch;           /* initial workspace capacity in latents (grown on demand) */
  int rope;                /* 1: 3D rotary position embedding on q and k (Appendix A.2). The head's dh/2
                              dimension pairs (2p, 2p+1) are split into level, latitude and longitude
                              groups, n_lon = ceil(P/3), n_lat = ceil((P - n_lon)/2), n_lev = P - n_lon - n_lat;
                              pair m of an axis rotates by pos * w_m with w_m = 10000^(-m/n_axis) for
                              level and latitude and w_m = 2 pi (m + 1) / W for longitude. 0: none. */
} wm_config;

typedef struct wm_ctx wm_ctx;
typedef struct wm_server wm_server;

/* ----------------------------------------------------------- context ---- */

/* Create a context on the current CUDA device and upload the weights of the
 * six-hour and one-hour processors (Section 2.1, Appendix A.2; the paper has 10
 * blocks per processor, here blocks_p6 and blocks_p1). The library copies the
 * weights; the caller keeps the file. weights_path: weight file = 8-byte magic "WM3WGT1\0", int32 C, blocks_p6,
 * blocks_p1, 0 (little endian), then float32 tensors: for the six-hour blocks
 * then the one-hour blocks, per block in this order
 *   ln1_g[C] ln1_b[C] wqkv[3C][C] bqkv[3C] wo[C][C] bo[C] ln2_g[C] ln2_b[C]
 *   w1[4C][C] b1[4C] w2[C][4C] b2[C]
 * (matrices [out][in], q/k/v row blocks of wqkv each head-major).
 * Errors: WM_ERR_INVALID_ARG (config), WM_ERR_IO (file), WM_ERR_OOM, WM_ERR_CUDA. */
wm_status wm_create(const wm_config* cfg, const char* weights_path, wm_ctx** out);

/* As wm_create, with the float32 tensors (no header) in host memory; n_floats
 * must equal (blocks_p6 + blocks_p1) * (12*C*C + 13*C). The buffer is copied. */
wm_status wm_create_from_host(const wm_config* cfg, const float* weights, size_t n_floats, wm_ctx** out);

/* Synchronises the device, frees everything the context owns. NULL is a no-op.
 * (Library service; no counterpart in the paper.) */
wm_status wm_destroy(wm_ctx* ctx);

/* Switch the precision used by later compute calls (weights for all precisions
 * are resident). The paper trains in half precision (Appendix A.3); the
 * precisions here are this library's. WM_ERR_INVALID_ARG for an unknown value. */
wm_status wm_set_precision(wm_ctx* ctx, int precision);

/* Sizes for `batch` latents at the context's current precision: floats per
 * latent (D*H*W*C) and bytes of the workspace the compute calls need (HOST
 * outputs, both required; WM_ERR_INVALID_ARG otherwise). (Library service.) */
wm_status wm_ctx_sizes(wm_ctx* ctx, int batch, size_t* latent_floats, size_t* workspace_bytes);

/* Allocate the workspace for `batch` latents now (at the current precision),
 * so that later calls, and graph captures, allocate nothing. WM_ERR_OOM if
 * it does not fit. (Library service.) */
wm_status wm_ctx_reserve(wm_ctx* ctx, int batch);

/* The tile plans the autotuner chose so far in this process (text, one line
 * per shape, NUL-terminated, truncated to len - 1 bytes; buf is HOST). The
 * attention kernel's plans are timed when a context's BF16 workspace is
 * allocated. (Library service.) */
wm_status wm_autotune_report(char* buf, size_t len);

/* ----------------------------------------------------------- compute ---- */

/* One neighborhood-attention transformer block (Section 2.1, Appendix A.2;
 * the formula at the top of this file), index `block` of processor `which`,
 * applied in place to latent (device, float32 [batch, D, H, W, C]).
 * WM_ERR_INVALID_ARG for which/block out of range, a NULL or misaligned latent
 * or batch < 1; WM_ERR_OOM, WM_ERR_CUDA, WM_ERR_TIMEOUT. */
wm_status wm_block_forward(wm_ctx* ctx, float* latent, int batch, int which, int block, void* stream);

/* One processor call (all of its blocks, in order) in place: a six-hour step
 * (WM_P6) or a one-hour step (WM_P1), Section 2.1. */
wm_status wm_processor_step(wm_ctx* ctx, float* latent, int batch, int which, void* stream);

/* Latent rollout to lead_hours (Section 2.1) in place on a device latent:
 * floor(T/6) six-hour steps then T mod 6 one-hour steps, replayed as one CUDA
 * graph captured on first use for (latent, batch, T, precision) and cached.
 * T = 0 is a no-op; T < 0 gives WM_ERR_INVALID_ARG. */
wm_status wm_latent_rollout(wm_ctx* ctx, float* latent, int batch, int lead_hours, void* stream);

/* End-to-end forecast from HOST memory (the problem statement of Section 2.1:
 * one state in, the state lead_hours later out): copies host_in (float32
 * [batch,D,H,W,C]) to a library-owned device latent, runs wm_latent_rollout,
 * copies the result to host_out (may equal host_in) and synchronises the
 * stream before returning, on the error path too. Pinned host buffers make
 * the copies asynchronous DMA. The caller guarantees the buffer sizes.
 * Errors: WM_ERR_INVALID_ARG (NULL, batch < 1, T < 0), WM_ERR_OOM, WM_ERR_CUDA. */
wm_status wm_forecast_host(wm_ctx* ctx, const float* host_in, float* host_out, int batch,
                           int lead_hours, void* stream);

/* A stream of n end-to-end forecasts from HOST memory (Section 2.1, as
 * wm_forecast_host): forecast i copies
 * host_in[i] to the device, rolls it out to lead_hours and copies the result
 * to host_out[i] (float32 [batch,D,H,W,C] each). A ring of three
 * library-owned device latents lets the upload of forecast i + 1 and the
 * download of forecast i - 1 run on library-owned copy streams while forecast
 * i computes on `stream`. Each result equals wm_forecast_host's bit for bit. Returns
 * once every result is in host memory. host_in[i] may repeat; host_out[i]
 * must not alias another forecast's input or output that is still in flight
 * (the same pointer for every output is fine: downloads are serialised).
 * Pinned host buffers make the copies asynchronous DMA. n = 0 is a no-op.
 * Errors as wm_forecast_host; every copy has finished before it returns. */
wm_status wm_forecast_host_many(wm_ctx* ctx, const float* const* host_in, float* const* host_out, int n, int batch,
                                int lead_hours, void* stream);

/* Batched uneven rollouts (the latent rollout of Section 2.1 for each request;
 * the batching is this library's): latents[i] (device, one float32 latent each) is
 * advanced in place to lead_hours[i]. All requests advance together one
 * processor step per tick; the requests due for the same processor in a tick
 * run as one batched step (row-independent kernels, so each result equals its
 * single-request rollout bit for bit). n >= 1; leads >= 0. */
wm_status wm_rollout_batch(wm_ctx* ctx, float* const* latents, const int* lead_hours, int n, void* stream);

/* Every hourly lead time 0..max_lead from one initial state (the hourly
 * forecasts of Section 4.1, Forecast Accessibility): out[t] (device, max_lead + 1 contiguous float32
 * latents) = the rollout of x (device, one latent) to t hours. By the greedy
 * schedule (Section 2.1) lead 6k + r is r one-hour steps after the k-th
 * six-hour anchor, so the anchors form one chain of six-hour steps and the
 * one-hour branches of all anchors advance together as batched steps of at
 * most max_batch latents. Each out[t] equals wm_latent_rollout(x, t) bit for
 * bit. Replayed from a CUDA graph captured per (x, out, max_lead, max_batch). */
wm_status wm_rollout_hourly(wm_ctx* ctx, const float* x, int max_lead, float* out, int max_batch, void* stream);

/* Greedy schedule of Section 2.1 (pure host): n6 = T div 6, n1 = T mod 6. */
wm_status wm_schedule(int lead_hours, int* n6, int* n1);

/* FP64 error reduction on the GPU (the relative-L2 metric of the parity
 * tolerances; library service): out[0] = sum (a-b)^2, out[1] = sum b^2 over n
 * float32 elements (device pointers); out is HOST memory of 2 doubles, filled
 * after an internal synchronisation of `stream`. rel-L2 = sqrt(out[0]/out[1]). */
wm_status wm_rel_l2(const float* a, const float* b, size_t n, double* out, void* stream);

/* Allocation-free variant of wm_rel_l2 (the paper has no counterpart; this is
 * a library service). Same inputs, outputs and result as wm_rel_l2, but it
 * allocates nothing: its scratch is a fixed 64 KiB device array inside the
 * library, present on every GPU that loads the library until the process
 * exits. For callers that cannot allocate device memory at the point of the
 * check -- a framework's caching allocator holds all free memory, or the
 * caller must not take cudaMalloc/cudaFree (cudaFree synchronises the whole
 * device and stalls every other stream).
 *   - n <= 268,435,456 elements (4096 partial sums of 65,536 elements each);
 *     larger n gives WM_ERR_INVALID_ARG and launches nothing.
 *   - Every call looks up the scratch array's device address on the current
 *     device (cudaGetSymbolAddress, which allocates nothing); the first call
 *     on a device also loads the library's device code there, so make it
 *     before any stream capture. n = 0 writes out = {0, 0} and launches
 *     nothing.
 *   - All calls share the one scratch array; calls whose kernels overlap on
 *     the GPU (e.g. from two streams at once) race and may return wrong sums.
 *     Every partial is rewritten on each call, so nothing needs clearing.
 *   - The sums are deterministic (fixed summation order), so they can differ
 *     from wm_rel_l2's atomically accumulated sums in the last bits. */
wm_status wm_rel_l2_noalloc(const float* a, const float* b, size_t n, double* out, void* stream);

/* NaN / infinity scan of the error check (library service; the paper has no
 * counterpart): *count (HOST) = the number of non-finite elements of x
 * (device, n float32), after an internal synchronisation of `stream`.
 * Allocates an 8-byte device counter per call. n = 0 gives 0 and reads
 * nothing (x may then be NULL); otherwise WM_ERR_INVALID_ARG for a NULL x. */
wm_status wm_count_nonfinite(const float* x, size_t n, unsigned long long* count, void* stream);

/* Reads (and clears) the device status word that bounded device-side waits
 * (and, in the debug build, the device-side index checks) write; synchronises
 * the device. WM_OK, WM_ERR_TIMEOUT or (debug build) WM_ERR_BOUNDS.
 * (Library service.) */
wm_status wm_device_status(void);

/* Self-test of the bounded-wait path: launches one kernel that waits on a
 * device flag that nothing sets, for at most timeout_us microseconds, then
 * returns. Expect WM_ERR_TIMEOUT, after which the context must stay usable. */
wm_status wm_selftest_wait_timeout(int timeout_us);

/* Per-launch kernel timing (library service). Between wm_timing_begin and wm_timing_end every
 * hot-path kernel launched by compute calls on this context is bracketed by a
 * CUDA event pair on its stream (rollouts then run eagerly instead of from a
 * graph). wm_timing_end synchronises the device and returns, per kernel kind
 * (wm_kernel_kind), the summed device milliseconds and the launch count.
 * At most max_launches launches are recorded; later ones are not timed. */
typedef enum { WM_K_LN1 = 0, WM_K_QKV = 1, WM_K_ATTN = 2, WM_K_PROJ = 3, WM_K_LN2 = 4, WM_K_FC1 = 5,
               WM_K_FC2 = 6, WM_KERNEL_KINDS = 7 } wm_kernel_kind;
wm_status wm_timing_begin(wm_ctx* ctx, int max_launches);
wm_status wm_timing_end(wm_ctx* ctx, double* ms_by_kind /* [WM_KERNEL_KINDS] */,
                        int* launches_by_kind /* [WM_KERNEL_KINDS] */);

/* Message of the last failed call on this thread ("" if none); the string is
 * owned by the library and valid until the thread's next failing call. */
const char* wm_last_error(void);

/* ----------------------------------------------------------- serving ---- */
/* Forecast server with continuous batching (one worker thread per server).
 * It serves the operational use of Section 4.1 (Forecast Accessibility): forecasts of one model to many
 * lead times. The paper describes no server; the policy below is this
 * library's.
 * Requests are a HOST latent (float32 [1, D, H, W, C], copied at submit) and a
 * lead time. They are admitted into device-resident latent slots in arrival
 * order while slots are free; the number of slots is set by the HBM budget:
 *   slots = (hbm_budget_bytes - workspace(max_batch) - max_batch latents of
 *            staging) / latent bytes.
 * Each tick, every admitted request with steps left takes one processor step
 * (greedy schedule, six-hour steps first); the requests due for the same
 * processor run as batched steps of at most max_batch latents; requests that
 * arrive meanwhile join at the next tick. A finished request keeps its result
 * in its slot until wm_server_poll collects it (which frees the slot).
 * Latency = submit call -> the host sees the tick that finished the request. */
/* While the server runs, ctx belongs to it (its worker issues the context's
 * compute calls on the server's own stream): use another context for other
 * work until wm_server_stop. */
wm_status wm_server_start(wm_ctx* ctx, size_t hbm_budget_bytes, int max_batch, wm_server** out);

/* Queue a request; WM_ERR_BUSY when the pending queue is full, WM_ERR_INVALID_ARG for T < 0. */
wm_status wm_server_submit(wm_server* srv, const float* host_latent, int lead_hours, uint64_t* req_id);

/* *done = 1 once the request has finished: its result is copied to host_out
 * (HOST, may be NULL to discard), latency_ms (may be NULL) is set, and the
 * request and its slot are released. *done = 0 while it is queued or running.
 * WM_ERR_NOT_FOUND for an unknown or already collected id; a poll that races
 * another poll of the same finished id gets WM_ERR_NOT_FOUND while the other
 * one copies the result out (each result is collected exactly once). If the
 * copy fails (WM_ERR_CUDA) the result stays collectable. */
wm_status wm_server_poll(wm_server* srv, uint64_t req_id, float* host_out, int* done, double* latency_ms);

/* out[11] (HOST): completed requests, p50 latency ms, p99 latency ms, mean
 * latency ms, forecasts/s (completed / (last completion - first arrival)),
 * most requests resident at once, ticks, batched steps launched, slots, most
 * requests advanced by one batched step, batched steps that advanced two or
 * more requests together. */
wm_status wm_server_stats(wm_server* srv, double* out);

/* Stops the worker after its current tick and frees the slots; pending and
 * uncollected requests are dropped. Returns the worker's error, if any. */
wm_status wm_server_stop(wm_server* srv);

/* ---------------------------------------------------------- op level ---- */
/* The individual hot-path kernels on caller device buffers, for parity tests
 * of each step against the oracle. Each is one step of the block at the top of
 * this file (Section 2.1, Appendix A.2): LayerNorm (LN1, LN2), the linear
 * layers (QKV, output projection, FC1, FC2) with their GELU and residual
 * epilogues, and the neighborhood attention. All are asynchronous on
 * `stream`; WM_ERR_INVALID_ARG for bad sizes, NULL or misaligned pointers,
 * WM_ERR_CUDA for a failed launch. */

/* LayerNorm over C of M float32 rows of x; out is float32 (out_bf16 = 0) or
 * bfloat16 (out_bf16 = 1) [M, C]. */
wm_status wm_op_layernorm(const float* x, const float* gamma, const float* beta, void* out, int out_bf16,
                          int M, int C, float eps, void* stream);

/* Linear layer D = A W^T + bias on A [M, K], W [N, K] (row major, K contiguous).
 * precision WM_PREC_FP32: A, W float32 (CUDA-core FP32 FMA);
 * precision WM_PREC_BF16: A, W bfloat16 (tcgen05, FP32 accumulate), K % 8 == 0.
 * epilogue 0: out = D (out float32 for FP32, bfloat16 for BF16)
 * epilogue 1: out = GELU(D) (same out types)
 * epilogue 2: out (float32 [M, N]) += D   (residual add)
 * epilogue 3: out (float32) = D. bias may be NULL. */
wm_status wm_op_linear(const void* A, const void* W, const float* bias, void* out, int M, int N, int K,
                       int precision, int epilogue, void* stream);

/* e4m3 linear layer (the FP8 MLP's GEMMs): A [M, K] and W [N, K] are E4M3 codes
 * (one byte each, OCP FP8 E4M3), D = alpha * (A W^T) + bias with FP32 accumulation.
 * epilogue 2: out (float32) += D;  3: out (float32) = D;
 * epilogue 4: out (E4M3 codes [M, N]) = e4m3(GELU(D) * out_scale), round to nearest
 *             even, saturating at +-448.  K % 16 == 0, N % 16 == 0. */
wm_status wm_op_linear_e4m3(const void* A, const void* W, float alpha, const float* bias, void* out, float out_scale,
                            int M, int N, int K, int epilogue, void* stream);

/* LayerNorm with E4M3 output: out[M, C] = e4m3(LN(x) * inv_scale) (RNE, saturating).
 * C in {128, 256, 384, 512, 768, 1024}. */
wm_status wm_op_layernorm_e4m3(const float* x, const float* gamma, const float* beta, void* out, int M, int C,
                               float eps, float inv_scale, void* stream);

/* The static per-tensor scales the FP8 MLP precision uses for block `block` of
 * processor `which` (HOST out[4]): s_u (LN2 output), s_w1, s_h (GELU output), s_w2.
 *   s_u  = max_c(|gamma2_c| sqrt(C-1) + |beta2_c|) / 448   (bound on |LN2(x)|)
 *   s_w1 = max|W1| / 448, s_w2 = max|W2| / 448
 *   s_h  = max(max_j(sum_c |W1_jc| (|gamma2_c| sqrt(C-1) + |beta2_c|) + |b1_j|), 0.17) / 448
 * (bound on |GELU(FC1)|). Bounds hold for every input, so no value saturates and
 * the scales do not depend on the batch or the request. */
wm_status wm_fp8_scales(wm_ctx* ctx, int which, int block, float* out);

/* Test hook for the tcgen05 GEMM tiles (process-wide, not thread-safe with
 * respect to launches in flight): mode 0 = the autotuner's plans (default),
 * 1 = 128-column tiles, 2 = 256-column tiles, 3 = 256 x 256 tiles on CTA pairs
 * (cta_group::2; shapes with N % 256 != 0 keep single-CTA tiles), 4 = 64-column
 * tiles (N % 64 == 0). Applies to every BF16 / FP8-MLP block GEMM launched or
 * captured afterwards and to wm_op_linear (BF16; pairs for epilogue 0 only).
 * Results are the same function of the inputs in every mode up to
 * accumulation rounding; the tile width also sets how the LayerNorm
 * statistics partials are split (two per tile). WM_ERR_INVALID_ARG for a
 * mode outside 0..4. */
wm_status wm_gemm_tile_override(int mode);

/* Process-wide switch: enable = 1 runs a BF16 block's MLP at C = 128 as one
 * fused kernel (FC1 with LayerNorm 2 folded, GELU, FC2 and the residual, the
 * hidden activations in shared memory; bit-identical to the two GEMMs),
 * enable = 0 (default) as two GEMMs, which were measured as fast or faster
 * inside captured rollouts (the fused kernel runs one CTA per 128 rows, the
 * first GEMM one per 128 x 128 output tile). Applies to blocks launched or
 * captured afterwards. WM_ERR_INVALID_ARG for another value. */
wm_status wm_set_fused_mlp(int enable);

/* Whole-rollout launches for narrow latents (Section 2.1 latent rollout,
 * Appendix A.2 blocks): 1 (the default) lets wm_latent_rollout and
 * wm_rollout_batch run BF16 contexts with C = 128, 4 heads, periodic
 * longitude, no rotary embedding, H % 8 == 0, W % 16 == 0, W >= 32 and
 * latitude / longitude windows of at most 5 as ONE kernel launch per group of
 * latents (as many as the device holds at once: 4 for the 4 x 24 x 48 latent).
 * Each CTA keeps an 8 x 16-token patch of its latent's residual stream in
 * shared memory for the whole rollout and runs every block's attention,
 * projection, MLP, LayerNorms and residual adds; the latent's CTAs meet once
 * per block at a counter in global memory. The result equals the per-kernel
 * path within the BF16 tolerance (LayerNorm is applied explicitly, not folded
 * into the GEMMs, so the two are not bit-identical). Latents of
 * wm_rollout_batch are read and written in place. 0: every rollout uses one
 * launch per GEMM / attention. WM_ERR_INVALID_ARG for another value. */
wm_status wm_set_fused_rollout(int enable);

/* ------------------------------------------------------------------------
 * Encoder and decoder (Section 2.1 "Encoder-processor-decoder architecture";
 * Appendix A.1 variables, A.2 architecture). The paper gives the grid (0.25
 * degrees -> 2-degree latent), the variables (5 atmospheric on 28 pressure
 * levels, 8 surface inputs, 17 surface outputs), the constant fields
 * concatenated with the input, and 2 NA blocks of width 1024 on each side; it
 * does not list the convolution layers. This library's reading:
 *   encoder: atmosphere zero-padded at the top (index 0 side) to level_pad
 *     levels; a strided convolution (kernel = stride = pd levels x p x p
 *     pixels) of the 5 variables -> Ce channels per latent token; a strided
 *     convolution (p x p) of surface inputs + constants -> Ce for the last
 *     latent level; `blocks` NA blocks at width Ce; a linear map Ce -> C.
 *   decoder: linear C -> Ce; `blocks` NA blocks; transposed convolutions
 *     (kernel = stride) back to the atmosphere (padding levels dropped) and
 *     the surface outputs. ResNet blocks are not built.
 * Physical fields (device, float32, contiguous, channel last):
 *   atm    [levels][H0][W0][v_atm]      sfc  [H0][W0][v_sfc_in]
 *   consts [H0][W0][n_const]            atm_out [levels][H0][W0][v_atm]
 *   sfc_out [H0][W0][v_sfc_out]
 * Latent: float32 [D][H][W][C], D = level_pad / pd + 1 (surface last),
 * H = H0 / p, W = W0 / p.
 * Weights (host float32 blob, n_floats long): matrices [out][in] with the
 * convolution kernels flattened as (level, row, column, channel):
 *   embed_atm_w [Ce][pd*p*p*v_atm], embed_atm_b [Ce],
 *   embed_sfc_w [Ce][p*p*(v_sfc_in+n_const)], embed_sfc_b [Ce],
 *   enc_out_w [C][Ce], enc_out_b [C], dec_in_w [Ce][C], dec_in_b [Ce],
 *   unembed_atm_w [pd*p*p*v_atm][Ce], unembed_atm_b [pd*p*p*v_atm],
 *   unembed_sfc_w [p*p*v_sfc_out][Ce], unembed_sfc_b [p*p*v_sfc_out],
 *   then the encoder's and the decoder's NA blocks in the processor blob
 *   layout (wm_create_from_host: encoder blocks first).
 * ------------------------------------------------------------------------ */
typedef struct wm_codec wm_codec;

typedef struct {
  int H0, W0;                  /* physical grid; multiples of p */
  int levels, level_pad, pd;   /* pressure levels, padded count (multiple of pd, >= levels), levels per token */
  int p;                       /* pixels per token along latitude and longitude */
  int v_atm, v_sfc_in, v_sfc_out, n_const;
  int Ce, heads, kd, kh, kw;   /* NA blocks of the encoder / decoder (window odd, dh = Ce/heads) */
  int blocks;                  /* NA blocks on each side (>= 1) */
  int C;                       /* latent width (the processor's C) */
  int lon_periodic;
  float ln_eps;
  int precision;               /* WM_PREC_FP32 or WM_PREC_BF16 */
} wm_codec_config;

/* Upload weights and allocate the workspace for one field set. Errors:
 * WM_ERR_INVALID_ARG for inconsistent sizes or a blob of the wrong length,
 * WM_ERR_OOM, WM_ERR_CUDA. Calls on one codec share its workspace: do not run
 * two of them concurrently (different streams or threads); use one codec per
 * concurrent caller. */
wm_status wm_codec_create(const wm_codec_config* cfg, const float* host_weights, size_t n_floats, wm_codec** out);
/* Synchronises the device and frees the codec (NULL is a no-op). */
wm_status wm_codec_destroy(wm_codec* codec);
/* Physical fields -> latent (all device pointers; asynchronous on stream). */
wm_status wm_encode(wm_codec* codec, const float* atm, const float* sfc, const float* consts, float* latent,
                    void* stream);
/* Latent -> physical fields (device pointers; the latent is not modified). */
wm_status wm_decode(wm_codec* codec, const float* latent, float* atm_out, float* sfc_out, void* stream);
/* Encode, roll the latent out to lead_hours with ctx's processors (ctx's latent
 * shape must equal the codec's), decode. latent_ws: device scratch of
 * D*H*W*C floats owned by the caller. */
wm_status wm_forecast_fields(wm_ctx* ctx, wm_codec* codec, const float* atm, const float* sfc, const float* consts,
                             int lead_hours, float* latent_ws, float* atm_out, float* sfc_out, void* stream);

/* 3D neighborhood attention (Section 2.1; window, bump edges and circular
 * longitude padding of Appendix A.2) on qkv [batch*D*H*W, 3C] (q | k | v, each head-major)
 * -> out [batch*D*H*W, C]. precision FP32: float32 in/out; BF16: bfloat16 in/out
 * (BF16 requires dh = C/heads in {16, 32, 48, 64}).
 * variant (BF16 only; FP32 takes 0): WM_NA_AUTO uses the plan tuned for this
 * shape, else the arithmetic family fixed for it, else the default. Otherwise
 * one of WM_NA_QK_CHUNK8, WM_NA_QK_CHUNK4, WM_NA_KQ picks the arithmetic
 * family, optionally OR-ed with WM_NA_PER_TILE or WM_NA_PERSISTENT to pick
 * the kernel kind (else the kind is chosen by a heuristic); or WM_NA_TCGEN05
 * alone, the tcgen05 kernel (tensor-memory accumulators, 16 x 8 query tiles;
 * head dim 32 or 48 with window 5x5 or 7x7 in latitude x longitude, or head
 * dim 64 with 5x5; at least kh + 3 latitudes; clamped longitude needs
 * W >= kw + 7), WM_ERR_INVALID_ARG for other shapes. Families round
 * differently (order of the softmax sums); the kernel kind and CTA shape do
 * not change any result. */
enum {
  WM_NA_AUTO = 0,
  WM_NA_QK_CHUNK8 = 1,   /* S = Q K^T, 16 queries per warp, softmax update every 8 key groups */
  WM_NA_QK_CHUNK4 = 2,   /* as above, update every 4 key groups */
  WM_NA_KQ = 3,          /* S^T = K Q^T, 8 queries per warp, update every 8 key groups */
  WM_NA_PER_TILE = 4,    /* one CTA per query tile */
  WM_NA_PERSISTENT = 8,  /* persistent CTAs with a producer warp */
  WM_NA_TCGEN05 = 16     /* S = Q K^T and O += P V on tcgen05, 128 queries per CTA tile, update per 8-longitude
                            half of a key level (its own family; alone, not combined with the bits above) */
};
wm_status wm_op_neighborhood_attention(const void* qkv, void* out, int batch, int D, int H, int W, int C,
                                       int heads, int kd, int kh, int kw, int lon_periodic, int precision,
                                       int variant, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* WM_H */
