// Whole-rollout persistent kernel for narrow latents (C = 128, 4 heads of 32
// channels): every block of the greedy schedule of every latent in ONE launch.
//
// Why: at C = 128 a block's five GEMM / attention launches are each a few
// microseconds of latency on a few dozen SMs, so a 14-day rollout (448 blocks)
// is bound by launch and memory round trips, not by arithmetic. Here each CTA
// owns one 8 x 16 (latitude x longitude) patch of 128 tokens of one level of
// one latent for the whole rollout; its residual rows stay in tensor memory,
// and per block (pre-LN transformer block, paper Sec. 2.1 and App. A.2):
//
//   attention   8 warps, mma.sync m16n8k16: each warp takes a 4 x 4 query
//               group and one head at a time and walks its 8 x 8 key
//               rectangle per key level (K/V slabs of the patch's halo brought
//               to shared memory by tensor copies from a producer warp, one
//               box per slab and two where the longitude wraps, three
//               stages), FP32 online softmax; O goes to shared memory as the
//               next GEMM's A operand
//   proj        tcgen05.mma (M = N = 128, K = 128) into TMEM; x += acc + b_o;
//               LayerNorm 2 of the new rows (two-pass, FP32) -> bf16 A operand
//   MLP         four 128-column hidden chunks: FC1 into two TMEM buffers,
//               bias + erf GELU -> bf16 chunk in shared memory, FC2 K slice
//               accumulated in TMEM; x += acc + b_2
//   LN1 + QKV   LayerNorm 1 of the next block -> A operand; Q, K, V (+ bias) to
//               a double-buffered bf16 [3C] array in global memory (L2)
//   barrier     the latent's CTAs meet at a counter in global memory (bounded
//               spin), then read their neighbours' K/V for the next block
//
// Roles (352 threads): warps 0-7 compute (attention, epilogues, LayerNorm),
// warp 8 one thread issuing the tcgen05 MMAs, warp 9 one thread streaming the
// block's weights (12 pre-swizzled 32 KB chunks per block, one bulk copy each,
// through a two-slot ring) and its biases and LayerNorm vectors (one bulk
// copy into a two-slot buffer), warp 10 one thread issuing the K/V tensor
// copies into a three-stage ring. Latents are independent: each has its own
// schedule (six-hour blocks, then one-hour blocks) and its own barrier, so
// latents with different lead times share the launch.
//
// Every mbarrier wait and the latent barrier are bounded in time; on a
// timeout the CTA records WM_ERR_TIMEOUT, the compute warps leave together
// (barrier with OR-reduction), copies and MMAs in flight are drained, TMEM
// is freed and the CTA returns.
#include "tc_gemm.cuh"

namespace wm {
namespace rs {

using namespace ptx;
using namespace tc;
using bf16 = __nv_bfloat16;
using Blk = RolloutBlock;

constexpr int C = 128, DH = 32, QKV = 3 * C;
constexpr int TH = 8, TW = 16;                 // query patch of one CTA
constexpr int SW = TW + 4;                     // slab columns: the patch's longitudes + 2 on each side
constexpr int SR_MAX = TH + 4;                 // slab rows (latitude windows of at most 5)
constexpr int THREADS = 352, MMA_WARP = 8, LOAD_WARP = 9, KV_WARP = 10;
constexpr int CHUNK = 128 * 128 * 2;           // 128 x 128 bf16 operand: two 64-column 128B-swizzled slices
constexpr int SLICE = CHUNK / 2;
constexpr int NSLOT = 2;                       // weight ring slots
constexpr int NKV = 3;                         // K/V stages
constexpr int VEC_FLOATS = 1664;               // a block's vectors (layout below)
constexpr int VEC_BYTES = VEC_FLOATS * 4;
constexpr int OFF_A = 0;                       // A operand: LN1(x), O or LN2(x)
constexpr int OFF_W = OFF_A + CHUNK;           // weight ring
constexpr int OFF_H = OFF_W + NSLOT * CHUNK;   // GELU chunks, 2 slots; K/V stages 0 and 1 alias it
constexpr int KV_SLAB = SR_MAX * SW * DH * 2;  // one head's K (or V) rows of a key level
constexpr int KV_STAGE = 2 * KV_SLAB;
constexpr int OFF_KV2 = OFF_H + 2 * CHUNK;     // the third K/V stage (the first two alias the GELU region)
constexpr int OFF_VEC = OFF_KV2 + KV_STAGE;    // vectors of two blocks
constexpr int SMEM_USED = OFF_VEC + 2 * VEC_BYTES;
constexpr int SMEM = SMEM_USED + 1024;         // + alignment slack
constexpr int OFF_RED = OFF_H + 2 * KV_STAGE;  // LayerNorm row partials [2 passes][2 halves][128]
static_assert(OFF_RED + 4 * 128 * 4 <= OFF_H + 2 * CHUNK, "LayerNorm exchange must fit in the GELU region");
static_assert(OFF_H % 1024 == 0 && OFF_KV2 % 512 == 0 && KV_SLAB % 512 == 0, "swizzled operands need aligned bases");
static_assert(SMEM <= 232448, "shared memory per CTA");
__device__ __forceinline__ uint32_t kv_stage_off(int b) { return (uint32_t)(b < 2 ? OFF_H + b * KV_STAGE : OFF_KV2); }
// TMEM columns: FC1 accumulators (and the projection's) at 0 and 128, FC2's at
// 256; QKV chunks at 0, 128, 256; the fp32 residual rows at 384
constexpr uint32_t T_ACC1 = 0, T_PROJ = 0, T_ACC2 = 256, T_X = 384;
// weight chunks of a block, in this order in memory, then the vectors
constexpr int W_QKV = 0, W_O = 3, W_1 = 4, W_2 = 8, W_VEC = 12;
// offsets of the vectors in floats
constexpr int V_BQKV = 0, V_BO = 384, V_LN1G = 512, V_LN1B = 640, V_LN2G = 768, V_LN2B = 896, V_B1 = 1024,
              V_B2 = 1536;

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// ---- compute-warp barriers (named barrier 1, the 256 compute threads)
__device__ __forceinline__ void bar_compute() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
// The same barrier, returning the OR of `p` over the compute threads: every
// compute warp takes the same decision from it.
__device__ __forceinline__ bool bar_compute_or(bool p) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, 256, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)p)
      : "memory");
  return r != 0;
}

// One box of a 4D tensor map (coordinates innermost first) into shared memory, completing on an mbarrier.
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                            int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, "
      "%6}], [%2];" ::"r"(dst),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
      : "memory");
}
__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&p);
}
// global -> shared bulk copy completing on an mbarrier (16-byte aligned, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// 32 consecutive TMEM columns of this warp's 32 lanes (one row per thread); the caller waits (tmem_wait_st)
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float (&v)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]), "f"(v[8]), "f"(v[9]),
      "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15]), "f"(v[16]), "f"(v[17]), "f"(v[18]),
      "f"(v[19]), "f"(v[20]), "f"(v[21]), "f"(v[22]), "f"(v[23]), "f"(v[24]), "f"(v[25]), "f"(v[26]), "f"(v[27]),
      "f"(v[28]), "f"(v[29]), "f"(v[30]), "f"(v[31])
      : "memory");
}

// byte offset of bf16 element (r, c) of a 128 x 128 operand (two 128B-swizzled 64-column slices)
__device__ __forceinline__ uint32_t op_off(int r, int c) {
  return (uint32_t)((c >> 6) * SLICE + r * 128 + ((((c & 63) >> 3) ^ (r & 7)) << 4) + (c & 7) * 2);
}

// Block i of latent g: six-hour blocks first, then one-hour blocks.
__device__ __forceinline__ const bf16* block_weights(const RolloutSmallArgs& a, int g, int i) {
  const int p6 = a.n6[g] * a.L6;
  return (i < p6 ? a.blk[i % a.L6] : a.blk[a.L6 + (i - p6) % a.L1]).w;
}

// LayerNorm of the thread's 64 columns (half hf of row r) with the partner
// half's partial sums exchanged through shared memory (two passes: mean, then
// the mean squared deviation), affine (gamma, beta: shared-memory vectors),
// rounded to bf16 into the A operand.
__device__ __forceinline__ void layernorm_to_a(uint8_t* smem, const float (&v)[64], int r, int hf,
                                               const float4* gamma, const float4* beta, float eps) {
  float* red = reinterpret_cast<float*>(smem + OFF_RED);
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < 64; ++j) s += v[j];
  red[hf * 128 + r] = s;
  bar_compute();
  const float mean = (red[r] + red[128 + r]) * (1.f / C);
  float q = 0.f;
#pragma unroll
  for (int j = 0; j < 64; ++j) {
    const float dv = v[j] - mean;
    q += dv * dv;
  }
  red[256 + hf * 128 + r] = q;
  bar_compute();
  const float rstd = rsqrtf((red[256 + r] + red[384 + r]) * (1.f / C) + eps);
  uint8_t* A = smem + OFF_A;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int j = 8 * k, c4 = (64 * hf + j) >> 2;
    const float4 g0 = gamma[c4], g1 = gamma[c4 + 1];
    const float4 b0 = beta[c4], b1 = beta[c4 + 1];
    const uint32_t w0 = pack_bf16((v[j] - mean) * rstd * g0.x + b0.x, (v[j + 1] - mean) * rstd * g0.y + b0.y);
    const uint32_t w1 = pack_bf16((v[j + 2] - mean) * rstd * g0.z + b0.z, (v[j + 3] - mean) * rstd * g0.w + b0.w);
    const uint32_t w2 = pack_bf16((v[j + 4] - mean) * rstd * g1.x + b1.x, (v[j + 5] - mean) * rstd * g1.y + b1.y);
    const uint32_t w3 = pack_bf16((v[j + 6] - mean) * rstd * g1.z + b1.z, (v[j + 7] - mean) * rstd * g1.w + b1.w);
    *reinterpret_cast<uint4*>(A + hf * SLICE + r * 128 + ((k ^ (r & 7)) << 4)) = make_uint4(w0, w1, w2, w3);
  }
}

// x += acc + bias over the thread's 64 columns (TMEM accumulator at acc_col,
// residual rows at T_X); the new values also into v.
__device__ __forceinline__ void residual_add(uint32_t tmem, uint32_t lane_off, uint32_t acc_col, int hf,
                                             const float4* bias, float (&v)[64]) {
#pragma unroll
  for (int sub = 0; sub < 2; ++sub) {
    const uint32_t col = (uint32_t)(64 * hf + 32 * sub);
    float acc[32], x[32];
    tmem_ld32(tmem + acc_col + col + lane_off, acc);
    tmem_ld32(tmem + T_X + col + lane_off, x);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float4 b = bias[(col >> 2) + q];
      x[4 * q] += acc[4 * q] + b.x;
      x[4 * q + 1] += acc[4 * q + 1] + b.y;
      x[4 * q + 2] += acc[4 * q + 2] + b.z;
      x[4 * q + 3] += acc[4 * q + 3] + b.w;
    }
    tmem_st32(tmem + T_X + col + lane_off, x);
#pragma unroll
    for (int j = 0; j < 32; ++j) v[32 * sub + j] = x[j];
  }
  tmem_wait_st();
}

// Bounded wait (all lanes of the warp take the result of lane 0's view).
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  return __all_sync(0xffffffffu, mbar_wait(bar, parity, abort_flag));
}

// Arrive on the latent's counter and wait until `target` CTAs have arrived,
// bounded in time. Every compute thread returns the same verdict.
__device__ __forceinline__ bool latent_barrier(unsigned int* counter, unsigned int target, int warp, int lane,
                                               volatile int* abort_flag) {
  bar_compute();   // every compute thread's global stores of this phase are issued
  int ok = 1;
  if (warp == 0) {
    if (lane == 0) {
      __threadfence();
      atomicAdd(counter, 1u);
      const unsigned long long t0 = globaltimer();
      while (true) {
        unsigned int v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(counter) : "memory");
        if (v >= target) break;
        if (*abort_flag || globaltimer() - t0 > kWaitLimitNs) {
          ok = 0;
          break;
        }
      }
      __threadfence();
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
  }
  return !bar_compute_or(!ok);
}

__global__ void __launch_bounds__(THREADS, 1) rollout_small_kernel(const __grid_constant__ RolloutSmallArgs a) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t w_full[NSLOT], w_empty[NSLOT], vec_full[2], vec_empty[2];
  __shared__ __align__(8) uint64_t a_full, mma_done, drain_bar, qkv_ready;
  __shared__ __align__(8) uint64_t acc1_full[2], acc1_empty[2], h_full[2], h_empty[2], kv_full[NKV], kv_empty[NKV];
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;

  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sbase = smem_u32(smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = blockIdx.x / a.T, tile = blockIdx.x % a.T;
  const int nb = a.n6[g] * a.L6 + a.n1[g] * a.L1;   // blocks of this latent's rollout (>= 1)
  const int steps = 4 * a.kd;                         // attention steps per block: (head, key level)

  // the patch: level d, latitudes h0 .. h0 + 7, longitudes w0 .. w0 + 15; its
  // key levels kd0 .. kd0 + kd - 1 and slab latitudes S0 .. S0 + SR - 1
  const int tpr = a.W / TW, tpl = (a.H / TH) * tpr;
  const int d = tile / tpl, h0 = ((tile % tpl) / tpr) * TH, w0 = (tile % tpr) * TW;
  const int rh = a.kh / 2;
  const int S0 = clampi(h0 - rh, 0, a.H - a.kh);
  const int SR = clampi(h0 + TH - 1 - rh, 0, a.H - a.kh) + a.kh - S0;
  const int kd0 = clampi(d - a.kd / 2, 0, a.D - a.kd);
  // K/V slab layout: 12 latitude rows x 20 longitudes of 64-byte key rows, one
  // box; where the patch's longitude halo wraps (w0 = 0 or W - 16), two boxes
  // side by side: columns 0-1 then 2-19, or 0-17 then 18-19
  const int wrap = w0 == 0 ? -1 : (w0 + TW + 2 > a.W ? 1 : 0);

  if (threadIdx.x == 0) {
    for (int b = 0; b < NSLOT; ++b) {
      mbar_init(&w_full[b], 1);
      mbar_init(&w_empty[b], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&vec_full[b], 1);
      mbar_init(&vec_empty[b], 8);
      mbar_init(&acc1_full[b], 1);
      mbar_init(&acc1_empty[b], 8);
      mbar_init(&h_full[b], 8);
      mbar_init(&h_empty[b], 1);
    }
    for (int b = 0; b < NKV; ++b) {
      mbar_init(&kv_full[b], 1);
      mbar_init(&kv_empty[b], 8);
    }
    mbar_init(&a_full, 8);
    mbar_init(&mma_done, 1);
    mbar_init(&drain_bar, 1);
    mbar_init(&qkv_ready, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == LOAD_WARP) {
    if (lane == 0) {
      // ---------------------------------------------- weights and vectors
      int slot = 0, par = 0;                // ring position and its use parity
      int last[NSLOT], last_vec[2] = {-1, -1};
      for (int b = 0; b < NSLOT; ++b) last[b] = -1;
      bool ok = true;
      auto load = [&](const bf16* src) -> bool {
        if (!mbar_wait(&w_empty[slot], (uint32_t)par ^ 1u, &abort_flag)) return false;
        mbar_expect_tx(&w_full[slot], CHUNK);
        bulk_g2s(sbase + OFF_W + slot * CHUNK, src, CHUNK, &w_full[slot]);
        last[slot] = par;
        if (++slot == NSLOT) {
          slot = 0;
          par ^= 1;
        }
        return true;
      };
      auto load_vec = [&](int j, const bf16* w) -> bool {
        const int b = j & 1;
        const uint32_t use = (uint32_t)(j >> 1) & 1u;
        if (!mbar_wait(&vec_empty[b], use ^ 1u, &abort_flag)) return false;
        mbar_expect_tx(&vec_full[b], VEC_BYTES);
        bulk_g2s(sbase + OFF_VEC + b * VEC_BYTES, w + (size_t)W_VEC * (CHUNK / 2), VEC_BYTES, &vec_full[b]);
        last_vec[b] = (int)use;
        return true;
      };
      constexpr int kOrder[9] = {W_O, W_1 + 0, W_1 + 1, W_2 + 0, W_1 + 2, W_2 + 1, W_1 + 3, W_2 + 2, W_2 + 3};
      const bf16* w0p = block_weights(a, g, 0);
      ok = load_vec(0, w0p);
      for (int c = 0; c < 3 && ok; ++c) ok = load(w0p + (size_t)(W_QKV + c) * (CHUNK / 2));
      for (int i = 0; i < nb && ok; ++i) {
        const bf16* w = block_weights(a, g, i);
#pragma unroll 1
        for (int q = 0; q < 9 && ok; ++q) ok = load(w + (size_t)kOrder[q] * (CHUNK / 2));
        if (ok && i + 1 < nb) {
          const bf16* wn = block_weights(a, g, i + 1);
          ok = load_vec(i + 1, wn);
          for (int c = 0; c < 3 && ok; ++c) ok = load(wn + (size_t)(W_QKV + c) * (CHUNK / 2));
        }
      }
      if (!ok) {
        abort_flag = 1;
        atomicExch(a.status, (int)WM_ERR_TIMEOUT);
        volatile int never = 0;
        for (int b = 0; b < NSLOT; ++b)
          if (last[b] >= 0) mbar_wait(&w_full[b], (uint32_t)last[b], &never);
        for (int b = 0; b < 2; ++b)
          if (last_vec[b] >= 0) mbar_wait(&vec_full[b], (uint32_t)last_vec[b], &never);
      }
    }
  } else if (warp == KV_WARP) {
    if (lane == 0) {
      // ------------------------------------------------- K/V tensor copies
      for (int k = 0; k < 3; ++k) asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&a.tm_kv[k]) : "memory");
      // boxes of 12 latitudes from S0 (rows past H read as zeros, rows past SR
      // are not used) x 20 longitudes, K and V
      const uint32_t kv_bytes = (uint32_t)(SR_MAX * SW * 64 * 2);
      int kst = 0, kpar = 0, last[NKV];   // ring position and its use parity
      for (int b = 0; b < NKV; ++b) last[b] = -1;
      bool ok = true;
      for (int i = 0; i < nb && ok; ++i) {
        // the latent's q, k, v of block i are complete
        if (!mbar_wait(&qkv_ready, (uint32_t)i & 1u, &abort_flag)) {
          ok = false;
          break;
        }
        // the q, k, v rows were written by generic stores (this and other CTAs);
        // the tensor copies below read them through the async proxy
        asm volatile("fence.proxy.async.global;" ::: "memory");
        for (int s = 0; s < steps; ++s) {
          const int b = kst;
          const uint32_t use = (uint32_t)kpar;
          if (!mbar_wait(&kv_empty[b], use ^ 1u, &abort_flag)) {
            ok = false;
            break;
          }
          const int h = s / a.kd, lev = ((i & 1) * a.G + g) * a.D + kd0 + s % a.kd;
          // debug builds: the boxes start inside the q, k, v array (a failed
          // check still issues the copies from coordinate 0, so the stage completes)
          const bool coords = WM_DCHECK(S0 >= 0 && S0 < a.H && lev >= 0 && lev < 2 * a.G * a.D &&
                                            (wrap != 0 || (w0 - 2 >= 0 && w0 - 2 + SW <= a.W)),
                                        a.status);
          mbar_expect_tx(&kv_full[b], kv_bytes);
          const uint32_t dst0 = sbase + kv_stage_off(b);
#pragma unroll
          for (int kv = 0; kv < 2; ++kv) {
            const int ch = C + kv * C + h * DH;
            const uint32_t dst = dst0 + kv * KV_SLAB;
            if (!coords) {
              tma_load_4d(dst, &a.tm_kv[0], &kv_full[b], ch, 0, 0, 0);
            } else if (wrap == 0) {
              tma_load_4d(dst, &a.tm_kv[0], &kv_full[b], ch, w0 - 2, S0, lev);
            } else if (wrap < 0) {
              tma_load_4d(dst, &a.tm_kv[2], &kv_full[b], ch, a.W - 2, S0, lev);
              tma_load_4d(dst + SR_MAX * 2 * 64, &a.tm_kv[1], &kv_full[b], ch, 0, S0, lev);
            } else {
              tma_load_4d(dst, &a.tm_kv[1], &kv_full[b], ch, a.W - 18, S0, lev);
              tma_load_4d(dst + SR_MAX * 18 * 64, &a.tm_kv[2], &kv_full[b], ch, 0, S0, lev);
            }
          }
          last[b] = (int)use;
          if (++kst == NKV) {
            kst = 0;
            kpar ^= 1;
          }
        }
      }
      if (!ok) {
        abort_flag = 1;
        atomicExch(a.status, (int)WM_ERR_TIMEOUT);
        volatile int never = 0;
        for (int b = 0; b < NKV; ++b)
          if (last[b] >= 0) mbar_wait(&kv_full[b], (uint32_t)last[b], &never);
      }
    }
  } else if (warp == MMA_WARP) {
    if (lane == 0) {
      // ------------------------------------------------------- MMA issuer
      constexpr uint32_t idesc = idesc_bf16(128, 128);
      int slot = 0, par = 0, a_cnt = 0;
      bool ok = true;
      // one 128 x 128 x 128 product: A operand at a_addr, the next weight chunk of the ring
      auto gemm = [&](uint32_t col, uint32_t a_addr, bool acc_in) -> bool {
        if (!mbar_wait(&w_full[slot], (uint32_t)par, &abort_flag)) return false;
        tc_fence_after();
        const uint32_t b_addr = sbase + OFF_W + slot * CHUNK;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          const uint64_t ad = sw128_desc(a_addr + s * SLICE), bd = sw128_desc(b_addr + s * SLICE);
#pragma unroll
          for (int k = 0; k < 4; ++k)
            umma_bf16<false>(tmem + col, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), idesc,
                             (acc_in || s || k) ? 1u : 0u);
        }
        umma_commit(&w_empty[slot]);
        if (++slot == NSLOT) {
          slot = 0;
          par ^= 1;
        }
        return true;
      };
      auto wait_a = [&]() -> bool {
        const bool r = mbar_wait(&a_full, (uint32_t)(a_cnt++) & 1u, &abort_flag);
        tc_fence_after();
        return r;
      };
      const uint32_t A = sbase + OFF_A;
      auto qkv = [&]() -> bool {
        if (!wait_a()) return false;
        for (int c = 0; c < 3; ++c)
          if (!gemm(T_ACC1 + 128 * c, A, false)) return false;
        umma_commit(&mma_done);
        return true;
      };
      auto fc1 = [&](int j) -> bool {
        const int b = j & 1;
        if (j >= 2 && !mbar_wait(&acc1_empty[b], 0u, &abort_flag)) return false;
        tc_fence_after();
        if (!gemm(T_ACC1 + 128 * b, A, false)) return false;
        umma_commit(&acc1_full[b]);
        return true;
      };
      auto fc2 = [&](int j) -> bool {
        const int b = j & 1;
        if (!mbar_wait(&h_full[b], (uint32_t)(j >> 1), &abort_flag)) return false;
        tc_fence_after();
        if (!gemm(T_ACC2, sbase + OFF_H + b * CHUNK, j > 0)) return false;
        umma_commit(&h_empty[b]);
        return true;
      };
      ok = qkv();
      for (int i = 0; i < nb && ok; ++i) {
        ok = wait_a() && gemm(T_PROJ, A, false);
        if (!ok) break;
        umma_commit(&mma_done);
        ok = wait_a() && fc1(0) && fc1(1) && fc2(0) && fc1(2) && fc2(1) && fc1(3) && fc2(2) && fc2(3);
        if (!ok) break;
        umma_commit(&mma_done);
        if (i + 1 < nb) ok = qkv();
      }
      if (!ok) {
        abort_flag = 1;
        atomicExch(a.status, (int)WM_ERR_TIMEOUT);
      }
      // every MMA issued so far completes before TMEM and shared memory are released
      umma_commit(&drain_bar);
      volatile int never = 0;
      mbar_wait(&drain_bar, 0u, &never);
    }
  } else if (warp < 8) {
    // ------------------------------------------------------ compute warps
    const int r = 32 * (warp & 3) + lane, hf = warp >> 2;   // epilogue row and column half
    const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
    const long N = (long)a.D * a.H * a.W;
    const int tok_r = (d * a.H + h0 + (r >> 4)) * a.W + w0 + (r & 15);
    float* xg = a.x[g] + (long)tok_r * C + 64 * hf;
    int md = 0;          // mma_done completions waited for
    bool ok = true;
    float v[64];

    // attention geometry of this warp: a 4 x 4 query group (rows g8, g8 + 8 of the m16 tile)
    const int gr = warp >> 2, gc = warp & 3, g8 = lane >> 2, t4 = lane & 3;
    const int rw = a.kw / 2;
    int R0 = min(clampi(h0 + 4 * gr - rh, 0, a.H - a.kh) - S0, SR - 8);
    const int qh0 = h0 + 4 * gr + (g8 >> 2), qh1 = qh0 + 2, qcl = g8 & 3;
    const uint32_t kmask = (1u << a.kh) - 1u;
    int sh0 = clampi(qh0 - rh, 0, a.H - a.kh) - S0 - R0, sh1 = clampi(qh1 - rh, 0, a.H - a.kh) - S0 - R0;
    // debug builds: the warp's 8-row key rectangle lies in the slab and holds
    // both query rows' latitude windows; on failure the warp reads rows 0-7
    if (!(WM_DCHECK(SR >= 8 && SR <= SR_MAX && R0 >= 0 && R0 + 8 <= SR, a.status) &&
          WM_DCHECK(sh0 >= 0 && sh0 + a.kh <= 8 && sh1 >= 0 && sh1 + a.kh <= 8, a.status))) {
      R0 = 0;
      sh0 = sh1 = 0;
    }
    const uint32_t lat0 = kmask << sh0;
    const uint32_t lat1 = kmask << sh1;
    const bool lon0 = abs(2 * t4 - 2 - qcl) <= rw, lon1 = abs(2 * t4 + 1 - 2 - qcl) <= rw;
    const int tq0 = (d * a.H + qh0) * a.W + w0 + 4 * gc + qcl, tq1 = tq0 + 2 * a.W;
    const int ri0 = (4 * gr + (g8 >> 2)) * TW + 4 * gc + qcl, ri1 = ri0 + 2 * TW;
    // byte offset in a K (or V) slab of 16-byte unit u of the key at slab row
    // lr, column c; the 64-byte swizzle of the tensor copies moves unit u of
    // the row at offset o to u ^ ((o >> 7) & 3)
    auto kv_off = [&](int lr, int c, int u) -> uint32_t {
      int o;
      if (wrap == 0) o = (lr * SW + c) * 64;
      else if (wrap < 0) o = c < 2 ? (lr * 2 + c) * 64 : SR_MAX * 2 * 64 + (lr * 18 + c - 2) * 64;
      else o = c < 18 ? (lr * 18 + c) * 64 : SR_MAX * 18 * 64 + (lr * 2 + c - 18) * 64;
      o += u * 16;
      return (uint32_t)(o ^ (((o >> 7) & 3) << 4));
    };
    // ldmatrix row addresses: K rows per n8 block, V rows per (k16 step, matrix pair)
    uint32_t koff[8], voff[4][2];
#pragma unroll
    for (int b = 0; b < 8; ++b) koff[b] = kv_off(R0 + b, 4 * gc + (lane & 7), lane >> 3);
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int np = 0; np < 2; ++np) {
        const int mi = lane >> 3;
        voff[q][np] = KV_SLAB + kv_off(R0 + 2 * q + (mi & 1), 4 * gc + (lane & 7), 2 * np + (mi >> 1));
      }
    int kst = 0, kpar = 0;   // K/V ring position and its use parity

    auto vec = [&](int j) -> const float4* { return reinterpret_cast<const float4*>(smem + OFF_VEC + (j & 1) * VEC_BYTES); };
    // QKV epilogue: + bias, bf16. The 128 x 384 tile is staged in shared memory
    // (chunk 0 in the A operand, chunks 1 and 2 in the GELU region, all free
    // once the QKV MMAs are done) in the operand layout, then written to the
    // global qkv array of block buffer `buf` in whole rows: the patch's 16
    // tokens of a latitude are 12 KB of consecutive memory.
    auto qkv_epilogue = [&](const float4* vb, int buf) {
      ok = warp_wait(&mma_done, (uint32_t)(md++) & 1u, &abort_flag) && ok;
      if (!ok) abort_flag = 1;
      tc_fence_after();
      const float4* bq = vb + V_BQKV / 4;
#pragma unroll 1
      for (int c = 0; c < 3; ++c) {
        uint8_t* stg = smem + (c == 0 ? OFF_A : OFF_H + (c - 1) * CHUNK) + hf * SLICE + r * 128;
#pragma unroll 1
        for (int sub = 0; sub < 2; ++sub) {
          const int col = 128 * c + 64 * hf + 32 * sub;
          float acc[32];
          tmem_ld32(tmem + T_ACC1 + (uint32_t)col + lane_off, acc);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float4 b0 = bq[(col >> 2) + 2 * k], b1 = bq[(col >> 2) + 2 * k + 1];
            const int j = 8 * k;
            *reinterpret_cast<uint4*>(stg + (((4 * sub + k) ^ (r & 7)) << 4)) =
                make_uint4(pack_bf16(acc[j] + b0.x, acc[j + 1] + b0.y), pack_bf16(acc[j + 2] + b0.z, acc[j + 3] + b0.w),
                           pack_bf16(acc[j + 4] + b1.x, acc[j + 5] + b1.y), pack_bf16(acc[j + 6] + b1.z, acc[j + 7] + b1.w));
          }
        }
      }
      tc_fence_before();
      bar_compute();
      // 16-byte piece p (0 .. 47) of tile row rr, consecutive threads along a row
      bf16* dst = a.qkv + ((long)buf * a.G + g) * N * QKV;
#pragma unroll 4
      for (int it = threadIdx.x; it < 128 * 48; it += 256) {
        const int rr = it / 48, p = it - rr * 48;
        const int c = p >> 4, sl = (p >> 3) & 1, u = p & 7;
        const uint8_t* src = smem + (c == 0 ? OFF_A : OFF_H + (c - 1) * CHUNK) + sl * SLICE + rr * 128 + ((u ^ (rr & 7)) << 4);
        const int tok = (d * a.H + h0 + (rr >> 4)) * a.W + w0 + (rr & 15);
        *reinterpret_cast<uint4*>(dst + (long)tok * QKV + 8 * p) = *reinterpret_cast<const uint4*>(src);
      }
    };
    auto a_ready = [&]() {
      fence_async_smem();   // generic-proxy stores, read by the tensor core next
      __syncwarp();
      if (lane == 0) mbar_arrive(&a_full);
    };

    // ---- prologue: residual rows into TMEM, LayerNorm 1 of block 0, QKV, latent barrier
    {
      const float4* src = reinterpret_cast<const float4*>(xg);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const float4 x = src[q];
        v[4 * q] = x.x;
        v[4 * q + 1] = x.y;
        v[4 * q + 2] = x.z;
        v[4 * q + 3] = x.w;
      }
#pragma unroll
      for (int sub = 0; sub < 2; ++sub) {
        float t[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) t[j] = v[32 * sub + j];
        tmem_st32(tmem + T_X + (uint32_t)(64 * hf + 32 * sub) + lane_off, t);
      }
      tmem_wait_st();
      ok = warp_wait(&vec_full[0], 0u, &abort_flag) && ok;
      layernorm_to_a(smem, v, r, hf, vec(0) + V_LN1G / 4, vec(0) + V_LN1B / 4, a.eps);
      a_ready();
      qkv_epilogue(vec(0), 0);
    }
    unsigned int epoch = 0;
    bool run = latent_barrier(a.bar + g, (++epoch) * (unsigned)a.T, warp, lane, &abort_flag) && !bar_compute_or(!ok);
    if (run && threadIdx.x == 0) mbar_arrive(&qkv_ready);

    for (int i = 0; i < nb && run; ++i) {
      const float4* vb = vec(i);
      const bf16* qkv_cur = a.qkv + ((long)(i & 1) * a.G + g) * N * QKV;
      // ------------------------------------------------ neighborhood attention
      {
        // this lane's query rows of head h (A fragments of the two k16 steps)
        auto load_q = [&](int h, uint32_t (&q)[2][4]) {
          const bf16* q0 = qkv_cur + (long)tq0 * QKV + h * DH + 2 * t4;
          const bf16* q1 = qkv_cur + (long)tq1 * QKV + h * DH + 2 * t4;
#pragma unroll
          for (int kk = 0; kk < 2; ++kk) {
            q[kk][0] = __ldcg(reinterpret_cast<const unsigned int*>(q0 + 16 * kk));
            q[kk][1] = __ldcg(reinterpret_cast<const unsigned int*>(q1 + 16 * kk));
            q[kk][2] = __ldcg(reinterpret_cast<const unsigned int*>(q0 + 16 * kk + 8));
            q[kk][3] = __ldcg(reinterpret_cast<const unsigned int*>(q1 + 16 * kk + 8));
          }
        };
        float o[4][4], l0 = 0.f, l1 = 0.f, m0 = -INFINITY, m1 = -INFINITY;
        uint32_t qa[2][4], qn[2][4];
        load_q(0, qn);
#pragma unroll 1
        for (int s = 0; s < steps; ++s) {
          const int h = s / a.kd, lv = s % a.kd;
          ok = warp_wait(&kv_full[kst], (uint32_t)kpar, &abort_flag) && ok;
          if (!ok) abort_flag = 1;
          if (lv == 0) {
#pragma unroll
            for (int kk = 0; kk < 2; ++kk)
#pragma unroll
              for (int e = 0; e < 4; ++e) qa[kk][e] = qn[kk][e];
            if (h + 1 < 4) load_q(h + 1, qn);   // the next head's queries, in flight during this head
#pragma unroll
            for (int nb8 = 0; nb8 < 4; ++nb8) o[nb8][0] = o[nb8][1] = o[nb8][2] = o[nb8][3] = 0.f;
            l0 = l1 = 0.f;
            m0 = m1 = -INFINITY;
          }
          const uint32_t kb = sbase + kv_stage_off(kst);
          // S = Q K^T over the 8 x 8 key rectangle (8 n8 blocks, one per rectangle row)
          float sc[8][4];
#pragma unroll
          for (int b = 0; b < 8; ++b) {
            uint32_t k0, k1, k2, k3;
            ldsm_x4(kb + koff[b], k0, k1, k2, k3);
            sc[b][0] = sc[b][1] = sc[b][2] = sc[b][3] = 0.f;
            mma16816(sc[b], qa[0], k0, k1);
            mma16816(sc[b], qa[1], k2, k3);
          }
          // mask (latitude row of the rectangle, longitude column) and scale to log2 units
          float mx0 = -INFINITY, mx1 = -INFINITY;
#pragma unroll
          for (int b = 0; b < 8; ++b) {
            const bool r0v = (lat0 >> b) & 1u, r1v = (lat1 >> b) & 1u;
            sc[b][0] = (r0v && lon0) ? sc[b][0] * a.scale_log2 : -INFINITY;
            sc[b][1] = (r0v && lon1) ? sc[b][1] * a.scale_log2 : -INFINITY;
            sc[b][2] = (r1v && lon0) ? sc[b][2] * a.scale_log2 : -INFINITY;
            sc[b][3] = (r1v && lon1) ? sc[b][3] * a.scale_log2 : -INFINITY;
            mx0 = fmaxf(mx0, fmaxf(sc[b][0], sc[b][1]));
            mx1 = fmaxf(mx1, fmaxf(sc[b][2], sc[b][3]));
          }
          mx0 = fmaxf(mx0, __shfl_xor_sync(0xffffffffu, mx0, 1));
          mx0 = fmaxf(mx0, __shfl_xor_sync(0xffffffffu, mx0, 2));
          mx1 = fmaxf(mx1, __shfl_xor_sync(0xffffffffu, mx1, 1));
          mx1 = fmaxf(mx1, __shfl_xor_sync(0xffffffffu, mx1, 2));
          const float mn0 = fmaxf(m0, mx0), mn1 = fmaxf(m1, mx1);   // finite: every level holds window keys
          const float al0 = ex2(m0 - mn0), al1 = ex2(m1 - mn1);
          m0 = mn0;
          m1 = mn1;
          l0 *= al0;
          l1 *= al1;
#pragma unroll
          for (int nb8 = 0; nb8 < 4; ++nb8) {
            o[nb8][0] *= al0;
            o[nb8][1] *= al0;
            o[nb8][2] *= al1;
            o[nb8][3] *= al1;
          }
          uint32_t pa[4][4];   // P as the A operand of the four k16 steps
#pragma unroll
          for (int b = 0; b < 8; ++b) {
            const float p0 = ex2(sc[b][0] - mn0), p1 = ex2(sc[b][1] - mn0);
            const float p2 = ex2(sc[b][2] - mn1), p3 = ex2(sc[b][3] - mn1);
            l0 += p0 + p1;
            l1 += p2 + p3;
            pa[b >> 1][(b & 1) * 2 + 0] = pack_bf16(p0, p1);
            pa[b >> 1][(b & 1) * 2 + 1] = pack_bf16(p2, p3);
          }
          // O += P V
#pragma unroll
          for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int np = 0; np < 2; ++np) {
              uint32_t v0, v1, v2, v3;
              ldsm_x4_t(kb + voff[q][np], v0, v1, v2, v3);
              mma16816(o[2 * np], pa[q], v0, v1);
              mma16816(o[2 * np + 1], pa[q], v2, v3);
            }
          // this warp is done with the stage
          __syncwarp();
          if (lane == 0) mbar_arrive(&kv_empty[kst]);
          if (++kst == NKV) {
            kst = 0;
            kpar ^= 1;
          }
          if (lv == a.kd - 1) {
            // head done: normalise, bf16 into the A operand (columns 32 h ..)
            float s0 = l0, s1 = l1;
            s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
            s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
            s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
            s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
            const float i0 = 1.f / s0, i1 = 1.f / s1;
#pragma unroll
            for (int nb8 = 0; nb8 < 4; ++nb8) {
              const int ch = h * DH + 8 * nb8 + 2 * t4;
              *reinterpret_cast<uint32_t*>(smem + OFF_A + op_off(ri0, ch)) = pack_bf16(o[nb8][0] * i0, o[nb8][1] * i0);
              *reinterpret_cast<uint32_t*>(smem + OFF_A + op_off(ri1, ch)) = pack_bf16(o[nb8][2] * i1, o[nb8][3] * i1);
            }
          }
        }
      }
      a_ready();
      // ------------------------------------------------ output projection + residual, LayerNorm 2
      ok = warp_wait(&mma_done, (uint32_t)(md++) & 1u, &abort_flag) && ok;
      if (!ok) abort_flag = 1;
      tc_fence_after();
      residual_add(tmem, lane_off, T_PROJ, hf, vb + V_BO / 4, v);
      tc_fence_before();
      layernorm_to_a(smem, v, r, hf, vb + V_LN2G / 4, vb + V_LN2B / 4, a.eps);
      a_ready();
      // ------------------------------------------------ MLP: FC1 chunks -> GELU -> shared memory
#pragma unroll 1
      for (int j = 0; j < 4; ++j) {
        const int b = j & 1;
        ok = warp_wait(&acc1_full[b], (uint32_t)(j >> 1), &abort_flag) && ok;
        if (!ok) abort_flag = 1;
        tc_fence_after();
        uint8_t* H = smem + OFF_H + b * CHUNK + hf * SLICE;
#pragma unroll 1
        for (int sub = 0; sub < 2; ++sub) {
          const int c = 64 * hf + 32 * sub;
          float acc[32];
          tmem_ld32(tmem + T_ACC1 + (uint32_t)(128 * b + c) + lane_off, acc);
          if (sub == 1) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc1_empty[b]);
          }
          const float4* b1 = vb + (V_B1 + 128 * j + c) / 4;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 bb = b1[q];
            acc[4 * q] += bb.x;
            acc[4 * q + 1] += bb.y;
            acc[4 * q + 2] += bb.z;
            acc[4 * q + 3] += bb.w;
          }
#pragma unroll
          for (int jj = 0; jj < 32; jj += 2) gelu_erf2(acc[jj], acc[jj + 1]);
          if (sub == 0 && j >= 2) {
            // this slot's previous chunk has been read by FC2
            ok = warp_wait(&h_empty[b], 0u, &abort_flag) && ok;
            if (!ok) abort_flag = 1;
          }
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            uint32_t w[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) w[e] = pack_bf16(acc[8 * k + 2 * e], acc[8 * k + 2 * e + 1]);
            *reinterpret_cast<uint4*>(H + r * 128 + (((4 * sub + k) ^ (r & 7)) << 4)) = make_uint4(w[0], w[1], w[2], w[3]);
          }
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&h_full[b]);
      }
      // ------------------------------------------------ FC2 + residual
      ok = warp_wait(&mma_done, (uint32_t)(md++) & 1u, &abort_flag) && ok;
      if (!ok) abort_flag = 1;
      tc_fence_after();
      residual_add(tmem, lane_off, T_ACC2, hf, vb + V_B2 / 4, v);
      tc_fence_before();
      // block i's vectors are no longer needed: their slot may take block i + 2's
      __syncwarp();
      if (lane == 0) mbar_arrive(&vec_empty[i & 1]);
      if (i + 1 < nb) {
        // ------------------------------------------------ next block: LayerNorm 1, QKV, latent barrier
        ok = warp_wait(&vec_full[(i + 1) & 1], (uint32_t)((i + 1) >> 1) & 1u, &abort_flag) && ok;
        if (!ok) abort_flag = 1;
        const float4* vn = vec(i + 1);
        layernorm_to_a(smem, v, r, hf, vn + V_LN1G / 4, vn + V_LN1B / 4, a.eps);
        a_ready();
        qkv_epilogue(vn, (i + 1) & 1);
        run = latent_barrier(a.bar + g, (++epoch) * (unsigned)a.T, warp, lane, &abort_flag);
        run = !bar_compute_or(!ok) && run;
        if (run && threadIdx.x == 0) mbar_arrive(&qkv_ready);
      } else {
        run = !bar_compute_or(!ok);
        if (run) {
          float4* dst = reinterpret_cast<float4*>(xg);
#pragma unroll
          for (int q = 0; q < 16; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        }
      }
    }
    if (!run) {
      abort_flag = 1;
      atomicCAS(a.status, 0, (int)WM_ERR_TIMEOUT);
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// One 128 x 128 chunk W[r0 + n][c0 + k] (row stride ld floats) as bf16 in the
// 128B-swizzled K-major layout the MMA reads: column k of row n in slice
// k / 64, 16-byte unit (k % 64) / 8 stored at unit ^ (n % 8).
__global__ void swizzle_chunk_kernel(const float* __restrict__ W, int ld, bf16* __restrict__ out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 128 * 16) return;
  const int n = idx >> 4, uk = idx & 15;
  const float* s = W + (size_t)n * ld + 8 * uk;
  uint32_t w[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) w[e] = pack_bf16(s[2 * e], s[2 * e + 1]);
  uint8_t* o = reinterpret_cast<uint8_t*>(out) + (uk >> 3) * SLICE + n * 128 + (((uk & 7) ^ (n & 7)) << 4);
  *reinterpret_cast<uint4*>(o) = make_uint4(w[0], w[1], w[2], w[3]);
}

}  // namespace rs

wm_status launch_swizzle_chunk(const float* W, int ld, __nv_bfloat16* out, cudaStream_t s) {
  rs::swizzle_chunk_kernel<<<8, 256, 0, s>>>(W, ld, out);
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

int rollout_small_capacity() {
  static int cap = -1;
  if (cap >= 0) return cap;
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaFuncSetAttribute(rs::rollout_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, rs::SMEM) !=
      cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, rs::rollout_small_kernel, rs::THREADS, rs::SMEM) !=
      cudaSuccess)
    return 0;
  cap = per * sms;
  return cap;
}

wm_status launch_rollout_small(const RolloutSmallArgs& a, cudaStream_t s) {
  const int grid = a.G * a.T;
  if (a.G < 1 || a.G > kRolloutSmallMaxLatents || grid > rollout_small_capacity())
    return fail(WM_ERR_INVALID_ARG, "small-latent rollout kernel: too many tiles for one cooperative launch");
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(rs::THREADS);
  cfg.dynamicSmemBytes = rs::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  WM_CUDA(cudaLaunchKernelEx(&cfg, rs::rollout_small_kernel, a));
  return WM_OK;
}

}  // namespace wm
