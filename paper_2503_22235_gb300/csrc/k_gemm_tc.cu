// BF16 GEMM on the 5th-generation tensor cores (tcgen05) for the processor's
// linear layers: out = epilogue(A[M,K] . W[N,K]^T + bias), FP32 accumulation
// in tensor memory.
//
// Persistent, warp-specialised kernel, one CTA per SM:
//   warp 0     TMA producer: A (128 x 64) and W (BN x 64) k-slices into a
//              STAGES-deep shared-memory ring (128-byte swizzle), mbarrier
//              expect-tx completion.
//   warp 1     MMA issuer: one thread issues tcgen05.mma (M=128, N=BN, K=16)
//              into one of two TMEM accumulators; tcgen05.commit frees the
//              smem stage and, after the last k-slice, hands the accumulator
//              to the epilogue.
//   warps 2-9  epilogue: tcgen05.ld (32x32b) rows out of TMEM, add bias, then
//              bf16 store, GELU + bf16 store, or FP32 residual add, while the
//              MMA warp already fills the other accumulator.
// Pair mode (BN = 256, PAIR): a cluster of two CTAs on two SMs computes a
// 256 x 256 tile with tcgen05.mma.cta_group::2 (M = 256). Each CTA loads its
// own 128 A rows and its own 128 of the tile's 256 W rows, so each SM's
// shared memory takes 32 KB per 64-deep k-slice instead of 48 KB and its
// tensor core reads the same, while each SM still produces a 128 x 256
// accumulator in its own TMEM for its own epilogue. The even CTA's MMA
// thread issues for both. Both CTAs' tensor copies (cta_group::2) complete
// on the even CTA's stage barrier, which expects the bytes of both; the even
// CTA's commits arrive on both CTAs' stage and accumulator barriers
// (multicast); every epilogue warp of both CTAs releases an accumulator on
// the even CTA's barrier.
// Every mbarrier wait is bounded in time; on a timeout the CTA records
// WM_ERR_TIMEOUT in the device status word, drains its own copies and MMAs,
// frees TMEM and returns.
#include <cuda_fp8.h>

#include "tc_gemm.cuh"

namespace wm {
namespace tc {

constexpr int BM = 128;
constexpr int BKB = 128;               // bytes per k-slice row (bf16: 64 elements, e4m3: 128)
constexpr int NUM_EPI_WARPS = 8;
constexpr int THREADS = 32 * (2 + NUM_EPI_WARPS);

// DUAL: a second (bf16) staging tile per epilogue warp; PAIR: this CTA holds half of the W tile
template <int BN, bool DUAL = false, bool PAIR = false>
struct Cfg {
  static constexpr int A_BYTES = BM * BKB;
  static constexpr int B_BYTES = (PAIR ? BN / 2 : BN) * BKB;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int STAGES = PAIR ? (DUAL ? 5 : 6) : (BN >= 256) ? (DUAL ? 3 : 4) : (DUAL ? 5 : 6);
  static constexpr int EPI_STRIDE = DUAL ? 6144 : 4096;     // per epilogue warp: 32x32 fp32 (+ 32x32 bf16)
  static constexpr int EPI_BYTES = NUM_EPI_WARPS * EPI_STRIDE;
  static constexpr int SMEM = STAGES * STAGE_BYTES + EPI_BYTES + 1024;   // + alignment slack
  static constexpr int TMEM_COLS = 2 * BN;                   // two accumulators
};

using namespace ptx;

// The same into this CTA's shared memory, completing on the mbarrier of either
// CTA of the pair (bar_cluster: a shared::cluster address).
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap* map, uint32_t bar_cluster, int c0,
                                                 int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
      "%4}], [%2];" ::"r"(dst),
      "l"((uint64_t)map), "r"(bar_cluster), "r"(c0), "r"(c1)
      : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
      ::"r"(dst), "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
      : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, uint32_t src, int c0, int c1) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"((uint64_t)map),
               "r"(src), "r"(c0), "r"(c1)
               : "memory");
}
__device__ __forceinline__ void tma_reduce_add_2d(const CUtensorMap* map, uint32_t src, int c0, int c1) {
  asm volatile("cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.tile.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                   (uint64_t)map),
               "r"(src), "r"(c0), "r"(c1)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// all but the most recent bulk group have finished reading shared memory
__device__ __forceinline__ void bulk_wait_read_1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Write this thread's row of a 32 x 32 output chunk into the warp's staging
// tile in the layout the output tensor map expects: bf16 rows of 64 bytes with
// the 64-byte swizzle (16-byte unit k of row r at k ^ ((r >> 1) & 3)), or fp32
// rows of 128 bytes with the 128-byte swizzle (unit k at k ^ (r & 7)). The
// swizzles keep the 32 row-parallel stores free of bank conflicts.
template <int EPI>
__device__ __forceinline__ void stage_row(uint8_t* buf, const float (&x)[32], int r) {
  if constexpr (EPI == EPI_GELU_F8) {
    // e4m3 rows of 32 bytes with the 32-byte swizzle (unit k of row r at k ^ ((r >> 2) & 1));
    // x is already divided by the output scale; RNE, saturating at +-448
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      uint32_t w[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int j = 16 * k + 4 * e;
        const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(x[j], x[j + 1]), __NV_SATFINITE, __NV_E4M3);
        const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(x[j + 2], x[j + 3]), __NV_SATFINITE, __NV_E4M3);
        w[e] = lo | (hi << 16);
      }
      *reinterpret_cast<uint4*>(buf + r * 32 + ((k ^ ((r >> 2) & 1)) << 4)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  } else if constexpr (EPI == EPI_STORE || EPI == EPI_GELU) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      uint32_t w[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        __nv_bfloat162 p = __floats2bfloat162_rn(x[8 * k + 2 * e], x[8 * k + 2 * e + 1]);
        w[e] = *reinterpret_cast<uint32_t*>(&p);
      }
      *reinterpret_cast<uint4*>(buf + r * 64 + ((k ^ ((r >> 1) & 3)) << 4)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k)
      *reinterpret_cast<float4*>(buf + r * 128 + ((k ^ (r & 7)) << 4)) =
          make_float4(x[4 * k], x[4 * k + 1], x[4 * k + 2], x[4 * k + 3]);
  }
}

template <int BN, int EPI, bool F8, bool DUAL = false, bool PAIR = false>
__global__ void __launch_bounds__(THREADS, 1)
    gemm_bf16_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                        const __grid_constant__ CUtensorMap tmC, const __grid_constant__ CUtensorMap tmC2, int M,
                        int N, int K, const EpiArgs e, int* __restrict__ status) {
  const float* __restrict__ bias = e.bias;
  const float alpha = e.alpha, out_scale = e.out_scale;
  constexpr bool kResLN = (EPI == EPI_RESID_LN);
  constexpr bool kLNF = (EPI == EPI_LNF_STORE || EPI == EPI_LNF_GELU);
  constexpr int BKE = F8 ? 128 : 64;     // elements per k-slice
  using CF = Cfg<BN, DUAL, PAIR>;
  static_assert(!PAIR || BN == 256, "pair tiles are 256 x 256");
  constexpr int TM = PAIR ? 2 * BM : BM;  // output rows per tile (of the CTA pair)
  constexpr int STAGES = CF::STAGES;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ __align__(8) uint64_t accf_bar[2];
  __shared__ __align__(8) uint64_t acce_bar[2];
  __shared__ __align__(8) uint64_t drain_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;

  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t smem_base = smem_u32(smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int num_n = (N + BN - 1) / BN;
  const int num_tiles = ((M + TM - 1) / TM) * num_n;
  const int nk = (K + BKE - 1) / BKE;
  // tiles are walked per CTA, or per CTA pair (both CTAs of a pair walk the same list)
  const uint32_t rank = PAIR ? cluster_ctarank() : 0u;
  const int unit = PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
  const int nunits = PAIR ? (int)(gridDim.x >> 1) : (int)gridDim.x;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      // (a pair's stage completes on the even CTA's barrier, with the bytes of both CTAs)
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf_bar[b], 1);
      mbar_init(&acce_bar[b], PAIR ? 2 * NUM_EPI_WARPS : NUM_EPI_WARPS);
    }
    mbar_init(&drain_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    if constexpr (PAIR) {
      // one warp of each CTA of the pair, collectively: the same columns in both SMs
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                   "r"(CF::TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                   "r"(CF::TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
  }
  tc_fence_before();
  __syncthreads();
  if constexpr (PAIR) cluster_sync();   // both CTAs' barriers and TMEM exist before any cross-CTA traffic
  tc_fence_after();
  const uint32_t tmem_base = tmem_slot;
  pdl_wait();      // the previous kernel's outputs (A, x, row statistics) are complete from here on
  pdl_trigger();

  if (warp == 0) {
    if (lane == 0) {
      // ---------------------------------------------------- TMA producer
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
      int stage = 0;
      uint32_t phase = 0;
      uint32_t issued_mask = 0, last_parity = 0;
      bool ok = true;
      for (int tile = unit; tile < num_tiles && ok; tile += nunits) {
        const int m0 = (tile / num_n) * TM + (int)rank * BM, n0 = (tile % num_n) * BN + (int)rank * (BN / 2);
        for (int kb = 0; kb < nk; ++kb) {
          if (!mbar_wait(&empty_bar[stage], phase ^ 1u, &abort_flag)) { ok = false; break; }
          const uint32_t sa = smem_base + stage * CF::STAGE_BYTES;
          if constexpr (PAIR) {
            if (rank == 0) mbar_expect_tx(&full_bar[stage], 2 * CF::STAGE_BYTES);
            const uint32_t fb = mapa_shared(smem_u32(&full_bar[stage]), 0);
            tma_load_2d_pair(sa, &tmA, fb, kb * BKE, m0);
            tma_load_2d_pair(sa + CF::A_BYTES, &tmB, fb, kb * BKE, n0);
          } else {
            mbar_expect_tx(&full_bar[stage], CF::STAGE_BYTES);
            tma_load_2d(sa, &tmA, &full_bar[stage], kb * BKE, m0);
            tma_load_2d(sa + CF::A_BYTES, &tmB, &full_bar[stage], kb * BKE, n0);
          }
          issued_mask |= 1u << stage;
          last_parity = (last_parity & ~(1u << stage)) | (phase << stage);
          if (++stage == STAGES) { stage = 0; phase ^= 1u; }
        }
      }
      if (!ok) {
        abort_flag = 1;
        atomicExch(status, (int)WM_ERR_TIMEOUT);
        // let our own copies land before the CTA's shared memory is released
        if (PAIR && rank != 0) {
          // they complete on the even CTA's barriers: give them a fixed 50 us
          const unsigned long long t0 = globaltimer();
          if (issued_mask != 0)
            while (globaltimer() - t0 < 50000ull) {
            }
        } else {
          for (int s = 0; s < STAGES; ++s)
            if (issued_mask & (1u << s)) {
              volatile int never = 0;
              mbar_wait(&full_bar[s], (last_parity >> s) & 1u, &never);
            }
        }
      }
    }
  } else if (warp == 1) {
    // (the odd CTA of a pair issues nothing here: the even CTA's thread issues the pair's MMAs)
    if (lane == 0 && !(PAIR && rank != 0)) {
      // ------------------------------------------------------ MMA issuer
      constexpr uint32_t idesc = F8 ? idesc_e4m3(TM, BN) : idesc_bf16(TM, BN);
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      int it = 0;
      for (int tile = unit; tile < num_tiles && ok; tile += nunits, ++it) {
        const int buf = it & 1;
        const uint32_t acc_par = (uint32_t)(it >> 1) & 1u;
        if (!(PAIR ? mbar_wait_cluster(&acce_bar[buf], acc_par ^ 1u, &abort_flag)
                   : mbar_wait(&acce_bar[buf], acc_par ^ 1u, &abort_flag))) { ok = false; break; }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(buf * BN);
        for (int kb = 0; kb < nk; ++kb) {
          if (!(PAIR ? mbar_wait_cluster(&full_bar[stage], phase, &abort_flag)
                     : mbar_wait(&full_bar[stage], phase, &abort_flag))) { ok = false; break; }
          tc_fence_after();
          const uint32_t sa = smem_base + stage * CF::STAGE_BYTES;
          const uint64_t adesc = sw128_desc(sa), bdesc = sw128_desc(sa + CF::A_BYTES);
#pragma unroll
          for (int k = 0; k < 4; ++k) {   // 4 MMAs of 32 bytes of K (16 bf16 / 32 e4m3) per slice
            if constexpr (F8)
              umma_e4m3<PAIR>(d_tmem, adesc + (uint64_t)(2 * k), bdesc + (uint64_t)(2 * k), idesc, (kb | k) != 0);
            else
              umma_bf16<PAIR>(d_tmem, adesc + (uint64_t)(2 * k), bdesc + (uint64_t)(2 * k), idesc, (kb | k) != 0);
          }
          if constexpr (PAIR) umma_commit_pair(&empty_bar[stage], 0x3);
          else umma_commit(&empty_bar[stage]);
          if (++stage == STAGES) { stage = 0; phase ^= 1u; }
        }
        if (!ok) break;
        if constexpr (PAIR) umma_commit_pair(&accf_bar[buf], 0x3);
        else umma_commit(&accf_bar[buf]);
      }
      if (!ok) {
        abort_flag = 1;
        atomicExch(status, (int)WM_ERR_TIMEOUT);
        // completes once every MMA issued above has finished
        if constexpr (PAIR) umma_commit_pair(&drain_bar, 0x1);
        else umma_commit(&drain_bar);
        volatile int never = 0;
        mbar_wait(&drain_bar, 0, &never);
      }
    }
  } else {
    // -------------------------------------------------------- epilogue
    const int quarter = warp & 3;                 // TMEM lane quarter this warp may access
    const int half = (warp - 2) >> 2;             // which half of the BN columns
    uint8_t* ebuf = smem + STAGES * CF::STAGE_BYTES + (warp - 2) * CF::EPI_STRIDE;
    const uint32_t ebuf32 = smem_u32(ebuf);
    uint8_t* ebuf2 = ebuf + 4096;                 // EPI_RESID_LN: the bf16 copy's staging tile
    const uint32_t ebuf2_32 = ebuf32 + 4096;
    // Narrow outputs (bf16: 2 KB per 32 x 32 chunk, e4m3: 1 KB) alternate
    // between two halves of the warp's 4 KB staging tile, so a chunk waits
    // only for the store of the chunk two before it.
    constexpr bool kPing = !kResLN && EPI != EPI_RESID_F32 && EPI != EPI_STORE_F32;
    constexpr int kChunkBytes = EPI == EPI_GELU_F8 ? 1024 : 2048;
    uint32_t staged = 0;                          // chunks this warp has staged (all tiles)
    int it = 0;
    for (int tile = unit; tile < num_tiles; tile += nunits, ++it) {
      const int buf = it & 1;
      const uint32_t acc_par = (uint32_t)(it >> 1) & 1u;
      if (!(PAIR ? mbar_wait_cluster(&accf_bar[buf], acc_par, &abort_flag)
                 : mbar_wait(&accf_bar[buf], acc_par, &abort_flag))) {
        abort_flag = 1;
        atomicExch(status, (int)WM_ERR_TIMEOUT);
        break;
      }
      tc_fence_after();
      const int m0 = (tile / num_n) * TM + (int)rank * BM, n0 = (tile % num_n) * BN;
      const int row0 = m0 + quarter * 32;
      const int m = row0 + lane;
      const uint32_t tbase = tmem_base + (uint32_t)(buf * BN) + ((uint32_t)(quarter * 32) << 16);
      const int c_begin = half * (BN / 2), c_end = (half + 1) * (BN / 2);
      // LayerNorm folded into this GEMM: merge the row's partial (mean, M2)
      // pairs (equal counts K / np each) into its mean and 1/sqrt(var + eps)
      float ln_mean = 0.f, ln_rstd = 0.f;
      if constexpr (kLNF) {
        if (m < M) {
          const float* st = e.stats + (size_t)m * e.np * 2;
          float mu = 0.f;
          for (int i = 0; i < e.np; ++i) mu += st[2 * i];
          mu /= (float)e.np;
          const float cnt = (float)K / (float)e.np;
          float m2 = 0.f;
          for (int i = 0; i < e.np; ++i) {
            const float d = st[2 * i] - mu;
            m2 += st[2 * i + 1] + cnt * d * d;
          }
          ln_mean = mu;
          ln_rstd = rsqrtf(m2 / (float)K + e.eps);
        }
      }
      // residual epilogue with row statistics: running Welford (count, mean, M2)
      float wn = 0.f, wmean = 0.f, wm2 = 0.f;
      float4 xa[kResLN ? 8 : 1];
      if constexpr (kResLN) {
#pragma unroll
        for (int q = 0; q < 8; ++q) xa[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        // debug builds: the tile's half lies inside the row (N % BN == 0 for this epilogue)
        if (row0 < M && m < M && n0 + c_begin < N && WM_DCHECK(n0 + c_end <= N, status)) {
          const float4* xo = reinterpret_cast<const float4*>(e.x + (size_t)m * N + n0 + c_begin);
#pragma unroll
          for (int q = 0; q < 8; ++q) xa[q] = xo[q];
        }
      }
#pragma unroll 1
      for (int c = c_begin; c < c_end; c += 32) {
        float v[32];
        tmem_ld32(tbase + (uint32_t)c, v);
        if (c + 32 >= c_end) {
          // last TMEM read of this tile: hand the accumulator back to the MMA warp
          // (of the even CTA, for a pair)
          tc_fence_before();
          __syncwarp();
          if (lane == 0) {
            if constexpr (PAIR) mbar_arrive_remote(mapa_shared(smem_u32(&acce_bar[buf]), 0));
            else mbar_arrive(&acce_bar[buf]);
          }
        }
        const int n = n0 + c;
        if (row0 >= M || n >= N) continue;   // whole chunk outside the output (warp-uniform)
        float lcs[kLNF ? 32 : 1], lbb[kLNF ? 32 : 1];
        if constexpr (kLNF) {   // column vectors of this chunk (N % 32 == 0 here)
          const float4* c4 = reinterpret_cast<const float4*>(e.colsum + n);
          const float4* b4 = reinterpret_cast<const float4*>(bias + n);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 a = __ldg(c4 + q), b = __ldg(b4 + q);
            lcs[4 * q] = a.x; lcs[4 * q + 1] = a.y; lcs[4 * q + 2] = a.z; lcs[4 * q + 3] = a.w;
            lbb[4 * q] = b.x; lbb[4 * q + 1] = b.y; lbb[4 * q + 2] = b.z; lbb[4 * q + 3] = b.w;
          }
        }
        if constexpr (kLNF) {
          // rstd (acc - mean colsum) + b', then GELU, two columns per instruction
          const uint64_t nmean2 = pack_f2(-ln_mean, -ln_mean), rstd2 = pack_f2(ln_rstd, ln_rstd);
#pragma unroll
          for (int j = 0; j < 32; j += 2) {
            float t0, t1;
            fma_f2(t0, t1, lcs[j], lcs[j + 1], nmean2, pack_f2(v[j], v[j + 1]));
            fma_f2(v[j], v[j + 1], t0, t1, rstd2, pack_f2(lbb[j], lbb[j + 1]));
            if constexpr (EPI == EPI_LNF_GELU) gelu_erf2(v[j], v[j + 1]);
          }
        } else if ((EPI == EPI_GELU || EPI == EPI_GELU_F8) && bias && n + 32 <= N) {
          // whole chunk with a bias: the same steps two columns per instruction
          const uint64_t alpha2 = pack_f2(alpha, alpha), oscale2 = pack_f2(out_scale, out_scale);
          const float4* b4 = reinterpret_cast<const float4*>(bias + n);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 b = __ldg(b4 + q);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int j = 4 * q + 2 * h;
              if constexpr (F8) mul_f2(v[j], v[j + 1], alpha2);
              add_f2(v[j], v[j + 1], v[j], v[j + 1], h ? b.z : b.x, h ? b.w : b.y);
              gelu_erf2(v[j], v[j + 1]);
              if constexpr (EPI == EPI_GELU_F8) mul_f2(v[j], v[j + 1], oscale2);
            }
          }
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            if constexpr (F8) v[j] *= alpha;
            v[j] += (bias && n + j < N) ? __ldg(bias + n + j) : 0.f;
            if constexpr (EPI == EPI_GELU || EPI == EPI_GELU_F8) v[j] = gelu_erf(v[j]);
            if constexpr (EPI == EPI_GELU_F8) v[j] *= out_scale;
          }
        }
        if constexpr (EPI == EPI_LNF_STORE) {
          if (e.rope != nullptr) {
            const RopeArgs& R = *e.rope;
            if (n < 2 * R.C && m < M) {
              // rotary embedding of q / k: this row's token position, then per pair
              const int tok = m % (R.D * R.H * R.W);
              const int pos[3] = {tok / (R.H * R.W), (tok / R.W) % R.H, tok % R.W};
#pragma unroll
              for (int jp = 0; jp < 16; ++jp) {
                const int p = ((n + 2 * jp) % R.C) % R.dh / 2;
                const int ax = p < R.n[0] ? 0 : (p < R.n[0] + R.n[1] ? 1 : 2);
                const int pm = p - (ax > 0 ? R.n[0] : 0) - (ax > 1 ? R.n[1] : 0);
                const float2 cs = __ldg(R.tab[ax] + pos[ax] * R.n[ax] + pm);
                const float a0 = v[2 * jp], a1 = v[2 * jp + 1];
                v[2 * jp] = a0 * cs.x - a1 * cs.y;
                v[2 * jp + 1] = a0 * cs.y + a1 * cs.x;
              }
            }
          }
        }
        if constexpr (kResLN) {
          // x_new = x_old + acc + bias (x_old loaded one chunk ahead), then the
          // chunk's mean / M2 merged into the row's (Chan et al.)
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            v[4 * q] += xa[q].x; v[4 * q + 1] += xa[q].y; v[4 * q + 2] += xa[q].z; v[4 * q + 3] += xa[q].w;
          }
          if (c + 32 < c_end && m < M) {
            const float4* xo = reinterpret_cast<const float4*>(e.x + (size_t)m * N + n + 32);
#pragma unroll
            for (int q = 0; q < 8; ++q) xa[q] = xo[q];
          }
          float cs = 0.f;
#pragma unroll
          for (int j = 0; j < 32; ++j) cs += v[j];
          const float cm = cs * (1.f / 32.f);
          float cq = 0.f;
#pragma unroll
          for (int j = 0; j < 32; ++j) cq += (v[j] - cm) * (v[j] - cm);
          const float nt = wn + 32.f, d = cm - wmean;
          wmean += d * (32.f / nt);
          wm2 += cq + d * d * (wn * 32.f / nt);
          wn = nt;
        }
        // the store that last used this staging buffer has read it
        if (lane == 0) {
          if constexpr (kPing) bulk_wait_read_1();
          else bulk_wait_read_all();
        }
        __syncwarp();
        const uint32_t soff = kPing ? (staged & 1u) * (uint32_t)kChunkBytes : 0u;
        ++staged;
        if constexpr (kResLN) stage_row<EPI_STORE_F32>(ebuf, v, lane);
        else if constexpr (kLNF) stage_row<EPI_STORE>(ebuf + soff, v, lane);
        else stage_row<EPI>(ebuf + soff, v, lane);
        fence_async_smem();
        __syncwarp();
        if (lane == 0) {
          if constexpr (EPI == EPI_RESID_F32)
            tma_reduce_add_2d(&tmC, ebuf32, n, row0);
          else
            tma_store_2d(&tmC, ebuf32 + soff, n, row0);
          bulk_commit();
        }
        if constexpr (kResLN) {
          // the bf16 copy of x_new for the next LayerNorm-folded GEMM: its own
          // staging tile (DUAL), or the fp32 one once its store has read it
          if constexpr (!DUAL) {
            if (lane == 0) bulk_wait_read_all();
            __syncwarp();
          }
          stage_row<EPI_STORE>(DUAL ? ebuf2 : ebuf, v, lane);
          fence_async_smem();
          __syncwarp();
          if (lane == 0) {
            tma_store_2d(&tmC2, DUAL ? ebuf2_32 : ebuf32, n, row0);
            bulk_commit();
          }
        }
      }
      if constexpr (kResLN) {
        if (row0 < M && m < M && wn > 0.f) {
          const int part = (n0 / BN) * 2 + half;
          float* st = e.stats + ((size_t)m * (2 * num_n) + part) * 2;
          st[0] = wmean;
          st[1] = wm2;
        }
      }
    }
    if (lane == 0) bulk_wait_all();
  }

  tc_fence_before();
  __syncthreads();
  // a pair leaves together: the even CTA's MMAs read the odd CTA's shared
  // memory, and both CTAs signal the even CTA's barriers
  if constexpr (PAIR) cluster_sync();
  if (warp == 0) {
    tc_fence_after();
    if constexpr (PAIR)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(CF::TMEM_COLS)
                   : "memory");
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(CF::TMEM_COLS)
                   : "memory");
  }
}

// How many two-CTA clusters of this kernel fit on the GPU at once (0 if none).
template <int BN, int EPI, bool F8, bool DUAL>
static int pair_capacity() {
  static int cap = -1;
  if (cap < 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * num_sms());
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = Cfg<BN, DUAL, true>::SMEM;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, gemm_bf16_tc_kernel<BN, EPI, F8, DUAL, true>, &cfg) != cudaSuccess) {
      cudaGetLastError();
      n = 0;
    }
    cap = n;
  }
  return cap;
}

template <int BN, int EPI, bool F8, bool DUAL = false, bool PAIR = false>
static wm_status launch_one(const GemmArgs& a, cudaStream_t s) {
  using CF = Cfg<BN, DUAL, PAIR>;
  auto kern = gemm_bf16_tc_kernel<BN, EPI, F8, DUAL, PAIR>;
  int grid;
  if constexpr (PAIR) {
    // persistent: every pair resident at once, each walking its share of the 256 x 256 tiles
    const int tiles = ((a.M + 2 * BM - 1) / (2 * BM)) * ((a.N + BN - 1) / BN);
    const int cap = pair_capacity<BN, EPI, F8, DUAL>();
    if (cap < 1) return fail(WM_ERR_CUDA, "no two-CTA cluster of the pair GEMM fits on this GPU");
    grid = 2 * (tiles < cap ? tiles : cap);
  } else {
    const int tiles = ((a.M + BM - 1) / BM) * ((a.N + BN - 1) / BN);
    grid = tiles < num_sms() ? tiles : num_sms();
  }
  EpiArgs e;
  e.bias = a.bias;
  e.colsum = a.colsum;
  e.x = a.x;
  e.stats = a.stats;
  e.np = a.np;
  e.eps = a.eps;
  e.alpha = a.alpha;
  e.out_scale = a.out_scale;
  e.rope = a.rope;
  if constexpr (PAIR)
    WM_CUDA(launch_pdl_pairs(kern, dim3(grid), dim3(THREADS), CF::SMEM, s, a.pdl, a.tmA, a.tmB, a.tmC, a.tmC2, a.M, a.N,
                             a.K, e, device_status_word()));
  else
    WM_CUDA(launch_pdl(kern, dim3(grid), dim3(THREADS), CF::SMEM, s, a.pdl, a.tmA, a.tmB, a.tmC, a.tmC2, a.M, a.N, a.K,
                       e, device_status_word()));
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

template <int BN, int EPI, bool F8, bool DUAL = false, bool PAIR = false>
static wm_status set_attr() {
  WM_CUDA(cudaFuncSetAttribute(gemm_bf16_tc_kernel<BN, EPI, F8, DUAL, PAIR>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<BN, DUAL, PAIR>::SMEM));
  return WM_OK;
}

template <int BN>
static wm_status set_attrs_bn() {
  wm_status st = WM_OK;
  auto chk = [&](wm_status x) { if (st == WM_OK) st = x; };
  chk(set_attr<BN, EPI_STORE, false>());
  chk(set_attr<BN, EPI_GELU, false>());
  chk(set_attr<BN, EPI_RESID_F32, false>());
  chk(set_attr<BN, EPI_STORE_F32, false>());
  chk(set_attr<BN, EPI_RESID_LN, false>());
  chk(set_attr<BN, EPI_RESID_LN, false, true>());
  chk(set_attr<BN, EPI_LNF_STORE, false>());
  chk(set_attr<BN, EPI_LNF_GELU, false>());
  chk(set_attr<BN, EPI_GELU_F8, true>());
  chk(set_attr<BN, EPI_RESID_F32, true>());
  chk(set_attr<BN, EPI_STORE_F32, true>());
  chk(set_attr<BN, EPI_RESID_LN, true>());
  chk(set_attr<BN, EPI_RESID_LN, true, true>());
  if constexpr (BN == 256) {
    // pair tiles: the epilogues of the processor block's GEMMs
    chk(set_attr<BN, EPI_RESID_LN, false, false, true>());
    chk(set_attr<BN, EPI_RESID_LN, false, true, true>());
    chk(set_attr<BN, EPI_LNF_STORE, false, false, true>());
    chk(set_attr<BN, EPI_LNF_GELU, false, false, true>());
    chk(set_attr<BN, EPI_GELU_F8, true, false, true>());
    chk(set_attr<BN, EPI_RESID_LN, true, false, true>());
    chk(set_attr<BN, EPI_RESID_LN, true, true, true>());
    chk(set_attr<BN, EPI_STORE, false, false, true>());
  }
  return st;
}

// The processor block's epilogues on 256 x 256 pair tiles (and a plain bf16
// store for the per-op tests).
static wm_status launch_pair(const GemmArgs& a, cudaStream_t s) {
  const bool dual = a.dual >= 0 ? a.dual == 1 : a.K <= 1024;
  if (a.f8) {
    switch (a.epi) {
      case EPI_GELU_F8: return launch_one<256, EPI_GELU_F8, true, false, true>(a, s);
      case EPI_RESID_LN:
        return dual ? launch_one<256, EPI_RESID_LN, true, true, true>(a, s)
                    : launch_one<256, EPI_RESID_LN, true, false, true>(a, s);
      default: return fail(WM_ERR_INVALID_ARG, "unsupported epilogue for the e4m3 pair GEMM");
    }
  }
  switch (a.epi) {
    case EPI_STORE: return launch_one<256, EPI_STORE, false, false, true>(a, s);
    case EPI_RESID_LN:
      return dual ? launch_one<256, EPI_RESID_LN, false, true, true>(a, s)
                  : launch_one<256, EPI_RESID_LN, false, false, true>(a, s);
    case EPI_LNF_STORE: return launch_one<256, EPI_LNF_STORE, false, false, true>(a, s);
    case EPI_LNF_GELU: return launch_one<256, EPI_LNF_GELU, false, false, true>(a, s);
    default: return fail(WM_ERR_INVALID_ARG, "unsupported epilogue for the bf16 pair GEMM");
  }
}

template <int BN>
static wm_status launch_bn(const GemmArgs& a, cudaStream_t s) {
  if (a.f8) {
    switch (a.epi) {
      case EPI_GELU_F8: return launch_one<BN, EPI_GELU_F8, true>(a, s);
      case EPI_RESID_F32: return launch_one<BN, EPI_RESID_F32, true>(a, s);
      case EPI_STORE_F32: return launch_one<BN, EPI_STORE_F32, true>(a, s);
      case EPI_RESID_LN:
        // short K: the epilogue dominates, give it a second staging tile (one stage fewer)
        return (a.dual >= 0 ? a.dual == 1 : a.K <= 1024) ? launch_one<BN, EPI_RESID_LN, true, true>(a, s)
                                                           : launch_one<BN, EPI_RESID_LN, true>(a, s);
      default: return fail(WM_ERR_INVALID_ARG, "unsupported epilogue for the e4m3 GEMM");
    }
  }
  switch (a.epi) {
    case EPI_STORE: return launch_one<BN, EPI_STORE, false>(a, s);
    case EPI_GELU: return launch_one<BN, EPI_GELU, false>(a, s);
    case EPI_RESID_F32: return launch_one<BN, EPI_RESID_F32, false>(a, s);
    case EPI_STORE_F32: return launch_one<BN, EPI_STORE_F32, false>(a, s);
    case EPI_RESID_LN:
      return (a.dual >= 0 ? a.dual == 1 : a.K <= 1024) ? launch_one<BN, EPI_RESID_LN, false, true>(a, s)
                                                         : launch_one<BN, EPI_RESID_LN, false>(a, s);
    case EPI_LNF_STORE: return launch_one<BN, EPI_LNF_STORE, false>(a, s);
    case EPI_LNF_GELU: return launch_one<BN, EPI_LNF_GELU, false>(a, s);
    default: return fail(WM_ERR_INVALID_ARG, "unsupported epilogue for the bf16 GEMM");
  }
}


// ------------------------------------------------------------ fused MLP ----
// The small latent's MLP (C = 128, hidden 4C = 512) in one persistent kernel
// per 128-row tile: FC1 with LayerNorm 2 folded into its epilogue and GELU,
// in four 128-column hidden chunks whose bf16 activations go to shared
// memory (never HBM), each chunk then the K slice of FC2 accumulating in
// tensor memory, and FC2's residual epilogue with the next LayerNorm's row
// statistics. Every output element is computed exactly as by the two
// separate GEMMs with 128-column tiles (the same K order in the MMAs, the
// same epilogue arithmetic, the same two statistics partials per row), so
// the results are bit for bit those of the unfused path.
//   warp 0     TMA producer: the tile's x rows (A of FC1), W1 and W2 chunks
//              (two-slot rings each).
//   warp 1     MMA issuer: FC1(0), FC1(1), then FC2(j) and FC1(j + 2).
//   warps 2-9  epilogue: lane quarter q = warp % 4 (rows 32q..32q+31), half
//              h = (warp - 2) / 4 (columns 64h..64h+63) of every chunk.
namespace mlp {
constexpr int C = 128, HID = 512, NCH = HID / C;
constexpr int SLICE = 128 * BKB;          // one 128-row x 64-column bf16 k-slice (16 KB)
constexpr int TILE = 2 * SLICE;           // 128 x 128 bf16 (32 KB)
constexpr int OFF_A = 0, OFF_W1 = TILE, OFF_H = 3 * TILE, OFF_W2 = 5 * TILE;
constexpr int SMEM = 7 * TILE + 1024;     // + alignment slack
constexpr uint32_t TMEM_ACC2 = 256;       // FC1 accumulators at columns 0 and 128, FC2's at 256
}  // namespace mlp

struct MlpEpi {
  const float* colsum1;   // column sums of the folded bf16 W1
  const float* bias1;     // folded FC1 bias
  const float* bias2;     // FC2 bias
  const float* stats_in;  // [M, np_in, 2] LayerNorm-2 partials (from the output projection)
  float* stats_out;       // [M, np_out, 2] LayerNorm-1 partials of the new residual
  float* x;               // fp32 residual [M, C], read and rewritten
  __nv_bfloat16* xb;      // bf16 copy of the new residual [M, C]
  int np_in;
  int np_out;             // 2: one partial per 64 columns; 4: one per 32 (as FC2 on 128- or 64-column tiles)
  float eps;
};

// bf16 rows of 32 columns into a 128-byte-swizzled K-major k-slice (the layout
// the MMA descriptors and a 128B-swizzled tensor copy use): 16-byte unit u
// of row r at u ^ (r & 7).
__device__ __forceinline__ void store_h_row(uint8_t* slice, int r, int unit0, const float (&v)[32]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    uint32_t w[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      __nv_bfloat162 pr = __floats2bfloat162_rn(v[8 * k + 2 * e], v[8 * k + 2 * e + 1]);
      w[e] = *reinterpret_cast<uint32_t*>(&pr);
    }
    *reinterpret_cast<uint4*>(slice + r * 128 + (((unit0 + k) ^ (r & 7)) << 4)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

__global__ void __launch_bounds__(THREADS, 1)
    mlp_small_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmW1,
                     const __grid_constant__ CUtensorMap tmW2, int M, const MlpEpi e, int* __restrict__ status) {
  using namespace mlp;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t a_full, a_empty, acc2_full, acc2_empty, drain_bar;
  __shared__ __align__(8) uint64_t w1_full[2], w1_empty[2], w2_full[2], w2_empty[2];
  __shared__ __align__(8) uint64_t acc1_full[2], acc1_empty[2], h_full[2], h_empty[2];
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;

  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sbase = smem_u32(smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int num_tiles = (M + BM - 1) / BM;

  if (threadIdx.x == 0) {
    mbar_init(&a_full, 1);
    mbar_init(&a_empty, 1);
    mbar_init(&acc2_full, 1);
    mbar_init(&acc2_empty, NUM_EPI_WARPS);
    mbar_init(&drain_bar, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&w1_full[b], 1);
      mbar_init(&w1_empty[b], 1);
      mbar_init(&w2_full[b], 1);
      mbar_init(&w2_empty[b], 1);
      mbar_init(&acc1_full[b], 1);
      mbar_init(&acc1_empty[b], NUM_EPI_WARPS);
      mbar_init(&h_full[b], NUM_EPI_WARPS);
      mbar_init(&h_empty[b], 1);
    }
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
  const uint32_t tmem_base = tmem_slot;
  pdl_wait();
  pdl_trigger();

  if (warp == 0) {
    if (lane == 0) {
      // ---------------------------------------------------- TMA producer
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmW1) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmW2) : "memory");
      // weight chunks in the order the MMA thread consumes them
      constexpr int kKind[8] = {1, 1, 2, 1, 2, 1, 2, 2};   // 1: W1 chunk, 2: W2 chunk
      constexpr int kChunk[8] = {0, 1, 0, 2, 1, 3, 2, 3};
      bool ok = true;
      // for the drain after a timeout: the parity of each barrier's last copies (-1: none)
      int last_a = -1, last_w1[2] = {-1, -1}, last_w2[2] = {-1, -1};
      int it = 0;
      for (int tile = blockIdx.x; tile < num_tiles && ok; tile += gridDim.x, ++it) {
        const int m0 = tile * BM;
        const uint32_t tp = (uint32_t)it & 1u;
        if (!mbar_wait(&a_empty, tp ^ 1u, &abort_flag)) { ok = false; break; }
        mbar_expect_tx(&a_full, TILE);
        for (int s = 0; s < 2; ++s) tma_load_2d(sbase + OFF_A + s * SLICE, &tmA, &a_full, s * 64, m0);
        last_a = (int)tp;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int j = kChunk[q], b = j & 1;
          const uint32_t use = (uint32_t)(2 * it + (j >> 1)) & 1u;
          uint64_t* full = kKind[q] == 1 ? &w1_full[b] : &w2_full[b];
          uint64_t* empty = kKind[q] == 1 ? &w1_empty[b] : &w2_empty[b];
          if (!mbar_wait(empty, use ^ 1u, &abort_flag)) { ok = false; break; }
          mbar_expect_tx(full, TILE);
          const uint32_t dst = sbase + (kKind[q] == 1 ? OFF_W1 : OFF_W2) + b * TILE;
          for (int s = 0; s < 2; ++s) {
            if (kKind[q] == 1) tma_load_2d(dst + s * SLICE, &tmW1, full, s * 64, j * C);
            else tma_load_2d(dst + s * SLICE, &tmW2, full, j * C + s * 64, 0);
          }
          if (kKind[q] == 1) last_w1[b] = (int)use;
          else last_w2[b] = (int)use;
        }
      }
      if (!ok) {
        abort_flag = 1;
        atomicExch(status, (int)WM_ERR_TIMEOUT);
        // let our own copies land before the CTA's shared memory is released
        volatile int never = 0;
        if (last_a >= 0) mbar_wait(&a_full, (uint32_t)last_a, &never);
        for (int b = 0; b < 2; ++b) {
          if (last_w1[b] >= 0) mbar_wait(&w1_full[b], (uint32_t)last_w1[b], &never);
          if (last_w2[b] >= 0) mbar_wait(&w2_full[b], (uint32_t)last_w2[b], &never);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------------ MMA issuer
      constexpr uint32_t idesc = idesc_bf16(BM, C);
      bool ok = true;
      int it = 0;
      for (int tile = blockIdx.x; tile < num_tiles && ok; tile += gridDim.x, ++it) {
        const uint32_t tp = (uint32_t)it & 1u;
        if (!mbar_wait(&a_full, tp, &abort_flag)) { ok = false; break; }
        tc_fence_after();
        // FC1 of hidden chunk j into accumulator j % 2 (K = C: two k-slices of 4 MMAs)
        auto fc1 = [&](int j) -> bool {
          const int b = j & 1;
          const uint32_t use = (uint32_t)(2 * it + (j >> 1)) & 1u;
          if (!mbar_wait(&w1_full[b], use, &abort_flag)) return false;
          if (!mbar_wait(&acc1_empty[b], use ^ 1u, &abort_flag)) return false;
          tc_fence_after();
          const uint32_t d = tmem_base + (uint32_t)(b * C);
#pragma unroll
          for (int s = 0; s < 2; ++s) {
            const uint64_t adesc = sw128_desc(sbase + OFF_A + s * SLICE);
            const uint64_t bdesc = sw128_desc(sbase + OFF_W1 + b * TILE + s * SLICE);
#pragma unroll
            for (int k = 0; k < 4; ++k)
              umma_bf16<false>(d, adesc + (uint64_t)(2 * k), bdesc + (uint64_t)(2 * k), idesc, (s | k) != 0);
          }
          umma_commit(&w1_empty[b]);
          umma_commit(&acc1_full[b]);
          if (j == NCH - 1) umma_commit(&a_empty);
          return true;
        };
        // FC2's K slice of hidden chunk j (the chunk's activations from shared memory)
        auto fc2 = [&](int j) -> bool {
          const int b = j & 1;
          const uint32_t use = (uint32_t)(2 * it + (j >> 1)) & 1u;
          if (j == 0 && !mbar_wait(&acc2_empty, tp ^ 1u, &abort_flag)) return false;
          if (!mbar_wait(&h_full[b], use, &abort_flag)) return false;
          if (!mbar_wait(&w2_full[b], use, &abort_flag)) return false;
          tc_fence_after();
          const uint32_t d = tmem_base + TMEM_ACC2;
#pragma unroll
          for (int s = 0; s < 2; ++s) {
            const uint64_t adesc = sw128_desc(sbase + OFF_H + b * TILE + s * SLICE);
            const uint64_t bdesc = sw128_desc(sbase + OFF_W2 + b * TILE + s * SLICE);
#pragma unroll
            for (int k = 0; k < 4; ++k)
              umma_bf16<false>(d, adesc + (uint64_t)(2 * k), bdesc + (uint64_t)(2 * k), idesc, (j | s | k) != 0);
          }
          umma_commit(&w2_empty[b]);
          umma_commit(&h_empty[b]);
          if (j == NCH - 1) umma_commit(&acc2_full);
          return true;
        };
        ok = fc1(0) && fc1(1);
        for (int j = 0; j < NCH && ok; ++j) {
          ok = fc2(j);
          if (ok && j + 2 < NCH) ok = fc1(j + 2);
        }
      }
      if (!ok) {
        abort_flag = 1;
        atomicExch(status, (int)WM_ERR_TIMEOUT);
        umma_commit(&drain_bar);  // completes once every MMA issued above has finished
        volatile int never = 0;
        mbar_wait(&drain_bar, 0, &never);
      }
    }
  } else {
    // -------------------------------------------------------- epilogue
    const int quarter = warp & 3;                 // TMEM lane quarter this warp may access
    const int half = (warp - 2) >> 2;             // columns 64 half .. 64 half + 63 of every chunk
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    const int r = quarter * 32 + lane;            // this thread's row in the tile
    int it = 0;
    for (int tile = blockIdx.x; tile < num_tiles; tile += gridDim.x, ++it) {
      const uint32_t tp = (uint32_t)it & 1u;
      const int m0 = tile * BM, row0 = m0 + quarter * 32, m = m0 + r;
      // LayerNorm 2 of the row from the projection's partial (mean, M2) pairs
      // (equal counts C / np each): its mean and 1 / sqrt(var + eps)
      float ln_mean = 0.f, ln_rstd = 0.f;
      if (m < M) {
        const float* st = e.stats_in + (size_t)m * e.np_in * 2;
        float mu = 0.f;
        for (int i = 0; i < e.np_in; ++i) mu += st[2 * i];
        mu /= (float)e.np_in;
        const float cnt = (float)C / (float)e.np_in;
        float m2 = 0.f;
        for (int i = 0; i < e.np_in; ++i) {
          const float d = st[2 * i] - mu;
          m2 += st[2 * i + 1] + cnt * d * d;
        }
        ln_mean = mu;
        ln_rstd = rsqrtf(m2 / (float)C + e.eps);
      }
      bool ok = true;
      // ---- FC1 chunks: rstd (acc - mean colsum) + b', GELU, bf16 into the H slot
      for (int j = 0; j < NCH && ok; ++j) {
        const int b = j & 1;
        const uint32_t use = (uint32_t)(2 * it + (j >> 1)) & 1u;
        if (!__all_sync(0xffffffffu, mbar_wait(&acc1_full[b], use, &abort_flag))) { ok = false; break; }
        tc_fence_after();
#pragma unroll 1
        for (int sub = 0; sub < 2; ++sub) {
          const int c = half * 64 + sub * 32;      // column in the chunk
          float v[32];
          tmem_ld32(tmem_base + (uint32_t)(b * C + c) + lane_off, v);
          if (sub == 1) {
            // last TMEM read of this chunk: the accumulator may be refilled
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc1_empty[b]);
          }
          const int n = j * C + c;                 // hidden column
          float lcs[32], lbb[32];
          {
            const float4* c4 = reinterpret_cast<const float4*>(e.colsum1 + n);
            const float4* b4 = reinterpret_cast<const float4*>(e.bias1 + n);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const float4 a = __ldg(c4 + q), bb = __ldg(b4 + q);
              lcs[4 * q] = a.x; lcs[4 * q + 1] = a.y; lcs[4 * q + 2] = a.z; lcs[4 * q + 3] = a.w;
              lbb[4 * q] = bb.x; lbb[4 * q + 1] = bb.y; lbb[4 * q + 2] = bb.z; lbb[4 * q + 3] = bb.w;
            }
          }
          const uint64_t nmean2 = pack_f2(-ln_mean, -ln_mean), rstd2 = pack_f2(ln_rstd, ln_rstd);
#pragma unroll
          for (int jj = 0; jj < 32; jj += 2) {
            float t0, t1;
            fma_f2(t0, t1, lcs[jj], lcs[jj + 1], nmean2, pack_f2(v[jj], v[jj + 1]));
            fma_f2(v[jj], v[jj + 1], t0, t1, rstd2, pack_f2(lbb[jj], lbb[jj + 1]));
            gelu_erf2(v[jj], v[jj + 1]);
          }
          if (sub == 0) {
            // the slot's previous chunk (j - 2) has been read by FC2
            if (!__all_sync(0xffffffffu, mbar_wait(&h_empty[b], use ^ 1u, &abort_flag))) { ok = false; break; }
          }
          store_h_row(smem + OFF_H + b * TILE + half * SLICE, r, sub * 4, v);
        }
        if (!ok) break;
        fence_async_smem();   // generic-proxy stores, read by the tensor core next
        __syncwarp();
        if (lane == 0) mbar_arrive(&h_full[b]);
      }
      if (ok && !__all_sync(0xffffffffu, mbar_wait(&acc2_full, tp, &abort_flag))) ok = false;
      if (!ok) {
        abort_flag = 1;
        atomicExch(status, (int)WM_ERR_TIMEOUT);
        break;
      }
      tc_fence_after();
      // ---- FC2: x_new = x_old + acc + b2, its bf16 copy, and Welford (count,
      // mean, M2) over this half's 64 columns: the next LayerNorm's partial
      float wn = 0.f, wmean = 0.f, wm2 = 0.f;
      float4 xa[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) xa[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (m < M) {
        const float4* xo = reinterpret_cast<const float4*>(e.x + (size_t)m * C + half * 64);
#pragma unroll
        for (int q = 0; q < 8; ++q) xa[q] = xo[q];
      }
#pragma unroll 1
      for (int sub = 0; sub < 2; ++sub) {
        const int c = half * 64 + sub * 32;
        float v[32];
        tmem_ld32(tmem_base + TMEM_ACC2 + (uint32_t)c + lane_off, v);
        if (sub == 1) {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&acc2_empty);
        }
        if (row0 >= M) continue;   // the whole 32-row group is past the end (warp-uniform)
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) v[jj] += __ldg(e.bias2 + c + jj);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          v[4 * q] += xa[q].x; v[4 * q + 1] += xa[q].y; v[4 * q + 2] += xa[q].z; v[4 * q + 3] += xa[q].w;
        }
        if (sub == 0 && m < M) {
          const float4* xo = reinterpret_cast<const float4*>(e.x + (size_t)m * C + c + 32);
#pragma unroll
          for (int q = 0; q < 8; ++q) xa[q] = xo[q];
        }
        float cs = 0.f;
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) cs += v[jj];
        const float cm = cs * (1.f / 32.f);
        float cq = 0.f;
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) cq += (v[jj] - cm) * (v[jj] - cm);
        const float nt = wn + 32.f, d = cm - wmean;
        wmean += d * (32.f / nt);
        wm2 += cq + d * d * (wn * 32.f / nt);
        wn = nt;
        if (e.np_out == 4 && m < M) {
          // one partial per 32 columns: this chunk's own (mean, M2), as a
          // residual epilogue on 64-column tiles writes it
          float* st = e.stats_out + ((size_t)m * 4 + half * 2 + sub) * 2;
          st[0] = wmean;
          st[1] = wm2;
          wn = 0.f;
          wmean = 0.f;
          wm2 = 0.f;
        }
        if (m < M) {
          float4* xd = reinterpret_cast<float4*>(e.x + (size_t)m * C + c);
#pragma unroll
          for (int q = 0; q < 8; ++q) xd[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
          uint4* bd = reinterpret_cast<uint4*>(e.xb + (size_t)m * C + c);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            uint32_t w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              __nv_bfloat162 pr = __floats2bfloat162_rn(v[8 * k + 2 * q], v[8 * k + 2 * q + 1]);
              w[q] = *reinterpret_cast<uint32_t*>(&pr);
            }
            bd[k] = make_uint4(w[0], w[1], w[2], w[3]);
          }
        }
      }
      if (e.np_out == 2 && row0 < M && m < M && wn > 0.f) {
        float* st = e.stats_out + ((size_t)m * 2 + half) * 2;
        st[0] = wmean;
        st[1] = wm2;
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem_base) : "memory");
  }
}

static wm_status launch_mlp(const MlpArgs& a, cudaStream_t s) {
  MlpEpi e;
  e.colsum1 = a.colsum1;
  e.bias1 = a.bias1;
  e.bias2 = a.bias2;
  e.stats_in = a.stats_in;
  e.stats_out = a.stats_out;
  e.x = a.x;
  e.xb = a.xb;
  e.np_in = a.np_in;
  e.np_out = a.np_out;
  e.eps = a.eps;
  const int tiles = (a.M + BM - 1) / BM;
  const int grid = tiles < num_sms() ? tiles : num_sms();
  WM_CUDA(launch_pdl(mlp_small_kernel, dim3(grid), dim3(THREADS), mlp::SMEM, s, a.pdl, a.tmA, a.tmW1, a.tmW2, a.M, e,
                     device_status_word()));
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}
}  // namespace tc

wm_status prepare_gemm_tc() {
  wm_status st = tc::set_attrs_bn<128>();
  if (st == WM_OK) st = tc::set_attrs_bn<256>();
  if (st == WM_OK) st = tc::set_attrs_bn<64>();
  if (st == WM_OK && cudaFuncSetAttribute(tc::mlp_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          tc::mlp::SMEM) != cudaSuccess)
    st = cuda_fail(cudaGetLastError(), "fused MLP shared-memory limit");
  return st;
}

wm_status launch_mlp_small(const MlpArgs& a, cudaStream_t s) {
  if (a.M <= 0) return WM_OK;
  if (!a.colsum1 || !a.bias1 || !a.bias2 || !a.stats_in || !a.stats_out || !a.x || !a.xb || a.np_in < 1 ||
      (a.np_out != 2 && a.np_out != 4))
    return fail(WM_ERR_INVALID_ARG, "fused MLP needs the LayerNorm statistics, biases, residual and its bf16 copy");
  if ((reinterpret_cast<uintptr_t>(a.x) | reinterpret_cast<uintptr_t>(a.xb)) & 15)
    return fail(WM_ERR_INVALID_ARG, "fused MLP needs 16-byte aligned residual buffers");
  return tc::launch_mlp(a, s);
}

wm_status launch_gemm_tc(const GemmArgs& a, cudaStream_t s) {
  if (a.M <= 0 || a.N <= 0) return WM_OK;
  if (a.epi == EPI_RESID_LN && (a.N % a.bn != 0 || !a.x || !a.stats))
    return fail(WM_ERR_INVALID_ARG, "residual+statistics epilogue needs N % tile == 0, x and stats");
  if ((a.epi == EPI_LNF_STORE || a.epi == EPI_LNF_GELU) &&
      (!a.stats || !a.colsum || !a.bias || a.np < 1 || a.N % 32 != 0))
    return fail(WM_ERR_INVALID_ARG, "LayerNorm-folded epilogue needs stats, colsum, bias, np >= 1, N % 32 == 0");
  if (a.K <= 0 || a.K % (a.f8 ? 16 : 8) != 0) return fail(WM_ERR_INVALID_ARG, "tcgen05 GEMM needs K > 0 and 16-byte rows");
  if (a.pair) {
    if (a.bn != 256 || a.N % 256 != 0) return fail(WM_ERR_INVALID_ARG, "pair GEMM tiles need BN = 256 and N % 256 == 0");
    return tc::launch_pair(a, s);
  }
  if (a.bn == 256) return tc::launch_bn<256>(a, s);
  if (a.bn == 128) return tc::launch_bn<128>(a, s);
  if (a.bn == 64) return tc::launch_bn<64>(a, s);
  return fail(WM_ERR_INVALID_ARG, "GEMM tile width must be 64, 128 or 256");
}

// ------------------------------------------------------------ TMA maps ----
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

bool make_tmap_e4m3(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, uint32_t box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || rows == 0 || cols == 0 || cols % 16 != 0 || (reinterpret_cast<uintptr_t>(base) & 15)) return false;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols};
  cuuint32_t box[2] = {128, box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool make_tmap_out_e4m3(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || rows == 0 || cols == 0 || cols % 16 != 0 || (reinterpret_cast<uintptr_t>(base) & 15)) return false;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols};
  cuuint32_t box[2] = {32, 32};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool make_tmap_out(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, bool f32) {
  EncodeTiledFn fn = encode_fn();
  const uint64_t el = f32 ? 4 : 2;
  if (!fn || rows == 0 || cols == 0 || (cols * el) % 16 != 0 || (reinterpret_cast<uintptr_t>(base) & 15)) return false;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols * el};
  cuuint32_t box[2] = {32, 32};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base),
                  dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  f32 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool make_tmap_qkv_slab(CUtensorMap* map, const void* qkv, uint64_t C3, uint64_t W, uint64_t H, uint64_t DB,
                        uint32_t box_c, uint32_t box_w, uint32_t box_h) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || (reinterpret_cast<uintptr_t>(qkv) & 15) || (C3 * 2) % 16 || (box_c * 2) % 16 || box_c > 256 ||
      box_w > 256 || box_h > 256)
    return false;
  cuuint64_t dims[4] = {C3, W, H, DB};
  cuuint64_t strides[3] = {C3 * 2, W * C3 * 2, H * W * C3 * 2};
  cuuint32_t box[4] = {box_c, box_w, box_h, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(qkv), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool make_tmap_kv_slab(CUtensorMap* map, const void* qkv, uint64_t C3, uint64_t W, uint64_t H, uint64_t levels,
                       uint32_t box_w, uint32_t box_h) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || (reinterpret_cast<uintptr_t>(qkv) & 15) || (C3 * 2) % 16 || box_w == 0 || box_w > W || box_h == 0 ||
      box_h > 256 || levels == 0)
    return false;
  cuuint64_t dims[4] = {C3, W, H, levels};
  cuuint64_t strides[3] = {C3 * 2, W * C3 * 2, H * W * C3 * 2};
  cuuint32_t box[4] = {32, box_w, box_h, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(qkv), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool make_tmap_bf16(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, uint32_t box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || rows == 0 || cols == 0 || (cols * 2) % 16 != 0 || (reinterpret_cast<uintptr_t>(base) & 15)) return false;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols * 2};
  cuuint32_t box[2] = {64, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace wm
