// Fused 3D neighborhood attention on the 5th-generation tensor cores
// (tcgen05): S = Q K^T and O += P V as tcgen05.mma with the accumulators in
// tensor memory, BF16 operands, FP32 accumulation and FP32 softmax
// statistics. The paper's attention is NATTEN's fused kernel (Section 2.1,
// "NATTEN"; Appendix A.2: window (5, 7, 7), bump windows at the poles,
// circular padding in longitude); this kernel computes the same function.
//
// Work unit ("tile"): batch element b, head, query level d and a block of
// 16 latitudes x 8 longitudes = 128 queries, one per tensor-memory lane
// (lane r = query (h0 + r / 8, w0 + r % 8)). All queries of a tile share
// their kd key levels. For every key level the CTA stages a K and a V slab
// of HR latitude rows x 16 longitude columns (the union of the tile's
// windows, HR = 16 + kh - 1, plus spare columns), split into two halves of 8
// longitude columns. Per (level, half) -- a "step" -- the tensor core
// computes S = Q K^T for all 128 queries against the half's HR x 8 keys
// (N = HR * 8, padded to 16), the softmax warps turn S into P in place, and
// the tensor core accumulates O += P V.
//
// Warp roles (persistent CTAs, one per SM, 12 warps, up to 168 registers a thread):
//   warps 0-7  softmax: warps q and q + 4 own tensor-memory lanes 32q..32q+31,
//              i.e. query rows 4q..4q+3 of the tile. Their windows cover
//              kh + 3 key rows; each of the two warps reads half of them
//              (8 columns per key row, one 8-column tcgen05.ld each), masks
//              keys outside its own window (bump rows, periodic or clamped
//              columns), and the pair combines its row maxima through shared
//              memory once per step, so both keep the same running max m
//              (which moves only when a row's maximum grows by more than
//              2^8; then O is rescaled in tensor memory). Each writes
//              P = 2^(S - m) as bf16 pairs over the first half of its rows'
//              S columns, and zeros in alternate key rows the quarter's
//              window does not reach. Warp q + 4 also copies the next tile's
//              queries into tensor memory (the A operand of Q K^T; loaded
//              one step ahead); warp q writes each finished tile's O / l to
//              global memory one step into the next tile.
//   warp 8     MMA issuer (one thread): QK(step + 2) is issued right after
//              PV(step), so the other S buffer's softmax overlaps both.
//   warps 9-11 loaders: cp.async 16-byte copies of the K/V slabs into a ring
//              of NS stages. Layout of one (K or V, half): [group of 8 keys]
//              [16-channel atom][8 keys x 32 bytes] with the 32-byte swizzle
//              (the two 16-byte units of keys 4..7 of a group swap places),
//              which K (the K-major B operand of Q K^T: one atom per MMA) and
//              V (the MN-major B operand of P V: atoms along N) share. Keys
//              past HR * 8 and the spare slab columns stay zero.
// Tensor memory (512 columns): S0, S1 (NPAD each), O0, O1 (dh each), Q0, Q1
// (dh / 2 each, bf16 pairs). Every mbarrier wait is bounded in time; on a
// timeout the CTA records WM_ERR_TIMEOUT, drains its own copies and MMAs,
// frees tensor memory and returns.
#include <algorithm>
#include <cmath>

#include "tc_ptx.cuh"

namespace wm {
namespace natc {

using namespace ptx;

// Two softmax warps per tensor-memory lane quarter (each takes half of the
// quarter's key rows), one MMA warp, three loader warps.
constexpr int kSoftWarps = 8, kMmaWarp = 8, kLoadWarps = 3;
constexpr int kThreads = 32 * (kSoftWarps + 1 + kLoadWarps);
constexpr int kMaxStages = 4;
constexpr float kLazyLog2 = 8.f;   // the running max moves when a row max grows by more than this

struct Params {
  const __nv_bfloat16* qkv;
  __nv_bfloat16* out;
  int* status;
  int B, D, H, W, C, heads, kd, periodic;
  int HR;      // key rows of a slab
  int NPAD;    // keys of a half as the MMA reads them: npad_for<KH>() ((16 + KH - 1) * 8, rounded up to 16)
  int NS;      // slab stages
  int tiles_h, tiles_w, ntiles;
  int colO, colQ;   // tensor-memory columns of O0 (O1 = +oStride) and Q0 (Q1 = +qStride)
  int oStride, qStride;
  float scale_log2;   // log2(e) / sqrt(dh)
};

struct TileGeo {
  int b, head, d, h0, w0;
  int ld0;      // first key level
  int s_lat;    // first slab latitude row
  int s_lon;    // longitude of slab column 0 (periodic: may be negative or wrap)
};

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

template <int KH, int KW>
__device__ __forceinline__ TileGeo tile_geo(const Params& p, int t) {
  TileGeo g;
  const int tw = t % p.tiles_w;
  t /= p.tiles_w;
  const int th = t % p.tiles_h;
  t /= p.tiles_h;
  g.d = t % p.D;
  t /= p.D;
  g.head = t % p.heads;
  g.b = t / p.heads;
  g.h0 = th * 16;
  g.w0 = tw * 8;
  g.ld0 = clampi(g.d - p.kd / 2, 0, p.D - p.kd);
  g.s_lat = clampi(g.h0 - KH / 2, 0, p.H - p.HR);
  g.s_lon = p.periodic ? g.w0 - KW / 2 : clampi(g.w0 - KW / 2, 0, p.W - (KW + 7));
  return g;
}

// Shared-memory matrix descriptor, 32-byte swizzle (layout type 6): rows of
// 32 bytes, 8-row groups. lbo, sbo: byte strides between atoms along the two
// dimensions as the tensor core reads them (for K-major operands sbo is the
// 8-row group stride along M/N and lbo is unused; for MN-major operands lbo is
// the stride between 16-element atoms along M/N and sbo the 8-row group
// stride along K).
__device__ __forceinline__ uint64_t desc_sw32(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)6 << 61);
}

// Instruction descriptor, kind::f16: D f32, A and B bf16, A K-major, B K-major
// (b_mn = 0) or MN-major (b_mn = 1).
__host__ __device__ constexpr uint32_t idesc_bf16_ab(int M, int N, int b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)b_mn << 16) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// D (tmem) (+)= A (tmem) * B (shared-memory descriptor)
__device__ __forceinline__ void umma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// 16-byte global -> shared copy through L1 (.ca: the lanes that share a
// 32-byte sector are served by one L2 request)
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// Byte offset of the (stage, K or V, half) region in the slab ring; NA =
// 16-channel atoms per head. A region is NPAD / 8 groups of NA atoms of
// 8 keys x 32 bytes.
__device__ __forceinline__ uint32_t region_off(const Params& p, int NA, int stage, int kv, int h) {
  return (uint32_t)((stage * 4 + kv * 2 + h) * NA * p.NPAD) * 32u;
}

// Softmax warps: this lane's query of tile ti (its dh channels as bf16
// pairs) from global memory into registers. Issued one step before the
// tensor-memory store, so the load latency is hidden behind a softmax step.
template <int DH, int KH, int KW>
__device__ __forceinline__ void softmax_load_q(const Params& p, int ti, int q, int lane, uint4 (&x)[DH / 8]) {
  const TileGeo G = tile_geo<KH, KW>(p, blockIdx.x + ti * gridDim.x);
  const int a = min(G.h0 + 4 * q + (lane >> 3), p.H - 1), w = min(G.w0 + (lane & 7), p.W - 1);
  const long tok = ((long)(G.b * p.D + G.d) * p.H + a) * p.W + w;
  const uint4* src = reinterpret_cast<const uint4*>(p.qkv + tok * (3L * p.C) + (long)G.head * DH);
#pragma unroll
  for (int c = 0; c < DH / 8; ++c) x[c] = __ldg(src + c);
}

// Softmax warps: the prefetched query into tensor-memory Q buffer ti & 1
// (the A operand of Q K^T), once the tile that used that buffer before has
// issued its last Q K^T.
template <int DH>
__device__ __forceinline__ bool softmax_store_q(const Params& p, int ti, int lane, uint32_t lane_base,
                                                const uint4 (&x)[DH / 8], uint64_t* q_empty, uint64_t* q_full,
                                                volatile int* abort_flag) {
  // the wait's outcome is made warp-uniform: the tcgen05 stores below are warp-collective
  if (!__all_sync(0xffffffffu, mbar_wait(&q_empty[ti & 1], ((uint32_t)(ti >> 1) & 1u) ^ 1u, abort_flag)))
    return false;
  tc_fence_after();
  const uint32_t qcol = lane_base + (uint32_t)(p.colQ + (ti & 1) * p.qStride);
#pragma unroll
  for (int c = 0; c < DH / 16; ++c) {   // 16 channels = 8 columns per store
    const uint32_t r[8] = {x[2 * c].x, x[2 * c].y, x[2 * c].z, x[2 * c].w,
                           x[2 * c + 1].x, x[2 * c + 1].y, x[2 * c + 1].z, x[2 * c + 1].w};
    tmem_st8(qcol + 8u * c, r);
  }
  tmem_wait_st();
  tc_fence_before();
  __syncwarp();
  if (lane == 0) mbar_arrive(&q_full[ti & 1]);
  return true;
}

// Softmax warps: O / l of tile ti (tensor-memory buffer ti & 1) to global
// memory as bf16; frees the O buffer for the tile after next.
template <int DH>
__device__ __noinline__ bool softmax_epilogue(const Params& p, int ti, int lane, uint32_t lane_base, float l,
                                              long orow, bool valid, uint64_t* o_full, uint64_t* o_empty,
                                              volatile int* abort_flag) {
  if (!__all_sync(0xffffffffu, mbar_wait(&o_full[ti & 1], (uint32_t)(ti >> 1) & 1u, abort_flag))) return false;
  tc_fence_after();
  uint32_t o[DH];
#pragma unroll
  for (int c = 0; c < DH / 8; ++c) {
    uint32_t r[8];
    tmem_ld8_nowait(lane_base + (uint32_t)(p.colO + (ti & 1) * p.oStride) + 8u * c, r);
#pragma unroll
    for (int i = 0; i < 8; ++i) o[8 * c + i] = r[i];
  }
  tmem_wait_ld();
  tc_fence_before();
  __syncwarp();
  if (lane == 0) mbar_arrive(&o_empty[ti & 1]);
  if (valid) {
    const float inv = 1.f / l;
    uint4* dst = reinterpret_cast<uint4*>(p.out + orow);
#pragma unroll
    for (int c = 0; c < DH / 8; ++c) {
      uint4 v;
      v.x = pack_bf16(__uint_as_float(o[8 * c + 0]) * inv, __uint_as_float(o[8 * c + 1]) * inv);
      v.y = pack_bf16(__uint_as_float(o[8 * c + 2]) * inv, __uint_as_float(o[8 * c + 3]) * inv);
      v.z = pack_bf16(__uint_as_float(o[8 * c + 4]) * inv, __uint_as_float(o[8 * c + 5]) * inv);
      v.w = pack_bf16(__uint_as_float(o[8 * c + 6]) * inv, __uint_as_float(o[8 * c + 7]) * inv);
      dst[c] = v;
    }
  }
  return true;
}

// Keys of a slab half as the MMAs read them: (16 + KH - 1) latitude rows x 8
// columns, rounded up to 16, whatever the grid's height (rows past a short
// grid's last latitude are zero padding, never in a window).
template <int KH>
constexpr int npad_for() { return ((16 + KH - 1) * 8 + 15) / 16 * 16; }

template <int DH, int KH, int KW>
__global__ void __launch_bounds__(kThreads, 1) na_tc_kernel(const Params p) {
  constexpr int NA = DH / 16;       // 16-channel (32-byte) atoms per head
  constexpr int kNpad = npad_for<KH>();   // p.NPAD, as a constant
  constexpr int WR = KH + 3;        // key rows a softmax warp reads
  constexpr int RH = KH / 2, RW = KW / 2;
  static_assert(DH % 16 == 0 && DH <= 64, "head dim");
  static_assert(KW + 7 <= 16, "a slab row holds 16 longitude columns");

  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t kv_full[kMaxStages], kv_empty[kMaxStages];
  __shared__ __align__(8) uint64_t s_full[2], p_ready[2], pv_done[2], q_full[2], q_empty[2], o_full[2], o_empty[2];
  __shared__ __align__(8) uint64_t drain_bar;
  __shared__ __align__(8) uint64_t xch_bar[4];   // per lane quarter: the two softmax warps' exchanges
  __shared__ float xch_val[2][2][128];           // [exchange parity][warp of the quarter][query]
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;

  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sbase = smem_u32(smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int my_tiles = blockIdx.x < p.ntiles ? (p.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int steps_per_tile = 2 * p.kd;
  const int nsteps = my_tiles * steps_per_tile;

  if (threadIdx.x == 0) {
    for (int s = 0; s < p.NS; ++s) {
      mbar_init(&kv_full[s], 32 * kLoadWarps);
      mbar_init(&kv_empty[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&s_full[i], 1);
      mbar_init(&p_ready[i], kSoftWarps);
      mbar_init(&pv_done[i], 1);
      mbar_init(&q_full[i], kSoftWarps / 2);     // the second warp of each quarter stores Q
      mbar_init(&q_empty[i], 1);
      mbar_init(&o_full[i], 1);
      mbar_init(&o_empty[i], kSoftWarps / 2);    // the first warp of each quarter writes O out
    }
    mbar_init(&drain_bar, 1);
    for (int i = 0; i < 4; ++i) mbar_init(&xch_bar[i], 64);   // every thread of a quarter's two warps
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // The MMA also reads keys the loaders never write (past HR * 8 in every
  // chunk, and the spare slab columns kw + 7 .. 15): masked scores, zero P,
  // so they must hold finite values. Zero the whole ring once.
  {
    const int items = p.NS * 4 * NA * p.NPAD * 2;   // 16-byte units
    for (int i = threadIdx.x; i < items; i += blockDim.x)
      *reinterpret_cast<uint4*>(smem + (uint32_t)i * 16u) = make_uint4(0, 0, 0, 0);
    fence_async_smem();
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  pdl_wait();      // qkv of the previous kernel is complete from here on
  pdl_trigger();

  // tensor-memory column of S buffer i (0 or 1)
  auto colS = [&](int i) -> uint32_t { return (uint32_t)(i * p.NPAD); };

  if (warp == kMmaWarp) {
    if (lane == 0) {
      // ------------------------------------------------------------ MMA issuer
      // One thread issues every MMA of the CTA. Its instruction stream is on
      // the critical path (an MMA waits for its operands' scalar arithmetic),
      // so the step indices advance incrementally, descriptors are offsets
      // from two precomputed ones, and both MMA loops are fully unrolled.
      constexpr int NKV = kNpad / 16;                          // P V MMAs per step (16 keys each)
      constexpr uint32_t GB = (uint32_t)NA * 256u;             // 8 keys x all atoms
      constexpr uint32_t REGION = (uint32_t)NA * kNpad * 32u;  // one (stage, K or V, half) region
      constexpr uint32_t idesc_pv = idesc_bf16_ab(128, DH, 1);
      constexpr uint32_t idesc_qk = idesc_bf16_ab(128, kNpad, 0);
      const uint64_t kdesc0 = desc_sw32(sbase, 16u, GB);       // region 0 as the K-major B of Q K^T
      const uint64_t vdesc0 = desc_sw32(sbase, 256u, GB);      // region 0 as the MN-major B of P V
      struct Cursor {   // a step: its tile, its index in the tile, the ring slot of its level
        int ti = 0, r = 0, stage = 0;
        uint32_t par = 0;
      };
      auto advance = [&](Cursor& c) {
        if (c.r & 1) {   // a level ends with its second half
          if (++c.stage == p.NS) {
            c.stage = 0;
            c.par ^= 1u;
          }
        }
        if (++c.r == steps_per_tile) {
          c.r = 0;
          ++c.ti;
        }
      };
      auto issue_qk = [&](const Cursor& c, int v) -> bool {
        const int h = c.r & 1;
        if (c.r == 0 && !mbar_wait(&q_full[c.ti & 1], (uint32_t)(c.ti >> 1) & 1u, &abort_flag)) return false;
        if (h == 0 && !mbar_wait(&kv_full[c.stage], c.par, &abort_flag)) return false;
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)((v & 1) * kNpad);
        const uint32_t a = tmem + (uint32_t)(p.colQ + (c.ti & 1) * p.qStride);
        const uint64_t kd = kdesc0 + (uint64_t)(((uint32_t)(c.stage * 4 + h) * REGION) >> 4);
#pragma unroll
        for (int k = 0; k < NA; ++k)   // one 16-channel atom (256 bytes along a group) per MMA
          umma_ts(d, a + 8u * k, kd + (uint64_t)(16 * k), idesc_qk, k > 0);
        umma_commit(&s_full[v & 1]);
        if (c.r == steps_per_tile - 1) umma_commit(&q_empty[c.ti & 1]);
        return true;
      };
      auto issue_pv = [&](const Cursor& c, int u) -> bool {
        const int h = c.r & 1;
        if (!mbar_wait(&p_ready[u & 1], (uint32_t)(u >> 1) & 1u, &abort_flag)) return false;
        if (c.r == 0 && !mbar_wait(&o_empty[c.ti & 1], ((uint32_t)(c.ti >> 1) & 1u) ^ 1u, &abort_flag)) return false;
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(p.colO + (c.ti & 1) * p.oStride);
        const uint32_t a = tmem + (uint32_t)((u & 1) * kNpad);
        const uint64_t vd = vdesc0 + (uint64_t)(((uint32_t)(c.stage * 4 + 2 + h) * REGION) >> 4);
        const uint32_t acc0 = c.r > 0 ? 1u : 0u;
#pragma unroll
        for (int k = 0; k < NKV; ++k)       // 16 keys = 2 groups per MMA
          umma_ts(d, a + 8u * k, vd + (uint64_t)((2u * GB * k) >> 4), idesc_pv, k > 0 ? 1u : acc0);
        umma_commit(&pv_done[u & 1]);
        if (h == 1) umma_commit(&kv_empty[c.stage]);
        if (c.r == steps_per_tile - 1) umma_commit(&o_full[c.ti & 1]);
        return true;
      };
      Cursor cq, cv;
      bool ok = true;
      if (nsteps > 0) {
        ok = issue_qk(cq, 0);
        advance(cq);
      }
      if (ok && nsteps > 1) {
        ok = issue_qk(cq, 1);
        advance(cq);
      }
      for (int u = 0; u < nsteps && ok; ++u) {
        ok = issue_pv(cv, u);
        advance(cv);
        if (ok && u + 2 < nsteps) {
          ok = issue_qk(cq, u + 2);
          advance(cq);
        }
      }
      if (!ok) {
        abort_flag = 1;
        atomicExch(p.status, (int)WM_ERR_TIMEOUT);
        umma_commit(&drain_bar);   // completes once every MMA issued above has finished
        volatile int never = 0;
        mbar_wait(&drain_bar, 0, &never);
      }
    }
  } else if (warp > kMmaWarp) {
    // --------------------------------------------------------------- loaders
    // lane = (atom, key of a quad, 16-byte unit): one instruction copies 4
    // consecutive keys (longitude columns) x the head's channels of K or V;
    // its 8-lane phases each write 4 keys x 32 bytes = 128 contiguous bytes.
    const int lw = warp - kMmaWarp - 1;
    const int la = lane >> 3, rk = (lane >> 1) & 3, lu = lane & 1;
    const bool active = la < NA;
    const long C3 = 3L * p.C;
    bool ok = true;
    int g = 0, prev_stage = -1;
    for (int ti = 0; ti < my_tiles && ok; ++ti) {
      const TileGeo G = tile_geo<KH, KW>(p, blockIdx.x + ti * gridDim.x);
      int lonoff[4];   // slab column 4 hq + rk (hq = 2 half + quad)
#pragma unroll
      for (int hq = 0; hq < 4; ++hq) {
        int lon = G.s_lon + 4 * hq + rk;
        if (p.periodic) {
          lon %= p.W;
          if (lon < 0) lon += p.W;
        } else {
          lon = min(lon, p.W - 1);   // columns past the grid are never loaded (spare) or masked
        }
        if (!WM_DCHECK(lon >= 0 && lon < p.W, p.status)) lon = 0;   // debug builds
        lonoff[hq] = lon * (int)C3;
      }
      const __nv_bfloat16* chan = p.qkv + (long)G.head * DH + la * 16 + lu * 8;
      const uint32_t lane_dst = (uint32_t)(la * 256 + rk * 32);
      for (int l = 0; l < p.kd; ++l, ++g) {
        const int stage = g % p.NS;
        if (!mbar_wait(&kv_empty[stage], ((uint32_t)(g / p.NS) & 1u) ^ 1u, &abort_flag)) {
          ok = false;
          break;
        }
        const long lev = (long)G.b * p.D + G.ld0 + l;
        const __nv_bfloat16* row0 = chan + ((lev * p.H + G.s_lat) * p.W) * C3;
        if (active) {
          for (int r = lw; r < p.HR; r += kLoadWarps) {
            const __nv_bfloat16* src = row0 + (long)r * p.W * C3;
            const uint32_t rdst = sbase + lane_dst + (uint32_t)r * (uint32_t)(NA * 256);
#pragma unroll
            for (int kv = 0; kv < 2; ++kv)
#pragma unroll
              for (int hq = 0; hq < 4; ++hq) {
                const int h = hq >> 1, qd = hq & 1;
                if (4 * hq + rk < KW + 7)   // spare columns stay zero
                  cp_async16(rdst + region_off(p, NA, stage, kv, h) + (uint32_t)(qd * 128 + ((lu ^ qd) << 4)),
                             src + lonoff[hq] + (long)(1 + kv) * p.C);
              }
          }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        // the previous level's copies have landed: publish it to the MMA
        if (prev_stage >= 0) {
          asm volatile("cp.async.wait_group 1;" ::: "memory");
          fence_async_smem();
          mbar_arrive(&kv_full[prev_stage]);
        }
        prev_stage = stage;
      }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (ok && prev_stage >= 0) {
      fence_async_smem();
      mbar_arrive(&kv_full[prev_stage]);
    }
    if (!ok) {
      abort_flag = 1;
      atomicExch(p.status, (int)WM_ERR_TIMEOUT);
    }
  } else {
    // --------------------------------------------------------------- softmax
    // Warp w: tensor-memory lane quarter q = w % 4 (query rows 4q..4q+3 of
    // the tile) and half `part` = w / 4 of the quarter's WR key rows. The two
    // warps of a quarter share the running max: they exchange their partial
    // row maxima once per step (and their row sums once per tile) through
    // shared memory and a bounded mbarrier. The first warp of a quarter
    // rescales O and writes it out; the second loads the next tile's Q.
    constexpr int WN = WR / 2;   // key rows of one warp (WR = KH + 3 is even)
    static_assert(WR % 2 == 0, "the two warps of a quarter split its key rows evenly");
    const int q = warp & 3, part = warp >> 2;
    const int RB = part * WN;    // this warp's first row among the quarter's WR
    const int qlane = 32 * q + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
    const uint64_t scale2 = pack_f2(p.scale_log2, p.scale_log2);
    const uint64_t neg2 = pack_f2(-INFINITY, -INFINITY);
    bool ok = true;
    uint32_t xcnt = 0;   // exchanges so far (the mbarrier's phase)
    // this lane's value against the other warp's for the same query
    auto exchange = [&](float v, float& other) -> bool {
      const int sl = (int)(xcnt & 1u);   // two slots: the partner is at most one exchange ahead
      xch_val[sl][part][qlane] = v;
      mbar_arrive(&xch_bar[q]);
      const bool got = __all_sync(0xffffffffu, mbar_wait(&xch_bar[q], xcnt & 1u, &abort_flag));
      ++xcnt;
      if (got) other = xch_val[sl][part ^ 1][qlane];
      return got;
    };
    // both warps of the quarter have passed this point (the same mbarrier)
    auto pair_sync = [&]() -> bool {
      mbar_arrive(&xch_bar[q]);
      const bool got = __all_sync(0xffffffffu, mbar_wait(&xch_bar[q], xcnt & 1u, &abort_flag));
      ++xcnt;
      return got;
    };

    uint4 qnext[DH / 8];   // the next tile's query, prefetched one step before its store
    if (my_tiles > 0 && part == 1) {
      softmax_load_q<DH, KH, KW>(p, 0, q, lane, qnext);
      ok = softmax_store_q<DH>(p, 0, lane, lane_base, qnext, q_empty, q_full, &abort_flag);
    }
    float prev_l = 1.f;
    long prev_orow = 0;
    bool prev_valid = false;
    for (int ti = 0; ti < my_tiles && ok; ++ti) {
      const TileGeo G = tile_geo<KH, KW>(p, blockIdx.x + ti * gridDim.x);
      // this lane's query and its window inside the slab
      const int a = G.h0 + 4 * q + (lane >> 3), w = G.w0 + (lane & 7);
      const int ac = min(a, p.H - 1), wc = min(w, p.W - 1);
      const int ra = clampi(ac - RH, 0, p.H - KH) - G.s_lat;                  // first window row in the slab
      const int cb = p.periodic ? wc - G.w0 : clampi(wc - RW, 0, p.W - KW) - G.s_lon;   // first window column
      const int a0 = min(G.h0 + 4 * q, p.H - 1);
      int R0 = min(clampi(a0 - RH, 0, p.H - KH) - G.s_lat, p.HR - WR);  // the quarter's first key row
      int rlo = ra - R0;                                                // 0 .. 3
      // debug builds: the quarter's key rows lie inside the slab and this
      // query's window inside them and inside the slab's 16 columns; on a
      // failure the rows are clamped into the slab and the query is not written
      const bool geo = WM_DCHECK(R0 >= 0 && R0 + WR <= p.HR && p.HR <= kNpad / 8, p.status) &&
                       WM_DCHECK(rlo >= 0 && rlo + KH <= WR && cb >= 0 && cb + KW <= 16, p.status);
      bool valid = a < p.H && w < p.W;
      if (!geo) {
        R0 = clampi(R0, 0, kNpad / 8 - WR);
        rlo = clampi(rlo, 0, WR - KH);
        valid = false;
      }
      uint64_t cbias[2][4];   // per half: (0 | -inf) pairs for the 8 columns of a key row
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int c0 = 8 * h + 2 * j;
          const float b0 = (c0 >= cb && c0 < cb + KW) ? 0.f : -INFINITY;
          const float b1 = (c0 + 1 >= cb && c0 + 1 < cb + KW) ? 0.f : -INFINITY;
          cbias[h][j] = pack_f2(b0, b1);
        }
      const long orow = (((long)(G.b * p.D + G.d) * p.H + ac) * p.W + wc) * p.C + (long)G.head * DH;
      float m = -INFINITY, lsum = 0.f;
      const uint32_t ocol = lane_base + (uint32_t)(p.colO + (ti & 1) * p.oStride);

      for (int r = 0; r < steps_per_tile && ok; ++r) {
        const int u = ti * steps_per_tile + r, h = r & 1;
        if (!__all_sync(0xffffffffu, mbar_wait(&s_full[u & 1], (uint32_t)(u >> 1) & 1u, &abort_flag))) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t scol = lane_base + colS(u & 1);
        uint64_t cbh[4];   // this half's column bias pairs
#pragma unroll
        for (int j = 0; j < 4; ++j) cbh[j] = h ? cbias[1][j] : cbias[0][j];
        // One pass over this warp's key rows of the step (read from tensor
        // memory in groups of RG rows): scale and mask, track the row max,
        // and -- when with_p -- P = 2^(t - mref) as bf16 pairs into pk with
        // its row sum.
        constexpr int RG = (WN + 1) / 2;
        uint32_t pk[WN][4];
        auto pass = [&](bool with_p, float mref, float& mx, float& ls) {
          const uint64_t mref2 = pack_f2(mref, mref);
          float ls0 = 0.f, ls1 = 0.f;
#pragma unroll
          for (int g0 = 0; g0 < WN; g0 += RG) {
            uint32_t sr[RG][8];
#pragma unroll
            for (int i = 0; i < RG; ++i)
              if (g0 + i < WN) tmem_ld8_nowait(scol + 8u * (uint32_t)(R0 + RB + g0 + i), sr[i]);
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < RG; ++i) {
              const int wi = g0 + i;
              if (wi < WN) {
                const bool rok = (unsigned)(RB + wi - rlo) < (unsigned)KH;
                float t[8];
#pragma unroll
                for (int j = 0; j < 4; ++j)
                  fma_f2(t[2 * j], t[2 * j + 1], __uint_as_float(sr[i][2 * j]), __uint_as_float(sr[i][2 * j + 1]),
                         scale2, rok ? cbh[j] : neg2);
                mx = max3(mx, max3(t[0], t[1], t[2]), max3(t[3], t[4], t[5]));
                mx = max3(mx, t[6], t[7]);
                if (with_p) {
#pragma unroll
                  for (int j = 0; j < 4; ++j) {
                    float d0, d1;
                    sub_f2(d0, d1, t[2 * j], t[2 * j + 1], mref2);
                    const float e0 = ex2(d0), e1 = ex2(d1);
                    add_f2(ls0, ls1, ls0, ls1, e0, e1);
                    pk[wi][j] = pack_bf16(e0, e1);
                  }
                }
              }
            }
          }
          ls = ls0 + ls1;
        };
        // Single pass against the current running max; the step is redone
        // only when some row's max grows by more than 2^kLazyLog2 (always on
        // a tile's first step, where the max is not set yet). The row max is
        // the two warps' combined one, so both warps of a quarter take the
        // same decisions; they are warp-uniform (the tensor-memory loads are
        // warp-collective), and a row whose max did not move recomputes the
        // same values.
        const bool first = (r == 0);
        float mx = -INFINITY, ls = 0.f;
        pass(!first, m == -INFINITY ? 0.f : m, mx, ls);
        float mo = -INFINITY;
        if (!exchange(mx, mo)) {
          ok = false;
          break;
        }
        mx = fmaxf(mx, mo);
        const bool grow = mx > m + kLazyLog2;
        if (first || __any_sync(0xffffffffu, grow)) {
          const bool rescale = grow && m != -INFINITY;
          if (__any_sync(0xffffffffu, rescale)) {
            const float alpha = rescale ? ex2(m - mx) : 1.f;
            if (part == 0) {
              // O already holds earlier steps of this tile: wait for the last
              // PV, then rescale O (alpha = 1 for rows that keep their max)
              const int up = u - 1;
              if (!__all_sync(0xffffffffu, mbar_wait(&pv_done[up & 1], (uint32_t)(up >> 1) & 1u, &abort_flag))) {
                ok = false;
                break;
              }
              tc_fence_after();
              const uint64_t alpha2 = pack_f2(alpha, alpha);
#pragma unroll
              for (int c = 0; c < DH / 8; ++c) {
                uint32_t v[8];
                tmem_ld8_nowait(ocol + 8u * c, v);
                tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 8; i += 2) {
                  float x0 = __uint_as_float(v[i]), x1 = __uint_as_float(v[i + 1]);
                  mul_f2(x0, x1, alpha2);
                  v[i] = __float_as_uint(x0);
                  v[i + 1] = __float_as_uint(x1);
                }
                tmem_st8(ocol + 8u * c, v);
              }
            }
            lsum *= alpha;
          }
          if (grow) m = mx;
          float mx2 = -INFINITY;
          pass(true, m == -INFINITY ? 0.f : m, mx2, ls);
        }
        lsum += ls;
        // P of key row k goes to the S columns of key row k / 2, and the zeros
        // of rows past the window land on S rows of this quarter too: both
        // warps must have read all their S rows first
        if (!pair_sync()) {
          ok = false;
          break;
        }
        // P over the first half of this step's S columns: key row R0 + RB + i
        // -> P columns 4 (R0 + RB + i) .. + 3
#pragma unroll
        for (int i = 0; i < WN; ++i)
          tmem_st4(scol + 4u * (uint32_t)(R0 + RB + i), pk[i][0], pk[i][1], pk[i][2], pk[i][3]);
        // zeros in the key rows outside the quarter's window (alternate rows per warp)
        for (int kr = part; kr < R0; kr += 2) tmem_st4(scol + 4u * kr, 0u, 0u, 0u, 0u);
        for (int kr = R0 + WR + ((R0 + WR + part) & 1); kr < p.NPAD / 8; kr += 2)
          tmem_st4(scol + 4u * kr, 0u, 0u, 0u, 0u);
        tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&p_ready[u & 1]);
        // the next tile's queries (second warp): loaded after step 0, stored
        // after step 1; the previous tile's output (first warp) after step 1
        // (its last P V is done by then)
        if (part == 1 && r == 0 && ti + 1 < my_tiles) softmax_load_q<DH, KH, KW>(p, ti + 1, q, lane, qnext);
        if (r == 1) {
          if (part == 0 && ti > 0 &&
              !softmax_epilogue<DH>(p, ti - 1, lane, lane_base, prev_l, prev_orow, prev_valid, o_full, o_empty,
                                    &abort_flag)) {
            ok = false;
            break;
          }
          if (part == 1 && ti + 1 < my_tiles &&
              !softmax_store_q<DH>(p, ti + 1, lane, lane_base, qnext, q_empty, q_full, &abort_flag)) {
            ok = false;
            break;
          }
        }
      }
      if (!ok) break;
      // the quarter's row sum: this warp's keys plus the other warp's
      float lo = 0.f;
      if (!exchange(lsum, lo)) {
        ok = false;
        break;
      }
      prev_l = lsum + lo;
      prev_orow = orow;
      prev_valid = valid;
    }
    if (ok && my_tiles > 0 && part == 0)
      ok = softmax_epilogue<DH>(p, my_tiles - 1, lane, lane_base, prev_l, prev_orow, prev_valid, o_full, o_empty,
                                &abort_flag);
    if (!ok) {
      abort_flag = 1;
      atomicExch(p.status, (int)WM_ERR_TIMEOUT);
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// ------------------------------------------------------------------ host ----

constexpr int kSmemLimit = 224 * 1024;   // dynamic shared memory; the rest of the 227 KB is static (barriers, exchanges)

struct Layout {
  int HR, NPAD, NS, colO, colQ, oStride, qStride;
  size_t smem;
};

int round_up(int v, int m) { return (v + m - 1) / m * m; }

// Tensor-memory and shared-memory layout for a shape; false if the kernel
// does not support it.
bool layout_for(int H, int W, int dh, int kh, int kw, bool periodic, Layout* L) {
  if (dh != 32 && dh != 48 && dh != 64) return false;
  if (!((kh == 5 && kw == 5) || (kh == 7 && kw == 7))) return false;
  L->HR = std::min(16 + kh - 1, H);
  if (L->HR < kh + 3) return false;                       // a warp's key rows must fit the slab
  if (!periodic && W < kw + 7) return false;
  L->NPAD = round_up((16 + kh - 1) * 8, 16);   // npad_for<kh>(): the kernel's constant
  if (L->NPAD > 256) return false;
  L->oStride = round_up(dh, 16);
  L->qStride = round_up(dh / 2, 16);
  L->colO = 2 * L->NPAD;
  L->colQ = L->colO + 2 * L->oStride;
  if (L->colQ + 2 * L->qStride > 512) return false;
  const size_t stage = (size_t)4 * (dh / 16) * L->NPAD * 32;
  // + 1024 bytes to align the base, + 1024 bytes past the last stage: a P V
  // descriptor read with the two strides interchanged would end at most 512
  // bytes past its region, so even that stays inside the allocation
  for (int ns = kMaxStages; ns >= 2; --ns) {
    const size_t need = (size_t)ns * stage + 2048;
    if (need <= (size_t)kSmemLimit) {
      L->NS = ns;
      L->smem = need;
      return true;
    }
  }
  return false;
}

template <int DH, int KH, int KW>
wm_status launch_t(const Params& p, const Layout& L, cudaStream_t s, bool pdl) {
  auto kern = na_tc_kernel<DH, KH, KW>;   // shared-memory limit set by prepare_na_tc
  const int grid = std::min(p.ntiles, num_sms());
  WM_CUDA(launch_pdl(kern, dim3(grid), dim3(kThreads), L.smem, s, pdl, p));
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

}  // namespace natc

bool na_tc_supported(int H, int W, int C, int heads, int kh, int kw, bool periodic) {
  natc::Layout L;
  return C % heads == 0 && natc::layout_for(H, W, C / heads, kh, kw, periodic, &L);
}

wm_status prepare_na_tc() {
  using namespace natc;
  WM_CUDA(cudaFuncSetAttribute(na_tc_kernel<32, 5, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit));
  WM_CUDA(cudaFuncSetAttribute(na_tc_kernel<48, 5, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit));
  WM_CUDA(cudaFuncSetAttribute(na_tc_kernel<64, 5, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit));
  WM_CUDA(cudaFuncSetAttribute(na_tc_kernel<32, 7, 7>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit));
  WM_CUDA(cudaFuncSetAttribute(na_tc_kernel<48, 7, 7>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit));
  return WM_OK;
}

wm_status launch_na_tc(const __nv_bfloat16* qkv, __nv_bfloat16* out, int B, int D, int H, int W, int C, int heads,
                       int kd, int kh, int kw, bool periodic, cudaStream_t s, bool pdl) {
  using namespace natc;
  if (B <= 0) return WM_OK;
  const int dh = C / heads;
  Layout L;
  if (C % heads != 0 || !layout_for(H, W, dh, kh, kw, periodic, &L))
    return fail(WM_ERR_INVALID_ARG, "shape not supported by the tcgen05 attention kernel");
  if ((reinterpret_cast<uintptr_t>(qkv) | reinterpret_cast<uintptr_t>(out)) & 15)
    return fail(WM_ERR_INVALID_ARG, "tcgen05 attention needs 16-byte aligned qkv and out");
  Params p{};
  p.qkv = qkv;
  p.out = out;
  p.status = device_status_word();
  p.B = B; p.D = D; p.H = H; p.W = W; p.C = C; p.heads = heads; p.kd = kd; p.periodic = periodic ? 1 : 0;
  p.HR = L.HR; p.NPAD = L.NPAD; p.NS = L.NS;
  p.colO = L.colO; p.colQ = L.colQ; p.oStride = L.oStride; p.qStride = L.qStride;
  p.tiles_h = (H + 15) / 16;
  p.tiles_w = (W + 7) / 8;
  const long nt = (long)p.tiles_h * p.tiles_w * D * heads * B;
  if (nt > (1L << 30)) return fail(WM_ERR_INVALID_ARG, "too many attention tiles");
  p.ntiles = (int)nt;
  p.scale_log2 = 1.4426950408889634f / sqrtf((float)dh);
  if (kh == 5 && kw == 5) {
    if (dh == 32) return launch_t<32, 5, 5>(p, L, s, pdl);
    if (dh == 48) return launch_t<48, 5, 5>(p, L, s, pdl);
    if (dh == 64) return launch_t<64, 5, 5>(p, L, s, pdl);
  } else {
    if (dh == 32) return launch_t<32, 7, 7>(p, L, s, pdl);
    if (dh == 48) return launch_t<48, 7, 7>(p, L, s, pdl);
  }
  return fail(WM_ERR_INVALID_ARG, "shape not supported by the tcgen05 attention kernel");
}

}  // namespace wm
