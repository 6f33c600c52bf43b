// Fused 3D neighborhood attention, BF16 operands, FP32 softmax statistics.
//
// CTA = (batch*head, query level, lat x lon query tile of TH x TW tokens).
// Every query of a CTA shares its level, hence its kd key levels. For each key
// level the CTA stages that level's K/V halo slab (the union of the tile's
// latitude windows x the tile's longitude span, wrapped modulo W when
// longitude is periodic) in shared memory with cp.async, double buffered.
// Each warp owns 16 queries (a WH x WW lat-lon patch) and walks only the key
// rectangle its own queries can see, 16 keys at a time:
//   S = Q K^T      mma.sync m16n8k16 (bf16 -> fp32), K fragments by ldmatrix
//   mask           bump (clamped) windows in level/latitude, periodic or
//                  clamped windows in longitude, evaluated per (query, key)
//   online softmax running max / sum in FP32, row max by quad warp shuffles
//   O += P V       P re-packed from the S accumulators, V by ldmatrix.trans
// The result is normalised once at the end and stored as bf16.
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <mutex>
#include <vector>

#include "wm_internal.cuh"

namespace wm {
namespace na {

struct Params {
  const __nv_bfloat16* qkv;
  __nv_bfloat16* out;
  int B, D, H, W, C, heads, kd, kh, kw, periodic;
  int WH, WW, NWH, NWW;  // warp patch and warp grid
  int HRmax, WC;          // smem slab rows / columns
  int log2span;           // columns of a warp's key rectangle = 1 << log2span (8, 16 or 32)
  int tiles_w;
  float scale_log2;       // log2(e) / sqrt(dh)
};

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

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
__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
// 2^x by the MUFU.EX2 hardware instruction (flush-to-zero; 2^-inf = 0).
__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&p);
}

template <int DH, int LS>   // LS = log2 of the key-rectangle width (3, 4 or 5)
__global__ void __launch_bounds__(384, 1) na_bf16_kernel(const Params p) {
  constexpr int DHP = DH + 8;   // padded key row: odd number of 16-byte units -> conflict-free ldmatrix
  constexpr int CH = DH / 8;    // 16-byte chunks per key row
  constexpr int KC = DH / 16;   // k16 steps of Q K^T
  constexpr int ND = DH / 8;    // n8 blocks of P V
  constexpr int GCH = 8;        // 16-key groups per softmax update
  extern __shared__ __align__(16) __nv_bfloat16 sm[];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, t4 = lane & 3;
  const int H = p.H, W = p.W, D = p.D;
  const int rh = p.kh / 2, rw = p.kw / 2;
  const int TH = p.NWH * p.WH, TW = p.NWW * p.WW;
  const int th = blockIdx.x / p.tiles_w, tw = blockIdx.x % p.tiles_w;
  const int h0 = th * TH, w0 = tw * TW;
  const int d = blockIdx.y;
  const int b = blockIdx.z / p.heads, head = blockIdx.z % p.heads;
  const long N = (long)D * H * W;
  const long C3 = 3L * p.C;
  const __nv_bfloat16* base = p.qkv + (long)b * N * C3;

  const int ld0 = clampi(d - p.kd / 2, 0, D - p.kd);
  const int hs0 = clampi(h0 - rh, 0, H - p.kh);
  const int HR = clampi(min(h0 + TH, H) - 1 - rh, 0, H - p.kh) + p.kh - hs0;
  const int ws0 = p.periodic ? (w0 - rw) : clampi(w0 - rw, 0, W - p.kw);
  const int WC = p.WC;
  const int slab = p.HRmax * WC * DHP;  // elements of one K (or V) slab

  // ---- stage one key level (K and V) into buffer `buf`. Each thread owns
  // fixed (K or V, slab column, 16-byte chunk) items and walks the slab rows,
  // so the per-copy work is two pointer increments.
  const int items = 2 * WC * CH;
  auto load_level = [&](int lev, int buf) {
    __nv_bfloat16* sbuf = sm + (size_t)buf * 2 * slab;
    const __nv_bfloat16* lbase = base + (long)lev * H * W * C3 + (long)hs0 * W * C3 + (1L * p.C) + head * DH;
    for (int it = tid; it < items; it += blockDim.x) {
      const int kv = it / (WC * CH);
      const int rem = it - kv * (WC * CH);
      const int c = rem / CH, ch = rem - c * CH;
      int lon = ws0 + c;
      bool ok = true;
      if (p.periodic) {
        if (lon < 0 || lon >= W) lon = ((lon % W) + W) % W;
      } else if (lon >= W) {
        ok = false;
        lon = 0;
      }
      const __nv_bfloat16* src = lbase + (long)lon * C3 + kv * p.C + ch * 8;
      uint32_t dst = (uint32_t)__cvta_generic_to_shared(sbuf + (size_t)kv * slab + (size_t)c * DHP + ch * 8);
      const long sstep = (long)W * C3;
      const uint32_t dstep = (uint32_t)(WC * DHP * 2);
      for (int r = 0; r < HR; ++r) {
        cp_async16(dst, ok ? (const void*)src : (const void*)p.qkv, ok ? 16 : 0);
        src += sstep;
        dst += dstep;
      }
    }
  };

  // ---- this warp's queries
  const int wy = warp / p.NWW, wx = warp % p.NWW;
  const int wh0 = h0 + wy * p.WH, ww0 = w0 + wx * p.WW;
  const bool warp_live = (wh0 < H) && (ww0 < W);
  int qh[2], qw[2], qsr[2], qsc[2];
  bool qvalid[2];
#pragma unroll
  for (int rr = 0; rr < 2; ++rr) {
    const int qi = g + 8 * rr;
    qh[rr] = wh0 + qi / p.WW;
    qw[rr] = ww0 + qi % p.WW;
    qvalid[rr] = (qh[rr] < H) && (qw[rr] < W);
    const int hc = min(qh[rr], H - 1), wc = min(qw[rr], W - 1);
    qsr[rr] = clampi(hc - rh, 0, H - p.kh) - hs0;                     // first key row (slab coords)
    qsc[rr] = p.periodic ? (wc - w0) : (clampi(wc - rw, 0, W - p.kw) - ws0);  // first key col (slab coords)
  }
  const int wr0 = clampi(min(wh0, H - 1) - rh, 0, H - p.kh) - hs0;
  const int wr1 = clampi(min(wh0 + p.WH - 1, H - 1) - rh, 0, H - p.kh) + p.kh - hs0;
  const int wc0 = p.periodic ? (ww0 - w0) : (clampi(min(ww0, W - 1) - rw, 0, W - p.kw) - ws0);
  constexpr int ls = LS, smask = (1 << LS) - 1;
  const int nkeys = (wr1 - wr0) << ls;
  const int ngroups = (nkeys + 15) / 16;
  // window of each of this thread's two queries inside the warp's key
  // rectangle: rows [rlo, rlo + kh), columns = set bits of colmask
  int rlo[2];
  uint32_t colmask[2];
#pragma unroll
  for (int rr = 0; rr < 2; ++rr) {
    rlo[rr] = qsr[rr] - wr0;
    colmask[rr] = (0xFFFFFFFFu >> (32 - p.kw)) << max(qsc[rr] - wc0, 0);
  }
  // column bias of accumulator entry (group parity, n8 block, query, e & 1)
  float cbias[2][2][2][2];
#pragma unroll
  for (int hf = 0; hf < 2; ++hf)
#pragma unroll
    for (int nb = 0; nb < 2; ++nb)
#pragma unroll
      for (int rr = 0; rr < 2; ++rr)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int col = (hf * 16 + nb * 8 + 2 * t4 + e) & smask;
          cbias[hf][nb][rr][e] = ((colmask[rr] >> col) & 1u) ? 0.f : -INFINITY;
        }

  // Q fragments (A operand), rows g and g+8 of the warp's 16 queries
  uint32_t qa[KC][4];
  {
    long tok0 = ((long)d * H + min(qh[0], H - 1)) * W + min(qw[0], W - 1);
    long tok1 = ((long)d * H + min(qh[1], H - 1)) * W + min(qw[1], W - 1);
    const __nv_bfloat16* q0 = base + tok0 * C3 + head * DH;
    const __nv_bfloat16* q1 = base + tok1 * C3 + head * DH;
#pragma unroll
    for (int kc = 0; kc < KC; ++kc) {
      qa[kc][0] = *reinterpret_cast<const uint32_t*>(q0 + kc * 16 + 2 * t4);
      qa[kc][1] = *reinterpret_cast<const uint32_t*>(q1 + kc * 16 + 2 * t4);
      qa[kc][2] = *reinterpret_cast<const uint32_t*>(q0 + kc * 16 + 8 + 2 * t4);
      qa[kc][3] = *reinterpret_cast<const uint32_t*>(q1 + kc * 16 + 8 + 2 * t4);
    }
  }

  float o[ND][4];
#pragma unroll
  for (int nd = 0; nd < ND; ++nd) o[nd][0] = o[nd][1] = o[nd][2] = o[nd][3] = 0.f;
  float mrow[2] = {-INFINITY, -INFINITY};
  float lrow[2] = {0.f, 0.f};

  load_level(ld0, 0);
  cp_async_commit();
  for (int li = 0; li < p.kd; ++li) {
    if (li + 1 < p.kd) load_level(ld0 + li + 1, (li + 1) & 1);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    const __nv_bfloat16* sK = sm + (size_t)(li & 1) * 2 * slab;
    const __nv_bfloat16* sV = sK + slab;
    const uint32_t sK32 = (uint32_t)__cvta_generic_to_shared(sK);
    const uint32_t sV32 = (uint32_t)__cvta_generic_to_shared(sV);
    if (warp_live) {
      // Up to GCH groups of 16 keys are scored before one online-softmax
      // update: their MMAs, masks and exponentials are independent, which
      // keeps the tensor and MUFU pipes busy with only a few warps per SM.
      for (int g0 = 0; g0 < ngroups; g0 += GCH) {
        const int mi = lane >> 3;
        float s[GCH][2][4];
#pragma unroll
        for (int gi = 0; gi < GCH; ++gi) {
#pragma unroll
          for (int nb = 0; nb < 2; ++nb) s[gi][nb][0] = s[gi][nb][1] = s[gi][nb][2] = s[gi][nb][3] = 0.f;
          if (g0 + gi < ngroups) {
            int jk = (g0 + gi) * 16 + (mi >> 1) * 8 + (lane & 7);
            if (jk >= nkeys) jk = 0;
            const int krow = (wr0 + (jk >> ls)) * WC + wc0 + (jk & smask);
#pragma unroll
            for (int kc = 0; kc < KC; ++kc) {
              uint32_t b0, b1, b2, b3;
              ldsm_x4(sK32 + (uint32_t)((krow * DHP + kc * 16 + (mi & 1) * 8) * 2), b0, b1, b2, b3);
              mma_bf16(s[gi][0], qa[kc][0], qa[kc][1], qa[kc][2], qa[kc][3], b0, b1);
              mma_bf16(s[gi][1], qa[kc][0], qa[kc][1], qa[kc][2], qa[kc][3], b2, b3);
            }
          }
        }
        // mask + scale + chunk row max. Key j sits at rectangle row j >> LS and
        // column j & smask. The column of each accumulator entry depends on
        // the group only through (g & 1) for 32-wide rectangles, so the column
        // test is a precomputed additive bias (0 or -inf); the row test is one
        // unsigned compare per n8 block.
        float gmx[GCH][2];
#pragma unroll
        for (int gi = 0; gi < GCH; ++gi) {
          const int gg = g0 + gi;
          const bool live = gg < ngroups;
#pragma unroll
          for (int nb = 0; nb < 2; ++nb) {
            const int row = (gg * 16 + nb * 8) >> LS;   // rectangle row of this n8 block
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
              const bool rok = live && ((unsigned)(row - rlo[rr]) < (unsigned)p.kh);
              const int half = (LS == 5) ? (gg & 1) : 0;
              const float cb0 = cbias[half][nb][rr][0], cb1 = cbias[half][nb][rr][1];
              s[gi][nb][2 * rr] = rok ? fmaf(s[gi][nb][2 * rr], p.scale_log2, cb0) : -INFINITY;
              s[gi][nb][2 * rr + 1] = rok ? fmaf(s[gi][nb][2 * rr + 1], p.scale_log2, cb1) : -INFINITY;
            }
          }
#pragma unroll
          for (int rr = 0; rr < 2; ++rr)
            gmx[gi][rr] = fmaxf(fmaxf(s[gi][0][2 * rr], s[gi][0][2 * rr + 1]),
                                fmaxf(s[gi][1][2 * rr], s[gi][1][2 * rr + 1]));
        }
        float mx[2];
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {   // tree over the groups
          float a = fmaxf(fmaxf(gmx[0][rr], gmx[1][rr]), fmaxf(gmx[2][rr], gmx[3][rr]));
          float b = fmaxf(fmaxf(gmx[4][rr], gmx[5][rr]), fmaxf(gmx[6][rr], gmx[7][rr]));
          mx[rr] = fmaxf(a, b);
        }
        float mref[2];
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
          mx[rr] = fmaxf(mx[rr], __shfl_xor_sync(0xffffffffu, mx[rr], 1));
          mx[rr] = fmaxf(mx[rr], __shfl_xor_sync(0xffffffffu, mx[rr], 2));
          const float mnew = fmaxf(mrow[rr], mx[rr]);
          mref[rr] = (mnew == -INFINITY) ? 0.f : mnew;
          const float alpha = ex2(mrow[rr] - mref[rr]);
          mrow[rr] = mnew;
          lrow[rr] *= alpha;
#pragma unroll
          for (int nd = 0; nd < ND; ++nd) {
            o[nd][2 * rr] *= alpha;
            o[nd][2 * rr + 1] *= alpha;
          }
        }
        // P = exp2(S - m), row sums (per thread; quad-reduced at the end), O += P V
        float lsum[GCH][2];
#pragma unroll
        for (int gi = 0; gi < GCH; ++gi) {
          if (g0 + gi >= ngroups) {
            lsum[gi][0] = lsum[gi][1] = 0.f;
            continue;
          }
          float pr[2][4];
#pragma unroll
          for (int nb = 0; nb < 2; ++nb)
#pragma unroll
            for (int e = 0; e < 4; ++e) pr[nb][e] = ex2(s[gi][nb][e] - mref[e >> 1]);
          lsum[gi][0] = (pr[0][0] + pr[0][1]) + (pr[1][0] + pr[1][1]);
          lsum[gi][1] = (pr[0][2] + pr[0][3]) + (pr[1][2] + pr[1][3]);
          const uint32_t pa0 = pack_bf16(pr[0][0], pr[0][1]);
          const uint32_t pa1 = pack_bf16(pr[0][2], pr[0][3]);
          const uint32_t pa2 = pack_bf16(pr[1][0], pr[1][1]);
          const uint32_t pa3 = pack_bf16(pr[1][2], pr[1][3]);
          int jv = (g0 + gi) * 16 + (mi & 1) * 8 + (lane & 7);
          if (jv >= nkeys) jv = 0;
          const int vrow = (wr0 + (jv >> ls)) * WC + wc0 + (jv & smask);
#pragma unroll
          for (int nd = 0; nd < ND; nd += 2) {
            uint32_t b0, b1, b2, b3;
            ldsm_x4_t(sV32 + (uint32_t)((vrow * DHP + nd * 8 + (mi >> 1) * 8) * 2), b0, b1, b2, b3);
            mma_bf16(o[nd], pa0, pa1, pa2, pa3, b0, b1);
            mma_bf16(o[nd + 1], pa0, pa1, pa2, pa3, b2, b3);
          }
        }
#pragma unroll
        for (int rr = 0; rr < 2; ++rr)
          lrow[rr] += ((lsum[0][rr] + lsum[1][rr]) + (lsum[2][rr] + lsum[3][rr])) +
                      ((lsum[4][rr] + lsum[5][rr]) + (lsum[6][rr] + lsum[7][rr]));
      }
    }
    __syncthreads();
  }

  if (!warp_live) return;
#pragma unroll
  for (int rr = 0; rr < 2; ++rr) {
    float l = lrow[rr];
    l += __shfl_xor_sync(0xffffffffu, l, 1);
    l += __shfl_xor_sync(0xffffffffu, l, 2);
    const float inv = 1.f / l;
    if (!qvalid[rr]) continue;
    const long tok = ((long)d * H + qh[rr]) * W + qw[rr];
    __nv_bfloat16* orow = p.out + ((long)b * N + tok) * p.C + head * DH;
#pragma unroll
    for (int nd = 0; nd < ND; ++nd)
      *reinterpret_cast<uint32_t*>(orow + nd * 8 + 2 * t4) = pack_bf16(o[nd][2 * rr] * inv, o[nd][2 * rr + 1] * inv);
  }
}

}  // namespace na

template <int DH>
static wm_status prep_dh(int lim) {
  WM_CUDA(cudaFuncSetAttribute(na::na_bf16_kernel<DH, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  WM_CUDA(cudaFuncSetAttribute(na::na_bf16_kernel<DH, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  WM_CUDA(cudaFuncSetAttribute(na::na_bf16_kernel<DH, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  return WM_OK;
}

wm_status prepare_na_bf16() {
  const int lim = 200 * 1024;  // the launcher never asks for more
  wm_status st = prep_dh<16>(lim);
  if (st == WM_OK) st = prep_dh<32>(lim);
  if (st == WM_OK) st = prep_dh<48>(lim);
  if (st == WM_OK) st = prep_dh<64>(lim);
  return st;
}

// smallest power of two >= max(8, v)
static int pow2span(int v) {
  int s = 8;
  while (s < v) s <<= 1;
  return s;
}

namespace {

struct NaPlan {
  int NWH, NWW;  // warp grid of a CTA (query tile = NWH*WH x NWW*WW)
};

using NaKey = std::array<int, 11>;
std::mutex g_na_mu;
std::map<NaKey, NaPlan> g_na_plans;  // autotuned plans

NaKey na_key(int B, int D, int H, int W, int C, int heads, int kd, int kh, int kw, bool per) {
  return NaKey{B, D, H, W, C, heads, kd, kh, kw, per ? 1 : 0, 0};
}

// Warp patch (WH x WW queries) with the fewest issued keys per query per
// level; fixed by the window alone, so a query's arithmetic (its key
// rectangle and the order it is walked in) never depends on the CTA plan.
bool warp_patch(int kh, int kw, int* WH, int* WW, int* span) {
  const int cand[5][2] = {{1, 16}, {2, 8}, {4, 4}, {8, 2}, {16, 1}};
  int best = -1, best_cost = 1 << 30;
  for (int i = 0; i < 5; ++i) {
    if (cand[i][1] + kw - 1 > 32) continue;
    const int cost = (cand[i][0] + kh - 1) * pow2span(cand[i][1] + kw - 1);
    if (cost < best_cost) {
      best_cost = cost;
      best = i;
    }
  }
  if (best < 0) return false;
  *WH = cand[best][0];
  *WW = cand[best][1];
  *span = pow2span(*WW + kw - 1);
  return true;
}

size_t plan_smem(const NaPlan& pl, int WH, int WW, int span, int kh, int H, int dh) {
  const int hr = std::min(pl.NWH * WH + kh - 1, H);
  const int wc = (pl.NWW - 1) * WW + span;
  return (size_t)2 * 2 * hr * wc * (dh + 8) * 2;
}

std::vector<NaPlan> na_candidates(int WH, int WW, int span, int kh, int H, int dh) {
  std::vector<NaPlan> out;
  for (int nw : {8, 12})
    for (int nwh = 1; nwh <= nw; ++nwh) {
      if (nw % nwh) continue;
      NaPlan pl{nwh, nw / nwh};
      if (plan_smem(pl, WH, WW, span, kh, H, dh) <= 200 * 1024) out.push_back(pl);
    }
  return out;
}

// Heuristic when no tuned plan exists: fewest staged keys per query times
// tile waste, over the candidates with the most warps that still give every
// SM a CTA.
NaPlan na_heuristic(int B, int D, int H, int W, int heads, int WH, int WW, int span, int kh, int dh) {
  NaPlan best{0, 0};
  double best_score = 1e30;
  for (const NaPlan& pl : na_candidates(WH, WW, span, kh, H, dh)) {
    const int TH = pl.NWH * WH, TW = pl.NWW * WW;
    const int th = (H + TH - 1) / TH, tw = (W + TW - 1) / TW;
    const int hr = std::min(TH + kh - 1, H), wc = (pl.NWW - 1) * WW + span;
    const long ctas = (long)th * tw * D * B * heads;
    double score = (double)hr * wc / (TH * TW) * ((double)th * TH / H) * ((double)tw * TW / W);
    if (ctas < num_sms()) score *= (double)num_sms() / ctas;   // idle SMs
    score /= std::sqrt((double)(pl.NWH * pl.NWW) / 8.0);      // more warps hide more latency
    if (score < best_score) {
      best_score = score;
      best = pl;
    }
  }
  return best;
}

template <int DH>
wm_status launch_plan(const NaPlan& pl, na::Params p, int WH, int WW, int span, cudaStream_t s) {
  p.WH = WH;
  p.WW = WW;
  p.log2span = 0;
  while ((1 << p.log2span) < span) ++p.log2span;
  p.NWH = pl.NWH;
  p.NWW = pl.NWW;
  p.HRmax = std::min(p.NWH * p.WH + p.kh - 1, p.H);
  p.WC = (p.NWW - 1) * p.WW + span;
  const int TH = p.NWH * p.WH, TW = p.NWW * p.WW;
  const int tiles_h = (p.H + TH - 1) / TH;
  p.tiles_w = (p.W + TW - 1) / TW;
  p.scale_log2 = 1.4426950408889634f / sqrtf((float)DH);
  if ((long)p.B * p.heads > 65535 || p.D > 65535) return fail(WM_ERR_INVALID_ARG, "batch*heads or D too large");
  dim3 grid(tiles_h * p.tiles_w, p.D, p.B * p.heads), block(32 * p.NWH * p.NWW);
  const int smem = (int)plan_smem(pl, WH, WW, span, p.kh, p.H, DH);
  switch (p.log2span) {
    case 3: na::na_bf16_kernel<DH, 3><<<grid, block, smem, s>>>(p); break;
    case 4: na::na_bf16_kernel<DH, 4><<<grid, block, smem, s>>>(p); break;
    case 5: na::na_bf16_kernel<DH, 5><<<grid, block, smem, s>>>(p); break;
    default: return fail(WM_ERR_INVALID_ARG, "unsupported key rectangle width");
  }
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

wm_status launch_with(const NaPlan& pl, const na::Params& p, int dh, int WH, int WW, int span, cudaStream_t s) {
  switch (dh) {
    case 16: return launch_plan<16>(pl, p, WH, WW, span, s);
    case 32: return launch_plan<32>(pl, p, WH, WW, span, s);
    case 48: return launch_plan<48>(pl, p, WH, WW, span, s);
    case 64: return launch_plan<64>(pl, p, WH, WW, span, s);
    default: return fail(WM_ERR_INVALID_ARG, "BF16 attention needs head dim 16, 32, 48 or 64");
  }
}

na::Params make_params(const __nv_bfloat16* qkv, __nv_bfloat16* out, int B, int D, int H, int W, int C, int heads,
                       int kd, int kh, int kw, bool periodic) {
  na::Params p{};
  p.qkv = qkv;
  p.out = out;
  p.B = B; p.D = D; p.H = H; p.W = W; p.C = C; p.heads = heads;
  p.kd = kd; p.kh = kh; p.kw = kw; p.periodic = periodic ? 1 : 0;
  return p;
}

}  // namespace

wm_status launch_na_bf16(const __nv_bfloat16* qkv, __nv_bfloat16* out, int B, int D, int H, int W, int C, int heads,
                         int kd, int kh, int kw, bool periodic, cudaStream_t s) {
  if (B <= 0) return WM_OK;
  const int dh = C / heads;
  int WH, WW, span;
  if (!warp_patch(kh, kw, &WH, &WW, &span))
    return fail(WM_ERR_INVALID_ARG, "longitude window too wide for the BF16 attention kernel");
  NaPlan pl{0, 0};
  {
    std::lock_guard<std::mutex> lk(g_na_mu);
    auto it = g_na_plans.find(na_key(B, D, H, W, C, heads, kd, kh, kw, periodic));
    if (it != g_na_plans.end()) pl = it->second;
  }
  if (!pl.NWH) pl = na_heuristic(B, D, H, W, heads, WH, WW, span, kh, dh);
  if (!pl.NWH) return fail(WM_ERR_INVALID_ARG, "attention window too large for the BF16 attention kernel");
  return launch_with(pl, make_params(qkv, out, B, D, H, W, C, heads, kd, kh, kw, periodic), dh, WH, WW, span, s);
}

// Time every candidate CTA plan for this shape (1 warm-up + 3 timed launches
// each, CUDA events on `s`) and keep the fastest for later launches. The
// outputs are written to `out`; results do not depend on the plan.
wm_status autotune_na_bf16(const __nv_bfloat16* qkv, __nv_bfloat16* out, int B, int D, int H, int W, int C,
                           int heads, int kd, int kh, int kw, bool periodic, cudaStream_t s, double* best_ms) {
  const int dh = C / heads;
  int WH, WW, span;
  if (!warp_patch(kh, kw, &WH, &WW, &span)) return fail(WM_ERR_INVALID_ARG, "window too wide");
  const na::Params p = make_params(qkv, out, B, D, H, W, C, heads, kd, kh, kw, periodic);
  cudaEvent_t e0, e1;
  WM_CUDA(cudaEventCreate(&e0));
  WM_CUDA(cudaEventCreate(&e1));
  NaPlan best{0, 0};
  float best_t = 1e30f;
  wm_status st = WM_OK;
  for (const NaPlan& pl : na_candidates(WH, WW, span, kh, H, dh)) {
    st = launch_with(pl, p, dh, WH, WW, span, s);
    if (st != WM_OK) break;
    cudaEventRecord(e0, s);
    for (int r = 0; r < 3 && st == WM_OK; ++r) st = launch_with(pl, p, dh, WH, WW, span, s);
    cudaEventRecord(e1, s);
    if (st != WM_OK) break;
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      st = fail(WM_ERR_CUDA, "autotune synchronisation failed");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_t) {
      best_t = ms;
      best = pl;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != WM_OK) return st;
  if (best.NWH) {
    std::lock_guard<std::mutex> lk(g_na_mu);
    g_na_plans[na_key(B, D, H, W, C, heads, kd, kh, kw, periodic)] = best;
  }
  if (best_ms) *best_ms = best_t / 3.0;
  return WM_OK;
}

}  // namespace wm
