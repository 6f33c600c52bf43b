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
#include <cstdio>
#include <string>
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
  int nbuf;               // slab ring depth of the persistent kernel (2 or 3)
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

// ----------------------------------------------------------------------------
// Pieces shared by both kernels. A "tile" is one CTA's unit of work: batch
// element b, head, query level d and a TH x TW lat-lon block of queries at
// (h0, w0). Its key levels are ld0 .. ld0 + kd - 1; each level's K/V slab
// covers latitudes hs0 .. hs0 + HR - 1 and WC longitudes from ws0 (wrapped
// modulo W when periodic).

struct Tile {
  int b, head, d, h0, w0;
  int ld0, hs0, HR, ws0;
};

__device__ __forceinline__ Tile make_tile(const Params& p, int t) {
  Tile T;
  const int TH = p.NWH * p.WH, TW = p.NWW * p.WW;
  const int tiles_h = (p.H + TH - 1) / TH;
  const int tw = t % p.tiles_w;
  t /= p.tiles_w;
  const int th = t % tiles_h;
  t /= tiles_h;
  T.d = t % p.D;
  const int bh = t / p.D;
  T.b = bh / p.heads;
  T.head = bh % p.heads;
  T.h0 = th * TH;
  T.w0 = tw * TW;
  const int rh = p.kh / 2, rw = p.kw / 2;
  T.ld0 = clampi(T.d - p.kd / 2, 0, p.D - p.kd);
  T.hs0 = clampi(T.h0 - rh, 0, p.H - p.kh);
  T.HR = clampi(min(T.h0 + TH, p.H) - 1 - rh, 0, p.H - p.kh) + p.kh - T.hs0;
  T.ws0 = p.periodic ? (T.w0 - rw) : clampi(T.w0 - rw, 0, p.W - p.kw);
  return T;
}

// cp.async one key level's K and V slabs into `sbuf` with threads
// [0, nthreads) of the caller's group (thread index `tid`). Each thread owns
// fixed (K or V, slab column, 16-byte chunk) items and walks the slab rows.
template <int DH>
__device__ __forceinline__ void load_level(const Params& p, const Tile& T, int lev, __nv_bfloat16* sbuf, int slab,
                                           int tid, int nthreads) {
  constexpr int DHP = DH + 8, CH = DH / 8;
  const long C3 = 3L * p.C;
  const long N = (long)p.D * p.H * p.W;
  const int WC = p.WC;
  const __nv_bfloat16* lbase = p.qkv + (long)T.b * N * C3 + ((long)lev * p.H + T.hs0) * p.W * C3 + (1L * p.C) +
                               T.head * DH;
  const long sstep = (long)p.W * C3;
  const uint32_t dstep = (uint32_t)(WC * DHP * 2);
  for (int it = tid; it < 2 * WC * CH; it += nthreads) {
    const int kv = it / (WC * CH);
    const int rem = it - kv * (WC * CH);
    const int c = rem / CH, ch = rem - c * CH;
    int lon = T.ws0 + c;
    bool ok = true;
    if (p.periodic) {
      if (lon < 0 || lon >= p.W) lon = ((lon % p.W) + p.W) % p.W;
    } else if (lon >= p.W) {
      ok = false;
      lon = 0;
    }
    const __nv_bfloat16* src = lbase + (long)lon * C3 + kv * p.C + ch * 8;
    uint32_t dst = (uint32_t)__cvta_generic_to_shared(sbuf + (size_t)kv * slab + (size_t)c * DHP + ch * 8);
    for (int r = 0; r < T.HR; ++r) {
      cp_async16(dst, ok ? (const void*)src : (const void*)p.qkv, ok ? 16 : 0);
      src += sstep;
      dst += dstep;
    }
  }
}

// Per-warp state: the warp's 16 queries (a WH x WW patch), its key rectangle
// inside the slab, the Q fragments, and the running softmax / output.
template <int DH, int LS>
struct WarpQ {
  static constexpr int KC = DH / 16, ND = DH / 8;
  uint32_t qa[KC][4];
  float o[ND][4];
  float mrow[2], lrow[2];
  int rlo[2];
  float cbias[2][2][2][2];
  int wr0, wc0, nkeys, ngroups;
  int qh[2], qw[2];
  bool qvalid[2];
  bool live;
};

template <int DH, int LS>
__device__ __forceinline__ void warp_begin(WarpQ<DH, LS>& q, const Params& p, const Tile& T, int warp, int lane) {
  constexpr int KC = DH / 16, ND = DH / 8;
  constexpr int smask = (1 << LS) - 1;
  const int g = lane >> 2, t4 = lane & 3;
  const int H = p.H, W = p.W;
  const int rh = p.kh / 2, rw = p.kw / 2;
  const int wy = warp / p.NWW, wx = warp % p.NWW;
  const int wh0 = T.h0 + wy * p.WH, ww0 = T.w0 + wx * p.WW;
  q.live = (wh0 < H) && (ww0 < W);
  int qsr[2], qsc[2];
#pragma unroll
  for (int rr = 0; rr < 2; ++rr) {
    const int qi = g + 8 * rr;
    q.qh[rr] = wh0 + qi / p.WW;
    q.qw[rr] = ww0 + qi % p.WW;
    q.qvalid[rr] = (q.qh[rr] < H) && (q.qw[rr] < W);
    const int hc = min(q.qh[rr], H - 1), wc = min(q.qw[rr], W - 1);
    qsr[rr] = clampi(hc - rh, 0, H - p.kh) - T.hs0;
    qsc[rr] = p.periodic ? (wc - T.w0) : (clampi(wc - rw, 0, W - p.kw) - T.ws0);
  }
  q.wr0 = clampi(min(wh0, H - 1) - rh, 0, H - p.kh) - T.hs0;
  const int wr1 = clampi(min(wh0 + p.WH - 1, H - 1) - rh, 0, H - p.kh) + p.kh - T.hs0;
  q.wc0 = p.periodic ? (ww0 - T.w0) : (clampi(min(ww0, W - 1) - rw, 0, W - p.kw) - T.ws0);
  q.nkeys = (wr1 - q.wr0) << LS;
  q.ngroups = (q.nkeys + 15) / 16;
  uint32_t colmask[2];
#pragma unroll
  for (int rr = 0; rr < 2; ++rr) {
    q.rlo[rr] = qsr[rr] - q.wr0;
    colmask[rr] = (0xFFFFFFFFu >> (32 - p.kw)) << max(qsc[rr] - q.wc0, 0);
  }
#pragma unroll
  for (int hf = 0; hf < 2; ++hf)
#pragma unroll
    for (int nb = 0; nb < 2; ++nb)
#pragma unroll
      for (int rr = 0; rr < 2; ++rr)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int col = (hf * 16 + nb * 8 + 2 * t4 + e) & smask;
          q.cbias[hf][nb][rr][e] = ((colmask[rr] >> col) & 1u) ? 0.f : -INFINITY;
        }
  const long N = (long)p.D * H * W;
  const long C3 = 3L * p.C;
  const __nv_bfloat16* base = p.qkv + (long)T.b * N * C3;
  const long tok0 = ((long)T.d * H + min(q.qh[0], H - 1)) * W + min(q.qw[0], W - 1);
  const long tok1 = ((long)T.d * H + min(q.qh[1], H - 1)) * W + min(q.qw[1], W - 1);
  const __nv_bfloat16* q0 = base + tok0 * C3 + T.head * DH;
  const __nv_bfloat16* q1 = base + tok1 * C3 + T.head * DH;
#pragma unroll
  for (int kc = 0; kc < KC; ++kc) {
    q.qa[kc][0] = *reinterpret_cast<const uint32_t*>(q0 + kc * 16 + 2 * t4);
    q.qa[kc][1] = *reinterpret_cast<const uint32_t*>(q1 + kc * 16 + 2 * t4);
    q.qa[kc][2] = *reinterpret_cast<const uint32_t*>(q0 + kc * 16 + 8 + 2 * t4);
    q.qa[kc][3] = *reinterpret_cast<const uint32_t*>(q1 + kc * 16 + 8 + 2 * t4);
  }
#pragma unroll
  for (int nd = 0; nd < ND; ++nd) q.o[nd][0] = q.o[nd][1] = q.o[nd][2] = q.o[nd][3] = 0.f;
  q.mrow[0] = q.mrow[1] = -INFINITY;
  q.lrow[0] = q.lrow[1] = 0.f;
}

// One key level: S = Q K^T over the warp's rectangle (up to GCH groups of 16
// keys before one online-softmax update), mask, softmax update, O += P V.
template <int DH, int LS, int GCH>
__device__ __forceinline__ void warp_level(WarpQ<DH, LS>& q, const Params& p, uint32_t sK32, uint32_t sV32, int lane) {
  constexpr int DHP = DH + 8, KC = DH / 16, ND = DH / 8;
  constexpr int ls = LS, smask = (1 << LS) - 1;
  const int WC = p.WC;
  const int mi = lane >> 3;
  for (int g0 = 0; g0 < q.ngroups; g0 += GCH) {
    float s[GCH][2][4];
#pragma unroll
    for (int gi = 0; gi < GCH; ++gi) {
#pragma unroll
      for (int nb = 0; nb < 2; ++nb) s[gi][nb][0] = s[gi][nb][1] = s[gi][nb][2] = s[gi][nb][3] = 0.f;
      if (g0 + gi < q.ngroups) {
        int jk = (g0 + gi) * 16 + (mi >> 1) * 8 + (lane & 7);
        if (jk >= q.nkeys) jk = 0;
        const int krow = (q.wr0 + (jk >> ls)) * WC + q.wc0 + (jk & smask);
#pragma unroll
        for (int kc = 0; kc < KC; ++kc) {
          uint32_t b0, b1, b2, b3;
          ldsm_x4(sK32 + (uint32_t)((krow * DHP + kc * 16 + (mi & 1) * 8) * 2), b0, b1, b2, b3);
          mma_bf16(s[gi][0], q.qa[kc][0], q.qa[kc][1], q.qa[kc][2], q.qa[kc][3], b0, b1);
          mma_bf16(s[gi][1], q.qa[kc][0], q.qa[kc][1], q.qa[kc][2], q.qa[kc][3], b2, b3);
        }
      }
    }
    // mask + scale + chunk row max. Key j sits at rectangle row j >> LS and
    // column j & smask. The column of each accumulator entry depends on the
    // group only through (g & 1) for 32-wide rectangles, so the column test
    // is a precomputed additive bias (0 or -inf); the row test is one
    // unsigned compare per n8 block.
    float gmx[GCH][2];
#pragma unroll
    for (int gi = 0; gi < GCH; ++gi) {
      const int gg = g0 + gi;
      const bool live = gg < q.ngroups;
#pragma unroll
      for (int nb = 0; nb < 2; ++nb) {
        const int row = (gg * 16 + nb * 8) >> LS;
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
          const bool rok = live && ((unsigned)(row - q.rlo[rr]) < (unsigned)p.kh);
          const int half = (LS == 5) ? (gg & 1) : 0;
          const float cb0 = q.cbias[half][nb][rr][0], cb1 = q.cbias[half][nb][rr][1];
          s[gi][nb][2 * rr] = rok ? fmaf(s[gi][nb][2 * rr], p.scale_log2, cb0) : -INFINITY;
          s[gi][nb][2 * rr + 1] = rok ? fmaf(s[gi][nb][2 * rr + 1], p.scale_log2, cb1) : -INFINITY;
        }
      }
#pragma unroll
      for (int rr = 0; rr < 2; ++rr)
        gmx[gi][rr] = fmaxf(fmaxf(s[gi][0][2 * rr], s[gi][0][2 * rr + 1]), fmaxf(s[gi][1][2 * rr], s[gi][1][2 * rr + 1]));
    }
    float mref[2];
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {   // tree over the groups, then the quad
      float mx = fmaxf(fmaxf(gmx[0][rr], gmx[1][rr]), fmaxf(gmx[2][rr], gmx[3][rr]));
      if constexpr (GCH == 8)
        mx = fmaxf(mx, fmaxf(fmaxf(gmx[4][rr], gmx[5][rr]), fmaxf(gmx[6][rr], gmx[7][rr])));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
      const float mnew = fmaxf(q.mrow[rr], mx);
      mref[rr] = (mnew == -INFINITY) ? 0.f : mnew;
      const float alpha = ex2(q.mrow[rr] - mref[rr]);
      q.mrow[rr] = mnew;
      q.lrow[rr] *= alpha;
#pragma unroll
      for (int nd = 0; nd < ND; ++nd) {
        q.o[nd][2 * rr] *= alpha;
        q.o[nd][2 * rr + 1] *= alpha;
      }
    }
    // P = exp2(S - m), row sums (per thread; quad-reduced at the end), O += P V
    float lsum[GCH][2];
#pragma unroll
    for (int gi = 0; gi < GCH; ++gi) {
      if (g0 + gi >= q.ngroups) {
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
      if (jv >= q.nkeys) jv = 0;
      const int vrow = (q.wr0 + (jv >> ls)) * WC + q.wc0 + (jv & smask);
#pragma unroll
      for (int nd = 0; nd < ND; nd += 2) {
        uint32_t b0, b1, b2, b3;
        ldsm_x4_t(sV32 + (uint32_t)((vrow * DHP + nd * 8 + (mi >> 1) * 8) * 2), b0, b1, b2, b3);
        mma_bf16(q.o[nd], pa0, pa1, pa2, pa3, b0, b1);
        mma_bf16(q.o[nd + 1], pa0, pa1, pa2, pa3, b2, b3);
      }
    }
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
      float t = (lsum[0][rr] + lsum[1][rr]) + (lsum[2][rr] + lsum[3][rr]);
      if constexpr (GCH == 8) t += (lsum[4][rr] + lsum[5][rr]) + (lsum[6][rr] + lsum[7][rr]);
      q.lrow[rr] += t;
    }
  }
}

template <int DH, int LS>
__device__ __forceinline__ void warp_end(const WarpQ<DH, LS>& q, const Params& p, const Tile& T, int lane) {
  constexpr int ND = DH / 8;
  const int t4 = lane & 3;
  const long N = (long)p.D * p.H * p.W;
#pragma unroll
  for (int rr = 0; rr < 2; ++rr) {
    float l = q.lrow[rr];
    l += __shfl_xor_sync(0xffffffffu, l, 1);
    l += __shfl_xor_sync(0xffffffffu, l, 2);
    const float inv = 1.f / l;
    if (!q.qvalid[rr]) continue;
    const long tok = ((long)T.d * p.H + q.qh[rr]) * p.W + q.qw[rr];
    __nv_bfloat16* orow = p.out + ((long)T.b * N + tok) * p.C + T.head * DH;
#pragma unroll
    for (int nd = 0; nd < ND; ++nd)
      *reinterpret_cast<uint32_t*>(orow + nd * 8 + 2 * t4) = pack_bf16(q.o[nd][2 * rr] * inv, q.o[nd][2 * rr + 1] * inv);
  }
}

// ---------------------------------------------------------------------------
// Kernel A: one CTA per tile; all threads load a level (cp.async, double
// buffered), then all warps consume it; one CTA-wide barrier per level.
template <int DH, int LS, int GCH, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) na_bf16_kernel(const Params p) {
  constexpr int DHP = DH + 8;
  extern __shared__ __align__(16) __nv_bfloat16 sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const Tile T = make_tile(p, blockIdx.x);
  const int slab = p.HRmax * p.WC * DHP;
  WarpQ<DH, LS> q;
  warp_begin<DH, LS>(q, p, T, warp, lane);
  load_level<DH>(p, T, T.ld0, sm, slab, tid, blockDim.x);
  cp_async_commit();
  for (int li = 0; li < p.kd; ++li) {
    if (li + 1 < p.kd) load_level<DH>(p, T, T.ld0 + li + 1, sm + (size_t)((li + 1) & 1) * 2 * slab, slab, tid, blockDim.x);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    const uint32_t sK32 = (uint32_t)__cvta_generic_to_shared(sm + (size_t)(li & 1) * 2 * slab);
    if (q.live) warp_level<DH, LS, GCH>(q, p, sK32, sK32 + (uint32_t)slab * 2, lane);
    __syncthreads();
  }
  if (q.live) warp_end<DH, LS>(q, p, T, lane);
}

// ---------------------------------------------------------------------------
// Kernel B: persistent, warp-specialised. Warps 0 .. NW-1 consume; warp NW
// produces: it streams the key levels of this CTA's tiles, one after the
// other, through an NBUF-deep ring of slabs. full[b] completes when the
// producer's cp.async copies into slab b land (cp.async.mbarrier.arrive);
// empty[b] completes when every consumer warp has finished with slab b. A
// fast warp therefore never waits for a slow one, and the next tile's first
// levels load while the current tile finishes. Waits are bounded.

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool na_mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t addr = smem_addr(bar);
  unsigned long long t0 = 0;
  for (int spin = 0;; ++spin) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    if (ok) return true;
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (spin == 0) t0 = t;
    else if (t - t0 > kWaitLimitNs) return false;
  }
}

template <int DH, int LS, int GCH, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) na_bf16_pipe_kernel(const Params p, int ntiles, int* status) {
  constexpr int DHP = DH + 8;
  extern __shared__ __align__(16) __nv_bfloat16 sm[];
  __shared__ __align__(8) uint64_t full_bar[3];
  __shared__ __align__(8) uint64_t empty_bar[3];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int NW = p.NWH * p.NWW;      // consumer warps
  const int NBUF = p.nbuf;
  const int slab = p.HRmax * p.WC * DHP;
  if (tid == 0) {
    for (int i = 0; i < NBUF; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&full_bar[i])), "r"(32) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&empty_bar[i])), "r"(NW) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == NW) {
    // ------------------------------------------------------------- producer
    int it = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const Tile T = make_tile(p, t);
      for (int li = 0; li < p.kd; ++li, ++it) {
        const int buf = it % NBUF;
        const uint32_t ph = (uint32_t)(it / NBUF) & 1u;
        if (!na_mbar_wait(&empty_bar[buf], ph ^ 1u)) {
          ok = false;
          break;
        }
        load_level<DH>(p, T, T.ld0 + li, sm + (size_t)buf * 2 * slab, slab, lane, 32);
        asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(&full_bar[buf]))
                     : "memory");
      }
    }
    if (!ok) atomicExch(status, (int)WM_ERR_TIMEOUT);
    asm volatile("cp.async.wait_all;" ::: "memory");   // own copies land before this warp leaves
    return;
  }
  // ------------------------------------------------------------- consumers
  int it = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const Tile T = make_tile(p, t);
    WarpQ<DH, LS> q;
    warp_begin<DH, LS>(q, p, T, warp, lane);
    for (int li = 0; li < p.kd; ++li, ++it) {
      const int buf = it % NBUF;
      const uint32_t ph = (uint32_t)(it / NBUF) & 1u;
      if (!na_mbar_wait(&full_bar[buf], ph)) {
        atomicExch(status, (int)WM_ERR_TIMEOUT);
        return;
      }
      const uint32_t sK32 = smem_addr(sm + (size_t)buf * 2 * slab);
      if (q.live) warp_level<DH, LS, GCH>(q, p, sK32, sK32 + (uint32_t)slab * 2, lane);
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&empty_bar[buf])) : "memory");
    }
    if (q.live) warp_end<DH, LS>(q, p, T, lane);
  }
}

}  // namespace na

template <int DH>
static wm_status prep_dh(int lim) {
  WM_CUDA(cudaFuncSetAttribute(na::na_bf16_kernel<DH, 3, 8, 384>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  WM_CUDA(cudaFuncSetAttribute(na::na_bf16_kernel<DH, 4, 8, 384>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  WM_CUDA(cudaFuncSetAttribute(na::na_bf16_kernel<DH, 5, 8, 384>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  WM_CUDA(cudaFuncSetAttribute(na::na_bf16_kernel<DH, 3, 4, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  WM_CUDA(cudaFuncSetAttribute(na::na_bf16_kernel<DH, 4, 4, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  WM_CUDA(cudaFuncSetAttribute(na::na_bf16_kernel<DH, 5, 4, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  WM_CUDA(cudaFuncSetAttribute(na::na_bf16_pipe_kernel<DH, 3, 8, 288>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  WM_CUDA(cudaFuncSetAttribute(na::na_bf16_pipe_kernel<DH, 4, 8, 288>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  WM_CUDA(cudaFuncSetAttribute(na::na_bf16_pipe_kernel<DH, 5, 8, 288>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  WM_CUDA(cudaFuncSetAttribute(na::na_bf16_pipe_kernel<DH, 3, 4, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  WM_CUDA(cudaFuncSetAttribute(na::na_bf16_pipe_kernel<DH, 4, 4, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  WM_CUDA(cudaFuncSetAttribute(na::na_bf16_pipe_kernel<DH, 5, 4, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  return WM_OK;
}

static constexpr int kNaSmemLimit = 220 * 1024;   // dynamic smem the launcher may ask for

wm_status prepare_na_bf16() {
  wm_status st = prep_dh<16>(kNaSmemLimit);
  if (st == WM_OK) st = prep_dh<32>(kNaSmemLimit);
  if (st == WM_OK) st = prep_dh<48>(kNaSmemLimit);
  if (st == WM_OK) st = prep_dh<64>(kNaSmemLimit);
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
  int NWH, NWW;  // consumer warp grid of a CTA (query tile = NWH*WH x NWW*WW)
  int kind;      // 0: one CTA per tile, CTA-wide barrier per level; 1: persistent producer/consumer
  int nbuf;      // slab buffers (kind 0: 2; kind 1: 2 or 3)
  int gch;       // 16-key groups scored per softmax update (8, or 4 for 16-warp CTAs)
};

using NaKey = std::array<int, 11>;
std::mutex g_na_mu;
std::map<NaKey, NaPlan> g_na_plans;  // autotuned plans
std::map<NaKey, double> g_na_ms;     // their measured time per launch
std::map<NaKey, int> g_na_gch;       // softmax chunk fixed per shape (key with B = 0) at its first tuning
std::string g_na_log;                 // every candidate's time, for the report

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
  return (size_t)pl.nbuf * 2 * hr * wc * (dh + 8) * 2;
}

// Candidate plans. gch = 0 allows both chunk sizes; otherwise only plans
// with that chunk size (the chunk size changes where the online softmax
// rescales, hence the rounding, so it is fixed per problem shape).
std::vector<NaPlan> na_candidates(int WH, int WW, int span, int kh, int H, int dh, int gch) {
  std::vector<NaPlan> out;
  if (gch != 4) {
    for (int nw : {8, 12})
      for (int nwh = 1; nwh <= nw; ++nwh) {
        if (nw % nwh) continue;
        NaPlan pl{nwh, nw / nwh, 0, 2, 8};
        if (plan_smem(pl, WH, WW, span, kh, H, dh) <= (size_t)kNaSmemLimit) out.push_back(pl);
      }
    for (int nbuf : {2, 3})
      for (int nwh = 1; nwh <= 8; nwh *= 2) {
        NaPlan pl{nwh, 8 / nwh, 1, nbuf, 8};
        if (plan_smem(pl, WH, WW, span, kh, H, dh) <= (size_t)kNaSmemLimit) out.push_back(pl);
      }
  }
  if (gch != 8) {
    for (int nwh = 1; nwh <= 16; nwh *= 2) {
      NaPlan pl{nwh, 16 / nwh, 0, 2, 4};
      if (plan_smem(pl, WH, WW, span, kh, H, dh) <= (size_t)kNaSmemLimit) out.push_back(pl);
    }
    for (int nw : {12, 15})
      for (int nbuf : {2, 3})
        for (int nwh = 1; nwh <= nw; ++nwh) {
          if (nw % nwh) continue;
          NaPlan pl{nwh, nw / nwh, 1, nbuf, 4};
          if (plan_smem(pl, WH, WW, span, kh, H, dh) <= (size_t)kNaSmemLimit) out.push_back(pl);
        }
  }
  return out;
}

// Heuristic when no tuned plan exists: fewest staged keys per query times
// tile waste; persistent plans are preferred when the tile count gives every
// SM several tiles.
NaPlan na_heuristic(int B, int D, int H, int W, int heads, int WH, int WW, int span, int kh, int dh) {
  NaPlan best{0, 0, 0, 2, 8};
  double best_score = 1e30;
  for (const NaPlan& pl : na_candidates(WH, WW, span, kh, H, dh, 8)) {
    const int TH = pl.NWH * WH, TW = pl.NWW * WW;
    const int th = (H + TH - 1) / TH, tw = (W + TW - 1) / TW;
    const int hr = std::min(TH + kh - 1, H), wc = (pl.NWW - 1) * WW + span;
    const long ctas = (long)th * tw * D * B * heads;
    double score = (double)hr * wc / (TH * TW) * ((double)th * TH / H) * ((double)tw * TW / W);
    if (ctas < num_sms()) score *= (double)num_sms() / ctas;   // idle SMs
    if (pl.kind == 1) score *= (ctas >= 4L * num_sms()) ? 0.8 : 1.5;
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
  p.nbuf = pl.nbuf;
  p.HRmax = std::min(p.NWH * p.WH + p.kh - 1, p.H);
  p.WC = (p.NWW - 1) * p.WW + span;
  const int TH = p.NWH * p.WH, TW = p.NWW * p.WW;
  const int tiles_h = (p.H + TH - 1) / TH;
  p.tiles_w = (p.W + TW - 1) / TW;
  p.scale_log2 = 1.4426950408889634f / sqrtf((float)DH);
  const long ntiles = (long)tiles_h * p.tiles_w * p.D * p.B * p.heads;
  if (ntiles > (1L << 30)) return fail(WM_ERR_INVALID_ARG, "too many attention tiles");
  const int smem = (int)plan_smem(pl, WH, WW, span, p.kh, p.H, DH);
  if (pl.kind == 0 && pl.gch == 8) {
    dim3 grid((unsigned)ntiles), block(32 * p.NWH * p.NWW);
    switch (p.log2span) {
      case 3: na::na_bf16_kernel<DH, 3, 8, 384><<<grid, block, smem, s>>>(p); break;
      case 4: na::na_bf16_kernel<DH, 4, 8, 384><<<grid, block, smem, s>>>(p); break;
      case 5: na::na_bf16_kernel<DH, 5, 8, 384><<<grid, block, smem, s>>>(p); break;
      default: return fail(WM_ERR_INVALID_ARG, "unsupported key rectangle width");
    }
  } else if (pl.kind == 0) {
    dim3 grid((unsigned)ntiles), block(32 * p.NWH * p.NWW);
    switch (p.log2span) {
      case 3: na::na_bf16_kernel<DH, 3, 4, 512><<<grid, block, smem, s>>>(p); break;
      case 4: na::na_bf16_kernel<DH, 4, 4, 512><<<grid, block, smem, s>>>(p); break;
      case 5: na::na_bf16_kernel<DH, 5, 4, 512><<<grid, block, smem, s>>>(p); break;
      default: return fail(WM_ERR_INVALID_ARG, "unsupported key rectangle width");
    }
  } else {
    const int grid = (int)std::min<long>(ntiles, num_sms());
    dim3 block(32 * (p.NWH * p.NWW + 1));
    int* st = device_status_word();
    if (pl.gch == 8) {
      switch (p.log2span) {
        case 3: na::na_bf16_pipe_kernel<DH, 3, 8, 288><<<grid, block, smem, s>>>(p, (int)ntiles, st); break;
        case 4: na::na_bf16_pipe_kernel<DH, 4, 8, 288><<<grid, block, smem, s>>>(p, (int)ntiles, st); break;
        case 5: na::na_bf16_pipe_kernel<DH, 5, 8, 288><<<grid, block, smem, s>>>(p, (int)ntiles, st); break;
        default: return fail(WM_ERR_INVALID_ARG, "unsupported key rectangle width");
      }
    } else {
      switch (p.log2span) {
        case 3: na::na_bf16_pipe_kernel<DH, 3, 4, 512><<<grid, block, smem, s>>>(p, (int)ntiles, st); break;
        case 4: na::na_bf16_pipe_kernel<DH, 4, 4, 512><<<grid, block, smem, s>>>(p, (int)ntiles, st); break;
        case 5: na::na_bf16_pipe_kernel<DH, 5, 4, 512><<<grid, block, smem, s>>>(p, (int)ntiles, st); break;
        default: return fail(WM_ERR_INVALID_ARG, "unsupported key rectangle width");
      }
    }
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
  NaPlan pl{0, 0, 0, 2, 8};
  int gch = 8;
  {
    std::lock_guard<std::mutex> lk(g_na_mu);
    auto it = g_na_plans.find(na_key(B, D, H, W, C, heads, kd, kh, kw, periodic));
    if (it != g_na_plans.end()) pl = it->second;
    auto ig = g_na_gch.find(na_key(0, D, H, W, C, heads, kd, kh, kw, periodic));
    if (ig != g_na_gch.end()) gch = ig->second;
  }
  if (!pl.NWH) {
    pl = na_heuristic(B, D, H, W, heads, WH, WW, span, kh, dh);
    if (gch == 4) {   // keep the shape's chunk size: the widest 16-warp plan that fits
      for (const NaPlan& c : na_candidates(WH, WW, span, kh, H, dh, 4)) pl = c;
    }
  }
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
  NaPlan best{0, 0, 0, 2, 8};
  float best_t = 1e30f;
  wm_status st = WM_OK;
  int gch_fixed = 0;
  {
    std::lock_guard<std::mutex> lk(g_na_mu);
    auto ig = g_na_gch.find(na_key(0, D, H, W, C, heads, kd, kh, kw, periodic));
    if (ig != g_na_gch.end()) gch_fixed = ig->second;
  }
  for (const NaPlan& pl : na_candidates(WH, WW, span, kh, H, dh, gch_fixed)) {
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
    {
      char line[160];
      std::snprintf(line, sizeof line, "  candidate B=%d %s warps=%dx%d buffers=%d chunk=%d: %.3f ms\n", B,
                    pl.kind ? "persistent" : "per-tile", pl.NWH, pl.NWW, pl.nbuf, pl.gch, ms / 3.0);
      std::lock_guard<std::mutex> lk(g_na_mu);
      g_na_log += line;
    }
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
    g_na_ms[na_key(B, D, H, W, C, heads, kd, kh, kw, periodic)] = best_t / 3.0;
    g_na_gch.emplace(na_key(0, D, H, W, C, heads, kd, kh, kw, periodic), best.gch);
  }
  if (best_ms) *best_ms = best_t / 3.0;
  return WM_OK;
}

std::string describe_na_plans() {
  std::lock_guard<std::mutex> lk(g_na_mu);
  std::string out;
  for (const auto& kv : g_na_plans) {
    const NaKey& k = kv.first;
    const NaPlan& pl = kv.second;
    char line[256];
    std::snprintf(line, sizeof line,
                  "attention B=%d D=%d H=%d W=%d C=%d heads=%d window=%dx%dx%d periodic=%d -> %s warps=%dx%d "
                  "buffers=%d chunk=%d %.3f ms\n",
                  k[0], k[1], k[2], k[3], k[4], k[5], k[6], k[7], k[8], k[9],
                  pl.kind ? "persistent" : "per-tile", pl.NWH, pl.NWW, pl.nbuf, pl.gch, g_na_ms[k]);
    out += line;
  }
  return out + g_na_log;
}

}  // namespace wm
