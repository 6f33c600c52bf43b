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
#include <type_traits>
#include <cmath>
#include <cstring>
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
  int slab;               // elements between the K and V slabs (and between ring buffers / 2); multiple of 64
  int tma;                // persistent kernel: non-wrapping slabs by one tensor copy each for K and V
  float scale_log2;       // log2(e) / sqrt(dh)
  int* dstatus;           // the device status word (debug builds record index-check failures there)
};

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// The online softmax moves its reference max only when a row's maximum grows
// by more than this many powers of two.
constexpr float kLazyLog2 = 8.f;

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


// First 128-byte aligned address at or after p (the launch adds 128 bytes).
__device__ __forceinline__ __nv_bfloat16* align128(__nv_bfloat16* p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  return p + (((128u - (a & 127u)) & 127u) >> 1);
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
  // debug builds: the key levels, the slab rows and its first column lie where
  // the loaders and the warps assume; a tile that fails loads nothing
  bool ok = WM_DCHECK(T.ld0 >= 0 && T.ld0 + p.kd <= p.D, p.dstatus);
  ok = WM_DCHECK(T.hs0 >= 0 && T.HR >= p.kh && T.HR <= p.HRmax && T.hs0 + T.HR <= p.H, p.dstatus) && ok;
  ok = WM_DCHECK(p.periodic ? (T.ws0 >= -rw && T.ws0 < p.W) : (T.ws0 >= 0 && T.ws0 + p.kw <= p.W), p.dstatus) && ok;
  if (!ok) T.HR = 0;
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
  uint64_t cbias[2][2][2];   // [half][n8 block][row]: packed (0 or -inf) pair for entries 2 t4, 2 t4 + 1
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
  // debug builds: the warp's key rectangle lies inside the slab, and each
  // query's window inside the rectangle; a warp that fails computes nothing
  if (q.live) {
    bool ok = WM_DCHECK(q.wr0 >= 0 && wr1 <= T.HR && q.wc0 >= 0 && q.wc0 + (1 << LS) <= p.WC, p.dstatus);
#pragma unroll
    for (int rr = 0; rr < 2; ++rr)
      ok = WM_DCHECK(qsr[rr] >= q.wr0 && qsr[rr] + p.kh <= wr1 && qsc[rr] >= q.wc0 &&
                         qsc[rr] + p.kw <= q.wc0 + (1 << LS),
                     p.dstatus) && ok;
    if (!ok) q.live = false;
  }
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
      for (int rr = 0; rr < 2; ++rr) {
        float cb[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int col = (hf * 16 + nb * 8 + 2 * t4 + e) & smask;
          cb[e] = ((colmask[rr] >> col) & 1u) ? 0.f : -INFINITY;
        }
        q.cbias[hf][nb][rr] = pack_f2(cb[0], cb[1]);
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

// Calls f(std::integral_constant<int, r>) for the runtime r in 1 .. R (no
// call for r = 0); r is warp-uniform.
template <int R, class F>
__device__ __forceinline__ void tail_chunk(int r, F& f) {
  if constexpr (R >= 1) {
    if (r == R) f(std::integral_constant<int, R>{});
    else tail_chunk<R - 1>(r, f);
  }
}

// One key level: S = Q K^T over the warp's rectangle (up to GCH groups of 16
// keys before one online-softmax update), mask, softmax update, O += P V.
template <int DH, int LS, int GCH>
__device__ __forceinline__ void warp_level(WarpQ<DH, LS>& q, const Params& p, uint32_t sK32, uint32_t sV32, int lane) {
  constexpr int DHP = DH + 8, KC = DH / 16, ND = DH / 8;
  constexpr int ls = LS, smask = (1 << LS) - 1;
  const int WC = p.WC;
  const int mi = lane >> 3;
  // Shared-memory byte address of this lane's ldmatrix row for key group gg.
  // For 8- and 16-wide rectangles a group is 2 or 1 whole rectangle rows, so
  // the address is the lane's row-0 address plus a row index clamped into the
  // rectangle (keys past it are masked). 32-wide rectangles use the general
  // row / column split.
  constexpr int RPG = LS == 3 ? 2 : 1;                   // rectangle rows per 16-key group (LS <= 4)
  const int last_row = (q.nkeys >> LS) - 1;
  const uint32_t rstride = (uint32_t)(WC * DHP * 2);
  const uint32_t kbase = sK32 + (uint32_t)(((q.wr0 * WC + q.wc0 +
                                             (LS == 3 ? (lane & 7) : (((mi >> 1) * 8 + (lane & 7)) & smask))) * DHP +
                                            (mi & 1) * 8) * 2);
  const uint32_t vbase = sV32 + (uint32_t)(((q.wr0 * WC + q.wc0 +
                                             (LS == 3 ? (lane & 7) : (((mi & 1) * 8 + (lane & 7)) & smask))) * DHP +
                                            (mi >> 1) * 8) * 2);
  auto k_addr = [&](int gg) -> uint32_t {
    if constexpr (LS <= 4) {
      return kbase + (uint32_t)min(RPG * gg + (LS == 3 ? (mi >> 1) : 0), last_row) * rstride;
    } else {
      int jk = gg * 16 + (mi >> 1) * 8 + (lane & 7);
      if (jk >= q.nkeys) jk = 0;
      const int krow = (q.wr0 + (jk >> ls)) * WC + q.wc0 + (jk & smask);
      return sK32 + (uint32_t)((krow * DHP + (mi & 1) * 8) * 2);
    }
  };
  auto v_addr = [&](int gg) -> uint32_t {
    if constexpr (LS <= 4) {
      return vbase + (uint32_t)min(RPG * gg + (LS == 3 ? (mi & 1) : 0), last_row) * rstride;
    } else {
      int jv = gg * 16 + (mi & 1) * 8 + (lane & 7);
      if (jv >= q.nkeys) jv = 0;
      const int vrow = (q.wr0 + (jv >> ls)) * WC + q.wc0 + (jv & smask);
      return sV32 + (uint32_t)((vrow * DHP + (mi >> 1) * 8) * 2);
    }
  };
  // One chunk of G groups starting at g0: S for all of them, one online
  // softmax update, O += P V. Full chunks have GCH groups; the level's last
  // chunk has exactly the groups left (a compile-time size 1 .. GCH - 1), so
  // no group is scored past the rectangle.
  int g0 = 0;
  auto chunk = [&](auto gsize) {
    constexpr int G = decltype(gsize)::value;
    // Every group of the chunk is scored, without a branch, so the groups'
    // MMA chains interleave.
    float s[G][2][4];
#pragma unroll
    for (int gi = 0; gi < G; ++gi) {
#pragma unroll
      for (int nb = 0; nb < 2; ++nb) s[gi][nb][0] = s[gi][nb][1] = s[gi][nb][2] = s[gi][nb][3] = 0.f;
    }
#pragma unroll
    for (int kc = 0; kc < KC; ++kc) {
#pragma unroll
      for (int gi = 0; gi < G; ++gi) {
        uint32_t b0, b1, b2, b3;
        ldsm_x4(k_addr(g0 + gi) + kc * 32, b0, b1, b2, b3);
        mma_bf16(s[gi][0], q.qa[kc][0], q.qa[kc][1], q.qa[kc][2], q.qa[kc][3], b0, b1);
        mma_bf16(s[gi][1], q.qa[kc][0], q.qa[kc][1], q.qa[kc][2], q.qa[kc][3], b2, b3);
      }
    }
    // mask + scale + chunk row max. Key j sits at rectangle row j >> LS and
    // column j & smask. The column of each accumulator entry depends on the
    // group only through (g & 1) for 32-wide rectangles, so the column test
    // is a precomputed additive bias (0 or -inf); the row test is one
    // unsigned compare per n8 block. Entries 2 t4 and 2 t4 + 1 of a row go
    // through the paired instructions together.
    const uint64_t scale2 = pack_f2(p.scale_log2, p.scale_log2);
    float gmx[G][2];
#pragma unroll
    for (int gi = 0; gi < G; ++gi) {
      const int gg = g0 + gi;
#pragma unroll
      for (int nb = 0; nb < 2; ++nb) {
        const int row = (gg * 16 + nb * 8) >> LS;
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
          const bool rok = (unsigned)(row - q.rlo[rr]) < (unsigned)p.kh;
          const int half = (LS == 5) ? (gg & 1) : 0;
          float t0, t1;
          fma_f2(t0, t1, s[gi][nb][2 * rr], s[gi][nb][2 * rr + 1], scale2, q.cbias[half][nb][rr]);
          s[gi][nb][2 * rr] = rok ? t0 : -INFINITY;
          s[gi][nb][2 * rr + 1] = rok ? t1 : -INFINITY;
        }
      }
#pragma unroll
      for (int rr = 0; rr < 2; ++rr)
        gmx[gi][rr] = max3(max3(s[gi][0][2 * rr], s[gi][0][2 * rr + 1], s[gi][1][2 * rr]), s[gi][1][2 * rr + 1],
                           -INFINITY);
    }
    float mx[2];
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {   // tree over the groups, then the quad
      float m = gmx[0][rr];
#pragma unroll
      for (int gi = 1; gi < G; gi += 2) m = gi + 1 < G ? max3(m, gmx[gi][rr], gmx[gi + 1][rr]) : fmaxf(m, gmx[gi][rr]);
      m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
      mx[rr] = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
    }
    // Lazy rescale: the reference max of the online softmax moves (and O and
    // the row sums are rescaled) only when some row of the warp sees its
    // maximum grow by more than kLazyLog2 (exponent units); otherwise the old
    // reference stays and the chunk's probabilities are at most 2^kLazyLog2,
    // well inside the FP32 accumulators and the bf16 P operand.
    const bool grow = (mx[0] > q.mrow[0] + kLazyLog2) || (mx[1] > q.mrow[1] + kLazyLog2);
    if (__any_sync(0xffffffffu, grow)) {
#pragma unroll
      for (int rr = 0; rr < 2; ++rr) {
        const float mnew = fmaxf(q.mrow[rr], mx[rr]);
        const float alpha = ex2(q.mrow[rr] - ((mnew == -INFINITY) ? 0.f : mnew));
        const uint64_t alpha2 = pack_f2(alpha, alpha);
        q.mrow[rr] = mnew;
        q.lrow[rr] *= alpha;
#pragma unroll
        for (int nd = 0; nd < ND; ++nd) mul_f2(q.o[nd][2 * rr], q.o[nd][2 * rr + 1], alpha2);
      }
    }
    float mref[2];
    uint64_t mref2[2];
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
      mref[rr] = (q.mrow[rr] == -INFINITY) ? 0.f : q.mrow[rr];
      mref2[rr] = pack_f2(mref[rr], mref[rr]);
    }
    // P = exp2(S - m), row sums (per thread; quad-reduced at the end), O += P V
    float lsum[G][2];
#pragma unroll
    for (int gi = 0; gi < G; ++gi) {
      float pr[2][4];
#pragma unroll
      for (int nb = 0; nb < 2; ++nb)
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
          float d0, d1;
          sub_f2(d0, d1, s[gi][nb][2 * rr], s[gi][nb][2 * rr + 1], mref2[rr]);
          pr[nb][2 * rr] = ex2(d0);
          pr[nb][2 * rr + 1] = ex2(d1);
        }
      // lsum[r] = (pr[0][2r] + pr[0][2r+1]) + (pr[1][2r] + pr[1][2r+1]), both rows at once
      float a0, a1, b0, b1;
      add_f2(a0, a1, pr[0][0], pr[0][2], pr[0][1], pr[0][3]);
      add_f2(b0, b1, pr[1][0], pr[1][2], pr[1][1], pr[1][3]);
      add_f2(lsum[gi][0], lsum[gi][1], a0, a1, b0, b1);
      const uint32_t pa0 = pack_bf16(pr[0][0], pr[0][1]);
      const uint32_t pa1 = pack_bf16(pr[0][2], pr[0][3]);
      const uint32_t pa2 = pack_bf16(pr[1][0], pr[1][1]);
      const uint32_t pa3 = pack_bf16(pr[1][2], pr[1][3]);
      const uint32_t va = v_addr(g0 + gi);
#pragma unroll
      for (int nd = 0; nd < ND; nd += 2) {
        uint32_t b0, b1, b2, b3;
        ldsm_x4_t(va + nd * 16, b0, b1, b2, b3);
        mma_bf16(q.o[nd], pa0, pa1, pa2, pa3, b0, b1);
        mma_bf16(q.o[nd + 1], pa0, pa1, pa2, pa3, b2, b3);
      }
    }
    // pairwise tree over the chunk's groups: ((0+1)+(2+3)) + ((4+5)+(6+7)) ...
#pragma unroll
    for (int w = 1; w < G; w *= 2)
#pragma unroll
      for (int i = 0; i + w < G; i += 2 * w)
        add_f2(lsum[i][0], lsum[i][1], lsum[i][0], lsum[i][1], lsum[i + w][0], lsum[i + w][1]);
    add_f2(q.lrow[0], q.lrow[1], q.lrow[0], q.lrow[1], lsum[0][0], lsum[0][1]);
  };
  for (; g0 + GCH <= q.ngroups; g0 += GCH) chunk(std::integral_constant<int, GCH>{});
  tail_chunk<GCH - 1>(q.ngroups - g0, chunk);
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
// Transposed formulation: a warp owns 8 queries (a WH x WW patch with
// WH * WW = 8) and computes S^T = K Q^T with 16 keys on the MMA's M side and
// the 8 queries on N, so the warp's key rectangle (the union of 8 windows) is
// smaller. Thread (g, t4) holds keys g and g + 8 of each 16-key group for
// queries 2 t4 and 2 t4 + 1. Row maxima and sums reduce over the 8 lanes that
// share t4. P^T is re-packed as bf16 8x8 blocks and transposed in registers
// (movmatrix) into the B operand of O^T += V^T P^T; V^T comes from the V slab
// by ldmatrix.trans.

__device__ __forceinline__ uint32_t movmatrix_t(uint32_t a) {
  uint32_t d;
  asm volatile("movmatrix.sync.aligned.m8n8.trans.b16 %0, %1;" : "=r"(d) : "r"(a));
  return d;
}

template <int DH, int LS>
struct WarpQT {
  static constexpr int KC = DH / 16, MD = DH / 16;
  uint32_t qb[KC][2];     // Q^T B fragments (query g)
  float o[MD][4];         // O^T: (dh g / g+8 of tile md) x (query 2t4 / 2t4+1)
  float mrow[2], lrow[2]; // queries 2t4, 2t4+1
  int rlo[2];
  uint64_t cbias2[2][2];  // [group parity][key row i = g / g + 8]: packed (0 or -inf) for queries 2 t4, 2 t4 + 1
  int wr0, wc0, nkeys, ngroups;
  int qh, qw;             // query g (the one this thread stores)
  bool qvalid, live;
};

template <int DH, int LS>
__device__ __forceinline__ void warp_begin_t(WarpQT<DH, LS>& q, const Params& p, const Tile& T, int warp, int lane) {
  constexpr int KC = DH / 16, MD = DH / 16;
  constexpr int smask = (1 << LS) - 1;
  const int g = lane >> 2, t4 = lane & 3;
  const int H = p.H, W = p.W;
  const int rh = p.kh / 2, rw = p.kw / 2;
  const int wy = warp / p.NWW, wx = warp % p.NWW;
  const int wh0 = T.h0 + wy * p.WH, ww0 = T.w0 + wx * p.WW;
  q.live = (wh0 < H) && (ww0 < W);
  q.wr0 = clampi(min(wh0, H - 1) - rh, 0, H - p.kh) - T.hs0;
  const int wr1 = clampi(min(wh0 + p.WH - 1, H - 1) - rh, 0, H - p.kh) + p.kh - T.hs0;
  q.wc0 = p.periodic ? (ww0 - T.w0) : (clampi(min(ww0, W - 1) - rw, 0, W - p.kw) - T.ws0);
  q.nkeys = (wr1 - q.wr0) << LS;
  q.ngroups = (q.nkeys + 15) / 16;
  // debug builds: the warp's key rectangle lies inside the slab (each query's
  // window is checked below); a warp that fails computes nothing
  if (q.live && !WM_DCHECK(q.wr0 >= 0 && wr1 <= T.HR && q.wc0 >= 0 && q.wc0 + (1 << LS) <= p.WC, p.dstatus))
    q.live = false;
  // the thread's two softmax queries (columns 2 t4, 2 t4 + 1)
  float cb[2][2][2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int qi = 2 * t4 + k;
    const int hc = min(wh0 + qi / p.WW, H - 1), wc = min(ww0 + qi % p.WW, W - 1);
    q.rlo[k] = clampi(hc - rh, 0, H - p.kh) - T.hs0 - q.wr0;
    const int qsc = p.periodic ? (wc - T.w0) : (clampi(wc - rw, 0, W - p.kw) - T.ws0);
    if (q.live && !WM_DCHECK(q.rlo[k] >= 0 && q.rlo[k] + p.kh <= wr1 - q.wr0 && qsc >= q.wc0 &&
                                 qsc + p.kw <= q.wc0 + (1 << LS),
                             p.dstatus))
      q.live = false;
    const uint32_t colmask = (0xFFFFFFFFu >> (32 - p.kw)) << max(qsc - q.wc0, 0);
#pragma unroll
    for (int hf = 0; hf < 2; ++hf)
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int col = (hf * 16 + g + 8 * i) & smask;
        cb[hf][i][k] = ((colmask >> col) & 1u) ? 0.f : -INFINITY;
      }
  }
#pragma unroll
  for (int hf = 0; hf < 2; ++hf)
#pragma unroll
    for (int i = 0; i < 2; ++i) q.cbias2[hf][i] = pack_f2(cb[hf][i][0], cb[hf][i][1]);
  // the query this thread loads and stores: query g
  q.qh = wh0 + g / p.WW;
  q.qw = ww0 + g % p.WW;
  q.qvalid = (q.qh < H) && (q.qw < W);
  const long N = (long)p.D * H * W;
  const long C3 = 3L * p.C;
  const long tok = ((long)T.d * H + min(q.qh, H - 1)) * W + min(q.qw, W - 1);
  const __nv_bfloat16* q0 = p.qkv + ((long)T.b * N + tok) * C3 + T.head * DH;
#pragma unroll
  for (int kc = 0; kc < KC; ++kc) {
    q.qb[kc][0] = *reinterpret_cast<const uint32_t*>(q0 + kc * 16 + 2 * t4);
    q.qb[kc][1] = *reinterpret_cast<const uint32_t*>(q0 + kc * 16 + 8 + 2 * t4);
  }
#pragma unroll
  for (int md = 0; md < MD; ++md) q.o[md][0] = q.o[md][1] = q.o[md][2] = q.o[md][3] = 0.f;
  q.mrow[0] = q.mrow[1] = -INFINITY;
  q.lrow[0] = q.lrow[1] = 0.f;
}

template <int DH, int LS, int GCH>
__device__ __forceinline__ void warp_level_t(WarpQT<DH, LS>& q, const Params& p, uint32_t sK32, uint32_t sV32,
                                             int lane) {
  constexpr int DHP = DH + 8, KC = DH / 16, MD = DH / 16;
  constexpr int smask = (1 << LS) - 1;
  const int WC = p.WC;
  const int mi = lane >> 3;
  const int g = lane >> 2;
  // Shared-memory byte address of this lane's ldmatrix row for key group gg
  // (as in the Q.K^T family: row-0 address plus a clamped row index for 8-
  // and 16-wide rectangles; keys past the rectangle are masked).
  constexpr int RPG = LS == 3 ? 2 : 1;
  const int last_row = (q.nkeys >> LS) - 1;
  const uint32_t rstride = (uint32_t)(WC * DHP * 2);
  const int lk = (mi & 1) * 8 + (lane & 7);            // key row this lane addresses in a K ldmatrix
  const int lv = (mi >> 1) * 8 + (lane & 7);           // ... in a V ldmatrix.trans
  const uint32_t kbase = sK32 + (uint32_t)(((q.wr0 * WC + q.wc0 + (LS == 3 ? (lane & 7) : (lk & smask))) * DHP +
                                            (mi >> 1) * 8) * 2);
  const uint32_t vbase = sV32 + (uint32_t)(((q.wr0 * WC + q.wc0 + (LS == 3 ? (lane & 7) : (lv & smask))) * DHP +
                                            (mi & 1) * 8) * 2);
  auto k_addr = [&](int gg) -> uint32_t {
    if constexpr (LS <= 4) {
      return kbase + (uint32_t)min(RPG * gg + (LS == 3 ? (mi & 1) : 0), last_row) * rstride;
    } else {
      int j = gg * 16 + lk;
      if (j >= q.nkeys) j = 0;
      return sK32 + (uint32_t)((((q.wr0 + (j >> LS)) * WC + q.wc0 + (j & smask)) * DHP + (mi >> 1) * 8) * 2);
    }
  };
  auto v_addr = [&](int gg) -> uint32_t {
    if constexpr (LS <= 4) {
      return vbase + (uint32_t)min(RPG * gg + (LS == 3 ? (mi >> 1) : 0), last_row) * rstride;
    } else {
      int j = gg * 16 + lv;
      if (j >= q.nkeys) j = 0;
      return sV32 + (uint32_t)((((q.wr0 + (j >> LS)) * WC + q.wc0 + (j & smask)) * DHP + (mi & 1) * 8) * 2);
    }
  };
  // Chunks of GCH groups, then one chunk of exactly the groups left, as in
  // the Q.K^T family.
  int g0 = 0;
  auto chunk = [&](auto gsize) {
    constexpr int G = decltype(gsize)::value;
    float s[G][4];
#pragma unroll
    for (int gi = 0; gi < G; ++gi) {
      s[gi][0] = s[gi][1] = s[gi][2] = s[gi][3] = 0.f;
      const uint32_t ka = k_addr(g0 + gi);
#pragma unroll
      for (int kc = 0; kc < KC; ++kc) {
        uint32_t a0, a1, a2, a3;
        ldsm_x4(ka + kc * 32, a0, a1, a2, a3);
        mma_bf16(s[gi], a0, a1, a2, a3, q.qb[kc][0], q.qb[kc][1]);
      }
    }
    // mask + scale, per-query chunk max; entries (key i, queries 2 t4 and
    // 2 t4 + 1) go through the paired instructions together
    const uint64_t scale2 = pack_f2(p.scale_log2, p.scale_log2);
    float mx[2] = {-INFINITY, -INFINITY};
#pragma unroll
    for (int gi = 0; gi < G; ++gi) {
      const int gg = g0 + gi;
      const int half = (LS == 5) ? (gg & 1) : 0;
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int row = (gg * 16 + 8 * i + g) >> LS;
        float t0, t1;
        fma_f2(t0, t1, s[gi][2 * i], s[gi][2 * i + 1], scale2, q.cbias2[half][i]);
        s[gi][2 * i] = ((unsigned)(row - q.rlo[0]) < (unsigned)p.kh) ? t0 : -INFINITY;
        s[gi][2 * i + 1] = ((unsigned)(row - q.rlo[1]) < (unsigned)p.kh) ? t1 : -INFINITY;
      }
      mx[0] = max3(mx[0], s[gi][0], s[gi][2]);
      mx[1] = max3(mx[1], s[gi][1], s[gi][3]);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      mx[k] = fmaxf(mx[k], __shfl_xor_sync(0xffffffffu, mx[k], 4));
      mx[k] = fmaxf(mx[k], __shfl_xor_sync(0xffffffffu, mx[k], 8));
      mx[k] = fmaxf(mx[k], __shfl_xor_sync(0xffffffffu, mx[k], 16));
    }
    // lazy rescale, as in the Q.K^T family
    const bool grow = (mx[0] > q.mrow[0] + kLazyLog2) || (mx[1] > q.mrow[1] + kLazyLog2);
    if (__any_sync(0xffffffffu, grow)) {
      float alpha[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const float mnew = fmaxf(q.mrow[k], mx[k]);
        alpha[k] = ex2(q.mrow[k] - ((mnew == -INFINITY) ? 0.f : mnew));
        q.mrow[k] = mnew;
      }
      const uint64_t alpha2 = pack_f2(alpha[0], alpha[1]);
      mul_f2(q.lrow[0], q.lrow[1], alpha2);
#pragma unroll
      for (int md = 0; md < MD; ++md) {
        mul_f2(q.o[md][0], q.o[md][1], alpha2);
        mul_f2(q.o[md][2], q.o[md][3], alpha2);
      }
    }
    const uint64_t mref2 = pack_f2(q.mrow[0] == -INFINITY ? 0.f : q.mrow[0], q.mrow[1] == -INFINITY ? 0.f : q.mrow[1]);
    float lsum[2] = {0.f, 0.f};
#pragma unroll
    for (int gi = 0; gi < G; ++gi) {
      float pr[4];
      float d0, d1;
      sub_f2(d0, d1, s[gi][0], s[gi][1], mref2);
      pr[0] = ex2(d0);
      pr[1] = ex2(d1);
      sub_f2(d0, d1, s[gi][2], s[gi][3], mref2);
      pr[2] = ex2(d0);
      pr[3] = ex2(d1);
      float e0, e1;
      add_f2(e0, e1, pr[0], pr[1], pr[2], pr[3]);
      add_f2(lsum[0], lsum[1], lsum[0], lsum[1], e0, e1);
      // P^T blocks (keys 0-7 / 8-15 x queries) transposed into the B operand
      const uint32_t b0 = movmatrix_t(pack_bf16(pr[0], pr[1]));
      const uint32_t b1 = movmatrix_t(pack_bf16(pr[2], pr[3]));
      const uint32_t va = v_addr(g0 + gi);
#pragma unroll
      for (int md = 0; md < MD; ++md) {
        uint32_t a0, a1, a2, a3;
        ldsm_x4_t(va + md * 32, a0, a1, a2, a3);
        mma_bf16(q.o[md], a0, a1, a2, a3, b0, b1);
      }
    }
    add_f2(q.lrow[0], q.lrow[1], q.lrow[0], q.lrow[1], lsum[0], lsum[1]);
  };
  for (; g0 + GCH <= q.ngroups; g0 += GCH) chunk(std::integral_constant<int, GCH>{});
  tail_chunk<GCH - 1>(q.ngroups - g0, chunk);
}

template <int DH, int LS>
__device__ __forceinline__ void warp_end_t(const WarpQT<DH, LS>& q, const Params& p, const Tile& T, int lane) {
  constexpr int MD = DH / 16;
  const int t4 = lane & 3;
  float inv[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    float l = q.lrow[k];
    l += __shfl_xor_sync(0xffffffffu, l, 4);
    l += __shfl_xor_sync(0xffffffffu, l, 8);
    l += __shfl_xor_sync(0xffffffffu, l, 16);
    inv[k] = 1.f / l;
  }
  const long N = (long)p.D * p.H * p.W;
  __nv_bfloat16* orow = p.out + ((long)T.b * N + ((long)T.d * p.H + min(q.qh, p.H - 1)) * p.W +
                                 min(q.qw, p.W - 1)) * p.C + T.head * DH;
#pragma unroll
  for (int md = 0; md < MD; ++md) {
    // (dh rows x queries) blocks transposed to (query g, dh 2 t4 .. 2 t4 + 1)
    const uint32_t lo = movmatrix_t(pack_bf16(q.o[md][0] * inv[0], q.o[md][1] * inv[1]));
    const uint32_t hi = movmatrix_t(pack_bf16(q.o[md][2] * inv[0], q.o[md][3] * inv[1]));
    if (q.qvalid) {
      *reinterpret_cast<uint32_t*>(orow + md * 16 + 2 * t4) = lo;
      *reinterpret_cast<uint32_t*>(orow + md * 16 + 8 + 2 * t4) = hi;
    }
  }
}

// The two arithmetic families behind one interface for the kernels.
template <int DH, int LS, int GCH>
struct ArithS {
  using State = WarpQ<DH, LS>;
  static __device__ __forceinline__ void begin(State& q, const Params& p, const Tile& T, int w, int l) {
    warp_begin<DH, LS>(q, p, T, w, l);
  }
  static __device__ __forceinline__ void level(State& q, const Params& p, uint32_t k, uint32_t v, int l) {
    warp_level<DH, LS, GCH>(q, p, k, v, l);
  }
  static __device__ __forceinline__ void end(const State& q, const Params& p, const Tile& T, int l) {
    warp_end<DH, LS>(q, p, T, l);
  }
};
template <int DH, int LS, int GCH>
struct ArithT {
  using State = WarpQT<DH, LS>;
  static __device__ __forceinline__ void begin(State& q, const Params& p, const Tile& T, int w, int l) {
    warp_begin_t<DH, LS>(q, p, T, w, l);
  }
  static __device__ __forceinline__ void level(State& q, const Params& p, uint32_t k, uint32_t v, int l) {
    warp_level_t<DH, LS, GCH>(q, p, k, v, l);
  }
  static __device__ __forceinline__ void end(const State& q, const Params& p, const Tile& T, int l) {
    warp_end_t<DH, LS>(q, p, T, l);
  }
};

// ---------------------------------------------------------------------------
// Kernel A: one CTA per tile; all threads load a level (cp.async, double
// buffered), then all warps consume it; one CTA-wide barrier per level.
template <int DH, int LS, int GCH, int MAXT, bool TR = false>
__global__ void __launch_bounds__(MAXT, 1) na_bf16_kernel(const Params p) {
  using A = typename std::conditional<TR, ArithT<DH, LS, GCH>, ArithS<DH, LS, GCH>>::type;
  extern __shared__ __align__(128) __nv_bfloat16 sm_raw[];
  __nv_bfloat16* sm = align128(sm_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const Tile T = make_tile(p, blockIdx.x);
  const int slab = p.slab;
  pdl_wait();      // qkv of the previous kernel is complete from here on
  pdl_trigger();
  typename A::State q;
  A::begin(q, p, T, warp, lane);
  load_level<DH>(p, T, T.ld0, sm, slab, tid, blockDim.x);
  cp_async_commit();
  for (int li = 0; li < p.kd; ++li) {
    if (li + 1 < p.kd) load_level<DH>(p, T, T.ld0 + li + 1, sm + (size_t)((li + 1) & 1) * 2 * slab, slab, tid, blockDim.x);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    const uint32_t sK32 = (uint32_t)__cvta_generic_to_shared(sm + (size_t)(li & 1) * 2 * slab);
    if (q.live) A::level(q, p, sK32, sK32 + (uint32_t)slab * 2, lane);
    __syncthreads();
  }
  if (q.live) A::end(q, p, T, lane);
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

template <int DH, int LS, int GCH, int MAXT, bool TR = false>
__global__ void __launch_bounds__(MAXT, 1)
    na_bf16_pipe_kernel(const Params p, int ntiles, int* status, const __grid_constant__ CUtensorMap tm_kv) {
  using A = typename std::conditional<TR, ArithT<DH, LS, GCH>, ArithS<DH, LS, GCH>>::type;
  constexpr int DHP = DH + 8;
  extern __shared__ __align__(128) __nv_bfloat16 sm_raw[];
  __nv_bfloat16* sm = align128(sm_raw);
  __shared__ __align__(8) uint64_t full_bar[3];
  __shared__ __align__(8) uint64_t empty_bar[3];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int NW = p.NWH * p.NWW;      // consumer warps
  const int NBUF = p.nbuf;
  const int slab = p.slab;
  if (tid == 0) {
    for (int i = 0; i < NBUF; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&full_bar[i])), "r"(32) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&empty_bar[i])), "r"(NW) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  pdl_wait();      // qkv of the previous kernel is complete from here on
  pdl_trigger();

  if (warp == NW) {
    // ------------------------------------------------------------- producer
    // A slab whose longitudes do not wrap around the grid is one tensor copy
    // for K and one for V (box = DH + 8 channels x WC x HRmax, which is the
    // padded slab layout; the extra channels and rows are never read). A
    // wrapping slab is copied 16 bytes at a time with cp.async. Either way
    // the 32 lanes arrive on full[b] once.
    if (p.tma && lane == 0) asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tm_kv) : "memory");
    const uint32_t box_bytes = (uint32_t)(p.HRmax * p.WC * DHP * 2);
    int it = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const Tile T = make_tile(p, t);
      const bool bulk = p.tma && !(p.periodic && (T.ws0 < 0 || T.ws0 + p.WC > p.W));
      for (int li = 0; li < p.kd; ++li) {
        const int buf = it % NBUF;
        const uint32_t ph = (uint32_t)(it / NBUF) & 1u;
        if (!na_mbar_wait(&empty_bar[buf], ph ^ 1u)) {
          ok = false;
          break;
        }
        const uint32_t fb = smem_addr(&full_bar[buf]);
        __nv_bfloat16* dst = sm + (size_t)buf * 2 * slab;
        if (bulk) {
          if (lane == 0) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(2 * box_bytes)
                         : "memory");
            const int c0 = p.C + T.head * DH, lev = T.b * p.D + T.ld0 + li;
#pragma unroll
            for (int kv = 0; kv < 2; ++kv)
              asm volatile(
                  "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
                  "[%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(smem_addr(dst + (size_t)kv * slab)),
                  "l"((uint64_t)&tm_kv), "r"(fb), "r"(c0 + kv * p.C), "r"(T.ws0), "r"(T.hs0), "r"(lev)
                  : "memory");
          } else {
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(fb) : "memory");
          }
        } else {
          load_level<DH>(p, T, T.ld0 + li, dst, slab, lane, 32);
          asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(fb) : "memory");
        }
        ++it;
      }
    }
    if (!ok) atomicExch(status, (int)WM_ERR_TIMEOUT);
    // own copies land before this warp leaves (the consumers may have given up)
    asm volatile("cp.async.wait_all;" ::: "memory");
    for (int j = max(it - NBUF, 0); j < it; ++j)
      if (!na_mbar_wait(&full_bar[j % NBUF], (uint32_t)(j / NBUF) & 1u)) atomicExch(status, (int)WM_ERR_TIMEOUT);
    return;
  }
  // ------------------------------------------------------------- consumers
  int it = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const Tile T = make_tile(p, t);
    typename A::State q;
    A::begin(q, p, T, warp, lane);
    for (int li = 0; li < p.kd; ++li, ++it) {
      const int buf = it % NBUF;
      const uint32_t ph = (uint32_t)(it / NBUF) & 1u;
      if (!na_mbar_wait(&full_bar[buf], ph)) {
        atomicExch(status, (int)WM_ERR_TIMEOUT);
        return;
      }
      const uint32_t sK32 = smem_addr(sm + (size_t)buf * 2 * slab);
      if (q.live) A::level(q, p, sK32, sK32 + (uint32_t)slab * 2, lane);
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&empty_bar[buf])) : "memory");
    }
    if (q.live) A::end(q, p, T, lane);
  }
}

}  // namespace na

template <int DH, bool TR>
static wm_status prep_dh_family(int lim) {
  constexpr int G = TR ? 8 : 4;   // the transposed family has one chunk size
  if (!TR) {
    WM_CUDA(cudaFuncSetAttribute(na::na_bf16_kernel<DH, 3, 8, 384>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    WM_CUDA(cudaFuncSetAttribute(na::na_bf16_kernel<DH, 4, 8, 384>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    WM_CUDA(cudaFuncSetAttribute(na::na_bf16_kernel<DH, 5, 8, 384>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    WM_CUDA(cudaFuncSetAttribute(na::na_bf16_pipe_kernel<DH, 3, 8, 288>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    WM_CUDA(cudaFuncSetAttribute(na::na_bf16_pipe_kernel<DH, 4, 8, 288>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    WM_CUDA(cudaFuncSetAttribute(na::na_bf16_pipe_kernel<DH, 5, 8, 288>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  }
  WM_CUDA(cudaFuncSetAttribute(na::na_bf16_kernel<DH, 3, G, 512, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  WM_CUDA(cudaFuncSetAttribute(na::na_bf16_kernel<DH, 4, G, 512, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  WM_CUDA(cudaFuncSetAttribute(na::na_bf16_kernel<DH, 5, G, 512, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  WM_CUDA(cudaFuncSetAttribute(na::na_bf16_pipe_kernel<DH, 3, G, 512, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  WM_CUDA(cudaFuncSetAttribute(na::na_bf16_pipe_kernel<DH, 4, G, 512, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  WM_CUDA(cudaFuncSetAttribute(na::na_bf16_pipe_kernel<DH, 5, G, 512, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  return WM_OK;
}

template <int DH>
static wm_status prep_dh(int lim) {
  wm_status st = prep_dh_family<DH, false>(lim);
  return st == WM_OK ? prep_dh_family<DH, true>(lim) : st;
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

// Arithmetic family of a plan: the formulation (S = Q K^T with 16 queries
// per warp, or S^T = K Q^T with 8) and the softmax chunk. Both change the
// rounding of a query's result, so a problem shape keeps the family it was
// first tuned with; the CTA shape and the kernel kind do not.
struct NaPlan {
  int NWH, NWW;  // consumer warp grid of a CTA (query tile = NWH*WH x NWW*WW)
  int kind;      // 0: one CTA per tile, CTA-wide barrier per level; 1: persistent producer/consumer
  int nbuf;      // slab buffers (kind 0: 2; kind 1: 2 or 3)
  int gch;       // 16-key groups scored per softmax update
  int tr;        // 1: transposed formulation
  int WH, WW, span;   // warp patch and key-rectangle width (fixed by tr and the window)
  int tc;        // 1: the tcgen05 kernel (k_na_tc.cu; the fields above are unused)
};

constexpr int kFamilyTc = 1024;
int family(const NaPlan& pl) { return pl.tc ? kFamilyTc : (pl.gch | (pl.tr << 8)); }

using NaKey = std::array<int, 11>;
std::mutex g_na_mu;
std::map<NaKey, NaPlan> g_na_plans;  // autotuned plans
std::map<NaKey, double> g_na_ms;     // their measured time per launch
std::map<NaKey, int> g_na_family;    // arithmetic family fixed per shape (key with B = 0) at its first tuning
std::string g_na_log;                 // every candidate's time, for the report

NaKey na_key(int B, int D, int H, int W, int C, int heads, int kd, int kh, int kw, bool per) {
  return NaKey{B, D, H, W, C, heads, kd, kh, kw, per ? 1 : 0, 0};
}

// Warp patch (WH x WW queries; 16 queries, or 8 for the transposed
// formulation) with the fewest issued keys per level; fixed by the window
// alone, so a query's arithmetic (its key rectangle and the order it is
// walked in) never depends on the CTA plan.
bool warp_patch(int tr, int kh, int kw, int* WH, int* WW, int* span) {
  static const int c16[5][2] = {{1, 16}, {2, 8}, {4, 4}, {8, 2}, {16, 1}};
  static const int c8[4][2] = {{1, 8}, {2, 4}, {4, 2}, {8, 1}};
  const int (*cand)[2] = tr ? c8 : c16;
  const int n = tr ? 4 : 5;
  int best = -1, best_cost = 1 << 30;
  for (int i = 0; i < n; ++i) {
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

// Elements of one K (or V) slab, rounded up to 128 bytes.
int plan_slab(const NaPlan& pl, int kh, int H, int dh) {
  const int hr = std::min(pl.NWH * pl.WH + kh - 1, H);
  const int wc = (pl.NWW - 1) * pl.WW + pl.span;
  return (hr * wc * (dh + 8) + 63) / 64 * 64;
}

// Dynamic shared memory of a plan: the slab ring plus 128 bytes of alignment slack.
size_t plan_smem(const NaPlan& pl, int kh, int H, int dh) {
  return (size_t)pl.nbuf * 2 * plan_slab(pl, kh, H, dh) * 2 + 128;
}

// Candidate plans of one arithmetic family (fam = 0: every family).
std::vector<NaPlan> na_candidates(int kh, int kw, int H, int W, int C, int heads, bool periodic, int fam) {
  const int dh = C / heads;
  std::vector<NaPlan> out;
  if ((fam == 0 || fam == kFamilyTc) && na_tc_supported(H, W, C, heads, kh, kw, periodic)) {
    NaPlan tc{};
    tc.NWH = tc.NWW = 1;
    tc.tc = 1;
    out.push_back(tc);
  }
  int WH, WW, span;
  auto add = [&](int nwh, int nww, int kind, int nbuf, int gch, int tr) {
    NaPlan pl{nwh, nww, kind, nbuf, gch, tr, WH, WW, span};
    if (plan_smem(pl, kh, H, dh) <= (size_t)kNaSmemLimit) out.push_back(pl);
  };
  if ((fam == 0 || fam == 8) && warp_patch(0, kh, kw, &WH, &WW, &span)) {
    for (int nw : {8, 12})
      for (int nwh = 1; nwh <= nw; ++nwh)
        if (nw % nwh == 0) add(nwh, nw / nwh, 0, 2, 8, 0);
    for (int nbuf : {2, 3})
      for (int nwh = 1; nwh <= 8; nwh *= 2) add(nwh, 8 / nwh, 1, nbuf, 8, 0);
  }
  if ((fam == 0 || fam == 4) && warp_patch(0, kh, kw, &WH, &WW, &span)) {
    for (int nwh = 1; nwh <= 16; nwh *= 2) add(nwh, 16 / nwh, 0, 2, 4, 0);
    for (int nw : {12, 15})
      for (int nbuf : {2, 3})
        for (int nwh = 1; nwh <= nw; ++nwh)
          if (nw % nwh == 0) add(nwh, nw / nwh, 1, nbuf, 4, 0);
  }
  if ((fam == 0 || fam == (8 | 256)) && warp_patch(1, kh, kw, &WH, &WW, &span)) {
    for (int nw : {8, 16})
      for (int nwh = 1; nwh <= nw; nwh *= 2) add(nwh, nw / nwh, 0, 2, 8, 1);
    for (int nw : {8, 12, 15})
      for (int nbuf : {2, 3})
        for (int nwh = 1; nwh <= nw; ++nwh)
          if (nw % nwh == 0) add(nwh, nw / nwh, 1, nbuf, 8, 1);
  }
  return out;
}

// Heuristic when no tuned plan exists, among the plans of family `fam` (and
// kernel kind `kind`, unless it is -1): fewest staged keys per query times
// tile waste; persistent plans are preferred when the tile count gives every
// SM several tiles.
NaPlan na_heuristic(int B, int D, int H, int W, int heads, int kh, int kw, int dh, bool periodic, int fam, int kind) {
  NaPlan best{};
  double best_score = 1e30;
  for (const NaPlan& pl : na_candidates(kh, kw, H, W, heads * dh, heads, periodic, fam)) {
    if (pl.tc) return pl;   // the tcgen05 family has one plan
    if (kind >= 0 && pl.kind != kind) continue;
    const int TH = pl.NWH * pl.WH, TW = pl.NWW * pl.WW;
    const int th = (H + TH - 1) / TH, tw = (W + TW - 1) / TW;
    const int hr = std::min(TH + kh - 1, H), wc = (pl.NWW - 1) * pl.WW + pl.span;
    const long ctas = (long)th * tw * D * B * heads;
    double score = (double)hr * wc / (TH * TW) * ((double)th * TH / H) * ((double)tw * TW / W);
    if (ctas < num_sms()) score *= (double)num_sms() / ctas;   // idle SMs
    if (pl.kind == 1 && kind < 0) score *= (ctas >= 4L * num_sms()) ? 0.8 : 1.5;
    score /= std::sqrt((double)(pl.NWH * pl.NWW * pl.WH * pl.WW) / 128.0);   // more warps hide more latency
    if (score < best_score) {
      best_score = score;
      best = pl;
    }
  }
  return best;
}

template <int DH, int LS, int G, int MT, bool TR>
void launch_tile(const na::Params& p, long ntiles, int smem, cudaStream_t s, bool pdl) {
  launch_pdl(na::na_bf16_kernel<DH, LS, G, MT, TR>, dim3((unsigned)ntiles), dim3(32 * p.NWH * p.NWW), smem, s, pdl, p);
}

template <int DH, int LS, int G, int MT, bool TR>
void launch_pipe(const na::Params& p, const CUtensorMap& tm, long ntiles, int smem, cudaStream_t s, bool pdl) {
  const int grid = (int)std::min<long>(ntiles, num_sms());
  launch_pdl(na::na_bf16_pipe_kernel<DH, LS, G, MT, TR>, dim3(grid), dim3(32 * (p.NWH * p.NWW + 1)), smem, s, pdl,
             p, (int)ntiles, device_status_word(), tm);
}

template <int DH, int LS>
void launch_family(const NaPlan& pl, const na::Params& p, const CUtensorMap& tm, long ntiles, int smem,
                   cudaStream_t s, bool pdl) {
  if (pl.tr) {
    if (pl.kind == 0) launch_tile<DH, LS, 8, 512, true>(p, ntiles, smem, s, pdl);
    else launch_pipe<DH, LS, 8, 512, true>(p, tm, ntiles, smem, s, pdl);
  } else if (pl.gch == 4) {
    if (pl.kind == 0) launch_tile<DH, LS, 4, 512, false>(p, ntiles, smem, s, pdl);
    else launch_pipe<DH, LS, 4, 512, false>(p, tm, ntiles, smem, s, pdl);
  } else {
    if (pl.kind == 0) launch_tile<DH, LS, 8, 384, false>(p, ntiles, smem, s, pdl);
    else launch_pipe<DH, LS, 8, 288, false>(p, tm, ntiles, smem, s, pdl);
  }
}

template <int DH>
wm_status launch_plan(const NaPlan& pl, na::Params p, cudaStream_t s, bool pdl) {
  p.WH = pl.WH;
  p.WW = pl.WW;
  p.log2span = 0;
  while ((1 << p.log2span) < pl.span) ++p.log2span;
  p.NWH = pl.NWH;
  p.NWW = pl.NWW;
  p.nbuf = pl.nbuf;
  p.HRmax = std::min(p.NWH * p.WH + p.kh - 1, p.H);
  p.WC = (p.NWW - 1) * p.WW + pl.span;
  const int TH = p.NWH * p.WH, TW = p.NWW * p.WW;
  const int tiles_h = (p.H + TH - 1) / TH;
  p.tiles_w = (p.W + TW - 1) / TW;
  p.scale_log2 = 1.4426950408889634f / sqrtf((float)DH);
  const long ntiles = (long)tiles_h * p.tiles_w * p.D * p.B * p.heads;
  if (ntiles > (1L << 30)) return fail(WM_ERR_INVALID_ARG, "too many attention tiles");
  const int nthreads = 32 * (p.NWH * p.NWW + (pl.kind == 1 ? 1 : 0));
  const int maxt = (pl.tr || pl.gch == 4) ? 512 : (pl.kind == 0 ? 384 : 288);
  if (nthreads > maxt) return fail(WM_ERR_INVALID_ARG, "attention plan exceeds its kernel's thread limit");
  const int smem = (int)plan_smem(pl, p.kh, p.H, DH);
  p.slab = plan_slab(pl, p.kh, p.H, DH);
  // The persistent kernel copies non-wrapping slabs with the tensor engine.
  CUtensorMap tm;
  std::memset(&tm, 0, sizeof tm);
  p.tma = pl.kind == 1 && make_tmap_qkv_slab(&tm, p.qkv, 3ull * p.C, p.W, p.H, (uint64_t)p.D * p.B, DH + 8, p.WC,
                                              p.HRmax) ? 1 : 0;
  switch (p.log2span) {
    case 3: launch_family<DH, 3>(pl, p, tm, ntiles, smem, s, pdl); break;
    case 4: launch_family<DH, 4>(pl, p, tm, ntiles, smem, s, pdl); break;
    case 5: launch_family<DH, 5>(pl, p, tm, ntiles, smem, s, pdl); break;
    default: return fail(WM_ERR_INVALID_ARG, "unsupported key rectangle width");
  }
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

wm_status launch_with(const NaPlan& pl, const na::Params& p, int dh, cudaStream_t s, bool pdl = false) {
  if (pl.tc)
    return launch_na_tc(p.qkv, p.out, p.B, p.D, p.H, p.W, p.C, p.heads, p.kd, p.kh, p.kw, p.periodic != 0, s, pdl);
  switch (dh) {
    case 16: return launch_plan<16>(pl, p, s, pdl);
    case 32: return launch_plan<32>(pl, p, s, pdl);
    case 48: return launch_plan<48>(pl, p, s, pdl);
    case 64: return launch_plan<64>(pl, p, s, pdl);
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
  p.dstatus = device_status_word();
  return p;
}

}  // namespace

wm_status launch_na_bf16(const __nv_bfloat16* qkv, __nv_bfloat16* out, int B, int D, int H, int W, int C, int heads,
                         int kd, int kh, int kw, bool periodic, cudaStream_t s, int variant, bool pdl) {
  if (B <= 0) return WM_OK;
  if ((reinterpret_cast<uintptr_t>(qkv) | reinterpret_cast<uintptr_t>(out)) & 15)
    return fail(WM_ERR_INVALID_ARG, "BF16 attention needs 16-byte aligned qkv and out");
  const int dh = C / heads;
  int WH, WW, span;
  if (!warp_patch(0, kh, kw, &WH, &WW, &span))
    return fail(WM_ERR_INVALID_ARG, "longitude window too wide for the BF16 attention kernel");
  NaPlan pl{};
  int fam = 8, kind = -1;
  if (variant == WM_NA_TCGEN05) {
    if (!na_tc_supported(H, W, C, heads, kh, kw, periodic))
      return fail(WM_ERR_INVALID_ARG, "shape not supported by the tcgen05 attention kernel");
    fam = kFamilyTc;
  } else if (variant != 0) {
    static const int fams[4] = {0, 8, 4, 8 | 256};
    fam = fams[variant & 3];
    kind = (variant & 4) ? 0 : (variant & 8) ? 1 : -1;
  } else {
    std::lock_guard<std::mutex> lk(g_na_mu);
    auto it = g_na_plans.find(na_key(B, D, H, W, C, heads, kd, kh, kw, periodic));
    if (it != g_na_plans.end()) pl = it->second;
    auto ig = g_na_family.find(na_key(0, D, H, W, C, heads, kd, kh, kw, periodic));
    if (ig != g_na_family.end()) fam = ig->second;
  }
  if (!pl.NWH) pl = na_heuristic(B, D, H, W, heads, kh, kw, dh, periodic, fam, kind);
  if (!pl.NWH) return fail(WM_ERR_INVALID_ARG, "attention window too large for the BF16 attention kernel");
  return launch_with(pl, make_params(qkv, out, B, D, H, W, C, heads, kd, kh, kw, periodic), dh, s, pdl);
}

// Time every candidate CTA plan for this shape (1 warm-up + 3 timed launches
// each, CUDA events on `s`) and keep the fastest for later launches. The
// outputs are written to `out`; results depend only on the arithmetic family,
// which the first tuning of a shape fixes for every later batch size.
wm_status autotune_na_bf16(const __nv_bfloat16* qkv, __nv_bfloat16* out, int B, int D, int H, int W, int C,
                           int heads, int kd, int kh, int kw, bool periodic, cudaStream_t s, double* best_ms) {
  const int dh = C / heads;
  int WH, WW, span;
  if (!warp_patch(0, kh, kw, &WH, &WW, &span)) return fail(WM_ERR_INVALID_ARG, "window too wide");
  const na::Params p = make_params(qkv, out, B, D, H, W, C, heads, kd, kh, kw, periodic);
  cudaEvent_t e0, e1;
  WM_CUDA(cudaEventCreate(&e0));
  WM_CUDA(cudaEventCreate(&e1));
  NaPlan best{};
  float best_t = 1e30f;
  wm_status st = WM_OK;
  int fam_fixed = 0;
  {
    std::lock_guard<std::mutex> lk(g_na_mu);
    auto ig = g_na_family.find(na_key(0, D, H, W, C, heads, kd, kh, kw, periodic));
    if (ig != g_na_family.end()) fam_fixed = ig->second;
  }
  for (const NaPlan& pl : na_candidates(kh, kw, H, W, C, heads, periodic, fam_fixed)) {
    st = launch_with(pl, p, dh, s);
    if (st != WM_OK) break;
    cudaEventRecord(e0, s);
    for (int r = 0; r < 3 && st == WM_OK; ++r) st = launch_with(pl, p, dh, s);
    cudaEventRecord(e1, s);
    if (st != WM_OK) break;
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      st = fail(WM_ERR_CUDA, "autotune synchronisation failed");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    {
      char line[200];
      if (pl.tc)
        std::snprintf(line, sizeof line, "  candidate B=%d tcgen05 persistent tile=16x8: %.3f ms\n", B, ms / 3.0);
      else
        std::snprintf(line, sizeof line, "  candidate B=%d %s %s warps=%dx%d patch=%dx%d buffers=%d chunk=%d: %.3f ms\n",
                      B, pl.tr ? "K.Q^T" : "Q.K^T", pl.kind ? "persistent" : "per-tile", pl.NWH, pl.NWW, pl.WH, pl.WW,
                      pl.nbuf, pl.gch, ms / 3.0);
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
    g_na_family.emplace(na_key(0, D, H, W, C, heads, kd, kh, kw, periodic), family(best));
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
    if (pl.tc)
      std::snprintf(line, sizeof line,
                    "attention B=%d D=%d H=%d W=%d C=%d heads=%d window=%dx%dx%d periodic=%d -> tcgen05 persistent "
                    "tile=16x8 %.3f ms\n",
                    k[0], k[1], k[2], k[3], k[4], k[5], k[6], k[7], k[8], k[9], g_na_ms[k]);
    else
      std::snprintf(line, sizeof line,
                    "attention B=%d D=%d H=%d W=%d C=%d heads=%d window=%dx%dx%d periodic=%d -> %s %s warps=%dx%d "
                    "patch=%dx%d buffers=%d chunk=%d %.3f ms\n",
                    k[0], k[1], k[2], k[3], k[4], k[5], k[6], k[7], k[8], k[9], pl.tr ? "K.Q^T" : "Q.K^T",
                    pl.kind ? "persistent" : "per-tile", pl.NWH, pl.NWW, pl.WH, pl.WW, pl.nbuf, pl.gch, g_na_ms[k]);
    out += line;
  }
  return out + g_na_log;
}

}  // namespace wm
