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

#include "wm_internal.cuh"

namespace wm {
namespace na {

struct Params {
  const __nv_bfloat16* qkv;
  __nv_bfloat16* out;
  int B, D, H, W, C, heads, kd, kh, kw, periodic;
  int WH, WW, NWH, NWW;  // warp patch and warp grid
  int HRmax, WC;          // smem slab rows / columns
  int span8;              // columns of a warp's key rectangle (multiple of 8)
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
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&p);
}

template <int DH>
__global__ void __launch_bounds__(256) na_bf16_kernel(const Params p) {
  constexpr int DHP = DH + 8;   // padded key row: odd number of 16-byte units -> conflict-free ldmatrix
  constexpr int CH = DH / 8;    // 16-byte chunks per key row
  constexpr int KC = DH / 16;   // k16 steps of Q K^T
  constexpr int ND = DH / 8;    // n8 blocks of P V
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

  // ---- stage one key level (K and V) into buffer `buf`
  auto load_level = [&](int lev, int buf) {
    __nv_bfloat16* dstK = sm + (size_t)buf * 2 * slab;
    const int per_kv = HR * WC * CH;
    for (int idx = tid; idx < 2 * per_kv; idx += blockDim.x) {
      const int kv = idx / per_kv;
      const int rem = idx - kv * per_kv;
      const int r = rem / (WC * CH);
      const int c = (rem / CH) % WC;
      const int ch = rem % CH;
      int lon = ws0 + c;
      bool ok = true;
      if (p.periodic) {
        lon %= W;
        if (lon < 0) lon += W;
      } else if (lon >= W) {
        ok = false;
        lon = 0;
      }
      const long tok = ((long)lev * H + (hs0 + r)) * W + lon;
      const __nv_bfloat16* src = base + tok * C3 + (1 + kv) * p.C + head * DH + ch * 8;
      const uint32_t dst = (uint32_t)__cvta_generic_to_shared(dstK + (size_t)kv * slab + (size_t)(r * WC + c) * DHP + ch * 8);
      cp_async16(dst, ok ? (const void*)src : (const void*)p.qkv, ok ? 16 : 0);
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
  const int span8 = p.span8;
  const int nkeys = (wr1 - wr0) * span8;
  const int ngroups = (nkeys + 15) / 16;

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
      for (int grp = 0; grp < ngroups; ++grp) {
        // ---- S = Q K^T for 16 keys
        // ldmatrix row address of this lane: key j = (mi>>1)*8 + (lane&7) for K, (mi&1)*8 + (lane&7) for V
        const int mi = lane >> 3;
        int jk = grp * 16 + (mi >> 1) * 8 + (lane & 7);
        int jv = grp * 16 + (mi & 1) * 8 + (lane & 7);
        if (jk >= nkeys) jk = 0;
        if (jv >= nkeys) jv = 0;
        const int krow = (wr0 + jk / span8) * WC + wc0 + jk % span8;
        const int vrow = (wr0 + jv / span8) * WC + wc0 + jv % span8;
        float s[2][4];
#pragma unroll
        for (int nb = 0; nb < 2; ++nb) s[nb][0] = s[nb][1] = s[nb][2] = s[nb][3] = 0.f;
#pragma unroll
        for (int kc = 0; kc < KC; ++kc) {
          uint32_t b0, b1, b2, b3;
          ldsm_x4(sK32 + (uint32_t)((krow * DHP + kc * 16 + (mi & 1) * 8) * 2), b0, b1, b2, b3);
          mma_bf16(s[0], qa[kc][0], qa[kc][1], qa[kc][2], qa[kc][3], b0, b1);
          mma_bf16(s[1], qa[kc][0], qa[kc][1], qa[kc][2], qa[kc][3], b2, b3);
        }
        // ---- mask + scale
#pragma unroll
        for (int nb = 0; nb < 2; ++nb)
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int j = grp * 16 + nb * 8 + 2 * t4 + (e & 1);
            const int rr = e >> 1;
            const int kr = wr0 + j / span8, kcn = wc0 + j % span8;
            const bool ok = (j < nkeys) && (kr >= qsr[rr]) && (kr < qsr[rr] + p.kh) && (kcn >= qsc[rr]) &&
                            (kcn < qsc[rr] + p.kw);
            s[nb][e] = ok ? s[nb][e] * p.scale_log2 : -INFINITY;
          }
        // ---- online softmax (rows g and g+8)
        float pr[2][4];
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
          float mx = fmaxf(fmaxf(s[0][2 * rr], s[0][2 * rr + 1]), fmaxf(s[1][2 * rr], s[1][2 * rr + 1]));
          mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
          mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
          const float mnew = fmaxf(mrow[rr], mx);
          const float mref = (mnew == -INFINITY) ? 0.f : mnew;
          const float alpha = exp2f(mrow[rr] - mref);
          mrow[rr] = mnew;
          float ls = 0.f;
#pragma unroll
          for (int nb = 0; nb < 2; ++nb)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const float v = exp2f(s[nb][2 * rr + e] - mref);
              pr[nb][2 * rr + e] = v;
              ls += v;
            }
          lrow[rr] = lrow[rr] * alpha + ls;
#pragma unroll
          for (int nd = 0; nd < ND; ++nd) {
            o[nd][2 * rr] *= alpha;
            o[nd][2 * rr + 1] *= alpha;
          }
        }
        // ---- O += P V
        const uint32_t pa0 = pack_bf16(pr[0][0], pr[0][1]);
        const uint32_t pa1 = pack_bf16(pr[0][2], pr[0][3]);
        const uint32_t pa2 = pack_bf16(pr[1][0], pr[1][1]);
        const uint32_t pa3 = pack_bf16(pr[1][2], pr[1][3]);
#pragma unroll
        for (int nd = 0; nd < ND; nd += 2) {
          uint32_t b0, b1, b2, b3;
          ldsm_x4_t(sV32 + (uint32_t)((vrow * DHP + nd * 8 + (mi >> 1) * 8) * 2), b0, b1, b2, b3);
          mma_bf16(o[nd], pa0, pa1, pa2, pa3, b0, b1);
          mma_bf16(o[nd + 1], pa0, pa1, pa2, pa3, b2, b3);
        }
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

wm_status prepare_na_bf16() {
  const int lim = 200 * 1024;  // the launcher never asks for more
  WM_CUDA(cudaFuncSetAttribute(na::na_bf16_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  WM_CUDA(cudaFuncSetAttribute(na::na_bf16_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  WM_CUDA(cudaFuncSetAttribute(na::na_bf16_kernel<48>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  WM_CUDA(cudaFuncSetAttribute(na::na_bf16_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  return WM_OK;
}

static int round8(int v) { return (v + 7) / 8 * 8; }

wm_status launch_na_bf16(const __nv_bfloat16* qkv, __nv_bfloat16* out, int B, int D, int H, int W, int C, int heads,
                         int kd, int kh, int kw, bool periodic, cudaStream_t s) {
  if (B <= 0) return WM_OK;
  const int dh = C / heads;
  na::Params p{};
  p.qkv = qkv;
  p.out = out;
  p.B = B; p.D = D; p.H = H; p.W = W; p.C = C; p.heads = heads;
  p.kd = kd; p.kh = kh; p.kw = kw; p.periodic = periodic ? 1 : 0;
  // warp patch: fewest keys per query per level
  const int cand[5][2] = {{1, 16}, {2, 8}, {4, 4}, {8, 2}, {16, 1}};
  int best = 0, best_cost = 1 << 30;
  for (int i = 0; i < 5; ++i) {
    const int cost = (cand[i][0] + kh - 1) * round8(cand[i][1] + kw - 1);
    if (cost < best_cost) { best_cost = cost; best = i; }
  }
  p.WH = cand[best][0];
  p.WW = cand[best][1];
  p.span8 = round8(p.WW + kw - 1);
  const int DHP = dh + 8;
  // warp grid (8 warps): least staged keys per query within the shared-memory budget
  int bestg = -1;
  double best_ratio = 1e30;
  size_t best_smem = 0;
  for (int nwh = 1; nwh <= 8; nwh *= 2) {
    const int nww = 8 / nwh;
    const int TH = nwh * p.WH;
    const int hr = std::min(TH + kh - 1, H);
    const int wc = (nww - 1) * p.WW + p.span8;
    const size_t smem = (size_t)2 * 2 * hr * wc * DHP * 2;
    if (smem > 200 * 1024) continue;
    const double ratio = (double)hr * wc / (TH * nww * p.WW);
    if (ratio < best_ratio) { best_ratio = ratio; bestg = nwh; best_smem = smem; }
  }
  if (bestg < 0) return fail(WM_ERR_INVALID_ARG, "attention window too large for the BF16 attention kernel");
  p.NWH = bestg;
  p.NWW = 8 / bestg;
  p.HRmax = std::min(p.NWH * p.WH + kh - 1, H);
  p.WC = (p.NWW - 1) * p.WW + p.span8;
  const int TH = p.NWH * p.WH, TW = p.NWW * p.WW;
  const int tiles_h = (H + TH - 1) / TH;
  p.tiles_w = (W + TW - 1) / TW;
  p.scale_log2 = 1.4426950408889634f / sqrtf((float)dh);
  if ((long)B * heads > 65535 || D > 65535) return fail(WM_ERR_INVALID_ARG, "batch*heads or D too large");
  dim3 grid(tiles_h * p.tiles_w, D, B * heads), block(256);
  const int smem = (int)best_smem;
#define WM_NA_CASE(DHV)                                \
  case DHV:                                           \
    na::na_bf16_kernel<DHV><<<grid, block, smem, s>>>(p); \
    break;
  switch (dh) {
    WM_NA_CASE(16)
    WM_NA_CASE(32)
    WM_NA_CASE(48)
    WM_NA_CASE(64)
    default:
      return fail(WM_ERR_INVALID_ARG, "BF16 attention needs head dim 16, 32, 48 or 64");
  }
#undef WM_NA_CASE
  WM_CUDA(cudaGetLastError());
  return WM_OK;
}

}  // namespace wm
