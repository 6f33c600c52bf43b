"""FP64 CPU oracle of the WeatherMesh-3 processor and its latent rollout.

TEST INFRASTRUCTURE ONLY. This module is the slow, plain reference that the GPU
library is checked against. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the library never calls it and
has no CPU fallback.

Everything is float64 numpy. Matrix products use ``@`` (a BLAS call serving as
one step of a definition); everything else is written as the definition reads.
The oracle shares no code with the CUDA path.

What the paper fixes, and the readings taken where it is silent:

* Section 2.1, "Encoder-processor-decoder architecture" and "latent rollout":
  the processor acts on the latent any number of times; one call advances 6 h
  (six-hour processor) or 1 h (one-hour processor); a lead time T is reached
  by a simple greedy schedule. Reading: greedy coin change, largest coin
  first -- floor(T/6) six-hour calls, then T mod 6 one-hour calls. T = 0 is
  the identity; T < 0 is an error.
* Section 2.1, "NATTEN" and Appendix A.2: each processor is a stack of
  neighborhood-attention transformer blocks over the (level, latitude,
  longitude) token grid. Reading of the block (the paper only says "NATTEN
  blocks"): pre-LayerNorm -> 3D neighborhood multi-head self-attention ->
  output projection -> residual add; pre-LayerNorm -> MLP (ratio 4, GELU) ->
  residual add. No final norm.
* Appendix A.2: "circular padding" in longitude -> periodic (mod W) windows;
  "bump" behaviour at the poles -> clamped windows that shift inward and keep
  their full size (also used along the level axis).
* Silent, read as PyTorch defaults: LayerNorm with biased variance, eps 1e-5,
  affine; exact erf GELU; softmax scale 1/sqrt(d_head); all linear layers
  carry a bias; no relative-position bias; dilation 1.
* Appendix A.2 also names rotary position embeddings without an axis split
  or frequencies: an optional 3D rotary embedding (``Shape.rope``) splits the
  rotation pairs over level / latitude / longitude (see ``rope_pairs``).
* Section 2.1 and Appendix A.2, encoder and decoder: convolution layers map
  the 0.25-degree grid to the 2-degree latent and back, with 2 NA blocks of
  hidden width 1024 on the latent side; constants are concatenated with the
  input. Readings (the layer list is not given): the convolutions are patch
  embeddings with kernel = stride (pd levels x 8 x 8 pixels for the
  atmosphere, zero-padded at the top to a multiple of pd levels; 8 x 8 for
  surface + constants), the surface is the last latent level, a linear map
  joins width 1024 to the processor's width, the decoder mirrors it with
  transposed convolutions (kernel = stride); ResNet blocks are not built.

Parity status: every function below is pinned by ``tests/test_oracle_pins.py``
(closed forms, library special cases, invariants, brute force on tiny grids,
and the step counts printed in Section 2.2). Physical forecast skill is not
reproducible without the paper's trained weights and data; that part is out
of reach and is not claimed.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf


# ---------------------------------------------------------------- schedule --

def greedy_schedule(lead_hours: int) -> tuple[int, int]:
    """(six-hour calls, one-hour calls) for an integer lead time (Section 2.1).

    Greedy coin change with coins {6, 1}: as many six-hour steps as fit, the
    remainder in one-hour steps, applied six-hour steps first.
    """
    if int(lead_hours) != lead_hours or lead_hours < 0:
        raise ValueError("lead time must be a non-negative integer number of hours")
    n6 = 0
    rest = int(lead_hours)
    while rest >= 6:
        rest -= 6
        n6 += 1
    return n6, rest


# ------------------------------------------------------------- primitives --

def layer_norm(x, gamma, beta, eps=1e-5):
    """LayerNorm over the last axis: (x - mean) / sqrt(biased var + eps) * gamma + beta."""
    x = np.asarray(x, dtype=np.float64)
    mean = x.mean(axis=-1, keepdims=True)
    var = ((x - mean) ** 2).mean(axis=-1, keepdims=True)
    return (x - mean) / np.sqrt(var + eps) * np.asarray(gamma, np.float64) + np.asarray(beta, np.float64)


def linear(x, weight, bias):
    """x @ weight^T + bias, weight stored [out_features, in_features]."""
    return np.asarray(x, np.float64) @ np.asarray(weight, np.float64).T + np.asarray(bias, np.float64)


def gelu(z):
    """Exact GELU: z * Phi(z) = 0.5 z (1 + erf(z / sqrt 2))."""
    z = np.asarray(z, np.float64)
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


# --------------------------------------------------- neighborhood windows --

def axis_window(n: int, k: int, periodic: bool) -> np.ndarray:
    """[n, k] indices of the window of every position along one axis.

    Clamped ("bump", Appendix A.2): the window of position i starts at
    clamp(i - k//2, 0, n - k) and covers k consecutive positions, so it
    shifts inward at the edges and never shrinks. Requires k <= n.
    Periodic ("circular padding", Appendix A.2): positions (i + o) mod n for
    o in [-k//2, k//2]. Requires k <= n so that the k positions are distinct.
    """
    if k % 2 != 1 or k < 1 or k > n:
        raise ValueError(f"window {k} must be odd and at most the axis length {n}")
    r = k // 2
    win = np.empty((n, k), dtype=np.int64)
    for i in range(n):
        if periodic:
            for o in range(k):
                win[i, o] = (i - r + o) % n
        else:
            start = min(max(i - r, 0), n - k)
            for o in range(k):
                win[i, o] = start + o
    return win


def neighbor_index(D, H, W, kd, kh, kw, lon_periodic=True) -> np.ndarray:
    """[N, kd*kh*kw] token ids of every token's 3D neighborhood.

    Token id n = (level * H + lat) * W + lon. Level and latitude windows are
    clamped; longitude is periodic when ``lon_periodic`` (else clamped).
    Neighbors are listed level-major, then latitude, then longitude.
    """
    wd = axis_window(D, kd, False)
    wh = axis_window(H, kh, False)
    ww = axis_window(W, kw, lon_periodic)
    nbr = np.empty((D, H, W, kd, kh, kw), dtype=np.int64)
    for a in range(kd):
        for b in range(kh):
            for c in range(kw):
                nbr[:, :, :, a, b, c] = ((wd[:, a][:, None, None] * H
                                          + wh[:, b][None, :, None]) * W
                                         + ww[:, c][None, None, :])
    return nbr.reshape(D * H * W, kd * kh * kw)


def neighborhood_attention(q, k, v, heads, nbr, return_weights=False, chunk=1024):
    """3D neighborhood multi-head attention (Section 2.1 "NATTEN").

    q, k, v: [B, N, C] float64; head h owns channels [h*dh, (h+1)*dh).
    nbr: [Nq, K] neighbor token ids for the queries q[:, :Nq] (normally all N).
    For each query t and head h:
        s(t') = q_h(t) . k_h(t') / sqrt(dh)  for t' in nbr[t]
        a = exp(s - max s) / sum exp(s - max s)
        o_h(t) = sum_t' a(t') v_h(t')
    Queries are processed ``chunk`` at a time only to bound memory.
    Returns o [B, Nq, C] (and the weights [B, Nq, heads, K] if asked).
    """
    q = np.asarray(q, np.float64)
    k = np.asarray(k, np.float64)
    v = np.asarray(v, np.float64)
    B, _, C = q.shape
    Nq, K = nbr.shape
    dh = C // heads
    scale = 1.0 / np.sqrt(dh)
    o = np.empty((B, Nq, C), dtype=np.float64)
    wts = np.empty((B, Nq, heads, K), dtype=np.float64) if return_weights else None
    for b in range(B):
        qb = q[b, :Nq].reshape(Nq, heads, dh)
        kb = k[b].reshape(-1, heads, dh)
        vb = v[b].reshape(-1, heads, dh)
        for t0 in range(0, Nq, chunk):
            t1 = min(t0 + chunk, Nq)
            idx = nbr[t0:t1]                        # [T, K]
            kn = kb[idx]                            # [T, K, heads, dh]
            vn = vb[idx]
            s = np.einsum("thd,tkhd->thk", qb[t0:t1], kn) * scale
            s = s - s.max(axis=-1, keepdims=True)
            e = np.exp(s)
            a = e / e.sum(axis=-1, keepdims=True)   # [T, heads, K]
            o[b, t0:t1] = np.einsum("thk,tkhd->thd", a, vn).reshape(t1 - t0, C)
            if return_weights:
                wts[b, t0:t1] = a
    return (o, wts) if return_weights else o


# ------------------------------------------------- rotary position embedding --
# Appendix A.2 states that tokens carry rotary position embeddings (RoFormer)
# but gives neither the split of the head dimension over the three axes nor
# the frequencies. Reading used here: the dh/2 rotation pairs (dims 2p, 2p+1)
# of every head are split into level, latitude and longitude groups (sizes
# n_lev, n_lat, n_lon with n_lon = ceil(P/3), n_lat = ceil((P - n_lon)/2),
# n_lev = the rest), in that order. Pair m of an axis with positions
# 0..n-1 rotates by angle pos * w_m with
#   level, latitude:  w_m = 10000^(-m / n_axis)        (RoFormer frequencies)
#   longitude:        w_m = 2 pi (m + 1) / W             (harmonics of the circle,
#                     so a rotation depends on longitude differences mod W)
# q and k are rotated after the QKV projection; v is not.

def rope_pairs(dh: int):
    """(n_lev, n_lat, n_lon) rotation pairs per axis for head dimension dh."""
    P = dh // 2
    n_lon = -(-P // 3)
    n_lat = -(-(P - n_lon) // 2)
    return P - n_lon - n_lat, n_lat, n_lon


def rope_angles(D, H, W, dh):
    """[N, dh/2] rotation angle of every (token, pair)."""
    n_lev, n_lat, n_lon = rope_pairs(dh)
    lev = np.arange(D, dtype=np.float64)
    lat = np.arange(H, dtype=np.float64)
    lon = np.arange(W, dtype=np.float64)
    ang = np.zeros((D, H, W, dh // 2))
    for m in range(n_lev):
        ang[:, :, :, m] = lev[:, None, None] * 10000.0 ** (-m / n_lev)
    for m in range(n_lat):
        ang[:, :, :, n_lev + m] = lat[None, :, None] * 10000.0 ** (-m / n_lat)
    for m in range(n_lon):
        ang[:, :, :, n_lev + n_lat + m] = lon[None, None, :] * (2.0 * np.pi * (m + 1) / W)
    return ang.reshape(D * H * W, dh // 2)


def rope_rotate(t, heads, angles):
    """Rotate pairs (2p, 2p+1) of every head of t [B, N, C] by angles [N, dh/2]."""
    t = np.asarray(t, np.float64)
    B, N, C = t.shape
    dh = C // heads
    x = t.reshape(B, N, heads, dh // 2, 2)
    c = np.cos(angles)[None, :, None, :]
    s = np.sin(angles)[None, :, None, :]
    out = np.empty_like(x)
    out[..., 0] = x[..., 0] * c - x[..., 1] * s
    out[..., 1] = x[..., 0] * s + x[..., 1] * c
    return out.reshape(B, N, C)


# ------------------------------------------------------ block / processor --

def _f64(w):
    return {name: np.asarray(val, dtype=np.float64) for name, val in w.items()}


def block(x, w, shape):
    """One neighborhood-attention transformer block on x [B, D, H, W, C] (reading A1 above)."""
    w = _f64(w)
    x = np.asarray(x, np.float64)
    B = x.shape[0]
    C = shape.C
    N = shape.D * shape.H * shape.W
    xf = x.reshape(B, N, C)
    nbr = neighbor_index(shape.D, shape.H, shape.W, shape.kd, shape.kh, shape.kw, shape.lon_periodic)
    # attention half
    u = layer_norm(xf, w["ln1_g"], w["ln1_b"], shape.ln_eps)
    qkv = linear(u, w["wqkv"], w["bqkv"])
    q, k, v = qkv[..., :C], qkv[..., C:2 * C], qkv[..., 2 * C:]
    if getattr(shape, "rope", False):
        ang = rope_angles(shape.D, shape.H, shape.W, C // shape.heads)
        q, k = rope_rotate(q, shape.heads, ang), rope_rotate(k, shape.heads, ang)
    o = neighborhood_attention(q, k, v, shape.heads, nbr)
    x1 = xf + linear(o, w["wo"], w["bo"])
    # MLP half
    u2 = layer_norm(x1, w["ln2_g"], w["ln2_b"], shape.ln_eps)
    hid = gelu(linear(u2, w["w1"], w["b1"]))
    x2 = x1 + linear(hid, w["w2"], w["b2"])
    return x2.reshape(x.shape)


def block_at_tokens(x, w, shape, tokens):
    """The block's output at the listed token ids only: [B, len(tokens), C].

    The same definition as ``block`` evaluated where asked: LayerNorm and the
    QKV projection are taken on the union of the listed tokens' neighborhoods,
    attention and the MLP on the listed tokens. Used for full-size latents,
    where evaluating every token in float64 would take hours.
    """
    w = _f64(w)
    x = np.asarray(x, np.float64)
    B = x.shape[0]
    C = shape.C
    N = shape.D * shape.H * shape.W
    xf = x.reshape(B, N, C)
    tokens = np.asarray(tokens, dtype=np.int64)
    nbr_all = neighbor_index(shape.D, shape.H, shape.W, shape.kd, shape.kh, shape.kw, shape.lon_periodic)
    nbr = nbr_all[tokens]                                  # [S, K]
    needed = np.unique(np.concatenate([nbr.ravel(), tokens]))
    pos = {int(t): i for i, t in enumerate(needed)}
    local_nbr = np.vectorize(pos.__getitem__)(nbr)         # [S, K] into `needed`
    local_tok = np.array([pos[int(t)] for t in tokens], dtype=np.int64)
    u = layer_norm(xf[:, needed], w["ln1_g"], w["ln1_b"], shape.ln_eps)
    qkv = linear(u, w["wqkv"], w["bqkv"])
    if getattr(shape, "rope", False):
        ang = rope_angles(shape.D, shape.H, shape.W, C // shape.heads)[needed]
        qkv = np.concatenate([rope_rotate(qkv[..., :C], shape.heads, ang),
                              rope_rotate(qkv[..., C:2 * C], shape.heads, ang), qkv[..., 2 * C:]], axis=-1)
    q = qkv[:, local_tok, :C]
    k, v = qkv[..., C:2 * C], qkv[..., 2 * C:]
    # queries first in a [B, S + ...] layout: neighborhood_attention reads q[:, :S]
    o = neighborhood_attention(q, k, v, shape.heads, local_nbr)
    x1 = xf[:, tokens] + linear(o, w["wo"], w["bo"])
    u2 = layer_norm(x1, w["ln2_g"], w["ln2_b"], shape.ln_eps)
    return x1 + linear(gelu(linear(u2, w["w1"], w["b1"])), w["w2"], w["b2"])


def processor(x, blocks, shape):
    """One processor call: its blocks in order, each with its own weights."""
    for w in blocks:
        x = block(x, w, shape)
    return x


def rollout(x, lead_hours, p6_blocks, p1_blocks, shape, per_step=None):
    """Latent rollout to ``lead_hours`` (Section 2.1): greedy schedule, six-hour steps first.

    If ``per_step`` is a list, the latent after every processor call is appended to it.
    """
    n6, n1 = greedy_schedule(lead_hours)
    x = np.asarray(x, np.float64)
    for _ in range(n6):
        x = processor(x, p6_blocks, shape)
        if per_step is not None:
            per_step.append(x)
    for _ in range(n1):
        x = processor(x, p1_blocks, shape)
        if per_step is not None:
            per_step.append(x)
    return x


# ---------------------------------------------------------- FP8 E4M3 codec --
# The FP8 MLP precision (a product-level choice, not a paper requirement)
# rounds MLP GEMM operands to E4M3 as defined by the OCP 8-bit floating point
# specification: 1 sign bit, 4 exponent bits with bias 7, 3 mantissa bits;
# exponent field 0 holds subnormals m/8 * 2^-6; S.1111.111 is NaN; there are
# no infinities, so the largest finite magnitude is 1.75 * 2^8 = 448.

def e4m3_decode(code: int) -> float:
    """Value of an E4M3 code (0..255)."""
    sign = -1.0 if code & 0x80 else 1.0
    e = (code >> 3) & 0xF
    m = code & 0x7
    if e == 0xF and m == 0x7:
        return float("nan")
    if e == 0:
        return sign * (m / 8.0) * 2.0 ** -6
    return sign * (1.0 + m / 8.0) * 2.0 ** (e - 7)


def e4m3_round(x):
    """Round to the nearest E4M3 value, ties to the even code, saturating at +-448."""
    x = np.asarray(x, dtype=np.float64)
    codes = np.arange(0, 0x7F)                       # non-negative finite codes, increasing values
    vals = np.array([e4m3_decode(int(c)) for c in codes])
    a = np.minimum(np.abs(x), 448.0)
    hi = np.clip(np.searchsorted(vals, a, side="left"), 0, len(vals) - 1)
    lo = np.clip(hi - 1, 0, len(vals) - 1)
    d_lo, d_hi = a - vals[lo], vals[hi] - a
    pick_hi = (d_hi < d_lo) | ((d_hi == d_lo) & (codes[hi] % 2 == 0))
    r = np.where(pick_hi, vals[hi], vals[lo])
    return np.sign(x) * r


def fp8_mlp_scales(w, C):
    """Static per-tensor E4M3 scales of the FP8-MLP precision for one block.

    Each scale is a bound on the magnitude of its tensor divided by 448 (the
    largest E4M3 value), so no value saturates for any input:
      LN2 output: |u_c| <= |gamma_c| sqrt(C - 1) + |beta_c|, because a biased
        standard deviation s over C values satisfies |x_c - mean| <= sqrt(C - 1) s;
      W1, W2: their largest magnitude;
      GELU(FC1) output: |z_j| <= sum_c |W1_jc| bound_u_c + |b1_j| (triangle
        inequality) and |GELU(z)| <= max(|z|, 0.17) (GELU's minimum is -0.16997).
    Returns (s_u, s_w1, s_h, s_w2).
    """
    g = np.abs(np.asarray(w["ln2_g"], np.float64))
    b = np.abs(np.asarray(w["ln2_b"], np.float64))
    W1 = np.abs(np.asarray(w["w1"], np.float64))
    W2 = np.abs(np.asarray(w["w2"], np.float64))
    b1 = np.abs(np.asarray(w["b1"], np.float64))
    bound_u = g * np.sqrt(C - 1.0) + b
    bound_z = W1 @ bound_u + b1
    return (bound_u.max() / 448.0, W1.max() / 448.0, max(bound_z.max(), 0.17) / 448.0, W2.max() / 448.0)


def block_fp8mlp(x, w, shape, rounding=None):
    """The block with its MLP operands rounded to E4M3 under the static scales.

    Same as ``block`` except: LN2's output, W1, the GELU output and W2 are each
    divided by their scale, rounded to E4M3 (``rounding``, default
    ``e4m3_round``) and the products rescaled. The attention half is exact.
    """
    q = e4m3_round if rounding is None else rounding
    w = _f64(w)
    x = np.asarray(x, np.float64)
    B = x.shape[0]
    C = shape.C
    N = shape.D * shape.H * shape.W
    xf = x.reshape(B, N, C)
    nbr = neighbor_index(shape.D, shape.H, shape.W, shape.kd, shape.kh, shape.kw, shape.lon_periodic)
    u = layer_norm(xf, w["ln1_g"], w["ln1_b"], shape.ln_eps)
    qkv = linear(u, w["wqkv"], w["bqkv"])
    o = neighborhood_attention(qkv[..., :C], qkv[..., C:2 * C], qkv[..., 2 * C:], shape.heads, nbr)
    x1 = xf + linear(o, w["wo"], w["bo"])
    s_u, s_w1, s_h, s_w2 = fp8_mlp_scales(w, C)
    u2 = q(layer_norm(x1, w["ln2_g"], w["ln2_b"], shape.ln_eps) / s_u)
    z = (u2 @ q(w["w1"] / s_w1).T) * (s_u * s_w1) + w["b1"]
    h = q(gelu(z) / s_h)
    x2 = x1 + (h @ q(w["w2"] / s_w2).T) * (s_h * s_w2) + w["b2"]
    return x2.reshape(x.shape)


def rel_l2(y, y_ref) -> float:
    """||y - y_ref||_2 / ||y_ref||_2 accumulated in float64."""
    y = np.asarray(y, np.float64).ravel()
    y_ref = np.asarray(y_ref, np.float64).ravel()
    return float(np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref))


# ------------------------------------------------------- encoder / decoder --
# Shapes: synth.Codec. Atmosphere [levels, H0, W0, v_atm], surface input
# [H0, W0, v_sfc_in], constants [H0, W0, n_const]; latent [D, H, W, C] with
# D = level_pad / pd + 1 (surface last), H = H0 / p, W = W0 / p.

def codec_patches_atm(atm, cd):
    """[D-1, H, W, pd*p*p*v_atm]: each token's input patch, ordered (level, row, column, variable).

    The atmosphere is zero-padded at the top (lowest level indices) to
    level_pad levels, so padded level i holds input level i - (level_pad - levels).
    """
    atm = np.asarray(atm, np.float64)
    pad = np.zeros((cd.level_pad, cd.H0, cd.W0, cd.v_atm))
    pad[cd.level_pad - cd.levels:] = atm
    t = pad.reshape(cd.D - 1, cd.pd, cd.H, cd.p, cd.W, cd.p, cd.v_atm)
    return t.transpose(0, 2, 4, 1, 3, 5, 6).reshape(cd.D - 1, cd.H, cd.W, cd.k_atm)


def codec_patches_sfc(sfc, const, cd):
    """[H, W, p*p*(v_sfc_in + n_const)]: surface fields then constants per pixel, ordered (row, column, channel)."""
    x = np.concatenate([np.asarray(sfc, np.float64), np.asarray(const, np.float64)], axis=-1)
    c = x.shape[-1]
    return x.reshape(cd.H, cd.p, cd.W, cd.p, c).transpose(0, 2, 1, 3, 4).reshape(cd.H, cd.W, cd.p * cd.p * c)


def codec_unpatch_atm(y, cd):
    """Inverse layout of codec_patches_atm: [D-1, H, W, k_atm] -> [levels, H0, W0, v_atm] (padding dropped)."""
    t = np.asarray(y, np.float64).reshape(cd.D - 1, cd.H, cd.W, cd.pd, cd.p, cd.p, cd.v_atm)
    full = t.transpose(0, 3, 1, 4, 2, 5, 6).reshape(cd.level_pad, cd.H0, cd.W0, cd.v_atm)
    return full[cd.level_pad - cd.levels:]


def codec_unpatch_sfc(y, cd):
    """[H, W, p*p*v_sfc_out] -> [H0, W0, v_sfc_out]."""
    t = np.asarray(y, np.float64).reshape(cd.H, cd.W, cd.p, cd.p, cd.v_sfc_out)
    return t.transpose(0, 2, 1, 3, 4).reshape(cd.H0, cd.W0, cd.v_sfc_out)


def encode(atm, sfc, const, w, cd):
    """Physical fields -> latent [D, H, W, C] (Section 2.1, Appendix A.2; readings above).

    Patch embeddings (convolutions with kernel = stride), the encoder's NA
    blocks at width Ce, then the linear map to the processor's width C.
    """
    w64 = {k: v for k, v in w.items() if not k.endswith("blocks")}
    x = np.empty((cd.D, cd.H, cd.W, cd.Ce))
    x[:cd.D - 1] = linear(codec_patches_atm(atm, cd), w64["embed_atm_w"], w64["embed_atm_b"])
    x[cd.D - 1] = linear(codec_patches_sfc(sfc, const, cd), w64["embed_sfc_w"], w64["embed_sfc_b"])
    x = processor(x[None], w["enc_blocks"], cd.block_shape())[0]
    return linear(x, w64["enc_out_w"], w64["enc_out_b"])


def decode(latent, w, cd):
    """Latent [D, H, W, C] -> (atmosphere [levels, H0, W0, v_atm], surface [H0, W0, v_sfc_out]).

    The linear map to width Ce, the decoder's NA blocks, then transposed
    convolutions with kernel = stride (one linear map per token, its outputs
    laid out over the token's pixels).
    """
    x = linear(latent, w["dec_in_w"], w["dec_in_b"])
    x = processor(x[None], w["dec_blocks"], cd.block_shape())[0]
    atm = codec_unpatch_atm(linear(x[:cd.D - 1], w["unembed_atm_w"], w["unembed_atm_b"]), cd)
    sfc = codec_unpatch_sfc(linear(x[cd.D - 1], w["unembed_sfc_w"], w["unembed_sfc_b"]), cd)
    return atm, sfc
