"""The FP8-MLP precision's static per-tensor scales against the tightest
per-tensor scales there are (each tensor's own max over the batch), on the
oracle's E4M3 emulation of one block.

The static scales are bounds that hold for every input (so nothing saturates
and a result does not depend on what it is batched with); they are looser
than the data's own maxima by up to ~27x. E4M3 keeps 3 mantissa bits at
every exponent, so a looser scale only moves values down the exponent range:
the block's error with the static scales stays within 5 % of its error with
the amax scales. The error itself (~2e-2 per block, ~5 % on the MLP output)
is E4M3's mantissa rounding, not the choice of scale.
"""
import numpy as np

import synth
from oracle import wm_oracle as orc


def _fp8_block(xf, x1, u2, W, scales):
    q = orc.e4m3_round
    su, sw1, sh, sw2 = scales
    z = (q(u2 / su) @ q(W["w1"] / sw1).T) * (su * sw1) + W["b1"]
    h = q(orc.gelu(z) / sh)
    return x1 + (h @ q(W["w2"] / sw2).T) * (sh * sw2) + W["b2"]


def test_static_fp8_scales_cost_no_accuracy_against_amax_scales():
    s = synth.SMALL
    x = synth.latent(s, 1, seed=1)
    w = synth.block_weights(s.C, 0, 0, 0, stress=True)
    W = orc._f64(w)
    C = s.C
    ref = orc.block(x, w, s).reshape(1, -1, C)
    xf = np.asarray(x, np.float64).reshape(1, -1, C)
    nbr = orc.neighbor_index(s.D, s.H, s.W, s.kd, s.kh, s.kw, True)
    qkv = orc.linear(orc.layer_norm(xf, W["ln1_g"], W["ln1_b"]), W["wqkv"], W["bqkv"])
    o = orc.neighborhood_attention(qkv[..., :C], qkv[..., C:2 * C], qkv[..., 2 * C:], s.heads, nbr)
    x1 = xf + orc.linear(o, W["wo"], W["bo"])
    u2 = orc.layer_norm(x1, W["ln2_g"], W["ln2_b"])
    h = orc.gelu(orc.linear(u2, W["w1"], W["b1"]))
    static = orc.fp8_mlp_scales(W, C)
    amax = (np.abs(u2).max() / 448, np.abs(W["w1"]).max() / 448, np.abs(h).max() / 448, np.abs(W["w2"]).max() / 448)
    assert all(st >= am * (1 - 1e-12) for st, am in zip(static, amax))   # the bounds hold on this data
    assert static[2] > 5 * amax[2]                                        # and are far from tight
    e_static = orc.rel_l2(_fp8_block(xf, x1, u2, W, static), ref)
    e_amax = orc.rel_l2(_fp8_block(xf, x1, u2, W, amax), ref)
    assert e_static <= 1.05 * e_amax, (e_static, e_amax)
    assert 5e-3 < e_amax < 5e-2, e_amax            # the E4M3 mantissa's own error
    # the emulation above is the oracle's FP8 block
    assert np.max(np.abs(_fp8_block(xf, x1, u2, W, static).reshape(x.shape) - orc.block_fp8mlp(x, w, s))) < 1e-12
