"""Pins of the oracle's encoder and decoder (Section 2.1, Appendix A.2).

The patch embedding is checked against a convolution written out as loops
over output cells and kernel taps (kernel tensor [out, level, row, column,
channel], stride = kernel, zero levels above the top); the decoder's
transposed convolution against loops over output pixels; the layouts against
exact round trips; the whole encoder / decoder against the longitude roll
symmetry that periodic windows imply.
"""
import dataclasses

import numpy as np
import pytest

import synth
from oracle import wm_oracle as orc

TINY = synth.Codec(H0=4, W0=6, levels=3, level_pad=4, pd=2, p=2, v_atm=2, v_sfc_in=2, v_sfc_out=3, n_const=1,
                   Ce=8, heads=2, kd=3, kh=1, kw=3, blocks=1)


def _rng_fields(cd, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((cd.levels, cd.H0, cd.W0, cd.v_atm)),
            rng.standard_normal((cd.H0, cd.W0, cd.v_sfc_in)),
            rng.standard_normal((cd.H0, cd.W0, cd.n_const)))


def test_codec_shapes_of_the_paper_grid():
    cd = synth.FULL_CODEC
    # 0.25 degrees -> 2 degrees is 8x per axis; 28 levels padded to 32 in slabs of 4, plus the surface
    assert (cd.D, cd.H, cd.W) == (9, 90, 180)
    assert (cd.v_atm, cd.levels, cd.v_sfc_in, cd.v_sfc_out, cd.n_const, cd.Ce) == (5, 28, 8, 17, 8, 1024)
    assert cd.k_atm == 4 * 8 * 8 * 5 and cd.k_sfc == 8 * 8 * 16 and cd.n_sfc_out == 8 * 8 * 17


def test_atmosphere_patch_embedding_is_a_strided_convolution():
    cd = TINY
    atm, _, _ = _rng_fields(cd, 1)
    rng = np.random.default_rng(2)
    K = rng.standard_normal((cd.Ce, cd.pd, cd.p, cd.p, cd.v_atm))     # conv kernel [out, level, row, col, var]
    b = rng.standard_normal(cd.Ce)
    got = orc.linear(orc.codec_patches_atm(atm, cd), K.reshape(cd.Ce, -1), b)
    top = cd.level_pad - cd.levels                                   # zero levels above the first input level
    ref = np.zeros((cd.D - 1, cd.H, cd.W, cd.Ce))
    for l in range(cd.D - 1):
        for h in range(cd.H):
            for w in range(cd.W):
                for o in range(cd.Ce):
                    acc = b[o]
                    for dl in range(cd.pd):
                        lev = l * cd.pd + dl - top
                        if lev < 0:
                            continue
                        for dy in range(cd.p):
                            for dx in range(cd.p):
                                for v in range(cd.v_atm):
                                    acc += K[o, dl, dy, dx, v] * atm[lev, h * cd.p + dy, w * cd.p + dx, v]
                    ref[l, h, w, o] = acc
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_surface_patch_embedding_is_a_strided_convolution_over_fields_and_constants():
    cd = TINY
    _, sfc, const = _rng_fields(cd, 3)
    cin = cd.v_sfc_in + cd.n_const
    rng = np.random.default_rng(4)
    K = rng.standard_normal((cd.Ce, cd.p, cd.p, cin))
    got = orc.linear(orc.codec_patches_sfc(sfc, const, cd), K.reshape(cd.Ce, -1), np.zeros(cd.Ce))
    ref = np.zeros((cd.H, cd.W, cd.Ce))
    for h in range(cd.H):
        for w in range(cd.W):
            for o in range(cd.Ce):
                for dy in range(cd.p):
                    for dx in range(cd.p):
                        px = np.concatenate([sfc[h * cd.p + dy, w * cd.p + dx], const[h * cd.p + dy, w * cd.p + dx]])
                        ref[h, w, o] += K[o, dy, dx] @ px
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_decoder_output_is_a_transposed_convolution():
    cd = TINY
    rng = np.random.default_rng(5)
    x = rng.standard_normal((cd.D - 1, cd.H, cd.W, cd.Ce))
    K = rng.standard_normal((cd.pd, cd.p, cd.p, cd.v_atm, cd.Ce))    # [level, row, col, var, in]
    b = rng.standard_normal((cd.pd, cd.p, cd.p, cd.v_atm))
    got = orc.codec_unpatch_atm(orc.linear(x, K.reshape(-1, cd.Ce), b.ravel()), cd)
    top = cd.level_pad - cd.levels
    for lev in range(cd.levels):
        for y in range(cd.H0):
            for xx in range(cd.W0):
                lp = lev + top
                tok = x[lp // cd.pd, y // cd.p, xx // cd.p]
                ref = K[lp % cd.pd, y % cd.p, xx % cd.p] @ tok + b[lp % cd.pd, y % cd.p, xx % cd.p]
                assert np.allclose(got[lev, y, xx], ref, rtol=1e-12, atol=1e-12)
    xs = rng.standard_normal((cd.H, cd.W, cd.Ce))
    Ks = rng.standard_normal((cd.p, cd.p, cd.v_sfc_out, cd.Ce))
    gs = orc.codec_unpatch_sfc(orc.linear(xs, Ks.reshape(-1, cd.Ce), np.zeros(Ks.shape[0] * 0 + cd.n_sfc_out)), cd)
    for y in range(cd.H0):
        for xx in range(cd.W0):
            assert np.allclose(gs[y, xx], Ks[y % cd.p, xx % cd.p] @ xs[y // cd.p, xx // cd.p], rtol=1e-12, atol=1e-12)


def test_patch_layouts_round_trip_exactly():
    cd = dataclasses.replace(TINY, v_sfc_out=TINY.v_sfc_in + TINY.n_const)
    atm, sfc, const = _rng_fields(cd, 6)
    assert np.array_equal(orc.codec_unpatch_atm(orc.codec_patches_atm(atm, cd), cd), atm)
    back = orc.codec_unpatch_sfc(orc.codec_patches_sfc(sfc, const, cd), cd)
    assert np.array_equal(back, np.concatenate([sfc, const], axis=-1))
    # the padding levels sit above the first input level and hold zeros
    pad = orc.codec_patches_atm(atm, cd)[0].reshape(cd.H, cd.W, cd.pd, cd.p, cd.p, cd.v_atm)
    assert np.all(pad[:, :, :cd.level_pad - cd.levels] == 0)


@pytest.mark.parametrize("stress", [False, True])
def test_encoder_and_decoder_commute_with_a_longitude_roll(stress):
    cd = TINY
    w = synth.codec_weights(cd, 6, seed=0, stress=stress)
    atm, sfc, const = _rng_fields(cd, 7)
    lat = orc.encode(atm, sfc, const, w, cd)
    lat_r = orc.encode(np.roll(atm, cd.p, axis=2), np.roll(sfc, cd.p, axis=1), np.roll(const, cd.p, axis=1), w, cd)
    assert np.allclose(lat_r, np.roll(lat, 1, axis=2), rtol=1e-10, atol=1e-10)
    a, s = orc.decode(lat, w, cd)
    a_r, s_r = orc.decode(np.roll(lat, 1, axis=2), w, cd)
    assert np.allclose(a_r, np.roll(a, cd.p, axis=2), rtol=1e-10, atol=1e-10)
    assert np.allclose(s_r, np.roll(s, cd.p, axis=1), rtol=1e-10, atol=1e-10)
    # and a shift by less than a patch is not a symmetry (the test can fail)
    lat_1 = orc.encode(np.roll(atm, 1, axis=2), np.roll(sfc, 1, axis=1), np.roll(const, 1, axis=1), w, cd)
    assert not np.allclose(lat_1, np.roll(lat, 1, axis=2), rtol=1e-3, atol=1e-3)


def test_encoder_with_identity_blocks_is_embedding_then_output_map():
    cd = TINY
    w = synth.codec_weights(cd, 6, seed=1, stress=True)
    for blk in w["enc_blocks"]:   # zero weights and biases: each block is the identity
        for k in blk:
            blk[k] = np.zeros_like(blk[k]) if not k.endswith("_g") else np.ones_like(blk[k])
    atm, sfc, const = _rng_fields(cd, 8)
    x = np.concatenate([orc.linear(orc.codec_patches_atm(atm, cd), w["embed_atm_w"], w["embed_atm_b"]),
                        orc.linear(orc.codec_patches_sfc(sfc, const, cd), w["embed_sfc_w"], w["embed_sfc_b"])[None]])
    ref = orc.linear(x, w["enc_out_w"], w["enc_out_b"])
    assert np.allclose(orc.encode(atm, sfc, const, w, cd), ref, rtol=1e-12, atol=1e-12)
    assert ref.shape == (cd.D, cd.H, cd.W, 6)
