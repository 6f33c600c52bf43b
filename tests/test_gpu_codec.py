"""Encoder and decoder on the GPU against the oracle (Section 2.1, Appendix A.2).

Small grid (192 x 384, 10 levels padded to 12, latent 4 x 24 x 48): encoder,
decoder and the whole field-to-field forecast in FP32 (<= 1e-5 relative L2,
FP32 accumulation order only) and BF16 (<= 2e-2, the per-block bound; the
encoder and decoder are 2 blocks plus 3 GEMMs each). Also: the longitude-roll
symmetry on the GPU and rejected configurations.
"""
import dataclasses

import numpy as np
import pytest
import torch

import paper_2503_22235_gb300 as wm
import synth
from oracle import wm_oracle as orc

pytestmark = pytest.mark.gpu
CD = synth.SMALL_CODEC
C = synth.SMALL.C
TOL = {wm.WM_PREC_FP32: 1e-5, wm.WM_PREC_BF16: 2e-2}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2503_22235_gb300 import build as wm_build
    wm_build.build()


@pytest.fixture(scope="module")
def weights():
    return synth.codec_weights(CD, C, seed=0, stress=True)


@pytest.fixture(scope="module")
def fields():
    return synth.codec_inputs(CD, seed=1)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _codec(weights, prec):
    return wm.wm_codec_create(wm.make_codec_config(CD, C, prec), synth.pack_codec_weights(weights))


@pytest.mark.parametrize("prec", [wm.WM_PREC_FP32, wm.WM_PREC_BF16])
def test_encoder_matches_oracle(weights, fields, prec):
    cd = _codec(weights, prec)
    try:
        atm, sfc, cst = fields
        lat = torch.empty(CD.D, CD.H, CD.W, C, device="cuda")
        wm.wm_encode(cd, _dev(atm), _dev(sfc), _dev(cst), lat)
        torch.cuda.synchronize()
        ref = orc.encode(atm, sfc, cst, weights, CD)
        err = orc.rel_l2(lat.cpu().numpy(), ref)
        print(f"encoder rel-L2 {err:.2e}")
        assert err <= TOL[prec], err
    finally:
        wm.wm_codec_destroy(cd)


@pytest.mark.parametrize("prec", [wm.WM_PREC_FP32, wm.WM_PREC_BF16])
def test_decoder_matches_oracle(weights, prec):
    cd = _codec(weights, prec)
    try:
        lat = synth.latent(synth.SMALL, 1, seed=3)[0]
        a_out = torch.empty(CD.levels, CD.H0, CD.W0, CD.v_atm, device="cuda")
        s_out = torch.empty(CD.H0, CD.W0, CD.v_sfc_out, device="cuda")
        lat_d = _dev(lat)
        wm.wm_decode(cd, lat_d, a_out, s_out)
        torch.cuda.synchronize()
        ra, rs = orc.decode(lat, weights, CD)
        ea, es = orc.rel_l2(a_out.cpu().numpy(), ra), orc.rel_l2(s_out.cpu().numpy(), rs)
        print(f"decoder rel-L2 atmosphere {ea:.2e} surface {es:.2e}")
        assert ea <= TOL[prec] and es <= TOL[prec], (ea, es)
        assert torch.equal(lat_d, _dev(lat))   # the latent is not modified
    finally:
        wm.wm_codec_destroy(cd)


@pytest.mark.parametrize("prec", [wm.WM_PREC_FP32, wm.WM_PREC_BF16])
def test_field_forecast_matches_oracle(weights, fields, prec):
    s = dataclasses.replace(synth.SMALL, blocks_p6=2, blocks_p1=1)
    p6, p1 = synth.processor_weights(s, seed=0, stress=True)
    ctx = wm.wm_create_from_host(wm.make_config(s, prec, 1), synth.pack_weights(p6, p1))
    cd = _codec(weights, prec)
    try:
        atm, sfc, cst = fields
        lead = 7
        ws = torch.empty(CD.D, CD.H, CD.W, C, device="cuda")
        a_out = torch.empty(CD.levels, CD.H0, CD.W0, CD.v_atm, device="cuda")
        s_out = torch.empty(CD.H0, CD.W0, CD.v_sfc_out, device="cuda")
        wm.wm_forecast_fields(ctx, cd, _dev(atm), _dev(sfc), _dev(cst), lead, ws, a_out, s_out)
        torch.cuda.synchronize()
        lat = orc.rollout(orc.encode(atm, sfc, cst, weights, CD)[None], lead, p6, p1, s)[0]
        ra, rs = orc.decode(lat, weights, CD)
        ea, es = orc.rel_l2(a_out.cpu().numpy(), ra), orc.rel_l2(s_out.cpu().numpy(), rs)
        print(f"forecast rel-L2 atmosphere {ea:.2e} surface {es:.2e}")
        tol = 1e-5 if prec == wm.WM_PREC_FP32 else 5e-2
        assert ea <= tol and es <= tol, (ea, es)
    finally:
        wm.wm_codec_destroy(cd)
        wm.wm_destroy(ctx)


def test_encoder_commutes_with_a_longitude_roll(weights, fields):
    cd = _codec(weights, wm.WM_PREC_FP32)
    try:
        atm, sfc, cst = fields
        a = torch.empty(CD.D, CD.H, CD.W, C, device="cuda")
        b = torch.empty_like(a)
        wm.wm_encode(cd, _dev(atm), _dev(sfc), _dev(cst), a)
        wm.wm_encode(cd, _dev(np.roll(atm, CD.p, axis=2)), _dev(np.roll(sfc, CD.p, axis=1)),
                     _dev(np.roll(cst, CD.p, axis=1)), b)
        torch.cuda.synchronize()
        assert orc.rel_l2(b.cpu().numpy(), np.roll(a.cpu().numpy(), 1, axis=2)) < 1e-5
    finally:
        wm.wm_codec_destroy(cd)


@pytest.mark.parametrize("change", [dict(H0=190), dict(level_pad=11), dict(levels=13), dict(kd=2), dict(blocks=0),
                                    dict(heads=3)])
def test_bad_codec_configs_are_rejected(weights, change):
    bad = dataclasses.replace(CD, **change)
    with pytest.raises(wm.WmError):
        wm.wm_codec_create(wm.make_codec_config(bad, C, wm.WM_PREC_BF16), synth.pack_codec_weights(weights))


def test_codec_weight_blob_length_is_checked(weights):
    blob = synth.pack_codec_weights(weights)
    with pytest.raises(wm.WmError):
        wm.wm_codec_create(wm.make_codec_config(CD, C, wm.WM_PREC_BF16), blob[:-1])


@pytest.mark.parametrize("prec", [wm.WM_PREC_FP32, wm.WM_PREC_BF16])
def test_clamped_longitude_codec_matches_oracle(fields, prec):
    """The same encoder and decoder with clamped (non-periodic) longitude windows."""
    cd = dataclasses.replace(CD, lon_periodic=False)
    w = synth.codec_weights(cd, C, seed=2, stress=True)
    codec = wm.wm_codec_create(wm.make_codec_config(cd, C, prec), synth.pack_codec_weights(w))
    try:
        atm, sfc, cst = fields
        lat = torch.empty(cd.D, cd.H, cd.W, C, device="cuda")
        wm.wm_encode(codec, _dev(atm), _dev(sfc), _dev(cst), lat)
        a_out = torch.empty(cd.levels, cd.H0, cd.W0, cd.v_atm, device="cuda")
        s_out = torch.empty(cd.H0, cd.W0, cd.v_sfc_out, device="cuda")
        wm.wm_decode(codec, lat, a_out, s_out)
        torch.cuda.synchronize()
        ref_lat = orc.encode(atm, sfc, cst, w, cd)
        ra, rs = orc.decode(lat.cpu().numpy(), w, cd)
        errs = (orc.rel_l2(lat.cpu().numpy(), ref_lat), orc.rel_l2(a_out.cpu().numpy(), ra),
                orc.rel_l2(s_out.cpu().numpy(), rs))
        print("clamped-longitude codec rel-L2", [f"{e:.2e}" for e in errs])
        assert max(errs) <= TOL[prec], errs
    finally:
        wm.wm_codec_destroy(codec)
