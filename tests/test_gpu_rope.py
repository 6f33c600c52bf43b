"""Blocks with the 3D rotary position embedding against the oracle."""
import dataclasses

import numpy as np
import pytest
import torch

import paper_2503_22235_gb300 as wm
import synth
from oracle import wm_oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2503_22235_gb300 import build as wm_build
    wm_build.build()


def _run_block(shape, prec, x, p6, p1):
    ctx = wm.wm_create_from_host(wm.make_config(shape, prec), synth.pack_weights(p6, p1))
    try:
        xt = torch.from_numpy(x).cuda()
        wm.wm_block_forward(ctx, xt, wm.WM_P6, 0)
        torch.cuda.synchronize()
        return xt.cpu().numpy()
    finally:
        wm.wm_destroy(ctx)


@pytest.mark.parametrize("prec,tol", [(wm.WM_PREC_FP32, 1e-5), (wm.WM_PREC_BF16, 2e-2)])
def test_rope_block_small_latent(prec, tol):
    s = dataclasses.replace(synth.SMALL, blocks_p6=1, blocks_p1=1, rope=True)
    p6, p1 = synth.processor_weights(s, seed=0, stress=True)
    x = synth.latent(s, 2, seed=1)
    got = _run_block(s, prec, x, p6, p1)
    ref = orc.block(x, p6[0], s)
    err = orc.rel_l2(got, ref)
    assert err <= tol, err
    # the embedding changes the result by far more than the kernel's error
    assert orc.rel_l2(ref, orc.block(x, p6[0], dataclasses.replace(s, rope=False))) > 5 * err


def test_rope_full_size_block_at_sampled_tokens():
    s = dataclasses.replace(synth.FULL, blocks_p6=1, blocks_p1=1, rope=True)
    p6, p1 = synth.processor_weights(s, seed=0, stress=True)
    x = synth.latent(s, 1, seed=2)
    got = _run_block(s, wm.WM_PREC_BF16, x, p6, p1).reshape(1, s.N, s.C)
    rng = np.random.default_rng(1)
    toks = np.unique(np.concatenate([[0, s.N - 1, s.W - 1], rng.integers(0, s.N, 12)]))
    ref = orc.block_at_tokens(x, p6[0], s, toks)
    assert orc.rel_l2(got[:, toks], ref) <= 2e-2
