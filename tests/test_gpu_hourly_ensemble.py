"""Hourly outputs from one initial state and ensemble batches.

Both reuse the batched processor step, whose kernels are row independent, so
every hourly output and every ensemble member must equal the corresponding
single-latent rollout bit for bit.
"""
import dataclasses

import numpy as np
import pytest
import torch

import paper_2503_22235_gb300 as wm
import synth
from oracle import wm_oracle as orc
from parity_util import assert_close

pytestmark = pytest.mark.gpu
SHAPE = dataclasses.replace(synth.SMALL, blocks_p6=2, blocks_p1=1)


@pytest.fixture(scope="module")
def ctx():
    from paper_2503_22235_gb300 import build as wm_build
    wm_build.build()
    p6, p1 = synth.processor_weights(SHAPE, seed=0, stress=True)
    c = wm.wm_create_from_host(wm.make_config(SHAPE, wm.WM_PREC_BF16, max_batch=4), synth.pack_weights(p6, p1))
    yield c
    wm.wm_destroy(c)


@pytest.mark.parametrize("max_lead,max_batch", [(20, 2), (13, 4), (5, 3), (0, 1)])
def test_hourly_outputs_equal_single_rollouts(ctx, max_lead, max_batch):
    x = torch.from_numpy(synth.latent(SHAPE, 1, seed=31)).cuda()
    out = torch.empty((max_lead + 1,) + tuple(x.shape[1:]), device="cuda")
    wm.wm_rollout_hourly(ctx, x, max_lead, out, max_batch)
    for t in range(max_lead + 1):
        alone = x.clone()
        wm.wm_latent_rollout(ctx, alone, t)
        torch.cuda.synchronize()
        assert torch.equal(out[t:t + 1], alone), t


@pytest.mark.parametrize("prec,tol_per_block", [(wm.WM_PREC_FP32, 1e-5), (wm.WM_PREC_BF16, 2e-2)])
def test_hourly_outputs_match_the_oracle(ctx, prec, tol_per_block):
    """Every hourly output out[t], t = 0..13, against the oracle's rollout to
    t hours (Section 2.1 greedy schedule; the hourly forecasts of Section 4.1),
    within the per-block tolerance times the blocks the rollout applies."""
    x = synth.latent(SHAPE, 1, seed=31)
    p6, p1 = synth.processor_weights(SHAPE, seed=0, stress=True)
    wm.wm_set_precision(ctx, prec)
    try:
        out = torch.empty((14,) + x.shape[1:], device="cuda")
        wm.wm_rollout_hourly(ctx, torch.from_numpy(x).cuda(), 13, out, 3)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.array_equal(got[0:1], x)
        for t in range(1, 14):
            n6, n1 = orc.greedy_schedule(t)
            blocks = n6 * SHAPE.blocks_p6 + n1 * SHAPE.blocks_p1
            ref = orc.rollout(x, t, p6, p1, SHAPE)
            assert_close(got[t:t + 1], ref, tol_per_block * blocks, SHAPE.C, (prec, t))
    finally:
        wm.wm_set_precision(ctx, wm.WM_PREC_BF16)


@pytest.mark.parametrize("prec", [wm.WM_PREC_BF16, wm.WM_PREC_BF16_FP8MLP])
def test_ensemble_members_equal_single_rollouts(ctx, prec):
    wm.wm_set_precision(ctx, prec)
    try:
        E = 5
        xs = synth.latent(SHAPE, E, seed=40)
        ens = torch.from_numpy(xs).cuda()
        wm.wm_latent_rollout(ctx, ens, 13)
        for e in range(E):
            alone = torch.from_numpy(xs[e:e + 1]).cuda()
            wm.wm_latent_rollout(ctx, alone, 13)
            torch.cuda.synchronize()
            assert torch.equal(ens[e:e + 1], alone), e
    finally:
        wm.wm_set_precision(ctx, wm.WM_PREC_BF16)
