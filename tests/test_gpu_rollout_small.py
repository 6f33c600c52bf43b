"""GPU parity of the whole-rollout kernel for narrow latents (C = 128, 4 heads):
one launch runs every block of the greedy schedule of up to four latents
(paper Sec. 2.1 latent rollout and greedy schedule; App. A.2 blocks).

* Against the FP64 oracle: rollouts of 1, 6, 7 and 13 hours on the
  4 x 24 x 48 latent with stress weights, and on grids that move the pole
  clamping, the window sizes and the level window (3 x 16 x 32 with 3x5x5;
  2 x 8 x 32 with 1x5x3; 2 x 8 x 48 with 1x3x3); relative L2 within 2e-2 per
  block and the per-token bound.
* Against the per-kernel path (wm_set_fused_rollout(0)): within the same
  tolerance (explicit LayerNorm here, folded into the GEMMs there).
* Bit for bit with itself: a rollout equals its chained processor steps (one
  launch per step) and its hourly outputs; latents batched in one launch
  (uneven leads through wm_rollout_batch, ensembles larger than one launch)
  equal the same latents alone.
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

CUDA = torch.device("cuda")
SMALL3 = dataclasses.replace(synth.SMALL, blocks_p6=2, blocks_p1=1)
GRIDS = [
    SMALL3,
    dataclasses.replace(SMALL3, D=3, H=16, W=32),
    dataclasses.replace(SMALL3, D=2, H=8, W=32, kd=1, kh=5, kw=3),
    dataclasses.replace(SMALL3, D=2, H=8, W=48, kd=1, kh=3, kw=3),
]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2503_22235_gb300 import build as wm_build
    wm_build.build()
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    yield
    wm.wm_set_fused_rollout(1)


def host(t):
    torch.cuda.synchronize()
    return t.detach().to("cpu", torch.float64).numpy()


def make_ctx(s, batch=1, seed=0):
    p6, p1 = synth.processor_weights(s, seed=seed, stress=True)
    ctx = wm.wm_create_from_host(wm.make_config(s, wm.WM_PREC_BF16, batch), synth.pack_weights(p6, p1))
    return ctx, p6, p1


def blocks(s, T):
    n6, n1 = orc.greedy_schedule(T)
    return n6 * s.blocks_p6 + n1 * s.blocks_p1


@pytest.mark.parametrize("s", GRIDS, ids=lambda s: f"{s.D}x{s.H}x{s.W}-{s.kd}{s.kh}{s.kw}")
def test_whole_rollout_matches_oracle(s):
    ctx, p6, p1 = make_ctx(s)
    try:
        x = synth.latent(s, 1, seed=5)
        for T in (1, 6, 7, 13):
            xt = torch.from_numpy(x).to(CUDA)
            wm.wm_latent_rollout(ctx, xt, T)
            wm.wm_device_status()   # raises on a recorded timeout
            ref = orc.rollout(x, T, p6, p1, s)
            assert_close(host(xt), ref, 2e-2 * blocks(s, T), s.C, ("lead", T))
    finally:
        wm.wm_destroy(ctx)


def test_whole_rollout_equals_per_kernel_path_within_tolerance():
    s = SMALL3
    ctx, _, _ = make_ctx(s)
    try:
        x = torch.from_numpy(synth.latent(s, 1, seed=6)).to(CUDA)
        out = {}
        for fused in (1, 0):
            wm.wm_set_fused_rollout(fused)
            xt = x.clone()
            wm.wm_latent_rollout(ctx, xt, 13)
            out[fused] = host(xt)
    finally:
        wm.wm_set_fused_rollout(1)
        wm.wm_destroy(ctx)
    assert not np.array_equal(out[1], out[0])   # the two paths really differ
    assert_close(out[1], out[0], 2e-2 * blocks(s, 13), s.C)


def test_rollout_equals_chained_steps_and_hourly_outputs():
    s = SMALL3
    ctx, _, _ = make_ctx(s)
    try:
        x = torch.from_numpy(synth.latent(s, 1, seed=7)).to(CUDA)
        a = x.clone()
        wm.wm_latent_rollout(ctx, a, 13)
        b = x.clone()
        for which in (wm.WM_P6, wm.WM_P6, wm.WM_P1):
            wm.wm_processor_step(ctx, b, which)
        torch.cuda.synchronize()
        assert torch.equal(a, b)
        hourly = torch.empty((14,) + tuple(x.shape[1:]), device=CUDA)
        wm.wm_rollout_hourly(ctx, x, 13, hourly, 3)
        for t in (1, 5, 6, 7, 12, 13):
            alone = x.clone()
            wm.wm_latent_rollout(ctx, alone, t)
            torch.cuda.synchronize()
            assert torch.equal(hourly[t:t + 1], alone), t
    finally:
        wm.wm_destroy(ctx)


def test_batched_latents_equal_alone():
    s = synth.SMALL
    ctx, _, _ = make_ctx(s, batch=4)
    try:
        xs = [torch.from_numpy(synth.latent(s, 1, seed=10 + i)).to(CUDA) for i in range(6)]
        # uneven leads: five latents in two launches (the lead-0 latent is untouched)
        leads = [13, 1, 0, 7, 6, 24]
        batch = [x.clone() for x in xs]
        wm.wm_rollout_batch(ctx, batch, leads)
        for x, b, t in zip(xs, batch, leads):
            alone = x.clone()
            wm.wm_latent_rollout(ctx, alone, t)
            torch.cuda.synchronize()
            assert torch.equal(b, alone), t
        # an ensemble of six members: launches of four and two
        ens = torch.stack([x[0] for x in xs])
        wm.wm_latent_rollout(ctx, ens, 7)
        for i, x in enumerate(xs):
            alone = x.clone()
            wm.wm_latent_rollout(ctx, alone, 7)
            torch.cuda.synchronize()
            assert torch.equal(ens[i:i + 1], alone), i
        wm.wm_device_status()
    finally:
        wm.wm_destroy(ctx)
