"""GPU parity of the fused small-latent MLP (C = 128: FC1 with LayerNorm 2
folded, GELU, FC2 and the residual in one kernel, the hidden activations in
shared memory). It computes every element as the two separate GEMMs do, so
blocks, processor steps and captured rollouts equal the unfused path bit
for bit (wm_set_fused_mlp switches between them), on the small latent
and on a grid whose token count leaves a ragged last tile; one block is also
checked against the FP64 oracle.
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
RAGGED = dataclasses.replace(synth.SMALL, D=3, H=20, W=30)   # 1800 tokens: 14 full tiles and a tail of 8 rows


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2503_22235_gb300 import build as wm_build
    wm_build.build()
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    yield
    wm.wm_set_fused_mlp(0)


def host(t):
    torch.cuda.synchronize()
    return t.detach().to("cpu", torch.float64).numpy()


def _run(shape, batch, fn, fused, stress=True):
    p6, p1 = synth.processor_weights(shape, seed=0, stress=stress)
    wm.wm_set_fused_mlp(fused)
    wm.wm_set_fused_rollout(0)   # processor steps and rollouts through the per-kernel path
    try:
        ctx = wm.wm_create_from_host(wm.make_config(shape, wm.WM_PREC_BF16, batch), synth.pack_weights(p6, p1))
        try:
            x = torch.from_numpy(synth.latent(shape, batch, seed=3)).to(CUDA)
            fn(ctx, x)
            return host(x), p6, p1
        finally:
            wm.wm_destroy(ctx)
    finally:
        wm.wm_set_fused_mlp(0)
        wm.wm_set_fused_rollout(1)


@pytest.mark.parametrize("shape,batch", [(synth.SMALL, 1), (synth.SMALL, 3), (RAGGED, 1)])
def test_fused_mlp_block_equals_two_gemms_and_oracle(shape, batch):
    blk = lambda ctx, x: wm.wm_block_forward(ctx, x, wm.WM_P6, 0)
    fused, p6, _ = _run(shape, batch, blk, 1)
    plain, _, _ = _run(shape, batch, blk, 0)
    assert np.array_equal(fused, plain)
    x = synth.latent(shape, batch, seed=3)
    assert_close(fused, orc.block(x, p6[0], shape), 2e-2, shape.C)


@pytest.mark.parametrize("shape", [synth.SMALL, RAGGED])
def test_fused_mlp_processor_steps_and_rollout_equal_two_gemms(shape):
    def steps(ctx, x):
        wm.wm_processor_step(ctx, x, wm.WM_P6)
        wm.wm_processor_step(ctx, x, wm.WM_P1)
        wm.wm_latent_rollout(ctx, x, 13)   # captured graph: 2 six-hour + 1 one-hour steps
    fused, _, _ = _run(shape, 2, steps, 1)
    plain, _, _ = _run(shape, 2, steps, 0)
    assert np.isfinite(fused).all()
    assert np.array_equal(fused, plain)
