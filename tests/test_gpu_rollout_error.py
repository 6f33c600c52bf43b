"""Latent rollout error against the FP64 oracle, step by step.

The default lead time is 49 h (eight six-hour steps and one one-hour step, 68
blocks) so the oracle finishes in about a minute; set WM_ROLLOUT_ERROR_HOURS=337
for the full 14-day-plus-one-hour rollout (452 blocks). With
WM_ERROR_CURVE_OUT=<path> the per-step curve is written there as JSON.
"""
import json
import os

import numpy as np
import pytest
import torch

import paper_2503_22235_gb300 as wm
import synth
from oracle import wm_oracle as orc

pytestmark = pytest.mark.gpu


def test_rollout_error_curve_against_oracle():
    from paper_2503_22235_gb300 import build as wm_build
    wm_build.build()
    T = int(os.environ.get("WM_ROLLOUT_ERROR_HOURS", "49"))
    s = synth.SMALL
    p6, p1 = synth.processor_weights(s, seed=0)
    x = synth.latent(s, 1, seed=1)
    ref_steps = []
    orc.rollout(x, T, p6, p1, s, per_step=ref_steps)
    n6, n1 = orc.greedy_schedule(T)
    ctx = wm.wm_create_from_host(wm.make_config(s, wm.WM_PREC_BF16), synth.pack_weights(p6, p1))
    curves = {}
    try:
        for prec, name in ((wm.WM_PREC_FP32, "fp32"), (wm.WM_PREC_BF16, "bf16"),
                           (wm.WM_PREC_BF16_FP8MLP, "fp8mlp")):
            wm.wm_set_precision(ctx, prec)
            xt = torch.from_numpy(x).cuda()
            errs = []
            for i in range(n6 + n1):
                wm.wm_processor_step(ctx, xt, wm.WM_P6 if i < n6 else wm.WM_P1)
                ref = torch.from_numpy(ref_steps[i].astype(np.float32)).cuda()
                errs.append(wm.wm_rel_l2(xt, ref))
            curves[name] = errs
            # the graph-captured rollout equals the chained steps
            xg = torch.from_numpy(x).cuda()
            wm.wm_latent_rollout(ctx, xg, T)
            torch.cuda.synchronize()
            assert torch.equal(xg, xt)
    finally:
        wm.wm_destroy(ctx)
    out = os.environ.get("WM_ERROR_CURVE_OUT")
    if out:
        with open(out, "w") as f:
            json.dump({"lead_hours": T, "steps": ["P6"] * n6 + ["P1"] * n1, "rel_l2": curves}, f)
    print("rollout rel-L2 per step:", {k: [f"{e:.2e}" for e in v] for k, v in curves.items()})
    # first step: 8 blocks, each within the per-block tolerance
    assert curves["fp32"][0] <= 8e-5
    assert curves["bf16"][0] <= 8 * 2e-2
    assert all(all(np.isfinite(v)) for v in curves.values())
    assert curves["fp32"][-1] < curves["bf16"][-1] < curves["fp8mlp"][-1]
