"""The debug build (libwm_debug.so: the same sources with WM_DEBUG_CHECKS=1,
i.e. device-side checks of the attention windows, slab geometry and tail
tiles that record WM_ERR_BOUNDS and skip the access) on the hot path: no
check fails on any attention family and kernel kind, on the FP32 attention,
on blocks at the small and the full-size latent, or on whole-rollout
launches (two latents, 7 h, on the small latent and on a 2 x 8 x 32 grid
with a 1 x 5 x 3 window). Every attention output (each family and kernel
kind named explicitly, and the FP32 kernel), the FP32 block and the
whole-rollout results equal the release build's bit for bit (the checks
change no arithmetic); the BF16 blocks, whose attention family the
autotuner picks per process by timing, agree within 2e-3.

The debug library runs in a child process (WM_LIBRARY=debug makes the
binding load it); this process runs the same cases on the release library.
"""
import dataclasses
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

# (B, D, H, W, C, heads, kd, kh, kw, periodic): ragged tiles, clamped and
# periodic longitude, the full-size window, dh 32 / 48 / 64
CASES = [
    (2, 4, 24, 48, 128, 4, 3, 5, 5, True),
    (1, 9, 20, 36, 96, 2, 5, 7, 7, True),
    (1, 9, 13, 29, 96, 2, 5, 7, 7, False),
    (1, 2, 11, 19, 64, 4, 1, 5, 3, True),
    (1, 5, 9, 23, 128, 2, 3, 9, 9, True),
]


def run_cases(out_path):
    """Every case through the library the binding loaded; outputs to out_path (.npz)."""
    import paper_2503_22235_gb300 as wm
    import synth
    dev = torch.device("cuda")
    variants = [wm.WM_NA_TCGEN05] + [fam | kind
                                                   for fam in (wm.WM_NA_QK_CHUNK8, wm.WM_NA_QK_CHUNK4, wm.WM_NA_KQ)
                                                   for kind in (wm.WM_NA_PER_TILE, wm.WM_NA_PERSISTENT)]
    res = {}
    for ci, (B, D, H, W, C, heads, kd, kh, kw, per) in enumerate(CASES):
        rng = np.random.default_rng(ci)
        qkv = torch.from_numpy((rng.standard_normal((B * D * H * W, 3 * C)) * 1.2).astype(np.float32)).to(dev)
        for v in variants:
            o = torch.empty(B * D * H * W, C, device=dev, dtype=torch.bfloat16)
            try:
                wm.wm_op_neighborhood_attention(qkv.to(torch.bfloat16), o, B, D, H, W, C, heads, kd, kh, kw, int(per),
                                                wm.WM_PREC_BF16, v)
            except wm.WmError as e:   # a variant this shape does not support: the same in both builds
                res[f"exact_na{ci}_v{v}"] = np.array([float(e.status)])
                continue
            res[f"exact_na{ci}_v{v}"] = o.float().cpu().numpy()
        o32 = torch.empty(B * D * H * W, C, device=dev)
        wm.wm_op_neighborhood_attention(qkv, o32, B, D, H, W, C, heads, kd, kh, kw, int(per), wm.WM_PREC_FP32,
                                        wm.WM_NA_AUTO)
        res[f"exact_na{ci}_fp32"] = o32.cpu().numpy()
    wm.wm_gemm_tile_override(wm.GEMM_TILES_256)   # the same GEMM tiles (and LayerNorm partials) in both builds
    for name, shape in (("small", synth.SMALL), ("full", dataclasses.replace(synth.FULL, blocks_p6=1, blocks_p1=1))):
        p6, p1 = synth.processor_weights(shape, seed=0, stress=True)
        ctx = wm.wm_create_from_host(wm.make_config(shape, wm.WM_PREC_BF16), synth.pack_weights(p6, p1))
        try:
            precs = (wm.WM_PREC_BF16, wm.WM_PREC_FP32) if name == "small" else (wm.WM_PREC_BF16,)
            for prec in precs:
                wm.wm_set_precision(ctx, prec)
                x = torch.from_numpy(synth.latent(shape, 1, seed=1)).to(dev)
                wm.wm_block_forward(ctx, x, wm.WM_P6, 0)
                kind = "exact" if prec == wm.WM_PREC_FP32 else "close"
                res[f"{kind}_block_{name}_{prec}"] = x.cpu().numpy()
        finally:
            wm.wm_destroy(ctx)
    wm.wm_gemm_tile_override(wm.GEMM_TILES_TUNED)
    grids = (dataclasses.replace(synth.SMALL, blocks_p6=2, blocks_p1=1),
             dataclasses.replace(synth.SMALL, D=2, H=8, W=32, kd=1, kh=5, kw=3, blocks_p6=2, blocks_p1=1))
    for gi, shape in enumerate(grids):
        p6, p1 = synth.processor_weights(shape, seed=0, stress=True)
        ctx = wm.wm_create_from_host(wm.make_config(shape, wm.WM_PREC_BF16, 2), synth.pack_weights(p6, p1))
        try:
            x = torch.from_numpy(synth.latent(shape, 2, seed=2)).to(dev)
            wm.wm_latent_rollout(ctx, x, 7)          # one whole-rollout launch of two latents
            res[f"exact_rollout{gi}"] = x.cpu().numpy()
        finally:
            wm.wm_destroy(ctx)
    wm.wm_device_status()   # raises WmError(WM_ERR_BOUNDS) if a debug check failed
    np.savez(out_path, **res)


@pytest.fixture(scope="module")
def debug_outputs(tmp_path_factory):
    from paper_2503_22235_gb300 import build as wm_build
    wm_build.build()
    wm_build.build(debug=True)
    out = str(tmp_path_factory.mktemp("debug") / "debug.npz")
    env = dict(os.environ, WM_LIBRARY="debug", PYTHONPATH=os.pathsep.join([ROOT, HERE]))
    r = subprocess.run([sys.executable, "-c", f"import test_gpu_debug_build as t; t.run_cases({out!r})"],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    return np.load(out)


def test_debug_build_checks_pass_and_results_equal_release(debug_outputs, tmp_path):
    import paper_2503_22235_gb300 as wm
    assert wm.LIB_PATH.endswith("libwm.so")
    out = str(tmp_path / "release.npz")
    run_cases(out)
    rel = np.load(out)
    assert sorted(rel.files) == sorted(debug_outputs.files)
    for k in rel.files:
        a, b = rel[k], debug_outputs[k]
        if k.startswith("exact_"):
            assert np.array_equal(a, b, equal_nan=True), k
        else:
            assert np.isfinite(b).all(), k
            assert np.linalg.norm(a - b) <= 2e-3 * np.linalg.norm(a), k
