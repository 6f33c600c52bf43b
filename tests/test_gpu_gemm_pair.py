"""GPU parity of the tcgen05 GEMM on CTA pairs (cta_group::2, 256 x 256 tiles).

A pair tile computes every output element with the same K-ordered sum as a
single-CTA 256-column tile, so the pair results are compared with the
single-CTA results bit for bit, and both with the float64 reference: at the
op level (plain bf16 store, ragged M, an odd count of 128-row tiles so that
the last pair's second CTA lies wholly past M, ragged K), for whole
processor steps whose four GEMMs all take pair tiles (C = 256: QKV, output
projection, FC1, FC2, in BF16 and in the FP8-MLP precision), and at the
full-size latent against the oracle at sampled tokens.
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


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2503_22235_gb300 import build as wm_build
    wm_build.build()
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    yield
    wm.wm_gemm_tile_override(wm.GEMM_TILES_TUNED)


def host(t):
    torch.cuda.synchronize()
    return t.detach().to("cpu", torch.float64).numpy()


def bf16_round(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


@pytest.mark.parametrize("M,N,K", [(1000, 256, 128), (300, 512, 136), (1, 256, 64), (4685, 768, 768),
                                   (257, 256, 3072), (20000, 3072, 768)])
def test_pair_tiles_equal_single_tiles_and_reference(M, N, K):
    rng = np.random.default_rng(M + 3 * N + 7 * K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    W = (rng.standard_normal((N, K)) / np.sqrt(K)).astype(np.float32)
    bias = (0.1 * rng.standard_normal(N)).astype(np.float32)
    Ah = torch.from_numpy(A).to(CUDA, torch.bfloat16)
    Wh = torch.from_numpy(W).to(CUDA, torch.bfloat16)
    bd = torch.from_numpy(bias).to(CUDA)
    outs = {}
    try:
        for mode in (wm.GEMM_TILES_256, wm.GEMM_TILES_PAIR):
            wm.wm_gemm_tile_override(mode)
            o = torch.full((M, N), float("nan"), device=CUDA, dtype=torch.bfloat16)
            wm.wm_op_linear(Ah, Wh, bd, o, wm.WM_PREC_BF16, wm.EPI_STORE)
            outs[mode] = host(o)
    finally:
        wm.wm_gemm_tile_override(wm.GEMM_TILES_TUNED)
    assert np.array_equal(outs[wm.GEMM_TILES_PAIR], outs[wm.GEMM_TILES_256])
    lin = orc.linear(bf16_round(A), bf16_round(W), bias)
    assert_close(outs[wm.GEMM_TILES_PAIR], lin, 4e-3, N)


@pytest.mark.parametrize("precision", ["bf16", "fp8mlp"])
def test_pair_tiles_processor_step(precision):
    s = dataclasses.replace(synth.SMALL, C=256, heads=4)
    prec = wm.WM_PREC_BF16 if precision == "bf16" else wm.WM_PREC_BF16_FP8MLP
    p6, p1 = synth.processor_weights(s, seed=0, stress=True)
    blob = synth.pack_weights(p6, p1)
    x = synth.latent(s, 2, seed=1)
    res = {}
    try:
        for mode in (wm.GEMM_TILES_256, wm.GEMM_TILES_PAIR):
            wm.wm_gemm_tile_override(mode)
            ctx = wm.wm_create_from_host(wm.make_config(s, prec, 2), blob)
            try:
                xt = torch.from_numpy(x).to(CUDA)
                wm.wm_processor_step(ctx, xt, wm.WM_P1)
                res[mode] = host(xt)
            finally:
                wm.wm_destroy(ctx)
    finally:
        wm.wm_gemm_tile_override(wm.GEMM_TILES_TUNED)
    assert np.array_equal(res[wm.GEMM_TILES_PAIR], res[wm.GEMM_TILES_256])
    if precision == "bf16":
        ref = orc.processor(x, p1, s)
        assert_close(res[wm.GEMM_TILES_PAIR], ref, 2e-2 * len(p1), s.C)
    else:
        ref = x
        for blk in p1:
            ref = orc.block_fp8mlp(ref, blk, s)
        assert_close(res[wm.GEMM_TILES_PAIR], ref, 2e-2 * len(p1), s.C)


def test_pair_tiles_full_size_block_at_sampled_tokens():
    s = dataclasses.replace(synth.FULL, blocks_p6=1, blocks_p1=1)
    p6, p1 = synth.processor_weights(s, seed=0, stress=True)
    x = synth.latent(s, 1, seed=1)
    rng = np.random.default_rng(1)
    N = s.N
    # the last rows sit in the final pair tile, whose second CTA runs past M
    toks = np.unique(np.concatenate([[0, s.W - 1, N - 257, N - 129, N - 1], rng.integers(0, N, 20)]))
    ref = orc.block_at_tokens(x, p6[0], s, toks)
    try:
        wm.wm_gemm_tile_override(wm.GEMM_TILES_PAIR)
        ctx = wm.wm_create_from_host(wm.make_config(s, wm.WM_PREC_BF16), synth.pack_weights(p6, p1))
        try:
            xt = torch.from_numpy(x).to(CUDA)
            wm.wm_block_forward(ctx, xt, wm.WM_P6, 0)
            got = host(xt).reshape(1, N, s.C)[:, toks]
        finally:
            wm.wm_destroy(ctx)
    finally:
        wm.wm_gemm_tile_override(wm.GEMM_TILES_TUNED)
    assert_close(got, ref, 2e-2, s.C)


@pytest.mark.parametrize("M,N,K", [(1000, 256, 128), (300, 512, 136), (1, 128, 64), (4685, 768, 768)])
def test_64_column_tiles_equal_wide_tiles_and_reference(M, N, K):
    """64-column tiles (more CTAs for narrow GEMMs) sum every element in the
    same K order as the wider tiles."""
    rng = np.random.default_rng(M + 5 * N + 11 * K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    W = (rng.standard_normal((N, K)) / np.sqrt(K)).astype(np.float32)
    bias = (0.1 * rng.standard_normal(N)).astype(np.float32)
    Ah = torch.from_numpy(A).to(CUDA, torch.bfloat16)
    Wh = torch.from_numpy(W).to(CUDA, torch.bfloat16)
    bd = torch.from_numpy(bias).to(CUDA)
    outs = {}
    try:
        for mode in (wm.GEMM_TILES_128, wm.GEMM_TILES_64):
            wm.wm_gemm_tile_override(mode)
            o = torch.full((M, N), float("nan"), device=CUDA, dtype=torch.bfloat16)
            wm.wm_op_linear(Ah, Wh, bd, o, wm.WM_PREC_BF16, wm.EPI_STORE)
            outs[mode] = host(o)
    finally:
        wm.wm_gemm_tile_override(wm.GEMM_TILES_TUNED)
    assert np.array_equal(outs[wm.GEMM_TILES_64], outs[wm.GEMM_TILES_128])
    assert_close(outs[wm.GEMM_TILES_64], orc.linear(bf16_round(A), bf16_round(W), bias), 4e-3, N)


@pytest.mark.parametrize("precision", ["bf16", "fp8mlp"])
def test_64_column_tiles_processor_step_small_latent(precision):
    """Every block GEMM of the small latent on 64-column tiles (four LayerNorm
    partials per row from the residual epilogues) against the oracle."""
    s = synth.SMALL
    prec = wm.WM_PREC_BF16 if precision == "bf16" else wm.WM_PREC_BF16_FP8MLP
    p6, p1 = synth.processor_weights(s, seed=0, stress=True)
    x = synth.latent(s, 2, seed=1)
    try:
        wm.wm_gemm_tile_override(wm.GEMM_TILES_64)
        wm.wm_set_fused_rollout(0)   # the step through the per-kernel GEMMs
        ctx = wm.wm_create_from_host(wm.make_config(s, prec, 2), synth.pack_weights(p6, p1))
        try:
            xt = torch.from_numpy(x).to(CUDA)
            wm.wm_processor_step(ctx, xt, wm.WM_P1)
            got = host(xt)
        finally:
            wm.wm_destroy(ctx)
    finally:
        wm.wm_gemm_tile_override(wm.GEMM_TILES_TUNED)
        wm.wm_set_fused_rollout(1)
    if precision == "bf16":
        ref = orc.processor(x, p1, s)
    else:
        ref = x
        for blk in p1:
            ref = orc.block_fp8mlp(ref, blk, s)
    assert_close(got, ref, 2e-2 * len(p1), s.C)
