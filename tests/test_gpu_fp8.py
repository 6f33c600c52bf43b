"""FP8 (E4M3) MLP precision: the e4m3 GEMM and LayerNorm kernels against the
oracle on the same codes, the static scales against the oracle's
definition, and the FP8-MLP block against the oracle's E4M3-emulated block.

Tolerances: the e4m3 GEMM with FP32 output multiplies exact E4M3 values, so
only FP32 accumulation order differs (<= 1e-5 relative L2). Quantised
outputs (LayerNorm, GELU) may differ by one E4M3 step where the FP32 and
FP64 pre-rounding values straddle a rounding boundary: >= 99 % of codes must
match and every mismatch must be one step. The FP8-MLP block is compared with
the oracle's emulated block at the BF16 per-block tolerance (2e-2).
"""
import dataclasses

import numpy as np
import pytest
import torch

import paper_2503_22235_gb300 as wm
import synth
from oracle import wm_oracle as orc

pytestmark = pytest.mark.gpu
CUDA = torch.device("cuda")
DECODE = np.array([orc.e4m3_decode(c) for c in range(256)])


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2503_22235_gb300 import build as wm_build
    wm_build.build()


def _codes(rng, shape):
    c = rng.integers(0, 256, shape).astype(np.uint8)
    c[(c & 0x7F) == 0x7F] = 0x38          # no NaN codes
    return c


def _encode(v):
    """E4M3 codes of already-representable values (oracle rounding, then table lookup)."""
    r = orc.e4m3_round(v)
    mag = np.searchsorted(DECODE[:0x7F], np.abs(r))
    return (mag | np.where(r < 0, 0x80, 0)).astype(np.uint8)


def _step_apart(a_codes, b_codes):
    """True where two codes are equal or adjacent E4M3 values."""
    va, vb = DECODE[a_codes], DECODE[b_codes]
    ia = np.searchsorted(DECODE[:0x7F], np.abs(va)) * np.sign(va)
    ib = np.searchsorted(DECODE[:0x7F], np.abs(vb)) * np.sign(vb)
    return np.abs(ia - ib) <= 1


@pytest.mark.parametrize("M,N,K", [(1000, 512, 128), (333, 768, 3072), (4608, 128, 512)])
def test_e4m3_linear_matches_oracle_on_the_same_codes(M, N, K):
    rng = np.random.default_rng(M + N + K)
    A, W = _codes(rng, (M, K)), _codes(rng, (N, K))
    alpha = 1.0 / 64
    bias = (0.1 * rng.standard_normal(N)).astype(np.float32)
    lin = orc.linear(DECODE[A], DECODE[W], np.zeros(N)) * alpha + bias
    At, Wt = torch.from_numpy(A).cuda(), torch.from_numpy(W).cuda()
    out = torch.empty(M, N, device=CUDA)
    wm.wm_op_linear_e4m3(At, Wt, alpha, torch.from_numpy(bias).cuda(), out, 1.0, wm.EPI_STORE_F32)
    torch.cuda.synchronize()
    assert orc.rel_l2(out.cpu().numpy(), lin) < 1e-5
    x0 = rng.standard_normal((M, N)).astype(np.float32)
    xr = torch.from_numpy(x0).cuda()
    wm.wm_op_linear_e4m3(At, Wt, alpha, torch.from_numpy(bias).cuda(), xr, 1.0, wm.EPI_RESID_F32)
    torch.cuda.synchronize()
    assert orc.rel_l2(xr.cpu().numpy(), x0 + lin) < 1e-5
    inv = 448.0 / np.abs(orc.gelu(lin)).max()
    hq = torch.empty(M, N, device=CUDA, dtype=torch.uint8)
    wm.wm_op_linear_e4m3(At, Wt, alpha, torch.from_numpy(bias).cuda(), hq, inv, wm.EPI_GELU_F8)
    torch.cuda.synchronize()
    got = hq.cpu().numpy()
    ref = _encode(orc.gelu(lin) * inv)
    assert np.mean(DECODE[got] == DECODE[ref]) > 0.99   # +0 and -0 compare equal
    assert np.all(_step_apart(got, ref))


def test_e4m3_layernorm_matches_oracle_codes():
    rng = np.random.default_rng(1)
    M, C = 777, 768
    x = (rng.standard_normal((M, C)) * 2 + 0.5).astype(np.float32)
    g = (1 + 0.1 * rng.standard_normal(C)).astype(np.float32)
    b = (0.1 * rng.standard_normal(C)).astype(np.float32)
    inv = 448.0 / (np.abs(g).max() * np.sqrt(C - 1) + np.abs(b).max())
    out = torch.empty(M, C, device=CUDA, dtype=torch.uint8)
    wm.wm_op_layernorm_e4m3(torch.from_numpy(x).cuda(), torch.from_numpy(g).cuda(), torch.from_numpy(b).cuda(),
                            out, 1e-5, inv)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    ref = _encode(orc.layer_norm(x, g, b, 1e-5) * inv)
    assert np.mean(DECODE[got] == DECODE[ref]) > 0.99   # +0 and -0 compare equal
    assert np.all(_step_apart(got, ref))


def _ctx(shape, stress=True, max_batch=1):
    p6, p1 = synth.processor_weights(shape, seed=0, stress=stress)
    ctx = wm.wm_create_from_host(wm.make_config(shape, wm.WM_PREC_BF16_FP8MLP, max_batch), synth.pack_weights(p6, p1))
    return ctx, p6, p1


def test_fp8_scales_match_oracle_definition():
    s = dataclasses.replace(synth.SMALL, blocks_p6=2, blocks_p1=1)
    ctx, p6, p1 = _ctx(s)
    try:
        for which, blocks in ((wm.WM_P6, p6), (wm.WM_P1, p1)):
            for i, w in enumerate(blocks):
                got = wm.wm_fp8_scales(ctx, which, i)
                ref = orc.fp8_mlp_scales(w, s.C)
                assert np.allclose(got, ref, rtol=1e-6, atol=0), (which, i, got, ref)
    finally:
        wm.wm_destroy(ctx)


@pytest.mark.parametrize("stress", [False, True])
def test_fp8_mlp_block_against_emulated_oracle(stress):
    s = dataclasses.replace(synth.SMALL, blocks_p6=1, blocks_p1=1)
    ctx, p6, _ = _ctx(s, stress=stress)
    try:
        x = synth.latent(s, 1, seed=1)
        xt = torch.from_numpy(x).cuda()
        wm.wm_block_forward(ctx, xt, wm.WM_P6, 0)
        torch.cuda.synchronize()
        got = xt.cpu().numpy()
        err_emul = orc.rel_l2(got, orc.block_fp8mlp(x, p6[0], s))
        err_exact = orc.rel_l2(got, orc.block(x, p6[0], s))
        print(f"fp8-mlp block: vs emulated {err_emul:.2e}, vs exact {err_exact:.2e}")
        assert err_emul <= 2e-2
        assert err_exact <= 5e-2
    finally:
        wm.wm_destroy(ctx)


def test_fp8_batched_rollouts_equal_single_rollouts():
    s = dataclasses.replace(synth.SMALL, blocks_p6=2, blocks_p1=1)
    ctx, _, _ = _ctx(s, max_batch=4)
    try:
        leads = [1, 6, 7, 13]
        xs = [synth.latent(s, 1, seed=20 + i) for i in range(len(leads))]
        batch = [torch.from_numpy(x).cuda() for x in xs]
        wm.wm_rollout_batch(ctx, batch, leads)
        for x, t, got in zip(xs, leads, batch):
            alone = torch.from_numpy(x).cuda()
            wm.wm_latent_rollout(ctx, alone, t)
            torch.cuda.synchronize()
            assert torch.equal(got, alone), t
    finally:
        wm.wm_destroy(ctx)
