"""GPU parity: every hot-path kernel and the composed block / processor /
rollout, called through the C ABI, against the FP64 oracle on the same seeded
inputs.

Tolerances (relative L2 unless noted; every oracle comparison also bounds
each token's largest channel error by 8x the tolerance times the token's
reference RMS, parity_util.assert_close):
  * FP32 plain path: <= 1e-5 per block (strict FP32 FMA, no TF32).
  * BF16 path:       <= 2e-2 per block. Linear layers are checked on
    bf16-rounded operands, where only FP32 accumulation order differs
    (<= 1e-5); attention on bf16-rounded q, k, v, where the bf16 rounding of
    the softmax weights adds ~2^-9 per weight (<= 1e-2).
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


def dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(CUDA, dtype)


def bf16_round(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def host(t):
    torch.cuda.synchronize()
    return t.detach().to("cpu", torch.float64).numpy()


def rel(a, b):
    return orc.rel_l2(a, b)


@pytest.fixture(scope="session", autouse=True)
def built():
    from paper_2503_22235_gb300 import build as wm_build
    wm_build.build()
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"


def make_ctx(shape, precision, seed=0, stress=False, max_batch=1):
    p6, p1 = synth.processor_weights(shape, seed=seed, stress=stress)
    blob = synth.pack_weights(p6, p1)
    ctx = wm.wm_create_from_host(wm.make_config(shape, precision, max_batch), blob)
    return ctx, p6, p1


# ------------------------------------------------------------- LayerNorm ---

@pytest.mark.parametrize("C", [128, 768, 40])
def test_layernorm_fp32_and_bf16(C):
    rng = np.random.default_rng(C)
    M = 257
    x = (rng.standard_normal((M, C)) * 3 + 1).astype(np.float32)
    g = (1 + 0.1 * rng.standard_normal(C)).astype(np.float32)
    b = (0.1 * rng.standard_normal(C)).astype(np.float32)
    ref = orc.layer_norm(x, g, b, 1e-5)
    out = torch.empty(M, C, device=CUDA)
    wm.wm_op_layernorm(dev(x), dev(g), dev(b), out, 1e-5)
    assert_close(host(out), ref, 1e-6, C)
    outh = torch.empty(M, C, device=CUDA, dtype=torch.bfloat16)
    wm.wm_op_layernorm(dev(x), dev(g), dev(b), outh, 1e-5)
    assert_close(host(outh), ref, 4e-3, C)


# ---------------------------------------------------------------- linear ---

@pytest.mark.parametrize("M,N,K", [(300, 384, 128), (1000, 512, 128), (77, 130, 24)])
@pytest.mark.parametrize("epi", [wm.EPI_STORE_F32, wm.EPI_GELU, wm.EPI_RESID_F32])
def test_linear_fp32(M, N, K, epi):
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    W = (rng.standard_normal((N, K)) / np.sqrt(K)).astype(np.float32)
    bias = (0.1 * rng.standard_normal(N)).astype(np.float32)
    x0 = rng.standard_normal((M, N)).astype(np.float32)
    out = dev(x0) if epi == wm.EPI_RESID_F32 else torch.empty(M, N, device=CUDA)
    wm.wm_op_linear(dev(A), dev(W), dev(bias), out, wm.WM_PREC_FP32, epi)
    lin = orc.linear(A, W, bias)
    ref = {wm.EPI_STORE_F32: lin, wm.EPI_GELU: orc.gelu(lin), wm.EPI_RESID_F32: x0 + lin}[epi]
    assert_close(host(out), ref, 1e-6, N)


@pytest.mark.parametrize("M,N,K", [(1000, 384, 128), (4608, 512, 128), (333, 256, 3072), (20000, 768, 768),
                                   (130, 136, 72), (4608, 128, 512)])
def test_linear_bf16_tcgen05(M, N, K):
    rng = np.random.default_rng(M * 7 + N + K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    W = (rng.standard_normal((N, K)) / np.sqrt(K)).astype(np.float32)
    bias = (0.1 * rng.standard_normal(N)).astype(np.float32)
    Ah, Wh = dev(A, torch.bfloat16), dev(W, torch.bfloat16)
    lin = orc.linear(bf16_round(A), bf16_round(W), bias)
    # fp32 output: only the accumulation order differs from the float64 reference
    out = torch.empty(M, N, device=CUDA)
    wm.wm_op_linear(Ah, Wh, dev(bias), out, wm.WM_PREC_BF16, wm.EPI_STORE_F32)
    assert_close(host(out), lin, 1e-5, N)
    # bf16 output, GELU epilogue, residual epilogue
    outh = torch.empty(M, N, device=CUDA, dtype=torch.bfloat16)
    wm.wm_op_linear(Ah, Wh, dev(bias), outh, wm.WM_PREC_BF16, wm.EPI_STORE)
    assert_close(host(outh), lin, 4e-3, N)
    wm.wm_op_linear(Ah, Wh, dev(bias), outh, wm.WM_PREC_BF16, wm.EPI_GELU)
    g_got = host(outh)
    assert_close(g_got, orc.gelu(lin), 4e-3, N)
    # per element against GELU of the GPU's own fp32 GEMM output: only the bf16
    # rounding (<= 2^-8 relative) and the epilogue's erf approximation
    # (A&S 7.1.26, |erf error| <= 1.5e-7, so |GELU error| <= 1e-7 (1 + |z|)) remain
    z32 = host(out)
    g32 = orc.gelu(z32)
    assert np.all(np.abs(g_got - g32) <= 2.0 ** -8 * np.abs(g32) + 1e-6 * (1 + np.abs(z32)))
    x0 = rng.standard_normal((M, N)).astype(np.float32)
    xr = dev(x0)
    wm.wm_op_linear(Ah, Wh, dev(bias), xr, wm.WM_PREC_BF16, wm.EPI_RESID_F32)
    assert_close(host(xr), x0 + lin, 1e-5, N)


# ------------------------------------------------- neighborhood attention ---

NA_CASES = [
    # (B, D, H, W, C, heads, kd, kh, kw, periodic)
    (1, 3, 5, 7, 32, 2, 3, 3, 5, True),
    (1, 3, 5, 7, 32, 2, 3, 3, 5, False),
    (2, 4, 24, 48, 128, 4, 3, 5, 5, True),       # small latent: dh 32, window 3x5x5
    (1, 9, 20, 36, 96, 2, 5, 7, 7, True),        # full-size window and dh 48 on a reduced grid
    (1, 9, 13, 29, 96, 2, 5, 7, 7, False),       # ragged tiles, clamped longitude
    (1, 2, 11, 19, 64, 4, 1, 5, 3, True),        # dh 16
    (1, 5, 9, 23, 128, 2, 3, 9, 9, True),        # dh 64
    (1, 3, 5, 7, 32, 2, 3, 5, 7, True),          # window = whole grid
]


def _na_inputs(B, D, H, W, C, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((B, D * H * W, 3 * C)) * 1.2).astype(np.float32)


@pytest.mark.parametrize("case", NA_CASES)
def test_neighborhood_attention_fp32(case):
    B, D, H, W, C, heads, kd, kh, kw, per = case
    qkv = _na_inputs(B, D, H, W, C, 1)
    out = torch.empty(B * D * H * W, C, device=CUDA)
    wm.wm_op_neighborhood_attention(dev(qkv), out, B, D, H, W, C, heads, kd, kh, kw, per, wm.WM_PREC_FP32)
    nbr = orc.neighbor_index(D, H, W, kd, kh, kw, per)
    ref = orc.neighborhood_attention(qkv[..., :C], qkv[..., C:2 * C], qkv[..., 2 * C:], heads, nbr)
    assert_close(host(out).reshape(B, -1, C), ref, 1e-6, C // heads, case)


_NA_REF = {}


def _na_bf16_ref(case):
    """Oracle attention on the bf16-rounded inputs of `case` (cached per case)."""
    if case not in _NA_REF:
        B, D, H, W, C, heads, kd, kh, kw, per = case
        q = bf16_round(_na_inputs(B, D, H, W, C, 2))
        nbr = orc.neighbor_index(D, H, W, kd, kh, kw, per)
        _NA_REF[case] = orc.neighborhood_attention(q[..., :C], q[..., C:2 * C], q[..., 2 * C:], heads, nbr)
    return _NA_REF[case]


def _na_bf16_run(case, variant):
    B, D, H, W, C, heads, kd, kh, kw, per = case
    qkv = _na_inputs(B, D, H, W, C, 2)
    out = torch.empty(B * D * H * W, C, device=CUDA, dtype=torch.bfloat16)
    wm.wm_op_neighborhood_attention(dev(qkv, torch.bfloat16), out, B, D, H, W, C, heads, kd, kh, kw, per,
                                    wm.WM_PREC_BF16, variant)
    torch.cuda.synchronize()
    return out


NA_VARIANTS = [wm.WM_NA_AUTO] + [fam | kind for fam in (wm.WM_NA_QK_CHUNK8, wm.WM_NA_QK_CHUNK4, wm.WM_NA_KQ)
                                 for kind in (wm.WM_NA_PER_TILE, wm.WM_NA_PERSISTENT)] + [wm.WM_NA_TCGEN05]


def _tc_supported(case):
    """Shapes the tcgen05 kernel takes (include/wm.h, WM_NA_TCGEN05)."""
    B, D, H, W, C, heads, kd, kh, kw, per = case
    dh = C // heads
    win = (kh, kw)
    if not ((dh in (32, 48) and win in ((5, 5), (7, 7))) or (dh == 64 and win == (5, 5))):
        return False
    return min(16 + kh - 1, H) >= kh + 3 and (per or W >= kw + 7)


@pytest.mark.parametrize("variant", NA_VARIANTS)
@pytest.mark.parametrize("case", NA_CASES)
def test_neighborhood_attention_bf16(case, variant):
    B, C = case[0], case[4]
    if variant == wm.WM_NA_TCGEN05 and not _tc_supported(case):
        with pytest.raises(wm.WmError) as e:
            _na_bf16_run(case, variant)
        assert e.value.status == wm.WM_ERR_INVALID_ARG
        return
    out = _na_bf16_run(case, variant)
    # tokens = (query, head) pairs: each head's output is its own softmax average
    assert_close(host(out).reshape(B, -1, C), _na_bf16_ref(case), 1e-2, C // case[5], (case, variant))


@pytest.mark.parametrize("fam", [wm.WM_NA_QK_CHUNK8, wm.WM_NA_QK_CHUNK4, wm.WM_NA_KQ])
@pytest.mark.parametrize("case", NA_CASES[2:5])
def test_neighborhood_attention_kernel_kind_does_not_change_results(case, fam):
    """Within one arithmetic family the per-tile and the persistent kernel,
    with any CTA shape, produce bit-identical outputs."""
    a = _na_bf16_run(case, fam | wm.WM_NA_PER_TILE)
    b = _na_bf16_run(case, fam | wm.WM_NA_PERSISTENT)
    assert torch.equal(a, b)


@pytest.mark.parametrize("case", [c for c in NA_CASES if _tc_supported(c)])
def test_tcgen05_attention_is_batch_independent(case):
    """A query's result depends only on its own position: the batch-2 launch
    equals two batch-1 launches bit for bit (the batched serving and ensemble
    paths rely on it)."""
    B, D, H, W, C, heads, kd, kh, kw, per = case
    qkv = torch.from_numpy(_na_inputs(2, D, H, W, C, 9)).to(CUDA, torch.bfloat16)
    both = torch.empty(2 * D * H * W, C, device=CUDA, dtype=torch.bfloat16)
    wm.wm_op_neighborhood_attention(qkv, both, 2, D, H, W, C, heads, kd, kh, kw, per, wm.WM_PREC_BF16,
                                    wm.WM_NA_TCGEN05)
    for b in range(2):
        one = torch.empty(D * H * W, C, device=CUDA, dtype=torch.bfloat16)
        wm.wm_op_neighborhood_attention(qkv[b].contiguous(), one, 1, D, H, W, C, heads, kd, kh, kw, per,
                                        wm.WM_PREC_BF16, wm.WM_NA_TCGEN05)
        torch.cuda.synchronize()
        assert torch.equal(one, both[b * D * H * W:(b + 1) * D * H * W]), b


def test_neighborhood_attention_rejects_bad_variants():
    case = NA_CASES[0]
    for v in (-1, 16, wm.WM_NA_PER_TILE, wm.WM_NA_KQ | 12):
        with pytest.raises(wm.WmError):
            _na_bf16_run(case, v)
    B, D, H, W, C, heads, kd, kh, kw, per = case
    out = torch.empty(B * D * H * W, C, device=CUDA)
    with pytest.raises(wm.WmError):
        wm.wm_op_neighborhood_attention(dev(_na_inputs(B, D, H, W, C, 1)), out, B, D, H, W, C, heads, kd, kh, kw,
                                        per, wm.WM_PREC_FP32, wm.WM_NA_KQ)


# ------------------------------------------------------- block / processor ---

@pytest.mark.parametrize("stress", [False, True])
def test_block_fp32_small_latent(stress):
    s = synth.SMALL
    ctx, p6, p1 = make_ctx(s, wm.WM_PREC_FP32, stress=stress)
    try:
        x = synth.latent(s, 1, seed=1)
        for which, blocks in ((wm.WM_P6, p6), (wm.WM_P1, p1)):
            for b in (0, len(blocks) - 1):
                xt = dev(x)
                wm.wm_block_forward(ctx, xt, which, b)
                assert_close(host(xt), orc.block(x, blocks[b], s), 1e-5, s.C, (which, b))
    finally:
        wm.wm_destroy(ctx)


@pytest.mark.parametrize("stress", [False, True])
def test_block_bf16_small_latent(stress):
    s = synth.SMALL
    ctx, p6, p1 = make_ctx(s, wm.WM_PREC_BF16, stress=stress)
    try:
        x = synth.latent(s, 2, seed=1)
        xt = dev(x)
        wm.wm_block_forward(ctx, xt, wm.WM_P6, 0)
        assert_close(host(xt), orc.block(x, p6[0], s), 2e-2, s.C)
    finally:
        wm.wm_destroy(ctx)


@pytest.mark.parametrize("fused", [1, 0])
def test_processor_steps_bf16_and_fp32_small_latent(fused):
    """P6 then P1 on the small latent against the oracle; in BF16 through the
    whole-rollout kernel (fused = 1) and through one launch per kernel (0)."""
    s = synth.SMALL
    ctx, p6, p1 = make_ctx(s, wm.WM_PREC_BF16, stress=True)
    wm.wm_set_fused_rollout(fused)
    try:
        x = synth.latent(s, 1, seed=3)
        ref6 = orc.processor(x, p6, s)
        ref61 = orc.processor(ref6, p1, s)
        for prec, tol in ((wm.WM_PREC_FP32, 1e-5 * 12), (wm.WM_PREC_BF16, 2e-2 * 12)):
            wm.wm_set_precision(ctx, prec)
            xt = dev(x)
            wm.wm_processor_step(ctx, xt, wm.WM_P6)
            assert_close(host(xt), ref6, tol, s.C, (prec, "P6"))
            wm.wm_processor_step(ctx, xt, wm.WM_P1)
            assert_close(host(xt), ref61, tol, s.C, (prec, "P6 then P1"))
    finally:
        wm.wm_set_fused_rollout(1)
        wm.wm_destroy(ctx)


# --------------------------------------------------------------- rollout ---

def test_rollout_equals_chained_processor_steps_and_oracle():
    s = synth.Shape(D=4, H=24, W=48, C=128, heads=4, kd=3, kh=5, kw=5, blocks_p6=3, blocks_p1=2)
    ctx, p6, p1 = make_ctx(s, wm.WM_PREC_BF16, stress=True)
    try:
        x = synth.latent(s, 1, seed=4)
        for prec in (wm.WM_PREC_BF16, wm.WM_PREC_FP32):
            wm.wm_set_precision(ctx, prec)
            a = dev(x)
            wm.wm_latent_rollout(ctx, a, 13)            # graph: 2 six-hour + 1 one-hour step
            b = dev(x)
            for which in (wm.WM_P6, wm.WM_P6, wm.WM_P1):
                wm.wm_processor_step(ctx, b, which)
            torch.cuda.synchronize()
            assert torch.equal(a, b)
            a2 = dev(x)
            wm.wm_latent_rollout(ctx, a2, 13)           # cached graph replay
            assert torch.equal(a, a2)
        ref = orc.rollout(x, 13, p6, p1, s)
        wm.wm_set_precision(ctx, wm.WM_PREC_FP32)
        c = dev(x)
        wm.wm_latent_rollout(ctx, c, 13)
        assert_close(host(c), ref, 1e-5 * 8, s.C)
        z = dev(x)
        wm.wm_latent_rollout(ctx, z, 0)
        assert torch.equal(z, dev(x))
        with pytest.raises(wm.WmError):
            wm.wm_latent_rollout(ctx, z, -1)
    finally:
        wm.wm_destroy(ctx)


def test_forecast_from_host_buffers_equals_device_rollout():
    s = synth.Shape(D=4, H=24, W=48, C=128, heads=4, kd=3, kh=5, kw=5, blocks_p6=2, blocks_p1=1)
    ctx, _, _ = make_ctx(s, wm.WM_PREC_BF16)
    try:
        x = synth.latent(s, 2, seed=5)
        hin = torch.from_numpy(x).pin_memory()
        hout = torch.empty_like(hin).pin_memory()
        wm.wm_forecast_host(ctx, hin, hout, 7)
        d = dev(x)
        wm.wm_latent_rollout(ctx, d, 7)
        assert torch.equal(hout, d.cpu())
    finally:
        wm.wm_destroy(ctx)


def test_forecast_stream_from_host_buffers_equals_single_calls():
    s = synth.Shape(D=4, H=24, W=48, C=128, heads=4, kd=3, kh=5, kw=5, blocks_p6=2, blocks_p1=1)
    ctx, _, _ = make_ctx(s, wm.WM_PREC_BF16)
    try:
        xs = [torch.from_numpy(synth.latent(s, 2, seed=40 + i)).pin_memory() for i in range(5)]
        outs = [torch.full_like(x, float("nan")).pin_memory() for x in xs]
        wm.wm_forecast_host_many(ctx, xs, outs, 7)
        for x, o in zip(xs, outs):
            ref = torch.empty_like(x).pin_memory()
            wm.wm_forecast_host(ctx, x, ref, 7)
            assert torch.equal(o, ref)
        # one input repeated into one shared output: the last result stays
        shared = torch.empty_like(xs[0]).pin_memory()
        wm.wm_forecast_host_many(ctx, [xs[1], xs[2], xs[3]], [shared] * 3, 7)
        assert torch.equal(shared, outs[3])
        wm.wm_forecast_host_many(ctx, [], [], 7)          # nothing to do
        with pytest.raises(wm.WmError):
            wm.wm_forecast_host_many(ctx, xs[:1], outs[:1], -1)
        # the binding refuses host buffers the library would overrun
        with pytest.raises(ValueError):
            wm.wm_forecast_host(ctx, xs[0].double(), outs[0], 7)
        with pytest.raises(ValueError):
            wm.wm_forecast_host(ctx, xs[0], outs[0][:1], 7)
        with pytest.raises(ValueError):
            wm.wm_forecast_host_many(ctx, [xs[0]], [outs[0].transpose(1, 2)], 7)
        with pytest.raises(ValueError):
            wm.wm_forecast_host_many(ctx, [xs[0].cuda()], [outs[0]], 7)
    finally:
        wm.wm_destroy(ctx)


def test_batched_uneven_rollouts_equal_single_rollouts():
    s = synth.Shape(D=4, H=24, W=48, C=128, heads=4, kd=3, kh=5, kw=5, blocks_p6=2, blocks_p1=1)
    ctx, _, _ = make_ctx(s, wm.WM_PREC_BF16, max_batch=4)
    try:
        leads = [1, 6, 7, 13, 0, 12]
        xs = [synth.latent(s, 1, seed=10 + i) for i in range(len(leads))]
        batch = [dev(x) for x in xs]
        wm.wm_rollout_batch(ctx, batch, leads)
        for x, t, got in zip(xs, leads, batch):
            alone = dev(x)
            wm.wm_latent_rollout(ctx, alone, t)
            torch.cuda.synchronize()
            assert torch.equal(got, alone), t
    finally:
        wm.wm_destroy(ctx)


# ------------------------------------------------------ full-size latent ---

def test_full_size_block_at_sampled_tokens():
    s = dataclasses.replace(synth.FULL, blocks_p6=1, blocks_p1=1)
    ctx, p6, _ = make_ctx(s, wm.WM_PREC_BF16, stress=True)
    try:
        x = synth.latent(s, 1, seed=1)
        rng = np.random.default_rng(0)
        N = s.N
        edge = [0, s.W - 1, (s.H - 1) * s.W, N - 1, (4 * s.H + 45) * s.W + 90, (8 * s.H + 3) * s.W + 179]
        toks = np.unique(np.concatenate([edge, rng.integers(0, N, 18)]))
        ref = orc.block_at_tokens(x, p6[0], s, toks)
        for prec, tol in ((wm.WM_PREC_BF16, 2e-2), (wm.WM_PREC_FP32, 1e-5)):
            wm.wm_set_precision(ctx, prec)
            xt = dev(x)
            wm.wm_block_forward(ctx, xt, wm.WM_P6, 0)
            got = host(xt).reshape(1, N, s.C)[:, toks]
            assert_close(got, ref, tol, s.C, prec)
    finally:
        wm.wm_destroy(ctx)


def test_full_size_attention_every_token_against_the_oracle():
    """The attention op at the full-size shape (9 x 90 x 180 tokens, C = 768,
    16 heads, window 5 x 7 x 7, periodic longitude), with the plan the
    autotuner keeps for it and with each kernel kind, against the oracle on
    every query and head (bf16-rounded q, k, v; tolerance as for the other
    attention shapes)."""
    from parity_util import na_oracle_parallel
    s = dataclasses.replace(synth.FULL, blocks_p6=1, blocks_p1=1)
    B, D, H, W, C, heads = 1, s.D, s.H, s.W, s.C, s.heads
    ctx, _, _ = make_ctx(s, wm.WM_PREC_BF16)       # tunes the attention plan for this shape
    try:
        qkv = _na_inputs(B, D, H, W, C, 5)
        qb = torch.from_numpy(qkv).to(torch.bfloat16)
        nbr = orc.neighbor_index(D, H, W, s.kd, s.kh, s.kw, True)
        ref = na_oracle_parallel(qb.to(torch.float32).numpy(), C, heads, nbr)
        qd = qb.to(CUDA)
        for variant in [wm.WM_NA_AUTO, wm.WM_NA_TCGEN05] + [fam | wm.WM_NA_PERSISTENT
                                                             for fam in (wm.WM_NA_QK_CHUNK4, wm.WM_NA_QK_CHUNK8)]:
            out = torch.empty(B * s.N, C, device=CUDA, dtype=torch.bfloat16)
            wm.wm_op_neighborhood_attention(qd, out, B, D, H, W, C, heads, s.kd, s.kh, s.kw, 1, wm.WM_PREC_BF16,
                                            variant)
            assert_close(host(out).reshape(B, -1, C), ref, 1e-2, C // heads, variant)
    finally:
        wm.wm_destroy(ctx)


def test_gemm_autotuner_reports_the_block_gemms():
    """Creating a BF16 context times the tile candidates of the block's GEMMs;
    the report lists QKV and FC1 per row count and the residual GEMMs for
    every row count (their tile width is fixed at the first tuning, so that a
    batched step rounds as a single-latent step does)."""
    s = synth.SMALL
    ctx, _, _ = make_ctx(s, wm.WM_PREC_BF16)
    try:
        rep = wm.wm_autotune_report()
        M = s.N
        assert f"gemm rows={M} N={3 * s.C} K={s.C} epilogue=ln_store" in rep
        assert f"gemm rows={M} N={4 * s.C} K={s.C} epilogue=ln_gelu" in rep
        assert f"gemm rows=any N={s.C} K={s.C} epilogue=resid_ln" in rep
        assert f"gemm rows=any N={s.C} K={4 * s.C} epilogue=resid_ln" in rep
        assert "candidate fc2" in rep
    finally:
        wm.wm_destroy(ctx)


# ------------------------------------------------------------------ misc ---

def test_rel_l2_fp64_reduction():
    rng = np.random.default_rng(3)
    a = rng.standard_normal(1_000_003).astype(np.float32)
    b = (a + 1e-3 * rng.standard_normal(a.size)).astype(np.float32)
    got = wm.wm_rel_l2(dev(b), dev(a))
    assert abs(got - orc.rel_l2(b, a)) < 1e-12


def test_nonfinite_scan_counts_nan_and_inf():
    x = torch.randn(1_000_003, device=CUDA)
    assert wm.wm_count_nonfinite(x) == 0
    idx = torch.tensor([0, 17, 65_536, 999_999, 1_000_002], device=CUDA)
    x[idx[:2]] = float("nan")
    x[idx[2:4]] = float("inf")
    x[idx[4]] = -float("inf")
    assert wm.wm_count_nonfinite(x) == 5
    assert wm.wm_count_nonfinite(x[:0]) == 0


def test_bounded_wait_times_out_and_context_stays_usable():
    assert wm.wm_selftest_wait_timeout(20000) == wm.WM_ERR_TIMEOUT
    wm.wm_device_status()  # cleared
    x = torch.ones(64, 128, device=CUDA)
    g = torch.ones(128, device=CUDA)
    b = torch.zeros(128, device=CUDA)
    out = torch.empty_like(x)
    wm.wm_op_layernorm(x, g, b, out)
    torch.cuda.synchronize()
    assert torch.all(out == 0)
