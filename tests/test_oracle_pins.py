"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test checks one definition against a value the paper prints, a closed
form, a library routine that computes a special case, an invariant of the
definition, or brute force on a tiny grid. A plausible slip in the oracle (a
dropped bias, a wrong sign, a transposed weight, an off-by-one window) breaks
at least one of them.
"""
import dataclasses
import math
import os

import numpy as np
import pytest
import torch
import torch.nn.functional as F

import synth
from oracle import wm_oracle as orc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TINY = synth.Shape(D=3, H=5, W=7, C=8, heads=2, kd=3, kh=3, kw=5, blocks_p6=2, blocks_p1=1)


# ------------------------------------------------------------ generator ---

def test_splitmix64_published_first_output():
    # SplitMix64 seeded with 0: first output 0xE220A8397B1DCDAF (Steele et al. 2014 reference code).
    u = synth.uniform(np.uint64(0), 1)[0]
    assert u == (0xE220A8397B1DCDAF >> 11) / 2.0 ** 53


def test_generator_is_deterministic_and_normal():
    a = synth.latent(TINY, 2, seed=1)
    b = synth.latent(TINY, 2, seed=1)
    assert np.array_equal(a, b)
    z = synth.normal(synth.stream_key(7, 3), 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01


# ------------------------------------------------------------- schedule ---

def _golden_schedule():
    rows = []
    with open(os.path.join(GOLDEN, "schedule_paper.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                t, n6, n1 = line.split()[:3]
                rows.append((int(t), int(n6), int(n1)))
    return rows


@pytest.mark.parametrize("T,n6,n1", _golden_schedule())
def test_schedule_paper_values(T, n6, n1):
    assert orc.greedy_schedule(T) == (n6, n1)


def test_schedule_is_minimal_coin_change():
    # dynamic-programming minimum number of {6 h, 1 h} calls for every T <= 1000
    best = [0] + [10 ** 9] * 1000
    for t in range(1, 1001):
        best[t] = min(best[t - 1] + 1, best[t - 6] + 1 if t >= 6 else 10 ** 9)
    for t in range(1001):
        n6, n1 = orc.greedy_schedule(t)
        assert 6 * n6 + n1 == t and 0 <= n1 < 6
        assert n6 + n1 == best[t]


@pytest.mark.parametrize("bad", [-1, -6, 2.5])
def test_schedule_rejects_bad_lead(bad):
    with pytest.raises(ValueError):
        orc.greedy_schedule(bad)


# ---------------------------------------------------- LN / linear / GELU ---

def test_layer_norm_linear_gelu_match_torch_fp64():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((5, 16)) * 3 + 1.5
    g = rng.standard_normal(16)
    b = rng.standard_normal(16)
    W = rng.standard_normal((24, 16))
    bias = rng.standard_normal(24)
    tx = torch.from_numpy(x)
    ln_t = F.layer_norm(tx, (16,), torch.from_numpy(g), torch.from_numpy(b), eps=1e-5).numpy()
    assert np.allclose(orc.layer_norm(x, g, b), ln_t, rtol=0, atol=1e-12)
    lin_t = F.linear(tx, torch.from_numpy(W), torch.from_numpy(bias)).numpy()
    assert np.allclose(orc.linear(x, W, bias), lin_t, rtol=0, atol=1e-12)
    ge_t = F.gelu(tx, approximate="none").numpy()
    assert np.allclose(orc.gelu(x), ge_t, rtol=0, atol=1e-14)


def test_layer_norm_moments():
    x = np.random.default_rng(1).standard_normal((7, 33)) * 5 - 2
    y = orc.layer_norm(x, np.ones(33), np.zeros(33), eps=0.0)
    assert np.allclose(y.mean(-1), 0, atol=1e-13)
    assert np.allclose((y ** 2).mean(-1), 1, atol=1e-12)   # biased variance -> exactly 1


def test_gelu_closed_form_points():
    # Phi(1) = 0.841344746068542948..., Phi(-1) = 1 - Phi(1)
    assert orc.gelu(0.0) == 0.0
    assert abs(orc.gelu(1.0) - 0.8413447460685429) < 1e-15
    assert abs(orc.gelu(-1.0) + (1 - 0.8413447460685429)) < 1e-15
    assert abs(orc.gelu(10.0) - 10.0) < 1e-12 and abs(orc.gelu(-10.0)) < 1e-12


# ------------------------------------------------------------- windows ---

def _bump_window_bruteforce(i, n, k):
    """The k consecutive positions inside [0, n) whose centre is nearest to i."""
    r = k // 2
    best = min(range(0, n - k + 1), key=lambda s: (abs(s + r - i), s))
    return set(range(best, best + k))


def _periodic_window_bruteforce(i, n, k):
    r = k // 2
    return {p for p in range(n) if min(abs(p - i), n - abs(p - i)) <= r}


@pytest.mark.parametrize("n,k", [(5, 3), (7, 7), (24, 5), (9, 5), (4, 3), (1, 1), (90, 7)])
def test_axis_window_clamped_matches_nearest_full_window(n, k):
    win = orc.axis_window(n, k, periodic=False)
    for i in range(n):
        assert len(set(win[i])) == k
        assert set(win[i]) == _bump_window_bruteforce(i, n, k)
        assert i in win[i]


@pytest.mark.parametrize("n,k", [(7, 5), (7, 7), (48, 5), (180, 7), (3, 3), (5, 1)])
def test_axis_window_periodic_matches_circular_distance(n, k):
    win = orc.axis_window(n, k, periodic=True)
    for i in range(n):
        assert len(set(win[i])) == k
        assert set(win[i]) == _periodic_window_bruteforce(i, n, k)


def test_axis_window_rejects_even_or_oversized():
    with pytest.raises(ValueError):
        orc.axis_window(8, 4, False)
    with pytest.raises(ValueError):
        orc.axis_window(4, 5, True)


def test_neighbor_sets_have_full_size_and_contain_self():
    nbr = orc.neighbor_index(4, 24, 48, 3, 5, 5, True)
    assert nbr.shape == (4 * 24 * 48, 75)
    for t in range(0, nbr.shape[0], 37):
        assert len(set(nbr[t])) == 75 and t in nbr[t]


# ------------------------------------------------ neighborhood attention ---

def _mask_bruteforce(D, H, W, kd, kh, kw, periodic):
    N = D * H * W
    mask = np.zeros((N, N), dtype=bool)
    for t in range(N):
        l, i, j = t // (H * W), (t // W) % H, t % W
        Ld = _bump_window_bruteforce(l, D, kd)
        Li = _bump_window_bruteforce(i, H, kh)
        Lj = _periodic_window_bruteforce(j, W, kw) if periodic else _bump_window_bruteforce(j, W, kw)
        for l2 in Ld:
            for i2 in Li:
                for j2 in Lj:
                    mask[t, (l2 * H + i2) * W + j2] = True
    return mask


def _sdpa_fp64(q, k, v, heads, mask=None):
    B, N, C = q.shape
    dh = C // heads
    tq = torch.from_numpy(q).reshape(B, N, heads, dh).transpose(1, 2)
    tk = torch.from_numpy(k).reshape(B, N, heads, dh).transpose(1, 2)
    tv = torch.from_numpy(v).reshape(B, N, heads, dh).transpose(1, 2)
    am = None if mask is None else torch.from_numpy(mask)
    o = F.scaled_dot_product_attention(tq, tk, tv, attn_mask=am)
    return o.transpose(1, 2).reshape(B, N, C).numpy()


def _qkv(B, N, C, seed):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((B, N, C)) * 1.5 for _ in range(3)]


@pytest.mark.parametrize("periodic", [False, True])
def test_whole_grid_window_equals_dense_attention(periodic):
    D, H, W = 3, 5, 7   # odd W so a periodic kw = W window holds every column once
    q, k, v = _qkv(2, D * H * W, 8, seed=3)
    nbr = orc.neighbor_index(D, H, W, D, H, W, periodic)
    o = orc.neighborhood_attention(q, k, v, 2, nbr)
    ref = _sdpa_fp64(q, k, v, 2)
    assert np.max(np.abs(o - ref)) < 1e-12


@pytest.mark.parametrize("periodic,win", [(True, (3, 3, 5)), (False, (1, 3, 3)), (True, (3, 5, 3))])
def test_windowed_attention_equals_masked_dense_attention(periodic, win):
    D, H, W = 3, 5, 7
    q, k, v = _qkv(1, D * H * W, 12, seed=4)
    nbr = orc.neighbor_index(D, H, W, *win, periodic)
    o = orc.neighborhood_attention(q, k, v, 3, nbr)
    ref = _sdpa_fp64(q, k, v, 3, _mask_bruteforce(D, H, W, *win, periodic))
    assert np.max(np.abs(o - ref)) < 1e-12


def test_attention_rows_sum_to_one():
    D, H, W = 4, 6, 9
    q, k, v = _qkv(1, D * H * W, 8, seed=5)
    nbr = orc.neighbor_index(D, H, W, 3, 5, 5, True)
    _, a = orc.neighborhood_attention(q * 4, k, v, 2, nbr, return_weights=True)
    assert np.max(np.abs(a.sum(-1) - 1.0)) < 1e-12
    assert a.min() >= 0


def test_unit_window_returns_values():
    q, k, v = _qkv(1, 3 * 5 * 7, 8, seed=6)
    nbr = orc.neighbor_index(3, 5, 7, 1, 1, 1, True)
    assert np.array_equal(orc.neighborhood_attention(q, k, v, 2, nbr), v)


def test_zero_query_gives_window_mean():
    D, H, W = 3, 5, 7
    _, k, v = _qkv(1, D * H * W, 8, seed=7)
    q = np.zeros_like(k)
    mask = _mask_bruteforce(D, H, W, 3, 3, 5, True)
    nbr = orc.neighbor_index(D, H, W, 3, 3, 5, True)
    o = orc.neighborhood_attention(q, k, v, 2, nbr)
    ref = (mask.astype(np.float64) @ v[0]) / mask.sum(1, keepdims=True)
    assert np.max(np.abs(o[0] - ref)) < 1e-13


def test_circular_padding_then_crop_equals_modular_longitude():
    # Appendix A.2 "circular padding": pad r_w columns each side by wrap, run the
    # clamped window on the padded grid, crop -- must equal mod-W windows.
    D, H, W, win = 3, 5, 9, (3, 3, 5)
    r = win[2] // 2
    q, k, v = _qkv(1, D * H * W, 8, seed=8)
    o_mod = orc.neighborhood_attention(q, k, v, 2, orc.neighbor_index(D, H, W, *win, True))

    def pad(a):
        g = a.reshape(1, D, H, W, 8)
        return np.concatenate([g[:, :, :, W - r:], g, g[:, :, :, :r]], axis=3).reshape(1, -1, 8)

    Wp = W + 2 * r
    o_pad = orc.neighborhood_attention(pad(q), pad(k), pad(v), 2,
                                       orc.neighbor_index(D, H, Wp, *win, False))
    o_crop = o_pad.reshape(1, D, H, Wp, 8)[:, :, :, r:r + W].reshape(1, -1, 8)
    assert np.max(np.abs(o_crop - o_mod)) < 1e-13


# ------------------------------------------------------ block / rollout ---

def _torch_block_dense(x, w, shape):
    """Independent float64 formulation: torch functional ops + dense masked attention."""
    t = {k: torch.from_numpy(np.asarray(v, np.float64)) for k, v in w.items()}
    B = x.shape[0]
    C = shape.C
    xt = torch.from_numpy(np.asarray(x, np.float64)).reshape(B, -1, C)
    mask = _mask_bruteforce(shape.D, shape.H, shape.W, shape.kd, shape.kh, shape.kw, shape.lon_periodic)
    u = F.layer_norm(xt, (C,), t["ln1_g"], t["ln1_b"], eps=shape.ln_eps)
    qkv = F.linear(u, t["wqkv"], t["bqkv"])
    q, k, v = qkv.split(C, dim=-1)
    o = torch.from_numpy(_sdpa_fp64(q.numpy(), k.numpy(), v.numpy(), shape.heads, mask))
    x1 = xt + F.linear(o, t["wo"], t["bo"])
    h = F.gelu(F.linear(F.layer_norm(x1, (C,), t["ln2_g"], t["ln2_b"], eps=shape.ln_eps),
                        t["w1"], t["b1"]), approximate="none")
    return (x1 + F.linear(h, t["w2"], t["b2"])).reshape(x.shape).numpy()


@pytest.mark.parametrize("stress", [False, True])
@pytest.mark.parametrize("periodic", [True, False])
def test_block_equals_dense_torch_formulation(stress, periodic):
    shape = synth.Shape(D=3, H=5, W=7, C=8, heads=2, kd=3, kh=3, kw=5, lon_periodic=periodic)
    x = synth.latent(shape, 2, seed=1)
    w = synth.block_weights(shape.C, 0, 0, 0, stress=stress)
    y = orc.block(x, w, shape)
    ref = _torch_block_dense(x, w, shape)
    assert np.max(np.abs(y - ref)) < 1e-11


def test_stress_weights_change_the_block():
    # the pins above would miss a dropped bias only if biases were all zero
    x = synth.latent(TINY, 1, seed=1)
    w0 = synth.block_weights(TINY.C, 0, 0, 0, stress=False)
    w1 = synth.block_weights(TINY.C, 0, 0, 0, stress=True)
    assert orc.rel_l2(orc.block(x, w1, TINY), orc.block(x, w0, TINY)) > 1e-3


def test_block_commutes_with_longitude_roll():
    x = synth.latent(TINY, 1, seed=2)
    w = synth.block_weights(TINY.C, 0, 0, 0, stress=True)
    for s in (1, 3):
        y1 = orc.block(np.roll(x, s, axis=3), w, TINY)
        y2 = np.roll(orc.block(x, w, TINY), s, axis=3)
        assert np.max(np.abs(y1 - y2)) < 1e-12


@pytest.mark.parametrize("axis", [1, 2])
def test_block_commutes_with_level_and_latitude_flip(axis):
    x = synth.latent(TINY, 1, seed=3)
    w = synth.block_weights(TINY.C, 0, 0, 0, stress=True)
    y1 = orc.block(np.flip(x, axis=axis), w, TINY)
    y2 = np.flip(orc.block(x, w, TINY), axis=axis)
    assert np.max(np.abs(y1 - y2)) < 1e-12


def test_block_output_is_not_flip_symmetric():
    # the flip pin above is not trivially true: the output itself is not symmetric
    x = synth.latent(TINY, 1, seed=3)
    w = synth.block_weights(TINY.C, 0, 0, 0, stress=True)
    y = orc.block(x, w, TINY)
    assert orc.rel_l2(np.flip(y, axis=2), y) > 1e-2


def test_block_at_tokens_matches_full_block():
    shape = synth.Shape(D=4, H=6, W=9, C=16, heads=2, kd=3, kh=5, kw=5)
    x = synth.latent(shape, 2, seed=4)
    w = synth.block_weights(shape.C, 0, 1, 2, stress=True)
    full = orc.block(x, w, shape).reshape(2, -1, shape.C)
    toks = np.array([0, 5, 17, 100, shape.N - 1])
    part = orc.block_at_tokens(x, w, shape, toks)
    assert np.max(np.abs(part - full[:, toks])) < 1e-12


def test_rollout_schedule_and_prefix_composition():
    x = synth.latent(TINY, 1, seed=5)
    p6, p1 = synth.processor_weights(TINY, seed=0, stress=True)
    assert np.array_equal(orc.rollout(x, 0, p6, p1, TINY), x.astype(np.float64))
    steps = []
    y13 = orc.rollout(x, 13, p6, p1, TINY, per_step=steps)
    assert len(steps) == 3                                 # 13 h = 2 x 6 h + 1 x 1 h
    y12 = orc.rollout(x, 12, p6, p1, TINY)
    assert np.max(np.abs(orc.processor(y12, p1, TINY) - y13)) < 1e-12
    assert np.max(np.abs(orc.processor(orc.processor(x, p6, TINY), p6, TINY) - y12)) < 1e-12
    # six-hour steps come first: P1(P6(x)) != P6(P1(x))
    y7 = orc.rollout(x, 7, p6, p1, TINY)
    other = orc.processor(orc.processor(x, p1, TINY), p6, TINY)
    assert np.max(np.abs(y7 - orc.processor(orc.processor(x, p6, TINY), p1, TINY))) < 1e-12
    assert orc.rel_l2(y7, other) > 1e-3


def _dense_chain(x, blocks, shape):
    for w in blocks:
        x = _torch_block_dense(x, w, shape)
    return x


def test_processor_is_its_blocks_in_order():
    """Appendix A.2: a processor is a stack of NA blocks, each with its own
    weights, applied in order. Pinned against the independent dense block
    chained by hand; the reversed order and a stack that reuses block 0's
    weights both give a different result, so an order or indexing slip in the
    oracle cannot pass."""
    shape = dataclasses.replace(TINY, blocks_p6=3)
    x = synth.latent(shape, 2, seed=6)
    p6, _ = synth.processor_weights(shape, seed=0, stress=True)
    y = orc.processor(x, p6, shape)
    assert np.max(np.abs(y - _dense_chain(x, p6, shape))) < 1e-11
    assert orc.rel_l2(y, _dense_chain(x, p6[::-1], shape)) > 1e-3
    assert orc.rel_l2(y, _dense_chain(x, [p6[0]] * 3, shape)) > 1e-3


def test_rollout_is_the_greedy_chain_of_dense_blocks():
    """Section 2.1: 13 h = two six-hour calls then one one-hour call, each
    call its processor's blocks in order (dense block chained by hand)."""
    x = synth.latent(TINY, 1, seed=7)
    p6, p1 = synth.processor_weights(TINY, seed=0, stress=True)
    ref = _dense_chain(x, list(p6) + list(p6) + list(p1), TINY)
    assert np.max(np.abs(orc.rollout(x, 13, p6, p1, TINY) - ref)) < 1e-11
    wrong_order = _dense_chain(x, list(p1) + list(p6) + list(p6), TINY)
    assert orc.rel_l2(ref, wrong_order) > 1e-3


def test_rel_l2():
    a = np.array([3.0, 4.0])
    assert orc.rel_l2(a, a) == 0.0
    assert math.isclose(orc.rel_l2(np.array([3.0, 5.0]), a), 1.0 / 5.0)


# ------------------------------------------------------------- FP8 codec ---

def test_e4m3_decode_matches_torch_on_all_codes():
    ref = torch.arange(256, dtype=torch.uint8).view(torch.float8_e4m3fn).double().numpy()
    got = np.array([orc.e4m3_decode(c) for c in range(256)])
    both_nan = np.isnan(ref) & np.isnan(got)
    assert np.all(both_nan | (ref == got))
    assert orc.e4m3_decode(0x7E) == 448.0 and orc.e4m3_decode(0x38) == 1.0
    assert orc.e4m3_decode(0x08) == 2.0 ** -6 and orc.e4m3_decode(0x01) == 2.0 ** -9
    assert np.isnan(orc.e4m3_decode(0x7F)) and np.isnan(orc.e4m3_decode(0xFF))


def test_e4m3_round_trips_every_finite_code_and_rounds_ties_to_even():
    finite = [orc.e4m3_decode(c) for c in range(256) if not np.isnan(orc.e4m3_decode(c))]
    assert np.array_equal(orc.e4m3_round(finite), np.array(finite))
    # ties: 1.0625 between 1.0 (even code) and 1.125; 1.1875 between 1.125 and 1.25 (even)
    assert orc.e4m3_round(1.0625) == 1.0 and orc.e4m3_round(1.1875) == 1.25
    assert orc.e4m3_round(-1.1875) == -1.25
    # saturation (OCP "satfinite"): beyond 448 clamps to 448
    assert orc.e4m3_round(1e6) == 448.0 and orc.e4m3_round(-500.0) == -448.0


def test_e4m3_round_matches_torch_in_range():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000) * 30, rng.uniform(-448, 448, 20000),
                        rng.standard_normal(5000) * 1e-3])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.float8_e4m3fn).double().numpy()
    assert np.array_equal(orc.e4m3_round(x.astype(np.float32)), ref)


# ------------------------------------------------------------ FP8 MLP ---

def test_fp8_scale_bounds_hold_and_are_reached_by_an_outlier():
    C = 64
    w = synth.block_weights(C, 0, 0, 0, stress=True)
    s_u, s_w1, s_h, s_w2 = orc.fp8_mlp_scales(w, C)
    rng = np.random.default_rng(5)
    x = rng.standard_normal((400, C)) * rng.uniform(0.1, 50, (400, 1))
    x[0] = 0.0
    x[0, 7] = 1e4                       # one-hot row: |x_c - mean| / std = sqrt(C - 1) at c = 7
    u = orc.layer_norm(x, w["ln2_g"], w["ln2_b"], 0.0)
    assert np.abs(u).max() <= s_u * 448.0 * (1 + 1e-12)
    assert np.abs(u[0, 7]) >= 0.5 * s_u * 448.0
    h = orc.gelu(orc.linear(u, w["w1"], w["b1"]))
    assert np.abs(h).max() <= s_h * 448.0 * (1 + 1e-12)
    assert s_w1 * 448.0 == np.abs(w["w1"]).max() and s_w2 * 448.0 == np.abs(w["w2"]).max()


def test_fp8_block_without_rounding_is_the_block():
    x = synth.latent(TINY, 1, seed=9)
    w = synth.block_weights(TINY.C, 0, 0, 1, stress=True)
    same = orc.block_fp8mlp(x, w, TINY, rounding=lambda v: v)
    assert np.max(np.abs(same - orc.block(x, w, TINY))) < 1e-12
    q = orc.block_fp8mlp(x, w, TINY)
    err = orc.rel_l2(q, orc.block(x, w, TINY))
    assert 1e-4 < err < 5e-2     # E4M3 keeps 3 mantissa bits


# ------------------------------------------------------------------ RoPE ---

ROPE = synth.Shape(D=3, H=5, W=7, C=24, heads=2, kd=3, kh=3, kw=5, rope=True)


def test_rope_pair_split_covers_the_head():
    for dh in (8, 16, 24, 32, 48, 64):
        a, b, c = orc.rope_pairs(dh)
        assert a + b + c == dh // 2 and min(a, b, c) >= 1 and c >= b >= a


def test_rope_rotation_matches_complex_multiplication():
    rng = np.random.default_rng(2)
    t = rng.standard_normal((1, 3 * 5 * 7, 24))
    ang = orc.rope_angles(3, 5, 7, 12)
    got = orc.rope_rotate(t, 2, ang)
    z = (t[..., 0::2] + 1j * t[..., 1::2]).reshape(1, -1, 2, 6) * np.exp(1j * ang)[None, :, None, :]
    ref = np.stack([z.real, z.imag], -1).reshape(1, -1, 24)
    assert np.max(np.abs(got - ref)) < 1e-12
    assert np.allclose(np.linalg.norm(got, axis=-1), np.linalg.norm(t, axis=-1))


def test_rope_scores_depend_only_on_relative_position():
    # q at p, k at p' and q at p + s, k at p' + s give the same rotated dot
    # product; along longitude the shift is taken modulo W
    rng = np.random.default_rng(3)
    D, H, W, dh = 4, 6, 7, 12
    ang = orc.rope_angles(D, H, W, dh).reshape(D, H, W, -1)
    q, k = rng.standard_normal((2, dh))

    def score(p, pp):
        a = orc.rope_rotate(q[None, None], 1, ang[p][None])[0, 0]
        b = orc.rope_rotate(k[None, None], 1, ang[pp][None])[0, 0]
        return a @ b

    base = score((1, 2, 3), (2, 0, 5))
    assert abs(score((2, 3, 3), (3, 1, 5)) - base) < 1e-12          # level and latitude shift
    assert abs(score((1, 2, 6), (2, 0, (5 + 3) % W)) - base) < 1e-12  # longitude shift, wrapped
    assert abs(score((1, 2, 3), (2, 1, 5)) - base) > 1e-6            # a different offset differs


def test_rope_block_keeps_longitude_roll_equivariance_and_breaks_flip():
    x = synth.latent(ROPE, 1, seed=4)
    w = synth.block_weights(ROPE.C, 0, 0, 0, stress=True)
    y = orc.block(x, w, ROPE)
    for s in (1, 4):
        assert np.max(np.abs(orc.block(np.roll(x, s, axis=3), w, ROPE) - np.roll(y, s, axis=3))) < 1e-12
    assert orc.rel_l2(orc.block(np.flip(x, axis=2), w, ROPE), np.flip(y, axis=2)) > 1e-4
    assert orc.rel_l2(y, orc.block(x, w, dataclasses.replace(ROPE, rope=False))) > 1e-4


def test_rope_block_at_tokens_matches_full_block():
    x = synth.latent(ROPE, 1, seed=5)
    w = synth.block_weights(ROPE.C, 0, 1, 0, stress=True)
    toks = np.array([0, 11, 52, ROPE.N - 1])
    full = orc.block(x, w, ROPE).reshape(1, -1, ROPE.C)
    assert np.max(np.abs(orc.block_at_tokens(x, w, ROPE, toks) - full[:, toks])) < 1e-12
