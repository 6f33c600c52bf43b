"""Serving loop: continuous batching with HBM-budget admission.

Requests with uneven lead times arrive while others run, share batched
processor steps, and each result must equal the same forecast computed alone
(wm_latent_rollout on one latent) bit for bit, in every precision (BF16,
FP8-MLP, FP32): the kernels are row independent, the FP8 scales static, and
the schedule per request does not depend on the mix.
"""
import dataclasses
import time

import numpy as np
import pytest
import torch

import paper_2503_22235_gb300 as wm
import synth

pytestmark = pytest.mark.gpu

SHAPE = dataclasses.replace(synth.SMALL, blocks_p6=2, blocks_p1=1)


@pytest.fixture(scope="module", params=[wm.WM_PREC_BF16, wm.WM_PREC_BF16_FP8MLP, wm.WM_PREC_FP32],
                ids=["bf16", "fp8mlp", "fp32"])
def ctx(request):
    from paper_2503_22235_gb300 import build as wm_build
    wm_build.build()
    p6, p1 = synth.processor_weights(SHAPE, seed=0, stress=True)
    c = wm.wm_create_from_host(wm.make_config(SHAPE, request.param), synth.pack_weights(p6, p1))
    yield c
    wm.wm_destroy(c)


def _budget(ctx, slots, max_batch):
    lat, ws = wm.wm_ctx_sizes(ctx, max_batch)
    return ws + (max_batch + slots) * lat * 4


def _alone(ctx, x, lead):
    d = torch.from_numpy(x).cuda()
    wm.wm_latent_rollout(ctx, d, lead)
    torch.cuda.synchronize()
    return d.cpu().numpy()


def test_server_results_equal_alone_and_in_the_mix(ctx):
    # the first two are long six-hour chains submitted back to back, so they
    # share batched six-hour steps whatever the worker's timing
    leads = [48, 42, 0, 7, 6, 24, 2, 19, 12, 5]
    xs = [synth.latent(SHAPE, 1, seed=100 + i) for i in range(len(leads))]
    srv = wm.wm_server_start(ctx, _budget(ctx, slots=4, max_batch=3), max_batch=3)
    try:
        ids = []
        for i, (x, t) in enumerate(zip(xs, leads)):
            ids.append(wm.wm_server_submit(srv, x, t))
            if i % 3 == 2:
                time.sleep(0.005)        # later requests arrive while earlier ones run
        outs = {}
        deadline = time.time() + 120
        while len(outs) < len(ids) and time.time() < deadline:
            for rid in ids:
                if rid in outs:
                    continue
                buf = np.empty_like(xs[0])
                done, lat_ms = wm.wm_server_poll(srv, rid, buf)
                if done:
                    assert lat_ms >= 0
                    outs[rid] = buf
            time.sleep(0.001)
        assert len(outs) == len(ids)
        st = wm.wm_server_stats(srv)
        assert st["completed"] == len(ids)
        assert st["slots"] == 4 and 2 <= st["max_active"] <= 4
        # the requests really were mixed: some batched steps advanced two or
        # more requests at once
        assert st["max_step_batch"] >= 2 and st["multi_request_steps"] >= 1, st
        assert st["max_step_batch"] <= 3
        assert st["p50_ms"] <= st["p99_ms"]
    finally:
        wm.wm_server_stop(srv)
    for rid, x, t in zip(ids, xs, leads):
        ref = _alone(ctx, x, t)
        assert np.array_equal(outs[rid], ref), t
    with pytest.raises(wm.WmError):
        wm.wm_server_poll(0, 1)  # a NULL server handle is rejected


def test_server_budget_and_arguments(ctx):
    with pytest.raises(wm.WmError) as e:
        wm.wm_server_start(ctx, 1024, max_batch=2)
    assert e.value.status == wm.WM_ERR_INVALID_ARG
    srv = wm.wm_server_start(ctx, _budget(ctx, slots=1, max_batch=1), max_batch=1)
    try:
        x = synth.latent(SHAPE, 1, seed=7)
        with pytest.raises(wm.WmError):
            wm.wm_server_submit(srv, x, -1)
        with pytest.raises(wm.WmError) as e:
            wm.wm_server_poll(srv, 12345)
        assert e.value.status == wm.WM_ERR_NOT_FOUND
        # one slot: requests queue and are admitted one after the other
        ids = [wm.wm_server_submit(srv, x, t) for t in (6, 1, 7)]
        got = {}
        deadline = time.time() + 60
        while len(got) < 3 and time.time() < deadline:
            for rid in ids:
                if rid not in got:
                    done, _ = wm.wm_server_poll(srv, rid, None)
                    if done:
                        got[rid] = True
            time.sleep(0.001)
        assert len(got) == 3
        assert wm.wm_server_stats(srv)["max_active"] == 1
    finally:
        wm.wm_server_stop(srv)


def test_concurrent_polls_collect_each_result_once(ctx):
    """Two threads poll every finished request at the same time: exactly one
    of them receives the result, the other sees the id as collected, and no
    slot is handed out twice (later requests in a full server still match
    their single-request rollouts)."""
    import threading
    srv = wm.wm_server_start(ctx, _budget(ctx, slots=3, max_batch=2), max_batch=2)
    try:
        xs = [synth.latent(SHAPE, 1, seed=200 + i) for i in range(12)]
        for round_ in range(4):
            batch = xs[3 * round_:3 * round_ + 3]
            ids = [wm.wm_server_submit(srv, x, 7) for x in batch]
            got = {rid: [] for rid in ids}
            lock = threading.Lock()

            def poller(rid):
                deadline = time.time() + 60
                while time.time() < deadline:
                    buf = np.empty_like(xs[0])
                    try:
                        done, _ = wm.wm_server_poll(srv, rid, buf)
                    except wm.WmError as e:
                        assert e.status == wm.WM_ERR_NOT_FOUND
                        return
                    if done:
                        with lock:
                            got[rid].append(buf)
                        return
                    time.sleep(0.0002)

            threads = [threading.Thread(target=poller, args=(rid,)) for rid in ids for _ in range(2)]
            for t in threads:
                t.start()
            for t in threads:
                t.join()
            for rid, x in zip(ids, batch):
                assert len(got[rid]) == 1, (round_, rid, len(got[rid]))
                assert np.array_equal(got[rid][0], _alone(ctx, x, 7))
    finally:
        wm.wm_server_stop(srv)
