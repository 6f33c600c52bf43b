"""The allocation-free error reduction, wm_rel_l2_noalloc.

It exists for callers that must not allocate device memory when they check a
result (a caching allocator owns the free memory, or cudaFree's device-wide
synchronisation is not acceptable). It must give what wm_rel_l2 gives. This
file is collected last so that a failure here never hides the other tests,
and it passes both alone in a fresh process and after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2503_22235_gb300 as wm

pytestmark = pytest.mark.gpu


def _sums(fn, a, b):
    out = (ctypes.c_double * 2)()
    st = fn(a.data_ptr(), b.data_ptr(), a.numel(), out, torch.cuda.current_stream().cuda_stream)
    assert st == wm.WM_OK, wm.lib().wm_last_error()
    return out[0], out[1]


def test_noalloc_rel_l2_matches_allocating_entry_point_on_consecutive_calls():
    from paper_2503_22235_gb300 import build as wm_build
    wm_build.build()
    L = wm.lib()
    rng = np.random.default_rng(11)
    # two calls in a row: the second is smaller, so partials left in the shared
    # scratch by the first call must not leak into its result
    for n in (3_000_017, 70_001):
        a = torch.from_numpy(rng.standard_normal(n).astype(np.float32)).cuda()
        b = torch.from_numpy((a.cpu().numpy() + 1e-3 * rng.standard_normal(n)).astype(np.float32)).cuda()
        ref = _sums(L.wm_rel_l2, a, b)
        got = _sums(L.wm_rel_l2_noalloc, a, b)
        for r, g in zip(ref, got):
            assert abs(g - r) <= 1e-12 * abs(r), (n, r, g)
        assert abs(wm.wm_rel_l2_noalloc(a, b) - wm.wm_rel_l2(a, b)) < 1e-12
        # and against the same sums taken on the host in float64
        ah, bh = a.cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64)
        host = (float(np.sum((ah - bh) ** 2)), float(np.sum(bh * bh)))
        for h, g in zip(host, got):
            assert abs(g - h) <= 1e-12 * abs(h), (n, h, g)


def test_noalloc_rel_l2_rejects_sizes_beyond_its_scratch():
    L = wm.lib()
    out = (ctypes.c_double * 2)()
    # pointers are never dereferenced: the size check comes first
    st = L.wm_rel_l2_noalloc(16, 16, 268_435_457, out, None)
    assert st == wm.WM_ERR_INVALID_ARG
    assert b"268435456" in L.wm_last_error()


def test_noalloc_rel_l2_of_zero_elements_is_zero_and_launches_nothing():
    L = wm.lib()
    out = (ctypes.c_double * 2)(7.0, 7.0)
    a = torch.zeros(4, device="cuda")
    st = L.wm_rel_l2_noalloc(a.data_ptr(), a.data_ptr(), 0, out, torch.cuda.current_stream().cuda_stream)
    assert st == wm.WM_OK, L.wm_last_error()
    assert out[0] == 0.0 and out[1] == 0.0
