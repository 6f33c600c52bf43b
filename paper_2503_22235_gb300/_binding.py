"""ctypes binding of libwm (include/wm.h). Argument marshalling only.

Every function here has the name of the C entry point it calls. Device
buffers are passed as torch CUDA tensors (only their data pointers are used);
streams default to torch's current stream. A missing library raises: there is
no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
# WM_LIBRARY=debug loads the debug build (device-side bounds checks, see build.py)
LIB_PATH = os.path.join(HERE, "libwm_debug.so" if os.environ.get("WM_LIBRARY") == "debug" else "libwm.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "wm.h")

WM_OK, WM_ERR_INVALID_ARG, WM_ERR_OOM, WM_ERR_CUDA, WM_ERR_TIMEOUT, WM_ERR_BUSY, WM_ERR_IO, WM_ERR_NOT_FOUND, \
    WM_ERR_BOUNDS = range(9)
WM_P6, WM_P1 = 0, 1
WM_PREC_FP32, WM_PREC_BF16, WM_PREC_BF16_FP8MLP = 0, 1, 2
EPI_STORE, EPI_GELU, EPI_RESID_F32, EPI_STORE_F32, EPI_GELU_F8 = 0, 1, 2, 3, 4
WM_NA_AUTO, WM_NA_QK_CHUNK8, WM_NA_QK_CHUNK4, WM_NA_KQ = 0, 1, 2, 3
WM_NA_PER_TILE, WM_NA_PERSISTENT = 4, 8
WM_NA_TCGEN05 = 16

_c_int, _c_float, _vp, _sz = ctypes.c_int, ctypes.c_float, ctypes.c_void_p, ctypes.c_size_t


class WmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"libwm status {status}: {message}")
        self.status = status


class wm_config(ctypes.Structure):
    _fields_ = [("D", _c_int), ("H", _c_int), ("W", _c_int), ("C", _c_int), ("heads", _c_int),
                ("kd", _c_int), ("kh", _c_int), ("kw", _c_int), ("blocks_p6", _c_int), ("blocks_p1", _c_int),
                ("lon_periodic", _c_int), ("ln_eps", _c_float), ("precision", _c_int), ("max_batch", _c_int),
                ("rope", _c_int)]


class wm_codec_config(ctypes.Structure):
    _fields_ = [("H0", _c_int), ("W0", _c_int), ("levels", _c_int), ("level_pad", _c_int), ("pd", _c_int),
                ("p", _c_int), ("v_atm", _c_int), ("v_sfc_in", _c_int), ("v_sfc_out", _c_int), ("n_const", _c_int),
                ("Ce", _c_int), ("heads", _c_int), ("kd", _c_int), ("kh", _c_int), ("kw", _c_int), ("blocks", _c_int),
                ("C", _c_int), ("lon_periodic", _c_int), ("ln_eps", _c_float), ("precision", _c_int)]


_SIGS = {
    "wm_create": (_c_int, [ctypes.POINTER(wm_config), ctypes.c_char_p, ctypes.POINTER(_vp)]),
    "wm_create_from_host": (_c_int, [ctypes.POINTER(wm_config), _vp, _sz, ctypes.POINTER(_vp)]),
    "wm_destroy": (_c_int, [_vp]),
    "wm_set_precision": (_c_int, [_vp, _c_int]),
    "wm_block_forward": (_c_int, [_vp, _vp, _c_int, _c_int, _c_int, _vp]),
    "wm_processor_step": (_c_int, [_vp, _vp, _c_int, _c_int, _vp]),
    "wm_latent_rollout": (_c_int, [_vp, _vp, _c_int, _c_int, _vp]),
    "wm_forecast_host": (_c_int, [_vp, _vp, _vp, _c_int, _c_int, _vp]),
    "wm_forecast_host_many": (_c_int, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _c_int, _c_int, _c_int, _vp]),
    "wm_rollout_batch": (_c_int, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_c_int), _c_int, _vp]),
    "wm_schedule": (_c_int, [_c_int, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int)]),
    "wm_rollout_hourly": (_c_int, [_vp, _vp, _c_int, _vp, _c_int, _vp]),
    "wm_rel_l2": (_c_int, [_vp, _vp, _sz, ctypes.POINTER(ctypes.c_double), _vp]),
    "wm_rel_l2_noalloc": (_c_int, [_vp, _vp, _sz, ctypes.POINTER(ctypes.c_double), _vp]),
    "wm_count_nonfinite": (_c_int, [_vp, _sz, ctypes.POINTER(ctypes.c_ulonglong), _vp]),
    "wm_device_status": (_c_int, []),
    "wm_selftest_wait_timeout": (_c_int, [_c_int]),
    "wm_last_error": (ctypes.c_char_p, []),
    "wm_timing_begin": (_c_int, [_vp, _c_int]),
    "wm_timing_end": (_c_int, [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_c_int)]),
    "wm_ctx_sizes": (_c_int, [_vp, _c_int, ctypes.POINTER(_sz), ctypes.POINTER(_sz)]),
    "wm_ctx_reserve": (_c_int, [_vp, _c_int]),
    "wm_autotune_report": (_c_int, [ctypes.c_char_p, _sz]),
    "wm_server_start": (_c_int, [_vp, _sz, _c_int, ctypes.POINTER(_vp)]),
    "wm_server_submit": (_c_int, [_vp, _vp, _c_int, ctypes.POINTER(ctypes.c_uint64)]),
    "wm_server_poll": (_c_int, [_vp, ctypes.c_uint64, _vp, ctypes.POINTER(_c_int), ctypes.POINTER(ctypes.c_double)]),
    "wm_server_stats": (_c_int, [_vp, ctypes.POINTER(ctypes.c_double)]),
    "wm_server_stop": (_c_int, [_vp]),
    "wm_op_layernorm": (_c_int, [_vp, _vp, _vp, _vp, _c_int, _c_int, _c_int, _c_float, _vp]),
    "wm_op_linear": (_c_int, [_vp, _vp, _vp, _vp, _c_int, _c_int, _c_int, _c_int, _c_int, _vp]),
    "wm_op_neighborhood_attention": (_c_int, [_vp, _vp] + [_c_int] * 12 + [_vp]),
    "wm_op_linear_e4m3": (_c_int, [_vp, _vp, _c_float, _vp, _vp, _c_float, _c_int, _c_int, _c_int, _c_int, _vp]),
    "wm_op_layernorm_e4m3": (_c_int, [_vp, _vp, _vp, _vp, _c_int, _c_int, _c_float, _c_float, _vp]),
    "wm_fp8_scales": (_c_int, [_vp, _c_int, _c_int, ctypes.POINTER(_c_float)]),
    "wm_gemm_tile_override": (_c_int, [_c_int]),
    "wm_set_fused_mlp": (_c_int, [_c_int]),
    "wm_set_fused_rollout": (_c_int, [_c_int]),
    "wm_codec_create": (_c_int, [ctypes.POINTER(wm_codec_config), _vp, _sz, ctypes.POINTER(_vp)]),
    "wm_codec_destroy": (_c_int, [_vp]),
    "wm_encode": (_c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "wm_decode": (_c_int, [_vp, _vp, _vp, _vp, _vp]),
    "wm_forecast_fields": (_c_int, [_vp, _vp, _vp, _vp, _vp, _c_int, _vp, _vp, _vp, _vp]),
}

_lib = None


def lib() -> ctypes.CDLL:
    """The loaded libwm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise WmError(WM_ERR_IO, f"{LIB_PATH} is missing: build it with paper_2503_22235_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name, None)
            if fn is None:
                continue
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def header_functions() -> list[str]:
    """Names of the functions include/wm.h declares."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(wm_[a-z0-9_]+)\s*\(", text)))


def _check(status: int):
    if status != WM_OK:
        msg = lib().wm_last_error()
        raise WmError(status, msg.decode() if msg else "")


def _ptr(t) -> int | None:
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if hasattr(t, "ctypes"):  # numpy
        return t.ctypes.data
    return int(t)


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def make_config(shape, precision=WM_PREC_BF16, max_batch=1) -> wm_config:
    """wm_config from an object with D, H, W, C, heads, kd, kh, kw, blocks_p6, blocks_p1, lon_periodic, ln_eps."""
    return wm_config(shape.D, shape.H, shape.W, shape.C, shape.heads, shape.kd, shape.kh, shape.kw,
                     shape.blocks_p6, shape.blocks_p1, int(bool(shape.lon_periodic)), float(shape.ln_eps),
                     int(precision), int(max_batch), int(bool(getattr(shape, "rope", False))))


# ------------------------------------------------------------------ context ---

def wm_create(cfg: wm_config, weights_path: str) -> int:
    out = _vp()
    _check(lib().wm_create(ctypes.byref(cfg), weights_path.encode(), ctypes.byref(out)))
    return out.value


def wm_create_from_host(cfg: wm_config, weights) -> int:
    """weights: contiguous float32 numpy array (the packed weight blob)."""
    import numpy as np
    w = np.ascontiguousarray(weights, dtype=np.float32)
    out = _vp()
    _check(lib().wm_create_from_host(ctypes.byref(cfg), w.ctypes.data, w.size, ctypes.byref(out)))
    return out.value


def wm_destroy(ctx: int) -> None:
    _check(lib().wm_destroy(ctx))


def wm_set_precision(ctx: int, precision: int) -> None:
    _check(lib().wm_set_precision(ctx, int(precision)))


# ------------------------------------------------------------------ compute ---

def wm_block_forward(ctx, latent, which, block, stream=None):
    _check(lib().wm_block_forward(ctx, _ptr(latent), latent.shape[0], int(which), int(block), _stream(stream)))


def wm_processor_step(ctx, latent, which, stream=None):
    _check(lib().wm_processor_step(ctx, _ptr(latent), latent.shape[0], int(which), _stream(stream)))


def wm_latent_rollout(ctx, latent, lead_hours, stream=None):
    _check(lib().wm_latent_rollout(ctx, _ptr(latent), latent.shape[0], int(lead_hours), _stream(stream)))


def _host_latents(ctx, tensors, batch):
    """Check that each host buffer holds `batch` whole float32 latents of this
    context, contiguous in host memory: the library trusts the sizes it is given."""
    per = wm_ctx_sizes(ctx, 1)[0]
    for t in tensors:
        if getattr(t, "is_cuda", False):
            raise ValueError("host buffer expected, got a CUDA tensor")
        dt = str(getattr(t, "dtype", ""))
        if dt not in ("torch.float32", "float32"):
            raise ValueError(f"float32 host buffer expected, got {dt or type(t).__name__}")
        contiguous = t.is_contiguous() if hasattr(t, "is_contiguous") else t.flags["C_CONTIGUOUS"]
        if not contiguous:
            raise ValueError("host buffer must be contiguous")
        n = t.numel() if hasattr(t, "numel") and callable(t.numel) else t.size
        if n != batch * per:
            raise ValueError(f"host buffer holds {n} floats, expected {batch} x {per}")


def wm_forecast_host(ctx, host_in, host_out, lead_hours, stream=None):
    batch = host_in.shape[0]
    _host_latents(ctx, [host_in, host_out], batch)
    _check(lib().wm_forecast_host(ctx, _ptr(host_in), _ptr(host_out), batch, int(lead_hours), _stream(stream)))


def wm_forecast_host_many(ctx, host_ins, host_outs, lead_hours, stream=None):
    n = len(host_ins)
    if len(host_outs) != n:
        raise ValueError("one output per input")
    batch = host_ins[0].shape[0] if n else 1
    _host_latents(ctx, list(host_ins) + list(host_outs), batch)
    ins = (_vp * max(n, 1))(*[_ptr(t) for t in host_ins])
    outs = (_vp * max(n, 1))(*[_ptr(t) for t in host_outs])
    _check(lib().wm_forecast_host_many(ctx, ins, outs, n, batch, int(lead_hours), _stream(stream)))


def wm_rollout_batch(ctx, latents, lead_hours, stream=None):
    n = len(latents)
    ptrs = (_vp * n)(*[_ptr(t) for t in latents])
    leads = (_c_int * n)(*[int(t) for t in lead_hours])
    _check(lib().wm_rollout_batch(ctx, ptrs, leads, n, _stream(stream)))


def wm_rollout_hourly(ctx, x, max_lead, out, max_batch=8, stream=None):
    """out: device tensor holding max_lead + 1 latents; out[t] = rollout of x to t hours."""
    _check(lib().wm_rollout_hourly(ctx, _ptr(x), int(max_lead), _ptr(out), int(max_batch), _stream(stream)))


def wm_schedule(lead_hours: int) -> tuple[int, int]:
    n6, n1 = _c_int(), _c_int()
    _check(lib().wm_schedule(int(lead_hours), ctypes.byref(n6), ctypes.byref(n1)))
    return n6.value, n1.value


def wm_rel_l2(a, b, stream=None) -> float:
    out = (ctypes.c_double * 2)()
    _check(lib().wm_rel_l2(_ptr(a), _ptr(b), a.numel(), out, _stream(stream)))
    return (out[0] / out[1]) ** 0.5 if out[1] > 0 else float(out[0] > 0)


def wm_rel_l2_noalloc(a, b, stream=None) -> float:
    """wm_rel_l2 without any device allocation (fixed in-library scratch, n <= 268,435,456)."""
    out = (ctypes.c_double * 2)()
    _check(lib().wm_rel_l2_noalloc(_ptr(a), _ptr(b), a.numel(), out, _stream(stream)))
    return (out[0] / out[1]) ** 0.5 if out[1] > 0 else float(out[0] > 0)


def wm_count_nonfinite(x, stream=None) -> int:
    """Number of NaN or infinite elements of the float32 device tensor x."""
    out = ctypes.c_ulonglong()
    _check(lib().wm_count_nonfinite(_ptr(x), x.numel(), ctypes.byref(out), _stream(stream)))
    return out.value


def wm_device_status() -> None:
    _check(lib().wm_device_status())


def wm_selftest_wait_timeout(timeout_us: int) -> int:
    """Returns the status code (WM_ERR_TIMEOUT expected) instead of raising."""
    return lib().wm_selftest_wait_timeout(int(timeout_us))


def wm_ctx_sizes(ctx, batch=1) -> tuple[int, int]:
    lat, ws = _sz(), _sz()
    _check(lib().wm_ctx_sizes(ctx, int(batch), ctypes.byref(lat), ctypes.byref(ws)))
    return lat.value, ws.value


def wm_autotune_report() -> str:
    size = 1 << 16
    while True:   # the library truncates to the buffer: grow until the report fits
        buf = ctypes.create_string_buffer(size)
        _check(lib().wm_autotune_report(buf, len(buf)))
        if len(buf.value) < size - 1 or size >= 1 << 26:
            return buf.value.decode()
        size *= 4


def wm_ctx_reserve(ctx, batch):
    _check(lib().wm_ctx_reserve(ctx, int(batch)))


# ------------------------------------------------------------------ serving ---

_server_ctx = {}   # server handle -> its context, for the host-buffer size checks


def wm_server_start(ctx, hbm_budget_bytes, max_batch) -> int:
    out = _vp()
    _check(lib().wm_server_start(ctx, int(hbm_budget_bytes), int(max_batch), ctypes.byref(out)))
    _server_ctx[out.value] = ctx
    return out.value


def wm_server_submit(srv, host_latent, lead_hours) -> int:
    """host_latent: contiguous float32 host array/tensor of one latent. Raises WmError (WM_ERR_BUSY) when full."""
    rid = ctypes.c_uint64()
    if srv in _server_ctx:
        _host_latents(_server_ctx[srv], [host_latent], 1)
    _check(lib().wm_server_submit(srv, _ptr(host_latent), int(lead_hours), ctypes.byref(rid)))
    return rid.value


def wm_server_poll(srv, req_id, host_out=None):
    """(done, latency_ms): copies the result into host_out when done."""
    done, lat = _c_int(), ctypes.c_double()
    if host_out is not None and srv in _server_ctx:
        _host_latents(_server_ctx[srv], [host_out], 1)
    _check(lib().wm_server_poll(srv, ctypes.c_uint64(req_id), _ptr(host_out), ctypes.byref(done), ctypes.byref(lat)))
    return bool(done.value), lat.value


SERVER_STATS = ("completed", "p50_ms", "p99_ms", "mean_ms", "forecasts_per_s", "max_active", "ticks",
                "batched_steps", "slots", "max_step_batch", "multi_request_steps")


def wm_server_stats(srv) -> dict:
    out = (ctypes.c_double * len(SERVER_STATS))()
    _check(lib().wm_server_stats(srv, out))
    return {k: out[i] for i, k in enumerate(SERVER_STATS)}


def wm_server_stop(srv):
    _server_ctx.pop(srv, None)
    _check(lib().wm_server_stop(srv))


KERNEL_KINDS = ("ln1", "qkv", "attn", "proj", "ln2", "fc1", "fc2")


def wm_timing_begin(ctx, max_launches=4096):
    _check(lib().wm_timing_begin(ctx, int(max_launches)))


def wm_timing_end(ctx) -> dict:
    """{kind: (total_ms, launches)} for the launches since wm_timing_begin."""
    n = len(KERNEL_KINDS)
    ms = (ctypes.c_double * n)()
    cnt = (_c_int * n)()
    _check(lib().wm_timing_end(ctx, ms, cnt))
    return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNEL_KINDS)}


# ----------------------------------------------------------------------- ops ---

def wm_op_layernorm(x, gamma, beta, out, eps=1e-5, stream=None):
    import torch
    M, C = x.shape[0], x.shape[-1]
    _check(lib().wm_op_layernorm(_ptr(x), _ptr(gamma), _ptr(beta), _ptr(out), int(out.dtype == torch.bfloat16),
                                 M, C, float(eps), _stream(stream)))


def wm_op_linear(A, W, bias, out, precision, epilogue, stream=None):
    M, K = A.shape
    N = W.shape[0]
    _check(lib().wm_op_linear(_ptr(A), _ptr(W), _ptr(bias), _ptr(out), M, N, K, int(precision), int(epilogue),
                              _stream(stream)))


def wm_op_neighborhood_attention(qkv, out, batch, D, H, W, C, heads, kd, kh, kw, lon_periodic, precision,
                                 variant=0, stream=None):
    _check(lib().wm_op_neighborhood_attention(_ptr(qkv), _ptr(out), batch, D, H, W, C, heads, kd, kh, kw,
                                              int(bool(lon_periodic)), int(precision), int(variant),
                                              _stream(stream)))


def wm_op_linear_e4m3(A, W, alpha, bias, out, out_scale, epilogue, stream=None):
    """A [M, K], W [N, K]: uint8 tensors of E4M3 codes."""
    M, K = A.shape
    N = W.shape[0]
    _check(lib().wm_op_linear_e4m3(_ptr(A), _ptr(W), float(alpha), _ptr(bias), _ptr(out), float(out_scale), M, N, K,
                                   int(epilogue), _stream(stream)))


def wm_op_layernorm_e4m3(x, gamma, beta, out, eps, inv_scale, stream=None):
    M, C = x.shape[0], x.shape[-1]
    _check(lib().wm_op_layernorm_e4m3(_ptr(x), _ptr(gamma), _ptr(beta), _ptr(out), M, C, float(eps), float(inv_scale),
                                      _stream(stream)))


def wm_fp8_scales(ctx, which, block) -> tuple:
    out = (_c_float * 4)()
    _check(lib().wm_fp8_scales(ctx, int(which), int(block), out))
    return tuple(out)


GEMM_TILES_TUNED, GEMM_TILES_128, GEMM_TILES_256, GEMM_TILES_PAIR, GEMM_TILES_64 = 0, 1, 2, 3, 4


def wm_set_fused_rollout(enable) -> None:
    """1 (default): narrow-latent rollouts as one whole-rollout launch; 0: one launch per kernel."""
    _check(lib().wm_set_fused_rollout(int(enable)))


def wm_set_fused_mlp(enable) -> None:
    """1 runs the C = 128 MLP as one fused kernel, 0 (default) as two GEMMs."""
    _check(lib().wm_set_fused_mlp(int(enable)))


def wm_gemm_tile_override(mode) -> None:
    """Test hook: force the block GEMMs' tiles (GEMM_TILES_*); GEMM_TILES_TUNED restores the tuned plans."""
    _check(lib().wm_gemm_tile_override(int(mode)))


# ------------------------------------------------------- encoder / decoder ---

def make_codec_config(codec, C, precision=WM_PREC_BF16) -> wm_codec_config:
    """wm_codec_config from an object with the fields of wm_codec_config (synth.Codec) and the latent width C."""
    return wm_codec_config(codec.H0, codec.W0, codec.levels, codec.level_pad, codec.pd, codec.p, codec.v_atm,
                           codec.v_sfc_in, codec.v_sfc_out, codec.n_const, codec.Ce, codec.heads, codec.kd,
                           codec.kh, codec.kw, codec.blocks, int(C), int(bool(codec.lon_periodic)),
                           float(codec.ln_eps), int(precision))


def wm_codec_create(cfg: wm_codec_config, weights) -> int:
    """weights: contiguous float32 host array (numpy)."""
    import numpy as np
    w = np.ascontiguousarray(weights, dtype=np.float32)
    out = _vp()
    _check(lib().wm_codec_create(ctypes.byref(cfg), w.ctypes.data, w.size, ctypes.byref(out)))
    return out.value


def wm_codec_destroy(codec) -> None:
    _check(lib().wm_codec_destroy(codec))


def wm_encode(codec, atm, sfc, consts, latent, stream=None) -> None:
    _check(lib().wm_encode(codec, _ptr(atm), _ptr(sfc), _ptr(consts), _ptr(latent), _stream(stream)))


def wm_decode(codec, latent, atm_out, sfc_out, stream=None) -> None:
    _check(lib().wm_decode(codec, _ptr(latent), _ptr(atm_out), _ptr(sfc_out), _stream(stream)))


def wm_forecast_fields(ctx, codec, atm, sfc, consts, lead_hours, latent_ws, atm_out, sfc_out, stream=None) -> None:
    _check(lib().wm_forecast_fields(ctx, codec, _ptr(atm), _ptr(sfc), _ptr(consts), int(lead_hours), _ptr(latent_ws),
                                    _ptr(atm_out), _ptr(sfc_out), _stream(stream)))
