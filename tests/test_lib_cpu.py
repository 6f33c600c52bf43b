"""Host-side checks of libwm that need no GPU: it builds, loads, exports every
declared entry point, and its host logic (schedule, argument validation)
agrees with the oracle and the header's error contract."""
import ctypes

import pytest

import paper_2503_22235_gb300 as wm
from paper_2503_22235_gb300 import build as wm_build
from oracle import wm_oracle as orc


@pytest.fixture(scope="module", autouse=True)
def built():
    wm_build.build()


def test_library_exports_every_declared_function():
    names = wm.header_functions()
    assert len(names) >= 15
    L = wm.lib()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_debug_build_exports_the_same_functions_and_status_codes():
    """libwm_debug.so (WM_DEBUG_CHECKS=1: device-side index checks) builds from
    the same sources, exports every declared function, and the header's
    WM_ERR_BOUNDS is the binding's."""
    path = wm_build.build(debug=True)
    assert path.endswith("libwm_debug.so")
    D = ctypes.CDLL(path)
    missing = [n for n in wm.header_functions() if not hasattr(D, n)]
    assert not missing, missing
    import os
    import re
    with open(os.path.join(os.path.dirname(wm_build.HERE), "include", "wm.h")) as f:
        hdr = f.read()
    assert int(re.search(r"WM_ERR_BOUNDS = (\d+)", hdr).group(1)) == wm.WM_ERR_BOUNDS


def test_schedule_matches_oracle():
    for T in range(0, 1001):
        assert wm.wm_schedule(T) == orc.greedy_schedule(T)


def test_schedule_rejects_negative_lead():
    with pytest.raises(wm.WmError) as e:
        wm.wm_schedule(-1)
    assert e.value.status == wm.WM_ERR_INVALID_ARG


def _cfg(**kw):
    base = dict(D=4, H=24, W=48, C=128, heads=4, kd=3, kh=5, kw=5, blocks_p6=8, blocks_p1=4, lon_periodic=1,
                ln_eps=1e-5, precision=wm.WM_PREC_BF16, max_batch=1, rope=0)
    base.update(kw)
    return wm.wm_config(*[base[f] for f, _ in wm.wm_config._fields_])


@pytest.mark.parametrize("bad", [dict(kd=4), dict(kh=0), dict(kw=49), dict(C=130), dict(heads=0),
                                 dict(blocks_p1=0), dict(precision=7), dict(kd=5)])
def test_create_rejects_bad_config_before_touching_the_gpu(bad):
    ctx = ctypes.c_void_p()
    st = wm.lib().wm_create_from_host(ctypes.byref(_cfg(**bad)), None, 0, ctypes.byref(ctx))
    assert st == wm.WM_ERR_INVALID_ARG
    assert ctx.value is None
    assert wm.lib().wm_last_error()


def test_create_reports_missing_weight_file():
    ctx = ctypes.c_void_p()
    st = wm.lib().wm_create(ctypes.byref(_cfg()), b"/nonexistent/weights.bin", ctypes.byref(ctx))
    assert st == wm.WM_ERR_IO


def test_null_arguments_are_rejected():
    L = wm.lib()
    assert L.wm_latent_rollout(None, None, 1, 6, None) == wm.WM_ERR_INVALID_ARG
    assert L.wm_processor_step(None, None, 1, 0, None) == wm.WM_ERR_INVALID_ARG
    assert L.wm_destroy(None) == wm.WM_OK
    assert L.wm_rollout_batch(None, None, None, 0, None) == wm.WM_ERR_INVALID_ARG
    assert L.wm_set_fused_rollout(2) == wm.WM_ERR_INVALID_ARG
    assert L.wm_set_fused_rollout(-1) == wm.WM_ERR_INVALID_ARG
    assert L.wm_set_fused_rollout(1) == wm.WM_OK


def _header_arity():
    import re
    with open(wm.HEADER if hasattr(wm, "HEADER") else wm._binding.HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for name, params in re.findall(r"\b(wm_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", text):
        params = params.strip()
        out[name] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_signatures_match_header_arity():
    from paper_2503_22235_gb300 import _binding
    arity = _header_arity()
    assert arity, "no declarations parsed"
    for name, (_, args) in _binding._SIGS.items():
        assert name in arity, name
        assert len(args) == arity[name], (name, len(args), arity[name])


def _header_struct_fields(name):
    """[(field, c type)] of `typedef struct { ... } name;` in include/wm.h, in order."""
    import re
    with open(wm.HEADER) as f:
        text = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
    m = re.search(r"typedef struct \{([^}]*)\}\s*" + name + r"\s*;", text)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if not decl:
            continue
        ctype, names = decl.split(None, 1)
        fields += [(n.strip(), ctype) for n in names.split(",")]
    return fields


@pytest.mark.parametrize("name", ["wm_config", "wm_codec_config"])
def test_binding_structs_mirror_the_header(name):
    """The ctypes structures have the header's fields, in order, with matching types."""
    import ctypes
    cls = getattr(wm, name)
    want = _header_struct_fields(name)
    got = [(f, t) for f, t in cls._fields_]
    assert [f for f, _ in got] == [f for f, _ in want]
    kinds = {"int": ctypes.c_int, "float": ctypes.c_float}
    for (f, t), (_, c) in zip(got, want):
        assert t is kinds[c], (f, t, c)


def test_binding_refuses_host_buffers_the_library_would_overrun(monkeypatch):
    # The host-copy calls trust the sizes they are given; the binding checks
    # dtype, device, contiguity and element count first (no GPU needed here).
    import numpy as np
    import torch
    from paper_2503_22235_gb300 import _binding as b
    per = 2 * 3 * 4 * 8
    monkeypatch.setattr(b, "wm_ctx_sizes", lambda ctx, batch=1: (per * batch, 0))
    good = torch.zeros(2, 2, 3, 4, 8)
    b._host_latents(None, [good, good.clone()], 2)
    b._host_latents(None, [np.zeros((1, 2, 3, 4, 8), np.float32)], 1)
    for bad, batch in [(good.double(), 2), (good[:1], 2), (good.transpose(2, 3), 2),
                       (np.zeros((2, 2, 3, 4, 8)), 2), (good, 3)]:
        with pytest.raises(ValueError):
            b._host_latents(None, [bad], batch)


def test_header_is_plain_c_and_a_c_program_links_against_the_library():
    # The boundary is a C ABI: wm.h must compile as strict C99 and a C program
    # must link against libwm.so and call it (wm_schedule is host-only).
    import os
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    libdir = os.path.join(root, "paper_2503_22235_gb300")
    if not os.path.exists(os.path.join(libdir, "libwm.so")):
        pytest.skip("libwm.so not built")
    work = os.path.join(root, "_build", "c_abi_check")
    os.makedirs(work, exist_ok=True)
    src = os.path.join(work, "main.c")
    with open(src, "w") as f:
        f.write('#include <stdio.h>\n#include "wm.h"\n'
                "int main(void) {\n"
                "  int n6 = -1, n1 = -1;\n"
                "  if (wm_schedule(337, &n6, &n1) != WM_OK || n6 != 56 || n1 != 1) return 1;\n"
                "  if (wm_schedule(-1, &n6, &n1) != WM_ERR_INVALID_ARG || wm_last_error()[0] == 0) return 2;\n"
                "  return 0;\n}\n")
    exe = os.path.join(work, "main")
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(root, "include"),
                    src, "-L", libdir, "-lwm", "-Wl,-rpath," + libdir, "-o", exe], check=True)
    assert subprocess.run([exe]).returncode == 0
