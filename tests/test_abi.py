"""The C-ABI library builds, loads, and exports every symbol include/coxgb.h
declares; argument checks and error strings work without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "coxgb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(cox_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2010_16114_gb300 import build
    from paper_2010_16114_gb300 import _lib as L
    build()
    return L.load()


def test_header_declares_the_boundary():
    names = _declared()
    for core in ("cox_setup", "cox_loss_grad", "cox_prox_step", "cox_path_fit", "cox_lipschitz",
                 "cox_lambda_max", "cox_get_state", "cox_set_state", "cox_strerror", "cox_destroy"):
        assert core in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2010_16114_gb300 import _lib as L
    names = _declared()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) <= set(L.EXPORTS) | set(names)
    for n in L.EXPORTS:
        assert n in names, f"binding exports {n} which the header does not declare"


def test_strerror_and_defaults(lib):
    from paper_2010_16114_gb300 import _lib as L
    assert L.strerror(0) == "ok"
    assert "timed out" in L.strerror(L.COX_ERR_TIMEOUT)
    assert L.strerror(12345) == "unknown error"
    o = L.cox_default_options()
    assert o.precision == L.COX_SPLIT_E4M3 and o.center == 1 and o.lag == 10 and o.wait_limit_s == 2.0
    assert o.tile_m == 0 and o.chunks == 0 and o.stages == 0


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the header's structs have the C sizes and offsets."""
    import subprocess
    from paper_2010_16114_gb300 import _lib as L
    structs = {"cox_options": L.cox_options, "cox_info": L.cox_info, "cox_tune_choice": L.cox_tune_choice,
               "cox_plan": L.cox_plan}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "coxgb.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                         check=True).stdout.split("\n") if l)
    for name, cls in structs.items():
        assert int(out[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(out[f"{name}.{f}"]) == getattr(cls, f).offset, (name, f)


def test_argument_errors_without_gpu(lib):
    """Bad arguments are rejected before any device work."""
    from paper_2010_16114_gb300 import _lib as L
    import numpy as np
    t = np.ones(4)
    e = np.ones(4, np.uint8)
    X = np.zeros((4, 3), np.uint8)
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    rc, h = L.cox_setup(vp(X), 0, 3, L.COX_X_INT8_HOST, vp(t), vp(e), None)
    assert rc == L.COX_ERR_ARG and not h.value
    rc, h = L.cox_setup(None, 4, 3, L.COX_X_INT8_HOST, vp(t), vp(e), None)
    assert rc == L.COX_ERR_ARG
    bad_t = np.array([1.0, np.nan, 2.0, 3.0])
    rc, h = L.cox_setup(vp(X), 4, 3, L.COX_X_INT8_HOST, vp(bad_t), vp(e), None)
    assert rc == L.COX_ERR_ARG
    bad_e = np.array([0, 1, 2, 0], np.uint8)
    rc, h = L.cox_setup(vp(X), 4, 3, L.COX_X_INT8_HOST, vp(t), vp(bad_e), None)
    assert rc == L.COX_ERR_ARG
    o = L.cox_default_options()
    o.precision = L.COX_FP64  # FP64 needs dense float64 X
    rc, h = L.cox_setup(vp(X), 4, 3, L.COX_X_INT8_HOST, vp(t), vp(e), o)
    assert rc == L.COX_ERR_UNSUPPORTED
    assert L.load().cox_loss_grad(None, None, 1, None, None, None) == L.COX_ERR_ARG
    assert L.load().cox_prox_step(None, None, None, 1, 1.0, None) == L.COX_ERR_ARG
    L.cox_destroy(None)


def test_no_device_is_reported_not_crashed(lib):
    """Without a usable sm_103 device, setup returns an error code."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2010_16114_gb300 import _lib as L
    import numpy as np
    t = np.arange(4.0)
    e = np.ones(4, np.uint8)
    X = np.zeros((4, 3), np.uint8)
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    rc, h = L.cox_setup(vp(X), 4, 3, L.COX_X_INT8_HOST, vp(t), vp(e), None)
    assert rc in (L.COX_ERR_CUDA, L.COX_ERR_UNSUPPORTED) and not h.value
