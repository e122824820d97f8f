"""The C-ABI library builds, loads, and exports every symbol include/coxgb.h
declares; argument checks and error strings work without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header: str = "coxgb.h", prefix: str = "cox"):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(" + prefix + r"_[a-z_0-9]+)\s*\(", src))
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


def test_nmf_header_symbols_are_exported(lib):
    from paper_2010_16114_gb300 import _lib as L
    names = _declared("nmfgb.h", "nmf")
    assert set(names) == set(L.NMF_EXPORTS), (names, L.NMF_EXPORTS)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_nmf_argument_errors_without_gpu(lib):
    """The NMF entry points reject bad arguments before any device work, and
    report a missing device as an error code."""
    import numpy as np
    from paper_2010_16114_gb300 import _lib as L
    X = np.ones((4, 3), np.float32)
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    h = ctypes.c_void_p()
    assert L.nmf_setup(vp(X), 4, 3, 0, -1, ctypes.byref(h)) == L.COX_ERR_ARG and not h.value
    assert L.nmf_setup(vp(X), 4, 3, L.NMF_MAX_RANK + 1, -1, ctypes.byref(h)) == L.COX_ERR_ARG
    assert L.nmf_setup(None, 4, 3, 2, -1, ctypes.byref(h)) == L.COX_ERR_ARG
    assert L.nmf_setup(vp(X), 0, 3, 2, -1, ctypes.byref(h)) == L.COX_ERR_ARG
    assert L.nmf_iterate(None, 0, 1, 1e-10, None) == L.COX_ERR_ARG
    assert L.nmf_objective(None, None, None) == L.COX_ERR_ARG
    assert L.nmf_destroy(None) == L.COX_OK
    import torch
    if not torch.cuda.is_available():
        rc = L.nmf_setup(vp(X), 4, 3, 2, -1, ctypes.byref(h))
        assert rc in (L.COX_ERR_CUDA, L.COX_ERR_UNSUPPORTED) and not h.value


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
               "cox_plan": L.cox_plan, "nmf_info": L.nmf_info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "coxgb.h"', '#include "nmfgb.h"',
             "int main(void) {"]
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


def test_plain_c_program_links_and_calls(lib, tmp_path):
    """A C11 program links libcoxgb.so through the header alone and calls the
    entry points that need no device: defaults, error names, a pipeline plan
    and the SNP ranking, and sees a handle-free argument error."""
    import subprocess
    src = tmp_path / "use.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "coxgb.h"
int main(void) {
    cox_options o;
    cox_default_options(&o);
    if (o.precision != COX_SPLIT_E4M3 || o.lag != 10) return 1;
    if (strcmp(cox_strerror(COX_OK), "ok") != 0) return 2;
    cox_plan pl;
    if (cox_plan_shape(16, 0, 0, 0, 0, &pl) != COX_OK || pl.ring < pl.decoder_groups) return 3;
    if (cox_plan_shape(0, 0, 0, 0, 0, &pl) != COX_ERR_ARG) return 4;
    const double lam[3] = {0.3, 0.2, 0.1};
    const float B[3 * 4] = {0.f, 0.5f, 0.f, 0.f,    /* lambda 0.3: SNP 1 */
                            0.1f, 0.7f, -0.3f, 0.f, /* lambda 0.2: SNPs 0, 2 join */
                            0.2f, 0.9f, -0.4f, 0.f};
    int64_t order[4], entry[4], count = -1;
    if (cox_rank_by_entry(4, 3, lam, B, 0, order, entry, &count) != COX_OK) return 5;
    if (count != 3 || order[0] != 1 || order[1] != 2 || order[2] != 0 || entry[3] != -1) return 6;
    if (cox_loss_grad(NULL, NULL, 1, NULL, NULL, NULL) != COX_ERR_ARG) return 7;
    cox_destroy(NULL);
    puts("ok");
    return 0;
}
''')
    exe = tmp_path / "use"
    libdir = os.path.join(ROOT, "paper_2010_16114_gb300")
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                    "-L", libdir, "-lcoxgb", f"-Wl,-rpath,{libdir}"], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout, r.stderr)
