"""SNP ranking by entry lambda (Section 6) in the library (cox_rank_by_entry,
host code, no GPU) against the FP64 oracle's: index work, so the order and
the entry lambdas must agree exactly, on coefficient paths with many zeros,
SNPs that leave and re-join, and ties in |beta|."""
import numpy as np
import pytest

from paper_2010_16114_gb300 import _lib as L


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2010_16114_gb300 import build
    build()
    return L.load()


def _path(seed, k, p, dtype):
    r = np.random.default_rng(seed)
    B = r.normal(0, 0.1, (k, p))
    B[r.random((k, p)) < 0.8] = 0.0
    # ties in |beta| at entry: quantised magnitudes, signs at random
    B = np.round(B, 2)
    lams = np.sort(r.uniform(0.1, 1.0, k))[::-1].copy()
    if seed % 2:
        perm = r.permutation(k)
        B, lams = B[perm], lams[perm]
    return lams, B.astype(dtype)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("seed", range(6))
def test_matches_the_oracle(orc, seed, dtype):
    from paper_2010_16114_gb300.cox import rank_by_entry
    lams, B = _path(seed, k=7 + seed, p=300, dtype=dtype)
    order, entry = rank_by_entry(lams, B)
    o_order, o_entry = orc.rank_by_entry(lams, B.astype(np.float64))
    assert np.array_equal(order, o_order)
    assert np.array_equal(entry, o_entry)
    assert 0 < len(order) < 300


def test_torch_input_and_shapes(orc):
    import torch
    from paper_2010_16114_gb300.cox import rank_by_entry
    lams, B = _path(3, k=5, p=40, dtype=np.float32)
    order, entry = rank_by_entry(lams, torch.from_numpy(B))
    o_order, o_entry = orc.rank_by_entry(lams, B.astype(np.float64))
    assert np.array_equal(order, o_order) and np.array_equal(entry, o_entry)
    with pytest.raises(ValueError):
        rank_by_entry(lams[:3], B)


def test_argument_errors():
    import ctypes
    lib = L.load()
    lams = np.array([0.5, np.nan])
    B = np.zeros((2, 4))
    out = np.zeros(4, np.int64)
    cnt = ctypes.c_int64()
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    assert lib.cox_rank_by_entry(4, 2, vp(lams), vp(B), 1, vp(out), vp(out.copy()), ctypes.byref(cnt)) == L.COX_ERR_ARG
    lams = np.array([0.5, 0.2])
    assert lib.cox_rank_by_entry(0, 2, vp(lams), vp(B), 1, vp(out), vp(out.copy()), ctypes.byref(cnt)) == L.COX_ERR_ARG
    assert lib.cox_rank_by_entry(4, 2, vp(lams), None, 1, vp(out), vp(out.copy()), ctypes.byref(cnt)) == L.COX_ERR_ARG
    e = np.zeros(4, np.int64)
    assert lib.cox_rank_by_entry(4, 2, vp(lams), vp(B), 1, vp(out), vp(e), ctypes.byref(cnt)) == 0
    assert cnt.value == 0 and np.all(e == -1)
