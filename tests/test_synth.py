"""The seeded input generators (synth/) that both the CUDA path and the FP64
oracle consume: the counter-based generator against its published
definition, the recipes' identities, the packed layouts, and the statistical
shape each recipe claims (genotype frequencies, event or censoring fraction,
whole-day ties).  CPU only."""
import ctypes

import numpy as np
import pytest

import synth

M64 = (1 << 64) - 1


def _splitmix64_output(z: int) -> int:
    """SplitMix64's output function (Steele, Lea & Flood, OOPSLA 2014): add the
    golden-ratio increment, then two xor-shift-multiply rounds and a final
    xor-shift."""
    z = (z + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


@pytest.fixture(scope="module")
def lib():
    synth.build_host()
    lib = synth._host()
    lib.syn_mix64.restype = ctypes.c_uint64
    lib.syn_mix64.argtypes = [ctypes.c_uint64]
    return lib


def test_splitmix64_known_answer_and_definition(lib):
    # the generator's first output from state 0
    assert _splitmix64_output(0) == 0xE220A8397B1DCDAF
    r = np.random.default_rng(5)
    for z in [0, 1, 2, M64, 0x9E3779B97F4A7C15] + [int(v) for v in r.integers(0, 1 << 63, 50)]:
        assert lib.syn_mix64(z) == _splitmix64_output(z)


def test_draw_is_keyed_by_seed_stream_and_counter(lib):
    def draw(seed, stream, a, b):
        key = _splitmix64_output(seed ^ ((stream * 0xD1B54A32D192ED03) & M64))
        return _splitmix64_output(_splitmix64_output((key + a) & M64) ^ b)
    for args in [(0, 0, 0, 0), (2010161141, 2, 7, 3), (2010161144, 5, 399999, 0), (1, 6, 123, 456)]:
        assert lib.syn_draw(*args) == draw(*args)
    assert lib.syn_draw(1, 2, 3, 4) != lib.syn_draw(1, 2, 4, 3)


def test_recipes_keep_their_identity():
    expect = {
        "normal_1k_2k": ("normal", 1000, 2000, 1, 2010161140),
        "geno_100k_50k": ("geno", 100_000, 50_000, 1, 2010161141),
        "geno_200k_10k": ("geno", 200_000, 10_000, 1, 2010161142),
        "geno_400k_100k_k32": ("geno", 400_000, 100_000, 32, 2010161143),
        "geno_400k_500k_k16": ("geno", 400_000, 500_000, 16, 2010161144),
    }
    assert set(synth.WORKLOADS) == set(expect)
    for name, (kind, n, p, k, seed) in expect.items():
        r = synth.WORKLOADS[name]
        assert (r.name, r.kind, r.n, r.p, r.k, r.seed) == (name, kind, n, p, k, seed)
        s = r.scaled(n=500, p=40)
        assert (s.seed, s.kind, s.n, s.p, s.k) == (seed, kind, 500, 40, k)
    r4 = synth.WORKLOADS["geno_400k_500k_k16"]
    assert (r4.maf_lo, r4.maf_hi, r4.event_frac, r4.dmax, r4.n_causal) == (0.01, 0.5, 0.05, 5000, 500)
    f = r4.lambda_fracs()
    assert len(f) == 16 and f[0] == pytest.approx(1.0) and f[-1] == pytest.approx(0.01)
    assert np.allclose(np.diff(np.log(f)), np.log(0.01) / 15)


def test_packed_rows_columns_and_dense_agree():
    w = synth.workload("geno_100k_50k", n=300, p=37)
    X = w.dense()
    assert X.dtype == np.uint8 and X.max() <= 2
    P = w.packed_rows()
    assert P.shape == (300, 10)
    j = np.arange(37)
    codes = (P[:, j // 4] >> (2 * (j % 4))) & 3
    assert np.array_equal(codes, X)
    assert np.all((P[:, 9] >> 2) == 0)  # the three code slots past p = 37 stay zero
    idx = np.array([0, 5, 36, 17])
    assert np.array_equal(w.cols(idx), X[:, idx].astype(np.float64))
    assert np.array_equal(w.packed_rows(100, 50), P[100:150])


def test_generation_is_deterministic():
    a = synth.workload("geno_200k_10k", n=2000, p=64)
    b = synth.workload("geno_200k_10k", n=2000, p=64)
    assert np.array_equal(a.dense(), b.dense()) and np.array_equal(a.y, b.y)
    assert np.array_equal(a.delta, b.delta) and np.array_equal(a.causal_idx, b.causal_idx)


def test_genotype_frequencies_follow_the_maf():
    w = synth.workload("geno_400k_500k_k16", n=20000, p=60)
    X = w.dense().astype(np.float64)
    assert np.all((w.maf >= 0.01) & (w.maf < 0.5))
    assert np.array_equal(w.thr, np.floor(w.maf * 2.0 ** 32).astype(np.uint32))
    se = np.sqrt(2 * w.maf * (1 - w.maf) / w.n)
    assert np.all(np.abs(X.mean(axis=0) - 2 * w.maf) <= 5 * se)
    # Hardy-Weinberg: P(x = 2) = MAF^2
    se2 = np.sqrt(w.maf ** 2 * (1 - w.maf ** 2) / w.n)
    assert np.all(np.abs((X == 2).mean(axis=0) - w.maf ** 2) <= 5 * se2 + 1e-12)


@pytest.mark.parametrize("name", ["geno_100k_50k", "geno_400k_100k_k32", "geno_400k_500k_k16"])
def test_day_times_hit_the_event_fraction_with_ties(name):
    w = synth.workload(name, n=20000, p=40)
    r = w.r
    assert int(w.delta.sum()) == round(r.event_frac * w.n)
    assert np.all(w.y == np.round(w.y)) and w.y.min() >= 1 and w.y.max() <= r.dmax
    assert len(np.unique(w.y)) < w.n  # whole days: tied times


def test_normal_times_hit_the_censoring_fraction_without_ties():
    w = synth.workload("normal_1k_2k")
    assert w.n - int(w.delta.sum()) == round(0.30 * w.n)
    assert len(np.unique(w.y)) == w.n and np.all(w.y > 0)
    assert len(w.causal_idx) == 20 and np.all(np.diff(w.causal_idx) > 0)


def test_nmf_inputs_grid_range_and_determinism():
    """NMF inputs: X on the grid k / 256 (exact in bf16), V and W in [0, 1),
    regenerable by rows."""
    X, V, W = synth.nmf_inputs(70, 90, 4)
    assert X.dtype == np.float32 and X.shape == (70, 90) and V.shape == (70, 4) and W.shape == (4, 90)
    k = X.astype(np.float64) * 256
    assert np.array_equal(k, np.round(k)) and k.min() >= 0 and k.max() <= 255
    assert len(np.unique(k)) > 200
    assert 0.45 < X.mean() < 0.55
    assert V.min() >= 0 and V.max() < 1 and W.min() >= 0 and W.max() < 1
    X2, V2, W2 = synth.nmf_inputs(70, 90, 4)
    assert np.array_equal(X, X2) and np.array_equal(V, V2) and np.array_equal(W, W2)
    assert np.array_equal(synth.nmf_x(10, 90, i0=30), X[30:40])
