"""GPU parity of the Section 5.1 NMF (multiplicative and alternating projected
gradient updates) against the FP64 oracle (oracle.nmf, oracle.nmf_objective),
through the C ABI in include/nmfgb.h.

Inputs: synth.nmf_inputs, X on the grid k / 256 (exact in the library's bf16
copy of X, so both sides factor the same matrix), V0 and W0 uniform on [0, 1)
in FP32.

Tolerances.  The library keeps V and W in FP32 and forms X W^T and V^T X from
FP32-exact bf16 limbs with FP32 tensor-core accumulation (512 K per
accumulator, then FP32 running sums; partial slots added in FP64); the Gram matrices are FP64
sums of FP32 block partials.  A numpy model of that arithmetic (FP32 products
and updates) stays within 1.1e-6 elementwise of the FP64 oracle after one
iteration and within 1.3e-6 relative L2 after 50 at 300 x 200, r = 20.  The
tests allow 10x: one iteration 2e-5 elementwise relative, ten iterations 2e-5
relative L2, the objective 1e-5 relative.  The APG step is a difference,
F - s (F G - P): its FP32 rounding is relative to the operands, so an APG entry
is compared relative to the larger of its new and its previous value (an entry
the step brings near zero from a large one carries the operands' error).
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    import paper_2010_16114_gb300 as P
    P.build()
    assert torch.cuda.is_available()
    from paper_2010_16114_gb300.nmf import NMF
    return NMF


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def max_rel(a, b, floor):
    a = np.asarray(a, np.float64)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), floor)))


def step_floor(algo, prev):
    """Per-entry floor of the relative error: none for the multiplicative
    update (a product of positive terms), the previous value for APG."""
    return 1e-30 if algo == "mult" else np.abs(np.asarray(prev, np.float64))


# (m, n, r): several row tiles with ragged tails in both products; a tall X whose
# CTAs each run three row tiles of X W^T (both TMEM accumulators reused) and whose
# X^T V is one row tile cut into ~130 partial slots; single ragged tiles; r = 1
# and the largest rank (N = 240, four pipeline stages); a wide X whose CTAs each sum
# ~130 K chunks of one row tile (17 accumulator windows per segment); degenerate
# X of one entry, one row and one column
SHAPES = [(300, 200, 5), (300, 200, 20), (51200, 128, 20), (97, 45, 3), (1000, 777, 1), (640, 520, 80),
          (1000, 3000, 60), (2560, 64000, 4), (1, 1, 1), (1, 300, 3), (130, 1, 2)]


@pytest.mark.parametrize("m,n,r", SHAPES)
@pytest.mark.parametrize("algo", ["mult", "apg"])
def test_one_iteration_elementwise(N, m, n, r, algo):
    X, V0, W0 = synth.nmf_inputs(m, n, r)
    Ve, We = oracle.nmf(X, V0, W0, 1, algo, 1e-10)
    h = N(X, r)
    h.set_factors(V0, W0)
    h.iterate(1, algo)
    V, W = h.factors()
    assert max_rel(V, Ve, step_floor(algo, V0)) <= 2e-5
    assert max_rel(W, We, step_floor(algo, W0)) <= 2e-5
    assert (V >= 0).all() and (W >= 0).all()
    h.close()


@pytest.mark.parametrize("algo", ["mult", "apg"])
def test_ten_iterations_and_objective(N, algo):
    m, n, r = 700, 450, 20
    X, V0, W0 = synth.nmf_inputs(m, n, r)
    h = N(X, r)
    h.set_factors(V0, W0)
    f0 = h.objective()
    assert abs(f0 - oracle.nmf_objective(X, V0, W0)) <= 1e-5 * oracle.nmf_objective(X, V0, W0)
    h.iterate(10, algo)
    V, W = h.factors()
    Ve, We = oracle.nmf(X, V0, W0, 10, algo, 1e-10)
    assert rel_l2(V, Ve) <= 2e-5
    assert rel_l2(W, We) <= 2e-5
    fe = oracle.nmf_objective(X, Ve, We)
    assert abs(h.objective() - fe) <= 1e-5 * fe
    h.close()


def test_multiplicative_objective_never_increases(N):
    """Lee and Seung: each multiplicative update leaves ||X - V W||^2 no larger."""
    X, V0, W0 = synth.nmf_inputs(500, 400, 10)
    h = N(X, 10)
    h.set_factors(V0, W0)
    f = [h.objective()]
    for _ in range(20):
        h.iterate(1, "mult")
        f.append(h.objective())
    f = np.array(f)
    assert np.all(np.diff(f) <= 1e-6 * f[:-1]), f
    assert f[-1] < 0.5 * f[0]
    h.close()


def test_deterministic(N):
    X, V0, W0 = synth.nmf_inputs(1000, 3000, 20)
    out = []
    for _ in range(2):
        h = N(X, 20)
        h.set_factors(V0, W0)
        h.iterate(5, "apg")
        out.append(h.factors())
        h.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_switching_algorithm_and_eps(N):
    """The captured iteration is rebuilt when the algorithm or eps changes."""
    m, n, r = 300, 200, 6
    X, V0, W0 = synth.nmf_inputs(m, n, r)
    h = N(X, r)
    h.set_factors(V0, W0)
    h.iterate(2, "mult", 1e-10)
    h.iterate(3, "apg", 1e-3)
    h.iterate(0, "apg", 1e-3)
    V, W = h.factors()
    Va, Wa = oracle.nmf(X, V0, W0, 2, "mult", 1e-10)
    Vb, Wb = oracle.nmf(X, Va, Wa, 3, "apg", 1e-3)
    assert rel_l2(V, Vb) <= 2e-5 and rel_l2(W, Wb) <= 2e-5
    info = h.info()
    assert info["launches"] >= 6 * 5 and info["limb_cols"] == 32
    h.close()


def test_bad_inputs(N):
    from paper_2010_16114_gb300 import _lib as L
    X, V0, W0 = synth.nmf_inputs(64, 48, 4)
    Xn = X.copy()
    Xn[3, 7] = -0.5
    with pytest.raises(L.CoxError) as e:
        N(Xn, 4)
    assert e.value.code == L.COX_ERR_ARG
    Xn[3, 7] = np.nan
    with pytest.raises(L.CoxError):
        N(Xn, 4)
    h = N(X, 4)
    Vb = V0.copy()
    Vb[0, 0] = -1.0
    with pytest.raises(L.CoxError):
        h.set_factors(Vb, W0)
    with pytest.raises(L.CoxError):
        h.iterate(-1, "mult")
    with pytest.raises(L.CoxError):
        h.iterate(1, "mult", eps=-1.0)
    h.close()


def test_full_size_one_iteration(N):
    """The benchmark workload, X 10,000 x 10,000 and r = 20 (Section 5.1's GPU
    experiment), one iteration of each algorithm against the oracle on every
    entry, and the objective."""
    m = n = 10_000
    r = 20
    X, V0, W0 = synth.nmf_inputs(m, n, r)
    h = N(X, r)
    for algo in ("mult", "apg"):
        h.set_factors(V0, W0)
        h.iterate(1, algo)
        V, W = h.factors()
        Ve, We = oracle.nmf(X, V0, W0, 1, algo, 1e-10)
        assert max_rel(V, Ve, step_floor(algo, V0)) <= 2e-5
        assert max_rel(W, We, step_floor(algo, W0)) <= 2e-5
        fe = oracle.nmf_objective(X, Ve, We)
        assert abs(h.objective() - fe) <= 1e-5 * fe
    h.close()
