"""The tensor-core products' barrier protocol in a model (pipeline_model.py), on
CPU: which plans the library launches could let an mbarrier parity wait return
on a stale phase, over every order the asynchronous loads and MMAs complete in
and every schedule of the warps.

* e2m1 form (a ring of code slots released after decoding, one of limb slots
  released after the MMAs): every plan of every k and shape is safe in any order.
* The depths its planner refuses (a code ring of 5, or a limb ring of 5, at three
  decoder groups and three TMEM slots) do alias; a build that planned a code ring
  of 5 faulted on the GPU.
* e4m3 form (one ring; one issuer per tile or two on alternate stages): the
  plans whose depth is at least G + R or a multiple of G are safe in any order.  The plans that rely on the TMEM ring being a multiple of
  G instead (one row tile at 64, 128 and 256 limb columns) are safe once the first
  S loads have landed; before that, a load of the first S stages that lands after
  later ones could let a decoder group's wait on its slot's second phase return
  early.  The model shows exactly that window and nothing past it.
"""
import pytest

from paper_2010_16114_gb300 import _lib as L
from pipeline_model import explore, random_runs

RUNS, N = 150, 36


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2010_16114_gb300 import build
    build()
    return L.load()


def _e2m1_plans():
    out = set()
    for k in range(1, 17):
        for t, c in ((2, 2), (1, 4)):
            rc, p = L.cox_plan_shape_prec(L.COX_SPLIT_E2M1, k, t, c, 0, 1)
            if rc == 0:
                out.add((p.decoder_groups, p.ring, p.stages, p.limb_stages))
    return sorted(out)


def _e4m3_plans():
    out = set()
    for k in range(1, 65):
        for t in (2, 1):
            for c in (3, 2, 1):
                for issue in (1, 3):  # per-tile issuers (pair commits share the protocol)
                    rc, p = L.cox_plan_shape(k, t, c, 0, issue)
                    if rc == 0:
                        out.add((p.decoder_groups, p.ring, p.stages))
    return sorted(out)


def test_e2m1_plans_never_alias():
    plans = _e2m1_plans()
    assert plans
    for G, R, S, S2 in plans:
        assert random_runs(G, R, S, S2, N, runs=RUNS, seed=11) is None, (G, R, S, S2)


def test_refused_e2m1_depths_alias():
    # the code ring of 5 that faulted on the GPU, and a limb ring of R + 2 = 5
    assert random_runs(3, 3, 5, 7, N, runs=RUNS, seed=11) is not None
    assert random_runs(3, 3, 7, 5, N, runs=RUNS, seed=11) is not None
    # exhaustively on a short pipeline as well
    assert explore(3, 3, 5, 7, N=14, limit=400_000) is not None
    # ... and neither aliases when every load lands in stage order
    assert random_runs(3, 3, 5, 7, N, runs=RUNS, seed=11, inorder=True) is None


def test_e4m3_plans():
    plans = _e4m3_plans()
    assert plans
    startup_only = []
    for G, R, S in plans:
        if S >= G + R or S % G == 0:
            assert random_runs(G, R, S, None, N, runs=RUNS, seed=11) is None, (G, R, S)
        else:
            assert R % G == 0, (G, R, S)  # the planner's third condition
            startup_only.append((G, R, S))
            assert random_runs(G, R, S, None, N, runs=RUNS, seed=11) is not None, (G, R, S)
            assert random_runs(G, R, S, None, N, runs=RUNS, seed=11, from_stage=S + G) is None, (G, R, S)
            assert random_runs(G, R, S, None, N, runs=RUNS, seed=11, inorder=True) is None, (G, R, S)
    assert sorted(startup_only) == [(3, 3, 5), (3, 6, 8)]


def test_single_ring_exhaustive_small():
    # every interleaving of a short pipeline: a depth meeting the first two
    # conditions never aliases
    assert explore(3, 3, 6, None, N=15, limit=400_000) is None
    assert explore(2, 2, 4, None, N=12, limit=400_000) is None


def test_alternating_issuer_plans():
    """e4m3 issue mode 2 (two issuers on alternate stages, two decoder groups):
    every plan is safe in any order; an odd ring of stages (which the planner
    refuses) aliases."""
    plans = set()
    for k in range(1, 65):
        for t in (2, 1):
            for c in (3, 2, 1):
                rc, p = L.cox_plan_shape(k, t, c, 0, 2)
                if rc == 0:
                    plans.add((p.decoder_groups, p.ring, p.stages))
    assert plans
    for G, R, S in sorted(plans):
        assert random_runs(G, R, S, None, N, runs=RUNS, seed=11, issuers=2) is None, (G, R, S)
        assert explore(G, R, S, None, N=12, limit=400_000, issuers=2) is None, (G, R, S)
    assert random_runs(2, 2, 5, None, N, runs=RUNS, seed=11, issuers=2) is not None


def test_ordered_start_closes_the_window_where_it_is_needed():
    """The fix for the start-up window of the third condition: each of the first S
    loads issued only once the load before it has landed.  For the plans that
    need it the model finds neither an aliasing wait nor a deadlock, in any load
    order; applied to a two-group ring of 4 it can deadlock (a producer warp that
    is late to look at the previous slot finds it already refilled by the other
    warp), so the fix belongs to those plans only."""
    for G, R, S in ((3, 3, 5), (3, 6, 8)):
        assert random_runs(G, R, S, None, N, runs=RUNS, seed=11, ordered_start=True) is None, (G, R, S)
        assert explore(G, R, S, None, N=2 * S + 3, limit=600_000, ordered_start=True) is None, (G, R, S)
    with pytest.raises(RuntimeError, match="deadlock"):
        for seed in range(1, 6):
            random_runs(2, 2, 4, None, N, runs=RUNS, seed=seed, ordered_start=True)
