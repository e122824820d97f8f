"""Host-side plans of the tensor-core products (cox_plan_shape, no GPU): for
every k and every compiled shape and depth, the plan keeps the pipeline's
invariants, which the kernel's hand-offs rely on:

* parity waits are unambiguous only when the phase before the awaited one is
  known to be complete; the hand-off chains guarantee that when ring >= decoder
  groups (TMEM-slot waits), when stages >= groups + ring or either is a multiple
  of the groups (shared-memory-stage waits), and when stages are even or
  >= ring + 2 (the two producer warps' release waits);
* ring < stages: the producer of stage i waits for the decoders of stage
  i - S + ring, who must not be waiting for that producer;
* lcm(groups, ring) x tiles <= 15 hardware named barriers (0 is __syncthreads);
* accumulators + slots <= 512 TMEM columns; shared memory within 227 KB and at
  least 120 KB (one CTA per SM owns all of TMEM).

With two issuers on alternate stages (issue 2) the stages of each parity form a
chain of their own, which needs two decoder groups, an even ring and an even
number of stages; each issuer holds an accumulator per row tile.
"""
import math

import pytest

from paper_2010_16114_gb300 import _lib as L

SHAPES = [(t, c, a) for a in (1, 2, 3) for t in (2, 1) for c in (3, 2, 1)]


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2010_16114_gb300 import build
    build()
    return L.load()


def _parity_safe(G, R, S):
    """The kernel's conditions for unambiguous parity waits: TMEM-slot waits
    need G <= R; shared-memory-stage waits need S >= G + R, S a multiple of G
    or R a multiple of G; the two producer warps' release waits need S even or
    S >= R + 2."""
    return G <= R and (S >= G + R or S % G == 0 or R % G == 0) and (S % 2 == 0 or S >= R + 2)


def _limb_cols(k):
    n = 4 * k
    return next(c for c in (16, 32, 64, 128, 256) if n <= c)


def _groups(t, c, a, np_cls):
    """Decoder groups: two for alternating issuers, for 2 tiles x 2 chunks at
    128 limb columns and 2 tiles x 3 chunks at 64 (no room for a third TMEM
    slot), else three."""
    return 2 if a == 2 or (t, c, np_cls) in ((2, 2, 128), (2, 3, 64)) else 3


def _some_safe_ring(t, c, a, np_cls, S):
    """Whether any TMEM ring the plan could take meets the parity rule at depth S."""
    G = _groups(t, c, a, np_cls)
    acc = (2 * t if a == 2 else t) * np_cls
    rmax = min(8, (512 - acc) // (t * c * 32), S - 1)
    for R in range(G, rmax + 1):
        if math.lcm(G, R) * t > 15:
            continue
        ok = (R % 2 == 0 and S % 2 == 0) if a == 2 else _parity_safe(G, R, S)
        if ok:
            return True
    return False


def _check(k, p):
    assert p.limb_cols >= 4 * k and p.limb_cols in (16, 32, 64, 128, 256)
    assert p.ring >= p.decoder_groups
    assert p.ring < p.stages
    assert p.stages >= p.decoder_groups + 1
    assert p.named_barriers == math.lcm(p.decoder_groups, p.ring) * p.tile_m <= 15
    if p.issue == 2:
        assert p.decoder_groups == 2 and p.ring % 2 == 0 and p.stages % 2 == 0
        assert p.issuers == 2 and p.mmas_per_commit == 4 * p.chunks * p.tile_m
        acc = 2 * p.tile_m * p.limb_cols
    else:
        assert p.issue in (1, 3)
        assert _parity_safe(p.decoder_groups, p.ring, p.stages)
        assert p.issuers == p.tile_m and p.mmas_per_commit == 4 * p.chunks * (2 if p.issue == 3 else 1)
        acc = p.tile_m * p.limb_cols
    assert p.tmem_cols == acc + p.ring * p.tile_m * p.chunks * 32 <= 512
    assert 120 * 1024 <= p.smem_bytes <= 227 * 1024


@pytest.mark.parametrize("k", range(1, 65))
def test_every_shape_and_depth_keeps_the_invariants(k):
    compiled = 0
    for t, c, a in SHAPES:
        rc, p = L.cox_plan_shape(k, t, c, 0, a)
        if rc != 0:
            assert rc == L.COX_ERR_ARG
            continue
        compiled += 1
        assert (p.tile_m, p.chunks, p.issue) == (t, c, a)
        _check(k, p)
        deepest = p.stages
        for s in range(1, 16):
            rc, q = L.cox_plan_shape(k, t, c, s, a)
            want = min(max(s, q.decoder_groups + 1 if rc == 0 else s), 12)  # the planner caps the depth at 12
            if rc != 0:
                # refused only beyond the shared-memory budget, or at a depth where no
                # ring meets the parity rule (an odd depth for alternating issuers)
                S = min(max(s, _groups(t, c, a, _limb_cols(k)) + 1), 12)
                assert rc == L.COX_ERR_ARG and (s > deepest or not _some_safe_ring(t, c, a, _limb_cols(k), S))
                continue
            _check(k, q)
            assert q.stages == want
    assert compiled >= 1


@pytest.mark.parametrize("k", [1, 4, 5, 8, 9, 16, 17, 32, 33, 64])
def test_default_shape(k):
    rc, p = L.cox_plan_shape(k)
    assert rc == 0
    _check(k, p)
    # the built-in default: two row tiles up to 128 limb columns, two K chunks up to 64
    assert p.tile_m == (2 if p.limb_cols <= 128 else 1)
    assert p.chunks == (2 if p.limb_cols <= 64 else 1)


def test_widest_limb_class_keeps_a_safe_ring():
    """256 limb columns (k > 32) fit five stages; four slots would leave the
    shared-memory waits without a guarantee (5 < 3 + 4, neither a multiple of
    3, 5 odd and < 4 + 2), so the planner takes three."""
    rc, p = L.cox_plan_shape(64)
    assert rc == 0 and (p.tile_m, p.chunks, p.stages, p.ring) == (1, 1, 5, 3)
    assert not _parity_safe(3, 4, 5) and _parity_safe(3, 3, 5)


def test_rejections():
    assert L.cox_plan_shape(0)[0] == L.COX_ERR_ARG
    assert L.cox_plan_shape(65)[0] == L.COX_ERR_ARG
    assert L.cox_plan_shape(16, 3, 0)[0] == L.COX_ERR_ARG      # three row tiles: not compiled
    assert L.cox_plan_shape(32, 0, 3)[0] == L.COX_ERR_ARG      # three K chunks: only at 64 limb columns
    assert L.cox_plan_shape(16, 1, 3)[0] == L.COX_ERR_ARG      # three K chunks: only with two row tiles
    assert L.cox_plan_shape(64, 2, 2)[0] == L.COX_ERR_ARG      # 256 limb columns take one tile, one chunk
    assert L.cox_plan_shape(16, -1, 0)[0] == L.COX_ERR_ARG
    assert L.load().cox_plan_shape(16, 0, 0, 0, 0, None) == L.COX_ERR_ARG
    assert L.cox_plan_shape(16, 2, 1, 0, 2)[0] == L.COX_ERR_ARG   # alternating issuers: not compiled for (2, 1)
    assert L.cox_plan_shape(16, 2, 2, 5, 2)[0] == L.COX_ERR_ARG   # alternating issuers need an even depth
    assert L.cox_plan_shape(16, 0, 0, 0, 4)[0] == L.COX_ERR_ARG


def test_front_end_wrapper():
    from paper_2010_16114_gb300.cox import plan_shape
    d = plan_shape(16)
    assert (d["tile_m"], d["chunks"], d["stages"], d["ring"], d["limb_cols"]) == (2, 2, 6, 3, 64)
    with pytest.raises(L.CoxError):
        plan_shape(32, chunks=3)


def test_alternating_issuers_plan():
    """k = 16 (64 limb columns) with two issuers on alternate stages: two row
    tiles x two K chunks per stage, 16 MMAs per commit, accumulators of 2 x 2 x 64
    columns and two 128-column slots fill TMEM, and six 32 KB stages."""
    rc, p = L.cox_plan_shape(16, 2, 2, 0, 2)
    assert rc == 0
    _check(16, p)
    assert (p.issuers, p.decoder_groups, p.ring, p.stages, p.mmas_per_commit, p.tmem_cols) == (2, 2, 2, 6, 16, 512)
    assert p.named_barriers == 4


def test_two_group_shape_at_128_limb_columns():
    """k = 17..32 (128 limb columns) with 2 row tiles x 2 K chunks: 256
    accumulator columns leave room for two 128-column slots only, so the shape
    runs two decoder groups (R = G = 2); at three stages no ring meets the
    shared-memory waits' rule (3 < 2 + 2, 3 odd), so the planner takes four
    stages (227 KB); 8 MMAs per commit per issuer.  Pair commits are not planned
    for it."""
    for k in (17, 32):
        rc, p = L.cox_plan_shape(k, 2, 2, 0, 1)
        assert rc == 0
        _check(k, p)
        assert (p.decoder_groups, p.ring, p.stages, p.named_barriers, p.tmem_cols, p.mmas_per_commit) == \
            (2, 2, 4, 4, 512, 8)
        assert not _parity_safe(2, 2, 3) and _parity_safe(2, 2, 4)
        assert L.cox_plan_shape(k, 2, 2, 3, 1)[0] == L.COX_ERR_ARG
        assert L.cox_plan_shape(k, 2, 2, 0, 3)[0] == L.COX_ERR_ARG


def test_two_group_shape_with_three_chunks():
    """k = 9..16 (64 limb columns) with 2 row tiles x 3 K chunks: 128
    accumulator columns and two 192-column slots fill TMEM, so two decoder
    groups (R = G = 2); 12 MMAs per commit per issuer; four 48 KB stages."""
    for k in (9, 16):
        rc, p = L.cox_plan_shape(k, 2, 3, 0, 1)
        assert rc == 0
        _check(k, p)
        assert (p.decoder_groups, p.ring, p.stages, p.named_barriers, p.tmem_cols, p.mmas_per_commit) == \
            (2, 2, 4, 4, 512, 12)
        assert L.cox_plan_shape(k, 2, 3, 0, 3)[0] == L.COX_ERR_ARG


# ---- the e2m1 operand form (COX_SPLIT_E2M1) ------------------------------------------

SHAPES4 = [(2, 2), (2, 4), (1, 2), (1, 4)]


def _limb_cols4(k):
    n = 8 * k
    return next(c for c in (64, 128) if n <= c)


def _check4(k, p):
    """e2m1 plans: eight limbs per coefficient in 64 or 128 columns;
    per-tile issuers, two MMAs (K = 64) per K chunk; 16 TMEM columns per tile
    and chunk beside 8 columns of scale factors.  Two shared-memory rings, each
    with one producer that reuses a slot only after its release: code slots
    (`stages`, at least G + 1) and limb slots (`limb_stages`, ring + 1 .. ring +
    3); a decoder group's parity wait on either ring is unambiguous when the
    ring's depth is at least G + ring or a multiple of G."""
    assert p.limb_cols == _limb_cols4(k)
    assert p.issue == 1 and p.issuers == p.tile_m and p.mmas_per_commit == 2 * p.chunks
    assert p.decoder_groups == 3 and p.chunks % 2 == 0
    G, R = p.decoder_groups, p.ring
    assert R >= G and R + 1 <= p.limb_stages <= R + 4
    for depth in (p.stages, p.limb_stages):
        assert depth >= G + R or depth % G == 0, (depth, G, R)
    assert p.stages >= p.decoder_groups + 1
    assert p.named_barriers == math.lcm(p.decoder_groups, p.ring) * p.tile_m <= 15
    assert p.tmem_cols == p.tile_m * p.limb_cols + p.ring * p.tile_m * p.chunks * 16 + 8 <= 512
    fold = p.tile_m * (p.limb_cols // 8) * 128 * 4 + 4 * (p.limb_cols // 8) * 4
    code_slot, limb_slot = p.tile_m * p.chunks * 4096, (p.chunks // 2) * p.limb_cols * 128
    assert p.smem_bytes == max(120 * 1024, p.stages * code_slot + p.limb_stages * limb_slot + 2048 + fold)
    assert p.smem_bytes <= 227 * 1024


@pytest.mark.parametrize("k", range(1, 17))
def test_e2m1_every_shape_and_depth_keeps_the_invariants(k):
    compiled = 0
    for t, c in SHAPES4:
        rc, p = L.cox_plan_shape_prec(L.COX_SPLIT_E2M1, k, t, c, 0, 1)
        if rc != 0:
            assert rc == L.COX_ERR_ARG
            continue
        compiled += 1
        assert (p.tile_m, p.chunks) == (t, c)
        _check4(k, p)
        for s in range(1, 16):
            rc, q = L.cox_plan_shape_prec(L.COX_SPLIT_E2M1, k, t, c, s, 1)
            want = max(s, p.decoder_groups + 1)
            if rc != 0:
                # refused only at a depth the parity rule forbids, or beyond 227 KB
                assert rc == L.COX_ERR_ARG
                unsafe = not (want >= p.decoder_groups + p.ring or want % p.decoder_groups == 0)
                assert unsafe or want > p.stages, (k, t, c, s)
                continue
            _check4(k, q)
            assert q.stages == want
    assert compiled >= 1


def test_e2m1_default_shapes_and_rejections():
    # two row tiles x two K chunks (k <= 16)
    for k, want in ((1, (2, 2, 64)), (8, (2, 2, 64)), (9, (2, 2, 128)), (16, (2, 2, 128))):
        rc, p = L.cox_plan_shape_prec(L.COX_SPLIT_E2M1, k, 0, 0, 0, 0)
        assert rc == 0
        _check4(k, p)
        assert (p.tile_m, p.chunks, p.limb_cols) == want
    E = L.COX_SPLIT_E2M1
    assert L.cox_plan_shape_prec(E, 17)[0] == L.COX_ERR_ARG          # 128 columns hold 16 coefficients
    assert L.cox_plan_shape_prec(E, 32)[0] == L.COX_ERR_ARG
    assert L.cox_plan_shape_prec(E, 16, 2, 1)[0] == L.COX_ERR_ARG    # chunk pairs only
    assert L.cox_plan_shape_prec(E, 16, 2, 3)[0] == L.COX_ERR_ARG
    assert L.cox_plan_shape_prec(E, 16, 2, 2, 0, 2)[0] == L.COX_ERR_ARG  # per-tile issuers only
    assert L.cox_plan_shape_prec(E, 16, 2, 2, 0, 3)[0] == L.COX_ERR_ARG
    assert L.cox_plan_shape_prec(E, 16, 2, 4)[0] == L.COX_ERR_ARG    # 2 x 4: not compiled
    assert L.cox_plan_shape_prec(E, 16, 1, 4)[0] == L.COX_ERR_ARG    # 1 x 4 at 128 columns: no safe depths fit
    assert L.cox_plan_shape_prec(E, 8, 1, 4)[0] == 0
    assert L.cox_plan_shape_prec(7, 16)[0] == L.COX_ERR_ARG          # not a tensor-core form
    # the e4m3 entry point is the e4m3 form of the general one
    for k in (1, 16, 64):
        a, b = L.cox_plan_shape(k)[1], L.cox_plan_shape_prec(L.COX_SPLIT_E4M3, k)[1]
        assert [getattr(a, f) for f, _ in L.cox_plan._fields_] == [getattr(b, f) for f, _ in L.cox_plan._fields_]
