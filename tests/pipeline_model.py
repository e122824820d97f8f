"""A model of the genotype-product kernel's barrier protocol, for checking that
no mbarrier parity wait can return on a stale phase.

An mbarrier's parity wait for parity p returns as soon as the barrier's number
of completed phases P has parity 1 - p; a wait meant for the k-th completion
(p = k mod 2) is correct only when P = k + 1 at that moment, and *aliases* when
P = k - 1 (the completion two phases back has the same parity).  The model runs
the kernel's agents as atomic steps in every order a scheduler picks:

* the code producer (e2m1 form) loads stage j into code slot j mod S once the
  decoders released stage j - S; the limb producer likewise into limb slot
  j mod S2 once stage j - S2's MMAs are complete (released by the decoders of
  stage j - S2 + R); loads complete asynchronously, in any order;
* decoder group g takes stages g, g + G, ...: it waits for the code load, the
  limb load and the TMEM slot (the MMAs of stage i - R), releases the limbs of
  stage i - R, decodes, releases the code slot, and hands stage i to the issuer;
* the issuer (one; per-tile issuers behave alike for these barriers) issues the
  stages' MMAs in order; MMAs complete in the order they were issued and free
  their TMEM slot.  With alternating issuers (the e4m3 form's issue mode 2) two
  issuers take the even and the odd stages, each in order, and the tensor pipe
  completes the MMAs in the interleaved order they were issued.

The e4m3 form's single ring (one slot per stage holding codes and limbs,
released by the decoders of stage i + R after the MMAs of stage i) is modelled
too, with its two producer warps on alternate stages.  Named barriers (decoders
to issuer) are modelled as exact per-stage hand-offs.

`explore` checks every interleaving of a small pipeline exhaustively (memoised
on the state), `random_runs` samples long schedules with biased schedulers.
Both return the first aliasing wait found, or None.  Test infrastructure only.
"""
from __future__ import annotations

import random


class Model:
    def __init__(self, G: int, R: int, S: int, S2: int | None, N: int, inorder: bool = False,
                 from_stage: int = 0, issuers: int = 1, ordered_start: bool = False):
        """S2 = None: the e4m3 single ring of S stages; else the e2m1 rings.
        inorder: loads complete in stage order (else in any order).
        from_stage: aliasing waits of decoders at earlier stages are not reported.
        issuers: 1, or 2 on alternate stages.
        ordered_start: (single ring) each of the first S loads is issued only
        once the load before it has landed."""
        self.G, self.R, self.S, self.S2, self.N = G, R, S, S2, N
        self.split = S2 is not None
        self.inorder = inorder
        self.from_stage = from_stage
        self.I = issuers
        self.ordered_start = ordered_start

    # state: (prod, loads_pending, dec, iss, handed, queue, P) with
    #   prod = tuple of next stage per producer (split: codes, limbs; single: two warps)
    #   loads_pending = frozenset of (kind, stage) loads issued and not complete
    #   dec = tuple of (next stage, substep) per decoder group
    #   iss = tuple of the next stage per issuer; handed = frozenset of stages handed over
    #   queue = stages whose MMAs are issued and not complete, in issue order
    #   P = dict-like tuple of completed phases per barrier
    def initial(self):
        G, S, R = self.G, self.S, self.R
        S2 = self.S2 if self.split else 0
        prod = (0, 0) if self.split else (0, 1)
        dec = tuple((g, 0) for g in range(G))
        P = {"full": (0,) * S, "empty": (0,) * S, "aempty": (0,) * R, "lfull": (0,) * S2, "lempty": (0,) * S2}
        return (prod, frozenset(), dec, tuple(range(self.I)), frozenset(), (), tuple(sorted(P.items())))

    @staticmethod
    def _bump(P, name, idx):
        d = dict(P)
        t = list(d[name])
        t[idx] += 1
        d[name] = tuple(t)
        return tuple(sorted(d.items()))

    @staticmethod
    def _get(P, name, idx):
        return dict(P)[name][idx]

    def _wait(self, P, name, idx, k):
        """(returns, aliased) for a wait meant for the k-th completion (0-based)."""
        got = self._get(P, name, idx)
        returns = got % 2 == (k + 1) % 2
        return returns, returns and got != k + 1

    def moves(self, st):
        """Yield (label, next_state) for every enabled step, or raise on aliasing."""
        prod, pend, dec, issued, handed, done, P = st  # issued: per issuer; done: the MMA queue
        G, R, S, N = self.G, self.R, self.S, self.N
        out = []
        # producers
        if self.split:
            S2 = self.S2
            for w, (ring, empty, n) in enumerate((("full", "empty", S), ("lfull", "lempty", S2))):
                j = prod[w]
                if j < N:
                    ok, alias = (True, False) if j < n else self._wait(P, empty, j % n, j // n - 1)
                    if alias:
                        return None, ("producer", w, j)
                    if ok:
                        np_ = list(prod)
                        np_[w] = j + 1
                        out.append((("load", w, j), (tuple(np_), pend | {(w, j)}, dec, issued, handed, done, P)))
        else:
            for w in (0, 1):
                j = prod[w]
                if j < N:
                    ok, alias = (True, False) if j < S else self._wait(P, "empty", j % S, j // S - 1)
                    if alias:
                        return None, ("producer", w, j)
                    if ok and self.ordered_start and 1 <= j < S:
                        ok, alias = self._wait(P, "full", j - 1, 0)
                        if alias:
                            return None, ("producer start", w, j)
                    if ok:
                        np_ = list(prod)
                        np_[w] = j + 2
                        out.append((("load", w, j), (tuple(np_), pend | {(0, j)}, dec, issued, handed, done, P)))
        # load completions (any order, or the oldest of each kind)
        if self.inorder:
            first = {}
            for (kind, j) in pend:
                first[kind] = min(first.get(kind, j), j)
            pend_moves = [(kind, j) for kind, j in first.items()]
        else:
            pend_moves = list(pend)
        for (kind, j) in pend_moves:
            name, n = ("full", S) if kind == 0 else ("lfull", self.S2)
            out.append((("landed", kind, j), (prod, pend - {(kind, j)}, dec, issued, handed, done,
                                               self._bump(P, name, j % n))))
        # decoder groups
        for g in range(G):
            i, sub = dec[g]
            if i >= N:
                continue
            nd = list(dec)
            if sub == 0:
                ok, alias = self._wait(P, "full", i % S, i // S)
                if alias and i >= self.from_stage:
                    return None, ("decoder full", g, i)
                ok = ok and not alias
                if ok:
                    nd[g] = (i, 1 if self.split else 2)
                    out.append((("dfull", g, i), (prod, pend, tuple(nd), issued, handed, done, P)))
            elif sub == 1:
                ok, alias = self._wait(P, "lfull", i % self.S2, i // self.S2)
                if alias and i >= self.from_stage:
                    return None, ("decoder lfull", g, i)
                ok = ok and not alias
                if ok:
                    nd[g] = (i, 2)
                    out.append((("dlfull", g, i), (prod, pend, tuple(nd), issued, handed, done, P)))
            elif sub == 2:
                ok, alias = (True, False) if i < R else self._wait(P, "aempty", i % R, i // R - 1)
                if alias:
                    return None, ("decoder aempty", g, i)
                if ok:
                    P2 = P
                    if i >= R:
                        # the MMAs of stage i - R are complete: release what they read
                        if self.split:
                            P2 = self._bump(P2, "lempty", (i - R) % self.S2)
                        else:
                            P2 = self._bump(P2, "empty", (i - R) % S)
                    if self.split:
                        P2 = self._bump(P2, "empty", i % S)  # codes read: slot free
                    nd[g] = (i + G, 0)
                    out.append((("decode", g, i), (prod, pend, tuple(nd), issued, handed | {i}, done, P2)))
        # issuers, each in stage order over its stages
        for j, i in enumerate(issued):
            if i < N and i in handed:
                ni = list(issued)
                ni[j] = i + self.I
                out.append((("issue", i), (prod, pend, dec, tuple(ni), handed, done + (i,), P)))
        # MMA completion, in issue order
        if done:
            out.append((("mma", done[0]), (prod, pend, dec, issued, handed, done[1:],
                                           self._bump(P, "aempty", done[0] % R))))
        return out, None

    def finished(self, st):
        return all(i >= self.N for i in st[3]) and not st[5]


def explore(G, R, S, S2, N, limit=400_000, inorder=False, from_stage=0, issuers=1, ordered_start=False):
    """Every interleaving (memoised); returns the first aliasing wait, or None.
    Raises RuntimeError when the state space exceeds `limit` or a state deadlocks."""
    m = Model(G, R, S, S2, N, inorder, from_stage, issuers, ordered_start)
    seen = set()
    stack = [m.initial()]
    while stack:
        st = stack.pop()
        if st in seen:
            continue
        seen.add(st)
        if len(seen) > limit:
            raise RuntimeError("state space beyond the limit")
        mv, bad = m.moves(st)
        if bad is not None:
            return bad
        if not mv:
            if not m.finished(st):
                raise RuntimeError(f"deadlock in state {st}")
            continue
        for _, nxt in mv:
            if nxt not in seen:
                stack.append(nxt)
    return None


def random_runs(G, R, S, S2, N, runs=300, seed=1, inorder=False, from_stage=0, issuers=1,
                ordered_start=False):
    """Random schedules, each biased towards one agent kind (so decoder groups
    race ahead of late loads, or loads of late MMAs); returns the first aliasing
    wait, or None."""
    m = Model(G, R, S, S2, N, inorder, from_stage, issuers, ordered_start)
    rng = random.Random(seed)
    kinds = ["load", "landed", "dfull", "dlfull", "decode", "issue", "mma"]
    for _ in range(runs):
        favour = {k: rng.choice([0.05, 1.0, 20.0]) for k in kinds}
        lead = rng.randrange(G)
        st = m.initial()
        while not m.finished(st):
            mv, bad = m.moves(st)
            if bad is not None:
                return bad
            if not mv:
                raise RuntimeError(f"deadlock in state {st}")
            w = [favour[lbl[0]] * (5.0 if lbl[0] in ("dfull", "dlfull", "decode") and lbl[1] == lead else 1.0)
                 for lbl, _ in mv]
            st = rng.choices([n for _, n in mv], weights=w)[0]
    return None
