"""CPU models of the strip kernels' data movement (no GPU): the strip and warp-run geometry
with the TMA copy rules, and the full/empty mbarrier row ring under random interleavings.

Both models restate, in plain integer arithmetic, what `csrc/step_pair.cuh` and
`csrc/ring.cuh` do: `warp_strip_width`, the copies of `issue_row` (a row of a strip plus
4 halo columns each side, in three pieces at the periodic x edges), the 60-column warp runs,
the columns `pull_pair` reads, and the ring protocol of `ring_produce` and the consumer loops
of `fe_step_pair` / `pp_pair_strip` with the parity semantics of `mbarrier.try_wait.parity`
(a wait on parity p returns once the barrier's current phase parity differs from p).
"""
import random

import pytest

NW, TXW, S = 4, 60, 6
TX = NW * TXW          # widest strip
W8 = TX + 8            # staged row width


def strip_width(nx, gx):
    return ((nx + gx - 1) // gx + 3) & ~3


def copies(nx, x0, w):
    """Source column ranges [a, b) of one staged row, in stage order (issue_row)."""
    if x0 >= 4 and x0 + w + 4 <= nx:
        return [(x0 - 4, x0 + w + 4)]
    xl = x0 - 4 if x0 >= 4 else nx - 4
    xr = x0 + w if x0 + w < nx else 0
    return [(xl, xl + 4), (x0, x0 + w), (xr, xr + 4)]


def test_strip_geometry_and_tma_rules_for_every_width():
    """For every nx = 8, 12, ..., 19996: the strips tile [0, nx) exactly, fit the 240-column
    ring, start and span multiples of 4 columns (16-byte TMA rule); every copy lies inside the
    row and lands the periodic neighbours in order; the warps' 60-column runs tile each strip
    (runs even, idle warps only beyond the strip); every staged column a lane reads lies inside
    the copied part of the stage."""
    for nx in range(8, 20000, 4):
        gx = (nx + TX - 1) // TX
        wb = strip_width(nx, gx)
        assert wb <= TX and wb % 4 == 0
        covered = 0
        for b in range(gx):
            x0 = b * wb
            w = min(wb, nx - x0)
            if w <= 0:
                continue
            assert x0 == covered and x0 % 4 == 0 and w % 4 == 0
            covered += w
            # copies: in bounds, 16-byte aligned, and staged column s holds source column
            # (x0 - 4 + s) mod nx
            staged = []
            for a, e in copies(nx, x0, w):
                assert 0 <= a < e <= nx and a % 4 == 0 and (e - a) % 4 == 0
                staged += list(range(a, e))
            assert staged == [(x0 - 4 + s) % nx for s in range(w + 8)]
            # warp runs
            nwa = min(NW, (w + 59) // 60)
            runs = []
            for warp in range(nwa):
                cw = warp * 60
                nw = min(60, w - cw)
                assert nw > 0 and nw % 2 == 0
                runs += list(range(cw, cw + nw))
                for lane in range(32):
                    if not 2 * lane <= nw + 2:  # act
                        continue
                    sc = cw - 2 + 2 * lane + 4
                    # pull_pair reads staged columns sc - 1 .. sc + 2 of rows q-1, q, q+1
                    assert 0 <= sc - 1 and sc + 2 < w + 8 <= W8
            assert runs == list(range(w))
        assert covered == nx


class Barrier:
    """An mbarrier: arrivals and expected transaction bytes; phase completes at zero pending."""

    def __init__(self, count):
        self.count = count
        self.pending = count
        self.tx = 0
        self.phase = 0

    def _maybe_complete(self):
        if self.pending == 0 and self.tx == 0:
            self.phase += 1
            self.pending = self.count

    def arrive(self):
        assert self.pending > 0
        self.pending -= 1
        self._maybe_complete()

    def arrive_expect_tx(self, nbytes):
        self.tx += nbytes
        self.arrive()

    def complete_tx(self, nbytes):
        self.tx -= nbytes
        assert self.tx >= 0
        self._maybe_complete()

    def try_wait_parity(self, p):
        return (self.phase & 1) != p


def simulate(model, nsrc, nwa, seed, max_events=200000):
    """Random interleaving of the producer, the copies in flight and nwa consumer warps.
    Returns the rows each consumer read from each stage; raises on a stale read or deadlock."""
    rng = random.Random(seed)
    full = [Barrier(1) for _ in range(S)]
    empty = [Barrier(nwa) for _ in range(S)]
    content = [None] * S    # ring index whose data sits in the stage (landed)
    in_flight = []          # (stage, ring index)
    # producer program counter
    prod = {"k": 0}
    # consumer state: FE iterates k = 2 .. nsrc-1, reads k-2..k and (k >= 6) k-4..k-2, releases
    # k-4; P iterates k = 2 .. nsrc-1, reads k-2..k and (k >= 4) k-3..k-1, releases k-3
    lag = 4 if model == "fe" else 3
    collide_from = 6 if model == "fe" else 4
    cons = [{"k": 2, "pre": 0} for _ in range(nwa)]

    def producer_enabled():
        k = prod["k"]
        if k >= nsrc:
            return False
        if k < S:
            return True
        return empty[k % S].try_wait_parity(((k // S) - 1) & 1)

    def producer_step():
        k = prod["k"]
        s = k % S
        full[s].arrive_expect_tx(1)
        in_flight.append((s, k))
        prod["k"] = k + 1

    def consumer_enabled(c):
        if c["pre"] < 2:  # the two waits before the loop: stages 0 and 1, parity 0
            return full[c["pre"]].try_wait_parity(0)
        k = c["k"]
        if k > nsrc - 1:
            return False
        return full[k % S].try_wait_parity((k // S) & 1)

    def read(j):
        assert content[j % S] == j, f"stale read: stage {j % S} holds {content[j % S]}, expected {j}"

    def consumer_step(c):
        if c["pre"] < 2:
            c["pre"] += 1
            return
        k = c["k"]
        for j in (k - 2, k - 1, k):
            read(j)
        if k >= collide_from:
            for j in range(k - lag, k - lag + 3):
                read(j)
        if k >= lag:
            empty[(k - lag) % S].arrive()
        c["k"] = k + 1

    for _ in range(max_events):
        actions = []
        if producer_enabled():
            actions.append(("p", None))
        for i, (s, j) in enumerate(in_flight):
            actions.append(("copy", i))
        for i, c in enumerate(cons):
            if consumer_enabled(c):
                actions.append(("c", i))
        if not actions:
            done = prod["k"] == nsrc and all(c["k"] == nsrc for c in cons) and not in_flight
            assert done, f"deadlock: producer k={prod['k']}, consumers {[c['k'] for c in cons]}"
            return
        kind, i = rng.choice(actions)
        if kind == "p":
            producer_step()
        elif kind == "copy":
            s, j = in_flight.pop(i)
            content[s] = j
            full[s].complete_tx(1)
        else:
            consumer_step(cons[i])
    raise AssertionError("no progress bound reached")


@pytest.mark.parametrize("model", ["fe", "pp"])
@pytest.mark.parametrize("nwa", [1, 2, 4])
def test_ring_protocol_random_interleavings(model, nwa):
    """Every staged row a consumer warp reads is the row it expects and has landed (no stale or
    overwritten stage), and every run ends (no deadlock), under 60 random schedules each of
    short and long strips (6-stage ring; release lag 4 for FE, 3 for P)."""
    rows_of = {"fe": lambda r: r + 6, "pp": lambda r: r + 4}
    for seed in range(60):
        for rows in (1, 2, 5, 16, 41):
            simulate(model, rows_of[model](rows), nwa, seed * 1000 + rows)


def test_ring_model_detects_a_short_ring():
    """The model is not vacuous: with the free-energy release lag (4) a 4-stage ring lets the
    producer overwrite a stage a warp still has to re-read."""
    global S
    old = S
    try:
        S = 4
        with pytest.raises(AssertionError):
            for seed in range(200):
                simulate("fe", 20, 2, seed)
    finally:
        S = old
