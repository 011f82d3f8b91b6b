"""The streaming sweep kernel's schedule, checked on the host.

The kernel (launch configurations 10 and 12) runs n_half half-sweeps in one
launch.  Item n is (half-sweep h, position k, group bx of a slice's tiles),
and half-sweep h visits slice t = (h S + k) mod nt at position k.
Configuration 10 numbers the items half-sweep after half-sweep,
n = (h * nt + k) * items_x + bx with S = 1 (items_x is called tiles_x below:
the model does not look inside an item); configuration 12 numbers the (h, k)
pairs in a rolling band, wave D h + k first and h second (the kernel's
stream_band_rank, restated here), with 1 <= S <= D - 1.  A block takes tickets in order; it looks once, without
waiting, whether its next item's slices are ready (the previous half-sweep has
finished slices t - 1, t, t + 1: done[t'] >= h * items_x) and stages it if so;
otherwise it waits for them only after finishing its current item.  This model replays that protocol with random
interleavings of the blocks and checks what the kernel relies on: every item
runs once; an item starts only after every item of the previous half-sweep on
its own and the neighbouring slices has finished; two items in flight at the
same time never touch the same links (a site of slice t touches links stored in
slices t and t - 1); and the launch never deadlocks, whatever the number of
blocks.
"""
import random

import pytest


def band_rank(h, k, nt, n_half, D):
    """Slot of (h, k) in the rolling band: pairs of earlier waves (wave D j + k'),
    then those of the same wave with smaller h."""
    w = D * h + k
    r = 0
    for j in range(n_half):
        c = w - D * j
        r += min(max(c, 0), nt)
        if j < h and c < nt:
            r += 1
    return r


class Order:
    """Ticket <-> (h, slice, group) of one launch: half-sweep after half-sweep
    (D None, S 1: configuration 10) or the rolling band (D, S: configuration 12)."""

    def __init__(self, nt, tiles_x, n_half, D=None, S=1):
        self.nt, self.tiles_x, self.n_half, self.S = nt, tiles_x, n_half, S
        if D is None:
            self.pairs = [(h, k) for h in range(n_half) for k in range(nt)]
        else:
            self.pairs = [None] * (nt * n_half)
            for h in range(n_half):
                for k in range(nt):
                    self.pairs[band_rank(h, k, nt, n_half, D)] = (h, k)
        self.slot = {}
        for i, (h, k) in enumerate(self.pairs):
            self.slot[(h, (h * S + k) % nt)] = i

    def item(self, n):
        h, k = self.pairs[n // self.tiles_x]
        return h, (h * self.S + k) % self.nt, n % self.tiles_x

    def ticket(self, h, t, bx):
        return self.slot[(h, t)] * self.tiles_x + bx


def item(n, tiles_x, nt):
    """Configuration 10's numbering in closed form."""
    per_half = tiles_x * nt
    h = n // per_half
    r = n - h * per_half
    k = r // tiles_x
    return h, (h % nt + k) % nt, r - k * tiles_x


def ready(done, h, t, tiles_x, nt):
    if h == 0:
        return True
    need = h * tiles_x
    return all(done[(t + d) % nt] >= need for d in (-1, 0, 1))


def run(nt, tiles_x, n_half, nblocks, seed, ready=ready, order=None):
    """Replays the blocks' protocol; returns the number of waits that found the
    slices not ready.  `ready` is the dependency rule (the kernel's by default);
    `order` the launch's numbering (configuration 10's by default)."""
    order = order or Order(nt, tiles_x, n_half)
    rng = random.Random(seed)
    total = tiles_x * nt * n_half
    done = [0] * nt
    finished = set()
    ticket = [0]
    in_flight = {}  # item -> (h, t)
    waits = 0

    def take():
        n = ticket[0]
        ticket[0] += 1
        staged = n < total and ready(done, *order.item(n)[:2], tiles_x, nt)
        return n, staged

    # a block: [state, cur, cur_staged, nxt, nxt_staged]
    blocks = []
    for _ in range(nblocks):
        n, st = take()
        blocks.append(["take", n, st, None, None])
    steps = 0
    while True:
        live = [b for b in blocks if b[1] < total]
        if not live:
            break
        movable = []
        for b in live:
            if b[0] == "start" and not b[2]:
                h, t, _ = order.item(b[1])
                if not ready(done, h, t, tiles_x, nt):
                    continue  # waiting
            movable.append(b)
        assert movable, "deadlock: every live block waits"
        b = rng.choice(movable)
        steps += 1
        assert steps < 100 * total + 1000
        if b[0] == "take":  # the next ticket, looked at once
            b[3], b[4] = take()
            b[0] = "start"
        elif b[0] == "start":
            h, t, bx = order.item(b[1])
            if not b[2]:
                waits += 1
            # an item starts only after the previous half-sweep finished t - 1, t, t + 1
            if h > 0:
                for d in (-1, 0, 1):
                    tt = (t + d) % nt
                    for x in range(tiles_x):
                        n_prev = order.ticket(h - 1, tt, x)
                        assert n_prev < b[1] and n_prev in finished
            # no two items in flight touch the same links
            mine = {t, (t - 1) % nt}
            for (h2, t2) in in_flight.values():
                if h2 != h:
                    assert not (mine & {t2, (t2 - 1) % nt}), (h, t, h2, t2)
            in_flight[b[1]] = (h, t)
            b[0] = "finish"
        else:  # finish: publish, move on to the taken ticket
            h, t = in_flight.pop(b[1])
            finished.add(b[1])
            done[t] += 1
            b[1], b[2] = b[3], b[4]
            b[0] = "take"
    assert finished == set(range(total))
    assert done == [tiles_x * n_half] * nt
    return waits


@pytest.mark.parametrize("nt,tiles_x,n_half,nblocks", [
    (2, 3, 5, 4), (4, 1, 7, 3), (6, 2, 6, 1), (8, 4, 9, 16), (12, 4, 20, 7), (32, 3, 6, 40)])
def test_schedule_is_race_free_and_terminates(nt, tiles_x, n_half, nblocks):
    for seed in range(6):
        run(nt, tiles_x, n_half, nblocks, seed)


def test_item_order_covers_every_tile_once():
    nt, tiles_x, n_half = 5, 3, 4
    seen = [item(n, tiles_x, nt) for n in range(nt * tiles_x * n_half)]
    assert len(set(seen)) == len(seen)
    for h in range(n_half):  # each half-sweep visits every slice, starting at slice h mod nt
        row = seen[h * nt * tiles_x:(h + 1) * nt * tiles_x]
        assert sorted((t, bx) for _, t, bx in row) == [(t, x) for t in range(nt) for x in range(tiles_x)]
        assert row[0][1] == h % nt


def test_skew_keeps_a_single_block_from_waiting():
    """One block takes every ticket in order: with the slice order shifted by one
    per half-sweep its next item is always ready when it looks (no waits), where
    an unshifted order would have to wait at every half-sweep boundary."""
    assert run(16, 4, 10, 1, 0) == 0


def test_a_weaker_rule_is_caught():
    """The model has teeth: waiting for the item's own slice only (not its two
    neighbours, whose sites share the temporal links) lets items of consecutive
    half-sweeps touch the same links at once, and the replay reports it."""
    def own_slice_only(done, h, t, tiles_x, nt):
        return h == 0 or done[t] >= h * tiles_x
    caught = 0
    for seed in range(20):
        try:
            run(8, 2, 6, 12, seed, ready=own_slice_only)
        except AssertionError:
            caught += 1
    assert caught > 0


def run_stalled(nt, tiles_x, n_half, nblocks, seed, skip, wait_limit):
    """The same protocol when the launch's first `skip` tickets are never taken (the
    host's fault injection) and each wait gives up after `wait_limit` looks: the
    block that gives up raises the abort flag, a block that finds the flag raised
    when it would wait ends, and the next ticket a block looks at is not staged
    once the flag is up.  Returns (aborted, started items)."""
    rng = random.Random(seed)
    total = tiles_x * nt * n_half
    done = [0] * nt
    finished, started = set(), set()
    ticket = [skip]
    abort = [False]
    in_flight = {}

    def take():
        n = ticket[0]
        ticket[0] += 1
        staged = n < total and not abort[0] and ready(done, *item(n, tiles_x, nt)[:2], tiles_x, nt)
        return n, staged

    blocks = []  # [state, cur, staged, nxt, nxt_staged, waits]
    for _ in range(nblocks):
        n, st = take()
        blocks.append(["start", n, st, None, None, 0])
    steps = 0
    while True:
        live = [b for b in blocks if b[0] != "exit" and b[1] < total]
        if not live:
            break
        b = rng.choice(live)
        steps += 1
        assert steps < 100 * total + 100 * nblocks * (wait_limit + 2), "the launch did not end"
        if b[0] == "take":
            b[3], b[4] = take()
            b[0] = "start"
            b[1], b[2] = b[3], b[4]
        elif b[0] == "start":
            h, t, _ = item(b[1], tiles_x, nt)
            if not b[2]:  # the bounded wait
                if abort[0]:
                    b[0] = "exit"
                    continue
                if not ready(done, h, t, tiles_x, nt):
                    b[5] += 1
                    if b[5] > wait_limit:
                        abort[0] = True
                        b[0] = "exit"
                    continue
            b[5] = 0
            if h > 0:  # dependencies as in the normal run
                for d in (-1, 0, 1):
                    tt = (t + d) % nt
                    for x in range(tiles_x):
                        n_prev = ((h - 1) * nt + ((tt - (h - 1)) % nt)) * tiles_x + x
                        assert n_prev in finished
            mine = {t, (t - 1) % nt}
            for (h2, t2) in in_flight.values():
                if h2 != h:
                    assert not (mine & {t2, (t2 - 1) % nt})
            in_flight[b[1]] = (h, t)
            started.add(b[1])
            b[0] = "finish"
        else:  # finish: publish; then the next ticket
            h, t = in_flight.pop(b[1])
            finished.add(b[1])
            done[t] += 1
            b[0] = "take"
    assert not in_flight
    return abort[0], started


@pytest.mark.parametrize("nt,tiles_x,n_half,nblocks,skip", [
    (8, 1, 2, 8, 1), (8, 1, 4, 3, 3), (6, 2, 5, 12, 2), (12, 4, 8, 40, 5), (4, 3, 6, 2, 1)])
def test_injected_stall_ends_the_launch_through_the_abort_flag(nt, tiles_x, n_half, nblocks, skip):
    """lgt_inject_stream_stall: the skipped items never run, so the half-sweep after
    them waits on slices that never become ready; a wait runs out, raises the
    abort flag, and every block ends (none is left waiting), with the items that
    did run still race-free and in dependency order."""
    for seed in range(8):
        aborted, started = run_stalled(nt, tiles_x, n_half, nblocks, seed, skip, wait_limit=5)
        assert aborted
        assert not (started & set(range(skip)))
        assert len(started) < tiles_x * nt * n_half - skip  # work was left undone


def test_band_order_with_whole_lattice_stagger_is_configuration_10s():
    """D = nt, S = 1 makes every wave hold one pair: the band's numbering is then
    configuration 10's, half-sweep after half-sweep."""
    nt, tiles_x, n_half = 6, 3, 5
    band = Order(nt, tiles_x, n_half, D=nt, S=1)
    assert [band.item(n) for n in range(nt * tiles_x * n_half)] == \
           [item(n, tiles_x, nt) for n in range(nt * tiles_x * n_half)]


@pytest.mark.parametrize("nt,n_half,D", [(2, 3, 2), (4, 7, 2), (6, 5, 3), (8, 9, 4), (32, 20, 8), (12, 4, 20)])
def test_band_ranks_are_a_permutation_in_wave_order(nt, n_half, D):
    """stream_band_rank numbers every (h, k) once, waves D h + k in increasing
    order and, within a wave, half-sweeps in increasing order."""
    ranks = {(h, k): band_rank(h, k, nt, n_half, D) for h in range(n_half) for k in range(nt)}
    assert sorted(ranks.values()) == list(range(nt * n_half))
    by_rank = sorted(ranks, key=ranks.get)
    assert by_rank == sorted(ranks, key=lambda hk: (D * hk[0] + hk[1], hk[0]))


def test_band_dependencies_hold_smaller_tickets():
    """Every S in 1 .. D - 1, for small lattices and any stagger (also D > nt):
    the three items of half-sweep h - 1 that item (h, slice t) waits for come
    earlier in the launch's order -- the property the deadlock argument needs."""
    for nt in (2, 4, 6, 10):
        for n_half in (1, 2, 5, 9):
            for D in range(2, 2 * nt + 2):
                for S in range(1, D):
                    o = Order(nt, 1, n_half, D=D, S=S)
                    for n in range(nt * n_half):
                        h, t, _ = o.item(n)
                        if h:
                            assert all(o.ticket(h - 1, (t + d) % nt, 0) < n for d in (-1, 0, 1)), (nt, n_half, D, S)


@pytest.mark.parametrize("nt,tiles_x,n_half,D,S,nblocks", [
    (4, 2, 6, 2, 1, 5), (6, 3, 7, 3, 1, 8), (6, 2, 9, 3, 2, 4), (8, 2, 10, 4, 2, 12), (10, 1, 12, 5, 3, 20),
    (12, 4, 8, 4, 3, 30), (32, 2, 8, 8, 6, 64), (8, 3, 5, 11, 4, 9)])
def test_band_schedule_is_race_free_and_terminates(nt, tiles_x, n_half, D, S, nblocks):
    """The rolling band under the blocks' protocol: every item once, dependencies
    finished first, no two in-flight items on the same links, no deadlock."""
    for seed in range(4):
        run(nt, tiles_x, n_half, nblocks, seed, order=Order(nt, tiles_x, n_half, D=D, S=S))


def test_band_brings_slices_back_soon():
    """What the band is for (32 slices, 20 half-sweeps, D 8, S 6: about four
    half-sweeps at once, two slices apart): half-sweep h returns to a slice at
    most (D - S) waves of at most ceil(nt / D) + 1 pairs after half-sweep h - 1
    left it (10 slices of work),
    except for the S slices h skips at its start; configuration 10's order
    returns after nt - 1 slices of work or more."""
    nt, n_half, D, S = 32, 20, 8, 6
    band = Order(nt, 1, n_half, D=D, S=S)
    near = far = 0
    for h in range(1, n_half):
        for t in range(nt):
            gap = band.ticket(h, t, 0) - band.ticket(h - 1, t, 0)
            assert gap > 0
            if gap <= (D - S) * (-(-nt // D) + 1):
                near += 1
            else:
                far += 1
    assert far == (n_half - 1) * S and near == (n_half - 1) * (nt - S)
    seq = Order(nt, 1, n_half)
    assert all(seq.ticket(h, t, 0) - seq.ticket(h - 1, t, 0) >= nt - 1 for h in range(1, n_half) for t in range(nt))
