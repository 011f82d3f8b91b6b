"""The streaming sweep kernel's schedule, checked on the host.

The kernel (launch configuration 10) runs n_half half-sweeps in one launch.
Item n is (half-sweep h, position k, group bx of a slice's tiles), with
n = (h * nt + k) * items_x + bx (items_x is called tiles_x below: the model
does not look inside an item), and half-sweep h visits slice t = (h + k) mod nt
at position k.  A block takes tickets in order; it looks once, without
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


def item(n, tiles_x, nt):
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


def run(nt, tiles_x, n_half, nblocks, seed, ready=ready):
    """Replays the blocks' protocol; returns the number of waits that found the
    slices not ready.  `ready` is the dependency rule (the kernel's by default)."""
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
        staged = n < total and ready(done, *item(n, tiles_x, nt)[:2], tiles_x, nt)
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
                h, t, _ = item(b[1], tiles_x, nt)
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
            h, t, bx = item(b[1], tiles_x, nt)
            if not b[2]:
                waits += 1
            # an item starts only after the previous half-sweep finished t - 1, t, t + 1
            if h > 0:
                for d in (-1, 0, 1):
                    tt = (t + d) % nt
                    for x in range(tiles_x):
                        n_prev = ((h - 1) * nt + ((tt - (h - 1)) % nt)) * tiles_x + x
                        assert n_prev in finished
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
