"""A sequential model of the batched kernel's sliced work queue, run under
random interleavings on the CPU.

The device protocol (genasm_align.cu, ring_take / ring_push and the loop of
batched_body): a ring of 2n slots, each with a sequence number; slot x < n
starts with hand-out position x published (seq x + 1), the others free (seq
x). A group without a pair reserves the next head position (atomic add) and
takes it once published (seq x + 1), marking the slot free for position
x + 2n; until then it polls, and it stops when the count of unfinished pairs
is zero. A group runs a pair for up to `slice` windows; at the end of a turn
it claims the next tail position (atomic add), waits (bounded) for that slot
to be free (seq == position), writes the pair and publishes it (seq + 1). A
push whose wait runs out keeps its pair for another turn and raises the
launch's flag; the reserver of the lost position leaves at the end.

Every memory access of the protocol is one step of the model; a random
scheduler picks which group steps next, with bursts that stall a group for a
long time (the adversarial case: a push stalled between its claim and its
publication while the other pairs cycle). Checked: a pair is never held by
two groups, every pair runs exactly its number of windows, every group
stops, the ring never holds more than n pairs, and the flag stays down
unless a wait was made to run out; with waits cut short, every group still
stops and every pair left unfinished is covered by the flag.
"""
from __future__ import annotations

import random

import pytest


class Ring:
    def __init__(self, windows, groups, slice_, push_polls=10**9, idle_polls=10**9, seed=0):
        self.n = n = len(windows)
        self.cap = 2 * n
        self.windows = list(windows)
        self.done = [0] * n
        self.seq = [x + 1 if x < n else x for x in range(self.cap)]
        self.slot = [x if x < n else -1 for x in range(self.cap)]
        self.head = 0
        self.tail = n
        self.unfinished = n
        self.flag = False
        self.slice = slice_
        self.push_polls = push_polls
        self.idle_polls = idle_polls
        self.holder = [None] * n  # group holding each pair
        self.rng = random.Random(seed)
        self.groups = [dict(state="want", resv=None, pair=None, budget=0, y=None, polls=0,
                            idle=0) for _ in range(groups)]

    def published(self, s):
        """Slot s holds a published position (seq = position + 1)."""
        return self.seq[s] % self.cap == (s + 1) % self.cap

    def step(self, g):
        G = self.groups[g]
        st = G["state"]
        if st == "want":
            if G["resv"] is None:
                G["resv"] = self.head  # atomicAdd on the head
                self.head += 1
                return
            x = G["resv"]
            s = x % self.cap
            if self.seq[s] == x + 1:  # published: take it
                p = self.slot[s]
                self.seq[s] = x + self.cap
                G["resv"] = None
                assert self.holder[p] is None, f"pair {p} taken twice"
                self.holder[p] = g
                G.update(state="busy", pair=p, budget=self.slice, idle=0)
            elif self.unfinished == 0:
                G["state"] = "stopped"
            else:
                G["idle"] += 1
                if G["idle"] >= self.idle_polls:
                    self.flag = True
                    G["state"] = "stopped"
        elif st == "busy":
            p = G["pair"]
            self.done[p] += 1  # one window
            assert self.done[p] <= self.windows[p]
            if self.done[p] == self.windows[p]:
                self.unfinished -= 1  # atomicSub
                self.holder[p] = None
                G.update(state="want", pair=None)
                return
            G["budget"] -= 1
            if G["budget"] == 0:
                G["y"] = self.tail  # atomicAdd on the tail
                self.tail += 1
                G.update(state="push", polls=0)
        elif st == "push":
            y = G["y"]
            s = y % self.cap
            if self.seq[s] != y:
                G["polls"] += 1
                if G["polls"] >= self.push_polls:  # the wait ran out: keep the pair
                    self.flag = True
                    G.update(state="busy", budget=self.slice)
                return
            self.slot[s] = G["pair"]
            G["state"] = "publish"
        elif st == "publish":
            y = G["y"]
            p = G["pair"]
            self.holder[p] = None
            self.seq[y % self.cap] = y + 1
            G.update(state="want", pair=None)

    def run(self, max_steps=10**6):
        live = list(range(len(self.groups)))
        stalled = {}
        for _ in range(max_steps):
            live = [g for g in live if self.groups[g]["state"] != "stopped"]
            if not live:
                return True
            # occasionally stall a group for a long burst of the others' steps
            if self.rng.random() < 0.02:
                stalled[self.rng.choice(live)] = self.rng.randint(10, 400)
            runnable = [g for g in live if stalled.get(g, 0) <= 0] or live
            g = self.rng.choice(runnable)
            for h in list(stalled):
                stalled[h] -= 1
            self.step(g)
            held = sum(1 for h in self.holder if h is not None)
            published = sum(1 for x in range(self.cap) if self.published(x))
            assert held + published <= self.n
        return False


@pytest.mark.parametrize("seed", range(300))
def test_ring_protocol_random_interleavings(seed):
    rng = random.Random(seed)
    n = rng.randint(1, 12)
    windows = [rng.randint(1, 7) for _ in range(n)]
    groups = rng.randint(1, 6)
    slice_ = rng.randint(1, 3)
    ring = Ring(windows, groups, slice_, seed=seed)
    assert ring.run(), "the groups did not all stop"
    assert ring.done == windows
    assert ring.unfinished == 0
    assert not ring.flag
    assert all(h is None for h in ring.holder)


@pytest.mark.parametrize("seed", range(100))
def test_ring_protocol_waits_run_out(seed):
    # Waits cut to a few polls (the device's bounds are seconds): a push that
    # gives up keeps its pair, a lost position's reserver and idle groups leave
    # when their wait runs out, so every group stops. No pair runs a window
    # twice or past its end; a pair left unfinished implies the flag (the
    # device reports such pairs as GA_PAIR_TIMED_OUT).
    rng = random.Random(1000 + seed)
    n = rng.randint(2, 10)
    windows = [rng.randint(2, 9) for _ in range(n)]
    ring = Ring(windows, rng.randint(2, 6), rng.randint(1, 2), push_polls=rng.randint(1, 3),
                idle_polls=rng.randint(1, 200), seed=seed)
    assert ring.run(), "the groups did not all stop"
    assert all(d <= w for d, w in zip(ring.done, windows))
    unfinished = sum(d < w for d, w in zip(ring.done, windows))
    assert unfinished == ring.unfinished
    assert unfinished == 0 or ring.flag


def test_ring_lost_position_strands_without_idle_bound():
    # Why the idle wait must be bounded too: with pushes that give up and
    # idle groups that never leave, a lost position's reserver can wait
    # forever while published pairs behind it have no reserver.
    stuck = 0
    for seed in range(40):
        rng = random.Random(1000 + seed)
        n = rng.randint(2, 10)
        windows = [rng.randint(2, 9) for _ in range(n)]
        ring = Ring(windows, rng.randint(2, 6), 1, push_polls=rng.randint(1, 3), seed=seed)
        stuck += not ring.run(max_steps=200_000)
    assert stuck > 0


def test_ring_push_slot_free_without_stalls():
    # Without stalls a claimed tail slot is already free (the wait is a guard).
    ring = Ring([5] * 8, 4, 1, seed=7)
    ring.rng = random.Random(7)
    waits = 0
    orig = ring.step

    def step(g):
        nonlocal waits
        G = ring.groups[g]
        if G["state"] == "push" and ring.seq[G["y"] % ring.cap] != G["y"]:
            waits += 1
        orig(g)

    ring.step = step
    # round-robin schedule: no group is stalled
    for _ in range(100000):
        live = [g for g in range(4) if ring.groups[g]["state"] != "stopped"]
        if not live:
            break
        for g in live:
            ring.step(g)
    assert ring.done == [5] * 8
    assert waits == 0
