"""A model of the joint sweep kernel's colour-step synchronisation (row
version flags), run under random interleavings on the CPU.

The model follows csrc/joint.cu: CTAs take the slots of a colour in rounds
of `warps` slots; each warp waits until both rows of its slot carry version
g = t P + c, reads them, and, if its block did not move (or the slot is a
bye), publishes g + 1 at once; the CTA then meets at its barrier; if any of
its blocks moved, the CTA applies their row updates, meets again, and the
moved blocks publish g + 1.  A grid barrier closes every sweep.

Checked for every interleaving drawn: the run never deadlocks, every read of
a row sees exactly the updates of all earlier colour steps (no stale read,
no update of the same colour step racing ahead), and every row carries every
colour step's update exactly once.
"""
import random

import pytest

from test_capi_cpu import _joint_slot_pair


class _Model:
    def __init__(self, p, grid, warps, sweeps, p_move, seed, publish_moved_early=False):
        self.p = p
        self.P = p + (p % 2) - 1
        self.half = (self.P + 1) // 2
        self.grid, self.warps, self.sweeps = grid, warps, sweeps
        self.rng = random.Random(seed)
        self.p_move = p_move
        self.publish_moved_early = publish_moved_early  # a planted protocol mistake
        self.ver = [0] * p    # published version of each row
        self.data = [0] * p   # colour steps whose update of the row is complete
        self.steps = self.sweeps * self.P

    def cta_program(self, b):
        """Generator of one CTA's actions; yields a predicate to wait on (or
        None) before each action."""
        rounds = [base for base in range(b * self.warps, self.half, self.grid * self.warps)]
        for t in range(self.sweeps):
            for c in range(self.P):
                g = t * self.P + c
                for base in rounds:
                    slots = []
                    for w in range(self.warps):
                        q = base + w
                        if q >= self.half:
                            continue
                        i, j, ra, rb = _joint_slot_pair(q, c, self.P, self.p)
                        rows = [r for r in (ra, rb) if r < self.p]
                        slots.append((i, rows))
                    # phase 0: warps independently wait, read and maybe publish
                    pending = list(range(len(slots)))
                    self.rng.shuffle(pending)
                    moved = {}
                    for k in pending:
                        i, rows = slots[k]
                        yield (lambda rows=rows, g=g: all(self.ver[r] >= g for r in rows))
                        for r in rows:  # the reads of this block
                            assert self.data[r] == g, ("stale or early read", r, g, self.data[r])
                        mv = i >= 0 and self.rng.random() < self.p_move
                        moved[k] = mv
                        if not mv:
                            for r in rows:
                                self.data[r] = g + 1
                                self.ver[r] = g + 1
                        elif self.publish_moved_early:
                            for r in rows:
                                self.ver[r] = g + 1
                        yield None
                    # CTA barrier; row updates of moved blocks; barrier; publish
                    if any(moved.values()):
                        for k, mv in moved.items():
                            if mv:
                                for r in slots[k][1]:
                                    assert self.data[r] == g
                                    self.data[r] = g + 1
                                yield None
                        for k, mv in moved.items():
                            if mv:
                                for r in slots[k][1]:
                                    self.ver[r] = g + 1
                        yield None
            yield ("grid", t)  # the diagonal step's grid barrier

    def run(self):
        progs = [self.cta_program(b) for b in range(self.grid)]
        waiting = [None] * self.grid  # predicate each CTA waits on
        done = [False] * self.grid
        for b in range(self.grid):
            waiting[b] = next(progs[b])
        while not all(done):
            runnable = []
            for b in range(self.grid):
                if done[b]:
                    continue
                w = waiting[b]
                if isinstance(w, tuple):  # at the sweep's grid barrier
                    continue
                if w is None or w():
                    runnable.append(b)
            if not runnable:
                # the sweep's grid barrier opens when every live CTA is there
                live = [b for b in range(self.grid) if not done[b]]
                if live and all(isinstance(waiting[b], tuple) for b in live):
                    for b in live:
                        waiting[b] = None
                    runnable = live
                else:
                    raise AssertionError("deadlock")
            b = self.rng.choice(runnable)
            try:
                waiting[b] = next(progs[b])
            except StopIteration:
                done[b] = True
        assert self.data == [self.steps] * self.p
        assert self.ver == [self.steps] * self.p


@pytest.mark.parametrize("p,grid,warps", [(2, 1, 1), (3, 2, 1), (5, 2, 2), (6, 3, 1),
                                          (13, 2, 3), (16, 3, 2), (33, 4, 2), (64, 2, 4)])
@pytest.mark.parametrize("p_move", [0.0, 0.3, 1.0])
def test_row_versions_never_deadlock_and_order_every_read(p, grid, warps, p_move):
    for seed in range(6):
        _Model(p, grid, warps, sweeps=2, p_move=p_move, seed=seed).run()


def test_publishing_a_moved_block_before_its_row_updates_is_caught():
    """The model detects the protocol's plausible mistake: a block that moved
    publishing its rows before the CTA has applied their updates."""
    caught = 0
    for p, grid, warps in [(13, 2, 3), (16, 3, 2), (33, 4, 2)]:
        for seed in range(4):
            try:
                _Model(p, grid, warps, 2, 0.3, seed, publish_moved_early=True).run()
            except AssertionError:
                caught += 1
    assert caught == 12
