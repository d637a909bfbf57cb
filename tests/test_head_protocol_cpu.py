"""The mbarrier protocol of the D = 64 tensor-core head (k_predict_tm), as a
model run under random interleavings on the CPU.

Roles, as in the kernel: P producer groups (tile li filled by group li mod P
into A slot li mod P, row metadata into slot li mod (P + 2)), two epilogue
groups of 4 warps (tile li read back by group li mod 2, whose first warp
issues the tile's first and second layers), and the tensor core, which
completes issued MMAs asynchronously in issue order.  Barriers: full and done
per tile modulo ring = lcm(P, 2); stored, out and empty per epilogue group.

A parity wait is modelled as mbarrier.try_wait.parity: it passes when the
barrier's completed-phase count has the other parity.  The model fails if a
wait passes for a phase not yet completed or after its barrier moved two
phases on, if an A slot is refilled while a first layer may still read it,
if the first layer runs on a slot that does not hold its tile, or if row
metadata is overwritten before all four warps of its tile have read it.
"""
import random

import pytest


class _Bar:
    def __init__(self, count):
        self.count, self.arrived, self.completed = count, 0, 0

    def arrive(self):
        self.arrived += 1
        if self.arrived == self.count:
            self.arrived = 0
            self.completed += 1

    def passed(self, phase):
        ok = (phase & 1) != (self.completed & 1)
        assert not (ok and self.completed < phase + 1), f"phase {phase} passed early"
        assert self.completed <= phase + 1, f"waiter for phase {phase} fell two phases behind"
        return ok


def _run(P, ntiles, seed, ring, meta):
    rng = random.Random(seed)
    full = [_Bar(1) for _ in range(ring)]
    done = [_Bar(1) for _ in range(ring)]
    stored, out, empty = [_Bar(4), _Bar(4)], [_Bar(1), _Bar(1)], [_Bar(4), _Bar(4)]
    slot_tile = [None] * P       # tile whose operand an A slot holds
    slot_reader = [None] * P     # tile whose first layer last read the slot
    meta_tile = [None] * meta
    meta_read = [set() for _ in range(meta)]
    issued, l1_done = [], set()

    def producer(g):
        for li in range(g, ntiles, P):
            if li >= P:
                while not done[(li - P) % ring].passed((li - P) // ring):
                    yield
            s, m = li % P, li % meta
            assert slot_reader[s] is None or slot_reader[s] in l1_done, "A slot refilled early"
            assert meta_tile[m] is None or len(meta_read[m]) == 4, "metadata overwritten early"
            slot_tile[s], meta_tile[m], meta_read[m] = li, li, set()
            yield
            full[li % ring].arrive()
            yield

    def epilogue(e, w):
        for li in range(e, ntiles, 2):
            if w == 0:
                while not full[li % ring].passed(li // ring):
                    yield
                if li >= 2:
                    while not empty[e].passed((li - 2) // 2):
                        yield
                assert slot_tile[li % P] == li, "first layer on a slot without its tile"
                slot_reader[li % P] = li
                issued.append(("l1", li))
                yield
            while not done[li % ring].passed(li // ring):
                yield
            assert meta_tile[li % meta] == li, "metadata of another tile"
            meta_read[li % meta].add(w)
            yield
            stored[e].arrive()
            if w == 0:
                while not stored[e].passed(li // 2):
                    yield
                issued.append(("l2", li))
            while not out[e].passed(li // 2):
                yield
            yield
            empty[e].arrive()
            yield

    def complete_one():
        kind, li = issued.pop(0)
        if kind == "l1":
            l1_done.add(li)
            done[li % ring].arrive()
        else:
            out[li % 2].arrive()

    live = [producer(g) for g in range(P)] + [epilogue(e, w) for e in range(2) for w in range(4)]
    for _ in range(100_000):
        if not live:
            break
        if issued and rng.random() < 0.2:
            complete_one()
            continue
        a = rng.choice(live)
        try:
            next(a)
        except StopIteration:
            live.remove(a)
    assert not live, "no progress"
    while issued:
        complete_one()


@pytest.mark.parametrize("P", [2, 3, 4])
def test_head_protocol_holds(P):
    ring = P if P % 2 == 0 else 2 * P
    for seed in range(60):
        for ntiles in (1, 2, 3, 7, 24):
            _run(P, ntiles, seed, ring, P + 2)


def test_model_catches_one_barrier_per_slot_with_odd_P():
    # consecutive phases of a slot's barrier alternate between the epilogue
    # groups; a group then takes the parity of a phase not yet completed
    with pytest.raises(AssertionError):
        for seed in range(60):
            _run(3, 24, seed, 3, 5)


def test_model_catches_too_few_metadata_slots():
    with pytest.raises(AssertionError):
        for seed in range(60):
            _run(4, 24, seed, 4, 5)
