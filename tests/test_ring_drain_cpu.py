"""Host model of the tensor-core kernels' shared-memory ring and of its drain after a
timeout (gemm_tc_kernel, wgrad_halo_kernel).

The kernels' protocol, restated: the producer fills stage it % S after waiting on
empty[s] with parity ((it / S) & 1) ^ 1, arms full[s] and issues the copy; the MMA thread
waits on full[s] with parity (it / S) & 1, issues its MMAs and commits them to empty[s].
Copies and MMAs complete asynchronously, in any order across stages. A wait that runs
out sets the abort flag and both roles leave their loops, recording `issued` (stages
loaded) and `consumed` (stages waited for). The drain then waits, for every it in
[consumed, issued), on full[it % S] with parity (it / S) & 1, and on one final commit of
the MMA thread.

Random interleavings check that at the drain every copy still in flight is covered by
exactly one of those waits, that each wait completes only once its own copy has landed
(not an earlier phase of the same stage), and that no more than S copies are ever
outstanding. An mbarrier phase wait on parity p returns once the barrier's completed-
phase count c has c & 1 != p (PTX ISA, mbarrier.try_wait.parity).
"""
import random

import pytest


class Bar:
    def __init__(self):
        self.completed = 0  # phases completed

    def ready(self, parity):
        return (self.completed & 1) != parity


def _run(S, total, seed, abort_at):
    rnd = random.Random(seed)
    full = [Bar() for _ in range(S)]
    empty = [Bar() for _ in range(S)]
    loads = []     # in-flight copies: (it, stage)
    mmas = []      # in-flight MMA groups: (it, stage)
    landed = set()
    issued = consumed = 0
    p_done = m_done = False
    abort = False
    ticks = 0
    while not (p_done and m_done):
        ticks += 1
        if ticks == abort_at:
            abort = True  # some wait ran out
        who = rnd.randrange(4)
        if who == 0 and not p_done:
            if abort or issued == total:
                p_done = True
            else:
                s = issued % S
                if empty[s].ready(((issued // S) & 1) ^ 1):
                    assert issued - consumed < S + 1
                    loads.append((issued, s))
                    issued += 1
        elif who == 1 and not m_done:
            if abort or consumed == total:
                m_done = True
            else:
                s = consumed % S
                if full[s].ready((consumed // S) & 1):
                    assert (consumed, s) in landed
                    mmas.append((consumed, s))
                    consumed += 1
        elif who == 2 and loads:
            i = rnd.randrange(len(loads))
            it, s = loads.pop(i)
            # copies of one stage complete in issue order: a stage has one copy in flight
            assert all(s2 != s for _, s2 in loads)
            full[s].completed += 1
            landed.add((it, s))
        elif who == 3 and mmas:
            it, s = mmas.pop(0)  # commits arrive in issue order
            empty[s].completed += 1
        assert issued - consumed <= S
    # drain: the waits the kernel makes, in its order
    pending = {it for it, _ in loads}
    waits = list(range(consumed, issued))
    assert set(waits) == pending | {it for it in waits if (it, it % S) in landed}
    assert pending <= set(waits)
    for it in waits:
        s, par = it % S, (it // S) & 1
        # the wait has not completed before its own copy lands...
        if (it, s) not in landed:
            assert not full[s].ready(par)
        # ...and completes once it has (the async engine runs on)
        while (it, s) not in landed:
            j = next(k for k, (it2, s2) in enumerate(loads) if s2 == s)
            it2, s2 = loads.pop(j)
            full[s2].completed += 1
            landed.add((it2, s2))
        assert full[s].ready(par)
    assert not loads  # every copy the CTA issued has landed before its memory is freed
    return issued, consumed


@pytest.mark.parametrize("S", [2, 3, 4, 16])
def test_drain_covers_every_copy_in_flight(S):
    saw_gap = False
    for seed in range(300):
        abort_at = 5 + (seed * 7) % 200
        issued, consumed = _run(S, total=40, seed=seed * 31 + S, abort_at=abort_at)
        saw_gap |= issued > consumed
    assert saw_gap  # some interleavings did leave copies in flight at the abort


def test_no_abort_leaves_nothing_to_drain():
    for seed in range(50):
        issued, consumed = _run(4, total=25, seed=seed, abort_at=10 ** 9)
        assert issued == consumed == 25
