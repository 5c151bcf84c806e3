"""The streaming backward's barrier protocol, checked on the CPU.

A model of one streaming CTA: the compute threads, the copy warp and the
update warp (each as one agent) and the copies in flight, run under random
interleavings. The model follows the kernel's waits and arrivals: stage
barriers full/empty, side-slot barriers sfull/sfree, partial-sum barriers
rfull/rempty. An mbarrier parity wait for phase k succeeds when phase k has
completed and the barrier has not completed phase k + 1 as well: had it, the
parity would match again and the wait would hold on until phase k + 2. The
checks: no wait ever sees its barrier two phases ahead, no interleaving
deadlocks, every copy issued lands before its agent is done with it, and
every agent finishes. A model with the update warp waiting on the stage
barrier instead of its own side-slot barrier shows the checker catching the
two-phases-ahead case.
"""
import random

import pytest

STAGES, SIDE = 2, 4  # the kernel's kStreamStages and kStreamSideSlots


class Hazard(AssertionError):
    pass


class Barrier:
    def __init__(self, name):
        self.name = name
        self.completed = 0  # phases completed

    def ready(self, k):
        """A parity wait for phase k: done when phase k completed; a barrier two
        phases ahead is a protocol error."""
        if self.completed >= k + 2:
            raise Hazard("%s: waiting for phase %d but %d phases completed" % (self.name, k, self.completed))
        return self.completed >= k + 1


def model(kinds, stages=STAGES, side=SIDE, seed=0, update_waits_on_stage=False):
    """kinds: per chunk of the CTA, 0 for a chance chunk or the number of set
    groups. Returns the number of scheduling steps; raises Hazard or a
    deadlock assertion."""
    rng = random.Random(seed)
    n = len(kinds)
    full = [Barrier("full[%d]" % s) for s in range(stages)]
    empty = [Barrier("empty[%d]" % s) for s in range(stages)]
    sfull = [Barrier("sfull[%d]" % k) for k in range(side)]
    sfree = [Barrier("sfree[%d]" % k) for k in range(side)]
    rfull = [Barrier("rfull[%d]" % p) for p in range(2)]
    rempty = [Barrier("rempty[%d]" % p) for p in range(2)]
    landing = []  # copies in flight: (barrier, chunk)
    stage_of = [None] * stages  # chunk whose copies target each stage
    side_of = [None] * side

    def issue(i):
        s, k = i % stages, i % side
        # a stage or side slot is refilled only once its previous chunk is consumed
        assert stage_of[s] is None or stage_of[s][1], "stage %d refilled while in use" % s
        assert side_of[k] is None or side_of[k][1], "side slot %d refilled while in use" % k
        stage_of[s] = [i, False]
        side_of[k] = [i, False]
        landing.append((full[s], i))
        if kinds[i] == 0:
            sfull[k].completed += 1  # no side bytes: the phase completes with the arrival
        else:
            landing.append((sfull[k], i))

    def copy_agent():
        for i in range(min(stages, n)):  # the prologue
            issue(i)
        yield None
        i = 0
        while i + stages < n:
            yield (empty[i % stages], i // stages)
            j = i + stages - side
            if j >= 0:
                yield (sfree[(i + stages) % side], j // side)
            issue(i + stages)
            i += 1

    def update_agent():
        grp = 0
        for i in range(n):
            k = i % side
            if update_waits_on_stage:  # the planted mistake: the stage barrier instead of the side slot's
                yield (full[i % stages], i // stages)
            else:
                yield (sfull[k], i // side)
            assert side_of[k][0] == i, "update warp reads side slot %d before chunk %d landed there" % (k, i)
            for _ in range(kinds[i]):
                p = grp & 1
                yield (rfull[p], grp // 2)
                rempty[p].completed += 1
                grp += 1
            side_of[k][1] = True
            sfree[k].completed += 1

    def compute_agent():
        grp = 0
        for i in range(n):
            s = i % stages
            yield (full[s], i // stages)
            assert stage_of[s][0] == i, "compute reads stage %d before chunk %d landed there" % (s, i)
            for g in range(kinds[i]):
                p = grp & 1
                if grp >= 2:
                    yield (rempty[p], (grp - 2) // 2)
                rfull[p].completed += 1
                grp += 1
            stage_of[s][1] = True
            empty[s].completed += 1

    agents = {"copy": copy_agent(), "update": update_agent(), "compute": compute_agent()}
    waiting = {}
    for name in list(agents):  # each agent up to its first wait (or to its end)
        try:
            waiting[name] = next(agents[name])
        except StopIteration:
            del agents[name]
    steps = 0
    while agents or landing:
        steps += 1
        runnable = [a for a in agents if waiting[a] is None or waiting[a][0].ready(waiting[a][1])]
        choices = [("agent", a) for a in runnable] + [("land", j) for j in range(len(landing))]
        assert choices, "deadlock: %s" % {a: (w[0].name, w[1]) for a, w in waiting.items() if w}
        what, x = rng.choice(choices)
        if what == "land":
            bar, _ = landing.pop(x)
            bar.completed += 1
            continue
        try:
            waiting[x] = next(agents[x])
        except StopIteration:
            del agents[x]
            del waiting[x]
    # every chunk's stage and side-slot phases completed exactly once
    assert sum(b.completed for b in full) == n and sum(b.completed for b in sfull) == n
    return steps


def random_kinds(rng, n):
    return [0 if rng.random() < 0.2 else rng.randint(1, 3) for _ in range(n)]


@pytest.mark.parametrize("stages,side", [(2, 4), (3, 6), (2, 6)])
def test_protocol_never_sees_a_barrier_two_phases_ahead_and_never_deadlocks(stages, side):
    rng = random.Random(stages * 100 + side)
    for trial in range(400):
        n = rng.randint(0, 30)
        model(random_kinds(rng, n), stages, side, seed=trial)


def test_protocol_edge_cases():
    for kinds in ([], [0], [1], [0] * 9, [3] * 9, [1, 0, 2, 0, 0, 3, 1]):
        for seed in range(50):
            model(kinds, seed=seed)


def test_the_checker_catches_the_update_warp_waiting_on_the_stage_barrier():
    # with the update warp on the stage barrier, a run where the compute
    # threads and the copy warp get two chunks ahead of it leaves the stage
    # barrier two phases past the one the update warp waits for
    rng = random.Random(7)
    caught = 0
    for trial in range(300):
        try:
            model([rng.randint(1, 2) for _ in range(12)], seed=trial, update_waits_on_stage=True)
        except Hazard:
            caught += 1
    assert caught > 0
