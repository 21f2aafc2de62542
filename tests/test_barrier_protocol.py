"""The scoring CTA's hand-over protocol (branch3_kernel), replayed on the host.

Warp 7 describes rounds of runs into two shared buffers; warps 0-6 score
them.  Named barriers (PTX bar.sync / bar.arrive, counted in threads, a warp
arriving as 32) carry the hand-over: FULL + b from the describing warp
(arrive) to the scoring warps (sync), EMPTY + b back (the scoring warps
arrive, the describing warp syncs before it rewrites buffer b two rounds
later), and CONS among the scoring warps alone (chunk staging and the end of
a round's reduction).  The replay steps the eight warps in random orders
and checks, for 0 to 40 rounds and any number of chunk changes per round:
every barrier phase completes (no deadlock), no warp arrives twice in one
phase, the describing warp never rewrites a buffer that a scoring warp still
reads, and every scoring warp scores every round exactly once, in order."""
import random

import pytest

FULL, EMPTY, CONS = 1, 3, 5
WARP = 32
N_ALL, N_CONS = 256, 224


class Barriers:
    def __init__(self):
        self.count = {}
        self.phase = {}
        self.members = {}

    def arrive(self, bid, n, who):
        """Arrive at barrier bid (n threads complete a phase); returns the
        phase arrived in.  A warp arriving twice in one phase is an error."""
        ph = self.phase.get(bid, 0)
        mem = self.members.setdefault((bid, ph), set())
        assert who not in mem, f"warp {who} arrived twice at barrier {bid} phase {ph}"
        mem.add(who)
        c = self.count.get(bid, 0) + WARP
        assert c <= n
        if c == n:
            self.count[bid] = 0
            self.phase[bid] = ph + 1
        else:
            self.count[bid] = c
        return ph

    def passed(self, bid, ph):
        return self.phase.get(bid, 0) > ph


def producer(rounds, state):
    """The describing warp (describe_rounds)."""
    r = 0
    while True:
        b = r & 1
        if r >= 2:
            yield ("sync", EMPTY + b, N_ALL)
        if r >= rounds:
            state["nrun"][b] = 0
            yield ("arrive", FULL + b, N_ALL)
            if r >= 1:
                yield ("sync", EMPTY + (b ^ 1), N_ALL)
            return
        assert not state["reading"][b], f"buffer {b} rewritten while read (round {r})"
        state["buf"][b] = r
        state["nrun"][b] = 1 + state["rng"].randrange(32)
        yield ("arrive", FULL + b, N_ALL)
        r += 1


def consumer(w, state, chunk_changes, prestage):
    """A scoring warp (warps 0-6 of branch3_kernel)."""
    staged = False
    if prestage:
        staged = True
        yield ("sync", CONS, N_CONS)
    r = 0
    while True:
        b = r & 1
        yield ("sync", FULL + b, N_ALL)
        if state["nrun"][b] == 0:
            return
        state["reading"][b].add(w)
        assert state["buf"][b] == r, (w, r, state["buf"][b])
        state["scored"][w].append(r)
        for _ in range(chunk_changes[r]):      # uniform over the scoring warps
            if staged:
                yield ("sync", CONS, N_CONS)   # the previous chunk's readers are done
            staged = True
            yield ("sync", CONS, N_CONS)       # staged points visible
        yield ("step", None, None)             # scoring
        assert state["buf"][b] == r
        yield ("sync", CONS, N_CONS)           # partial sums in
        yield ("step", None, None)             # reduction flushed
        state["reading"][b].discard(w)
        yield ("arrive", EMPTY + b, N_ALL)
        r += 1


def replay(rounds, seed, prestage):
    rng = random.Random(seed)
    state = {"nrun": [None, None], "buf": [None, None], "reading": [set(), set()],
             "scored": {w: [] for w in range(7)}, "rng": rng}
    chunk_changes = [rng.choice([0, 0, 0, 1, 1, 2]) for _ in range(rounds + 1)]
    actors = {w: consumer(w, state, chunk_changes, prestage) for w in range(7)}
    actors[7] = producer(rounds, state)
    bars = Barriers()
    waiting = {}            # warp -> (barrier, phase) it waits on
    pending = {w: next(g) for w, g in actors.items()}
    done = set()
    for _ in range(200000):
        runnable = [w for w in actors if w not in done and
                    (w not in waiting or bars.passed(*waiting[w]))]
        if not runnable:
            break
        w = rng.choice(runnable)
        if w in waiting:
            del waiting[w]
        else:
            kind, bid, n = pending[w]
            if kind in ("sync", "arrive"):
                ph = bars.arrive(bid, n, w)
                if kind == "sync" and not bars.passed(bid, ph):
                    waiting[w] = (bid, ph)
                    continue
        try:
            pending[w] = next(actors[w])
        except StopIteration:
            done.add(w)
    assert done == set(actors), f"deadlock: done {sorted(done)}, waiting {waiting}"
    assert all(v == 0 for v in bars.count.values()), bars.count
    for w in range(7):
        assert state["scored"][w] == list(range(rounds)), (w, state["scored"][w])


@pytest.mark.parametrize("prestage", [True, False])
def test_protocol_completes_for_any_schedule(prestage):
    for rounds in list(range(0, 12)) + [25, 40]:
        for seed in range(40):
            replay(rounds, 1000 * rounds + seed, prestage)


def test_replay_catches_a_missing_empty_wait():
    """A describing warp that skips its EMPTY wait rewrites a buffer still
    being read (or scores a round twice): the replay must see it."""
    global producer
    keep = producer

    def bad(rounds, state):
        r = 0
        while True:
            b = r & 1
            if r >= rounds:
                state["nrun"][b] = 0
                yield ("arrive", FULL + b, N_ALL)
                return
            assert not state["reading"][b], "rewritten while read"
            state["buf"][b] = r
            state["nrun"][b] = 1
            yield ("arrive", FULL + b, N_ALL)
            r += 1

    producer = bad
    try:
        failed = 0
        for seed in range(60):
            try:
                replay(6, seed, True)
            except AssertionError:
                failed += 1
        assert failed > 0
    finally:
        producer = keep
