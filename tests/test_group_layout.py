"""The task layout of a round scored in one launch, restated on the host.

The engine lays a round's tasks out by rotation group: the popped parents of
one search that share level and rotation (group G, P_G parents, T_G
rotational children each, Eq. (13)) hold tasks off(G) + j P_G + i for child
rotation j and the group's parent i, off(G) the search's task offset plus
the exclusive prefix of P T over its groups in creation order.  These tests
restate that layout in Python (group creation in any order, parents joining
in any order within a group) and check the properties the scoring kernel and
the survivor pass rely on: every search's tasks fill exactly its own range,
each (parent, child rotation) appears once, and the tasks of one child
rotation of a group are consecutive."""
import random


def layout(parents, toff, rng):
    """parents: list of (search, rl, T); returns {position: (parent, j)}."""
    groups = {}          # (search, rl) -> [parent indices] in joining order
    order = {}           # search -> [keys] in creation order
    for p in rng.sample(range(len(parents)), len(parents)):   # the compaction's arbitrary order
        s, rl, T = parents[p]
        key = (s, rl)
        if key not in groups:
            groups[key] = []
            order.setdefault(s, []).append(key)
        groups[key].append(p)
    pos = {}
    for s, keys in order.items():
        run = toff[s]
        for key in keys:       # the exclusive scan over the search's groups
            members = groups[key]
            T = parents[members[0]][2]
            P = len(members)
            for i, p in enumerate(members):
                for j in range(T):
                    at = run + j * P + i
                    assert at not in pos
                    pos[at] = (p, j)
            run += P * T
    return pos, groups


def test_grouped_layout_fills_each_search_range_once():
    rng = random.Random(5)
    for trial in range(300):
        nsearch = rng.randint(1, 5)
        parents = []
        for s in range(nsearch):
            nrot = rng.randint(1, 12)
            for _ in range(rng.randint(0, 60)):
                rl = rng.randrange(nrot)
                parents.append((s, rl, 1 + (rl * 7) % 5))   # T depends on the rotation only
        if not parents:
            continue
        ntask = [sum(T for s2, _, T in parents if s2 == s) for s in range(nsearch)]
        toff = [sum(ntask[:s]) for s in range(nsearch)]
        pos, groups = layout(parents, toff, rng)
        assert sorted(pos) == list(range(sum(ntask)))
        seen = set(pos.values())
        assert len(seen) == len(pos) == sum(T for _, _, T in parents)
        for at, (p, j) in pos.items():   # each task in its own search's range
            s = parents[p][0]
            assert toff[s] <= at < toff[s] + ntask[s]
        for key, members in groups.items():   # one child rotation's tasks are consecutive
            T = parents[members[0]][2]
            for j in range(T):
                ats = sorted(at for at, (p, jj) in pos.items() if jj == j and p in members)
                assert ats == list(range(ats[0], ats[0] + len(members)))
