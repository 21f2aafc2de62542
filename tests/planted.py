"""The planted-pose check of the tests (test helper): translation within one
finest voxel of the returned leaf's dilated cell centre (T + 1/2) r per
axis, and each angle within one finest angular step of the planted angle,
unless the returned leaf ties the best leaf within that box -- the Eq. (11)
score cannot tell such leaves apart and the tie rule picks the
lexicographically smallest, which may lie one or two steps away in roll,
pitch or yaw (a one-step rotation moves most scan points by less than a
voxel: Eq. (2) ties the step to the farthest point)."""
import itertools
import math

import numpy as np


def box_leaves(r, g, pose):
    """Leaves within one voxel (of the cell centre) and one step of the pose."""
    T = [[t for t in range(int(math.floor(pose[i] / r - 1.5)), int(math.floor(pose[i] / r + 0.5)) + 1)
          if abs((t + 0.5) * r - pose[i]) <= r] for i in range(3)]
    A = []
    for i in range(3):
        cs = []
        for c in range(g.N(0)[i]):
            d = g.angle(0, i, c) - pose[3 + i]
            if i == 2:
                d = (d + math.pi) % (2 * math.pi) - math.pi
            if abs(d) <= g.dprime(0)[i] * (1 + 1e-12):
                cs.append(c)
        A.append(cs)
    return np.array([[*t, *a, 0] for t in itertools.product(*T) for a in itertools.product(*A)], np.int32)


def check_planted(r, g, om, scan, pose, node, best, res_pose):
    """Assert the planted-pose bar; returns the angular errors in steps."""
    for i in range(3):
        assert abs((node[i] + 0.5) * r - pose[i]) <= r, ("translation", i)
    steps = []
    for i in range(3):
        d = res_pose[3 + i] - pose[3 + i]
        if i == 2:
            d = (d + math.pi) % (2 * math.pi) - math.pi
        steps.append(abs(d) / g.dprime(0)[i])
    if max(steps) > 1 + 1e-9:
        box = box_leaves(r, g, pose)
        assert len(box) > 0
        assert int(om.score_nodes(g, scan, box).max()) == best, ("angles", steps)
    return steps
