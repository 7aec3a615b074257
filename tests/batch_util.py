"""Helpers shared by the batched-form tests: seeded instance sets and the map
from node ids of a batched plan's tree to ids in each instance's own tree."""
import numpy as np

import workloads as w


def instances(sides, seed=3):
    """2D upwind convection-diffusion instances: side N, velocity direction
    uniform on the circle and Peclet number uniform in [1, 100], both seeded."""
    angles = w.uniform01(seed, len(sides)) * 2.0 * np.pi
    pe = 1.0 + 99.0 * w.uniform01(seed + 1, len(sides))
    return [w.convdiff2d_upwind(int(N), float(a), float(p)) for N, a, p in zip(sides, angles, pe)]


def records(flat):
    """[id, count, ids...] records of plan exports 3 / 4 as (id, tuple(ids))."""
    out, i = [], 0
    while i < len(flat):
        node, cnt = int(flat[i]), int(flat[i + 1])
        out.append((node, tuple(int(x) for x in flat[i + 2:i + 2 + cnt])))
        i += 2 + cnt
    return out


class Layout:
    """Maps node ids (4 h + kind, h = 2^level + j) of the union's tree to
    (instance, id in the instance's tree), or (None, None) outside them."""

    def __init__(self, inst, L):
        self.inst = np.asarray(inst).reshape(-1, 4)   # [first row, rows, first leaf, depth]
        self.L = L

    def local(self, node):
        h, kind = node >> 2, node & 3
        lev = h.bit_length() - 1
        j = h - (1 << lev)
        for k, (_, _, base, d) in enumerate(self.inst):
            top = self.L - int(d)
            if lev < top:
                continue
            lo = int(base) >> (self.L - lev)
            if lo <= j < lo + (1 << (lev - top)):
                return k, 4 * ((1 << (lev - top)) + (j - lo)) + kind
        return None, None
