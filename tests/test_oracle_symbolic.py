"""Symbolic pins of the oracle: the nested partitioning, the per-level node
counts of Algorithm 1 and the sparsity-preservation theorem (Thm. sparse)."""
from collections import deque

import numpy as np
import pytest

import oracle
import workloads as w


def parse_records(flat):
    out, i = [], 0
    while i < len(flat):
        node, deg = int(flat[i]), int(flat[i + 1])
        out.append((node, [int(v) for v in flat[i + 2:i + 2 + deg]]))
        i += 2 + deg
    return out


def parse_batches(flat):
    levels, i = {}, 0
    while i < len(flat):
        lev, nb = int(flat[i]), int(flat[i + 1])
        i += 2
        bl = []
        for _ in range(nb):
            c = int(flat[i])
            bl.append([int(v) for v in flat[i + 1:i + 1 + c]])
            i += 1 + c
        levels[lev] = bl
    return levels


def cluster_graphs(A, perm, leaf_off, L):
    """Adjacency sets of every level, from the CSR pattern (Def. adj)."""
    leaf_of = np.empty(A.n, dtype=np.int64)
    for j in range(len(leaf_off) - 1):
        leaf_of[perm[leaf_off[j]:leaf_off[j + 1]]] = j
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    a, b = leaf_of[rows], leaf_of[A.colind]
    adj = []
    for i in range(L + 1):
        ca, cb = a >> (L - i), b >> (L - i)
        g = [set() for _ in range(1 << i)]
        for x, y in zip(ca[ca != cb], cb[ca != cb]):
            g[x].add(int(y)); g[y].add(int(x))
        adj.append(g)
    return adj


def distance(g, x, y, cap=4):
    if x == y:
        return 0
    seen, dq = {x: 0}, deque([x])
    while dq:
        u = dq.popleft()
        if seen[u] >= cap:
            break
        for v in g[u]:
            if v not in seen:
                seen[v] = seen[u] + 1
                if v == y:
                    return seen[v]
                dq.append(v)
    return cap + 1


def cl(node):
    h = node >> 2
    lev = h.bit_length() - 1
    return lev, h - (1 << lev)


@pytest.mark.parametrize("make,leaf,eps", [
    (lambda: w.poisson2d(32, 32), 16, 1e-4),
    (lambda: w.poisson3d(8, 8, 8), 16, 1e-2),
    (lambda: w.convdiff2d_upwind(20, 1.0, 40.0), 8, 1e-3),
])
def test_sparsity_theorem_and_counts(make, leaf, eps):
    A = make()
    o = oracle.Oracle(A, leaf_size=leaf)
    o.factor(eps)
    L = o.depth
    perm, leaf_off = o.export(oracle.EXPORT_PERM), o.export(oracle.EXPORT_LEAF_OFF)
    adj = cluster_graphs(A, perm, leaf_off, L)
    # Compress: every well-separated neighbour is at distance exactly 2
    # (Def. wellSep / Cor. dist: > 1; Thm. sparse: never > 2).
    comps = parse_records(o.export(oracle.EXPORT_COMPRESS))
    for s, ws in comps:
        ls, js = cl(s)
        for p in ws:
            lp, jp = cl(p)
            assert lp == ls
            assert distance(adj[ls], js, jp) == 2
    # Eliminate: after compression every neighbour is adjacent (distance <= 1)
    elims = parse_records(o.export(oracle.EXPORT_ELIM))
    for p, nb in elims:
        lp, jp = cl(p)
        for q in nb:
            lq, jq = cl(q)
            assert lq == lp and distance(adj[lp], jp, jq) <= 1
    # Alg. 1: 2^(i-1) super-nodes at level i, each compressed once and
    # eliminated with its black-node right after it
    batches = parse_batches(o.export(oracle.EXPORT_BATCHES))
    assert sorted(batches) == list(range(1, L + 1))
    order = []
    for i in range(L, 0, -1):
        supers = [s for b in batches[i] for s in b]
        assert sorted(cl(s)[1] for s in supers) == list(range(1 << (i - 1)))
        for s in supers:
            order += [s, s + 1]          # black(i, j) id = super(i, j) id + 1
    assert [p for p, _ in elims] == order
    assert [s for s, _ in comps] == order[0::2]
    # batch members share no edge: none is a neighbour of another at its
    # elimination
    nbrs = dict(elims)
    for i in range(L, 0, -1):
        for b in batches[i]:
            for s in b:
                assert not (set(nbrs[s]) & set(b))


@pytest.mark.parametrize("shape,leaf,box", [
    ((32, 32), 16, (4, 4)),
    ((64, 64, 64), 64, (4, 4, 4)),
    ((16, 16, 8), 64, (4, 4, 4)),
])
def test_bisection_gives_boxes(shape, leaf, box):
    A = w.poisson2d(*shape) if len(shape) == 2 else w.poisson3d(*shape)
    o = oracle.Oracle(A, leaf_size=leaf)
    assert 2 ** o.depth == A.n // leaf
    perm, off = o.export(oracle.EXPORT_PERM), o.export(oracle.EXPORT_LEAF_OFF)
    assert sorted(perm.tolist()) == list(range(A.n))
    for j in range(len(off) - 1):
        c = A.coords[perm[off[j]:off[j + 1]]]
        ext = tuple(int(v) for v in c.max(0) - c.min(0) + 1)
        assert ext == box and len(c) == int(np.prod(box))
    # leaf 0 holds the lowest corner; siblings split the longest axis
    c0 = A.coords[perm[off[0]:off[1]]]
    assert c0.min(0).tolist() == [0.0] * len(shape)


@pytest.mark.parametrize("make,leaf", [
    (lambda: w.poisson2d(32, 32), 8),
    (lambda: w.poisson3d(8, 8, 8), 8),
])
def test_separation3_distances(make, leaf):
    # the variant of Sec. 7: every compressed interaction is at cluster
    # distance >= 3 (Def. distance), and after compression every neighbour of
    # an eliminated node is within distance 2 -- the analogue of Thm. sparse
    A = make()
    o = oracle.Oracle(A, leaf_size=leaf, separation=3)
    o.factor(1e-2)
    L = o.depth
    adj = cluster_graphs(A, o.export(oracle.EXPORT_PERM), o.export(oracle.EXPORT_LEAF_OFF), L)
    n_ws = 0
    for s, ws in parse_records(o.export(oracle.EXPORT_COMPRESS)):
        ls, js = cl(s)
        for p in ws:
            lp, jp = cl(p)
            assert lp == ls and distance(adj[ls], js, jp) >= 3
            n_ws += 1
    assert n_ws > 0
    for p, nb in parse_records(o.export(oracle.EXPORT_ELIM)):
        lp, jp = cl(p)
        for q in nb:
            lq, jq = cl(q)
            assert lq == lp and distance(adj[lp], jp, jq) <= 2
