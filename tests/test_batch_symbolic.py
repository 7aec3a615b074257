"""CPU tests of the batched form's host analysis (lrs_analyze_batch): every
instance keeps the partitioning, batches, well-separated sets and
elimination neighbours it has alone -- checked record by record against the
oracle's analysis of that instance -- and clusters outside the instances'
subtrees carry no work.  No GPU call is made here."""
import numpy as np
import pytest

import oracle
import paper_1510_07363_gb300 as lrs
import workloads as w
from batch_util import Layout, instances as _instances, records as _records
from paper_1510_07363_gb300 import build as lrs_build


@pytest.fixture(scope="module", autouse=True)
def built():
    lrs_build.build()
    lrs.load()


SIDES = [9, 16, 12, 20, 7, 13]


@pytest.mark.parametrize("leaf,separation", [(8, 2), (16, 2), (8, 3)])
def test_batch_plan_is_the_instances_plans(leaf, separation):
    As = _instances(SIDES)
    plan = lrs.lrs_analyze_batch(As, leaf_size=leaf, separation=separation)
    inst = plan.export(lrs.EXPORT_INSTANCES).reshape(-1, 4)
    leaf_off = plan.export(lrs.EXPORT_LEAF_OFF)
    perm = plan.export(lrs.EXPORT_PERM)
    L = int(np.log2(len(leaf_off) - 1))
    singles = [oracle.Oracle(A, leaf_size=leaf, separation=separation) for A in As]
    for o in singles:
        o.factor(1e-3)
    # placement: rows in order, depths of the single analyses, aligned and disjoint leaf ranges
    assert np.array_equal(inst[:, 0], np.concatenate([[0], np.cumsum([A.n for A in As])[:-1]]))
    assert np.array_equal(inst[:, 1], [A.n for A in As])
    depths = [int(np.log2(len(o.export(oracle.EXPORT_LEAF_OFF)) - 1)) for o in singles]
    assert np.array_equal(inst[:, 3], depths)
    assert (1 << L) >= sum(1 << d for d in depths) > (1 << (L - 1))
    ranges = sorted((int(b), int(b) + (1 << int(d))) for _, _, b, d in inst)
    for (b, e), (_, d) in zip(ranges, sorted((int(b), int(d)) for _, _, b, d in inst)):
        assert b % (1 << d) == 0
    assert all(e0 <= b1 for (_, e0), (b1, _) in zip(ranges, ranges[1:]))
    # partition: each instance's positions and leaves are its own analysis, shifted
    for k, (r0, nk, base, d) in enumerate(inst):
        p0 = leaf_off[base]
        ref_off = singles[k].export(oracle.EXPORT_LEAF_OFF)
        assert np.array_equal(leaf_off[base:base + (1 << d) + 1] - p0, ref_off)
        assert np.array_equal(perm[p0:p0 + nk] - r0, singles[k].export(oracle.EXPORT_PERM))
    lay = Layout(inst, L)
    # compressions and eliminations: the union's records restricted to an
    # instance, in order, are that instance's records; the rest carry no work
    for what in (lrs.EXPORT_COMPRESS, lrs.EXPORT_ELIM):
        per = [[] for _ in As]
        for node, nbrs in _records(plan.export(what)):
            k, loc = lay.local(node)
            if k is None:
                h = node >> 2
                if what == lrs.EXPORT_COMPRESS:
                    assert nbrs == ()
                else:   # a structural zero-size node: super -> its black, black -> its red
                    assert nbrs in ((), (4 * h + (2 if node & 3 == 1 else 0),))
                continue
            mapped = []
            for v in nbrs:
                kv, lv = lay.local(v)
                assert kv == k
                mapped.append(lv)
            per[k].append((loc, tuple(sorted(mapped))))
        for k, o in enumerate(singles):
            ref = [(n, tuple(sorted(v))) for n, v in _records(o.export(what))]
            assert per[k] == ref, (what, k)


def test_batch_of_one_is_lrs_analyze():
    A = w.convdiff2d_upwind(20, 1.0, 40.0)
    one = lrs.lrs_analyze_batch([A], leaf_size=8)
    ref = lrs.lrs_analyze(A, leaf_size=8)
    for what in (lrs.EXPORT_PERM, lrs.EXPORT_LEAF_OFF, lrs.EXPORT_BATCHES, lrs.EXPORT_COMPRESS,
                 lrs.EXPORT_ELIM):
        assert np.array_equal(one.export(what), ref.export(what)), what
    assert np.array_equal(ref.export(lrs.EXPORT_INSTANCES), [0, A.n, 0, 6])   # 2^6 >= 400 / 8


def test_batch_rejects_bad_input():
    A = w.poisson2d(8, 8)
    bad = w.CSR(A.rowptr, A.colind.copy(), A.val, A.coords)
    bad.colind[3] = A.n
    with pytest.raises(lrs.LrsError) as e:
        lrs.lrs_analyze_batch([A, bad], leaf_size=8)
    assert e.value.code == lrs.LRS_ERR_INVALID_ARG
    with pytest.raises(lrs.LrsError):
        lrs.lrs_analyze_batch([A], leaf_size=0)


def test_batch_mixes_dimensions_and_tiny_instances():
    # a 3D instance, a 2D one and one smaller than two leaves (depth 1): each
    # keeps its own analysis, and the placement stays aligned and disjoint
    As = [w.poisson3d(6, 5, 4), w.convdiff2d_upwind(11, 0.3, 20.0), w.poisson2d(3, 4)]
    plan = lrs.lrs_analyze_batch(As, leaf_size=8)
    inst = plan.export(lrs.EXPORT_INSTANCES).reshape(-1, 4)
    leaf_off = plan.export(lrs.EXPORT_LEAF_OFF)
    perm = plan.export(lrs.EXPORT_PERM)
    for k, A in enumerate(As):
        one = lrs.lrs_analyze(A, leaf_size=8)
        r0, nk, base, d = (int(v) for v in inst[k])
        ref_off = one.export(lrs.EXPORT_LEAF_OFF)
        assert d == len(ref_off).bit_length() - 1 and base % (1 << d) == 0
        p0 = leaf_off[base]
        assert np.array_equal(leaf_off[base:base + (1 << d) + 1] - p0, ref_off)
        assert np.array_equal(perm[p0:p0 + nk] - r0, one.export(lrs.EXPORT_PERM))
    assert int(inst[2][3]) == 1                    # 12 unknowns, leaf 8: depth 1
