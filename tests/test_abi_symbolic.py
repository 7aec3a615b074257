"""CPU tests of the C-ABI boundary: the library loads, exports every symbol
that include/lrs.h declares, rejects bad arguments, and its host analysis
(nested partitioning, batches, well-separated sets, elimination neighbours)
equals the oracle's bit for bit.  No GPU call is made here."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_1510_07363_gb300 as lrs
import workloads as w
from paper_1510_07363_gb300 import build as lrs_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    lrs_build.build()
    lrs.load()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "lrs.h")).read()
    return sorted(set(re.findall(r"LRS_API\s+[\w\s\*]+?\b(lrs_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    names = declared_symbols()
    assert len(names) >= 10
    assert sorted(lrs.ABI_SYMBOLS) == names
    lib = ctypes.CDLL(lrs.LIB_PATH)
    for name in names:
        assert hasattr(lib, name), name


def test_status_strings():
    for code in range(0, 9):
        assert lrs.status_string(code) != "unknown status"
    assert lrs.status_string(99) == "unknown status"


def test_analyze_rejects_bad_input():
    A = w.poisson2d(8, 8)
    bad = w.CSR(A.rowptr, A.colind.copy(), A.val, A.coords)
    bad.colind[3] = A.n            # column out of range
    with pytest.raises(lrs.LrsError) as e:
        lrs.lrs_analyze(bad, leaf_size=8)
    assert e.value.code == lrs.LRS_ERR_INVALID_ARG
    dup = w.CSR(A.rowptr, A.colind.copy(), A.val, A.coords)
    dup.colind[1] = dup.colind[0]  # repeated column in row 0
    with pytest.raises(lrs.LrsError):
        lrs.lrs_analyze(dup, leaf_size=8)
    with pytest.raises(lrs.LrsError):
        lrs.lrs_analyze(A, leaf_size=0)
    with pytest.raises(lrs.LrsError):
        lrs.lrs_analyze(A, depth=30)
    nan = w.CSR(A.rowptr, A.colind, A.val, A.coords.copy())
    nan.coords[5, 1] = np.nan      # bisection needs ordered coordinates
    with pytest.raises(lrs.LrsError) as e:
        lrs.lrs_analyze(nan, leaf_size=8)
    assert e.value.code == lrs.LRS_ERR_INVALID_ARG


CASES = [
    ("poisson2d_32x32_leaf16", lambda: w.poisson2d(32, 32), 16),
    ("poisson2d_12x10_leaf8", lambda: w.poisson2d(12, 10), 8),
    ("poisson3d_8x8x8_leaf16", lambda: w.poisson3d(8, 8, 8), 16),
    ("poisson3d_16x16x16_leaf64", lambda: w.poisson3d(16, 16, 16), 64),
    ("convdiff_20_leaf8", lambda: w.convdiff2d_upwind(20, 1.0, 40.0), 8),
    ("varcoef_6x7x5_leaf8", lambda: w.varcoef3d(6, 7, 5, seed=2), 8),
]


@pytest.mark.parametrize("name,make,leaf", CASES, ids=[c[0] for c in CASES])
def test_symbolic_plan_equals_oracle(name, make, leaf):
    A = make()
    plan = lrs.lrs_analyze(A, leaf_size=leaf)
    o = oracle.Oracle(A, leaf_size=leaf)
    o.factor(1e-3)          # the oracle's symbolic records come out of its factorization
    for what in (oracle.EXPORT_PERM, oracle.EXPORT_LEAF_OFF, oracle.EXPORT_BATCHES,
                 oracle.EXPORT_COMPRESS, oracle.EXPORT_ELIM):
        mine, ref = plan.export(what), o.export(what)
        assert mine.shape == ref.shape, what
        assert np.array_equal(mine, ref), what


def test_symbolic_plan_full_size_3d_partition():
    # the 64^3 leaf-64 workload: partition and leaf offsets equal the oracle's
    A = w.poisson3d(64, 64, 64)
    plan = lrs.lrs_analyze(A, leaf_size=64)
    o = oracle.Oracle(A, leaf_size=64)
    assert np.array_equal(plan.export(lrs.EXPORT_PERM), o.export(oracle.EXPORT_PERM))
    assert np.array_equal(plan.export(lrs.EXPORT_LEAF_OFF), o.export(oracle.EXPORT_LEAF_OFF))



@pytest.mark.parametrize("name,make,leaf", [c for c in CASES if c[0] in
                                            ("poisson2d_32x32_leaf16", "poisson3d_8x8x8_leaf16", "convdiff_20_leaf8")],
                         ids=["poisson2d_32x32_leaf16", "poisson3d_8x8x8_leaf16", "convdiff_20_leaf8"])
def test_symbolic_plan_equals_oracle_separation3(name, make, leaf):
    # the separation variant (cluster distance >= 3): both sides' plans agree
    A = make()
    plan = lrs.lrs_analyze(A, leaf_size=leaf, separation=3)
    o = oracle.Oracle(A, leaf_size=leaf, separation=3)
    o.factor(1e-3)
    for what in (oracle.EXPORT_BATCHES, oracle.EXPORT_COMPRESS, oracle.EXPORT_ELIM):
        assert np.array_equal(plan.export(what), o.export(what)), what
    base = lrs.lrs_analyze(A, leaf_size=leaf)
    assert not np.array_equal(plan.export(lrs.EXPORT_COMPRESS), base.export(lrs.EXPORT_COMPRESS))
    with pytest.raises(lrs.LrsError):
        lrs.lrs_analyze(A, leaf_size=leaf, separation=1)


@pytest.mark.parametrize("seed,separation", [(1, 2), (2, 2), (3, 3), (4, 3)])
def test_symbolic_plan_equals_oracle_on_random_graphs(seed, separation):
    A = w.knn_graph(500, 5, seed)
    plan = lrs.lrs_analyze(A, leaf_size=12, separation=separation)
    o = oracle.Oracle(A, leaf_size=12, separation=separation)
    o.factor(1e-2)
    for what in (oracle.EXPORT_PERM, oracle.EXPORT_LEAF_OFF, oracle.EXPORT_BATCHES,
                 oracle.EXPORT_COMPRESS, oracle.EXPORT_ELIM):
        assert np.array_equal(plan.export(what), o.export(what)), what
