"""The serving form's GPU executor (lrs_server_* without executor hooks):
factorizations resident on the device, solves against them merged into
multi-column GMRES runs on several worker threads.  Every result must be the
one lrs_solve gives for the same right-hand sides alone: true residual
<= 1e-10 per column and the solution within 1e-9 of the lone solve (in norm
and in every column's largest entry; merged and lone runs may pick different
traversal kernels for their column counts, so they agree to rounding, not
bit for bit)."""
import gc

import numpy as np
import pytest

import paper_1510_07363_gb300 as lrs
import workloads as w
from test_gpu_parity import assert_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_07363_gb300 import build
    build.build()
    lrs.load()


def test_serving_gpu_executor_matches_lrs_solve():
    As = [w.poisson3d(12, 12, 12), w.convdiff2d_upwind(40, 0.4, 30.0)]
    plans = [lrs.lrs_analyze(A, leaf_size=16) for A in As]
    srv = lrs.Server(hbm_budget=8 << 30, workers=3, max_batch_rhs=8)
    fs = [srv.factor(p, A.val, 1e-3) for p, A in zip(plans, As)]
    for f in fs:
        _, info = srv.wait(f)
        assert info.status == 0 and info.bytes > 0
    reqs = []
    for k in range(10):
        i = k % 2
        B = w.rhs_uniform(As[i].n, range(10 * k + 1, 10 * k + 2 + k % 3))
        reqs.append((i, srv.solve(fs[i], B, tol=1e-10), B))
    alone = [lrs.lrs_factor(p, A.val, 1e-3) for p, A in zip(plans, As)]
    merged = 0
    for i, t, B in reqs:
        X, info = srv.wait(t)
        assert info.status == 0 and info.rel_res <= 1e-10
        merged += info.batch_rhs > B.shape[1]
        for c in range(B.shape[1]):
            r = np.linalg.norm(w.spmv(As[i], X[:, c]) - B[:, c]) / np.linalg.norm(B[:, c])
            assert r <= 1e-10
        X1, info1, _ = alone[i].solve(B, restart=30, maxit=300, tol=1e-10)
        assert info1.status == 0
        assert_close(X, X1, 1e-9)
    st = srv.stats()
    assert st["resident"] == 2 and st["queued"] == 0
    for f in fs:
        srv.evict(f)
    assert srv.stats()["held_bytes"] == 0
    srv.close()


def test_serving_factor_outlives_a_dropped_plan():
    """A resident factor holds its own reference to the plan it was built
    from: the caller may drop the plan right after submitting the
    factorization, and later solves still read a live plan."""
    A = w.poisson3d(10, 10, 10)
    srv = lrs.Server(hbm_budget=4 << 30, workers=2, max_batch_rhs=4)
    t = srv.factor(lrs.lrs_analyze(A, leaf_size=16), A.val, 1e-3)   # no reference kept here
    gc.collect()
    _, info = srv.wait(t)
    assert info.status == 0
    gc.collect()
    B = w.rhs_uniform(A.n, [3, 4])
    X, sinfo = srv.wait(srv.solve(t, B, tol=1e-10))
    assert sinfo.status == 0
    f1 = lrs.lrs_factor(lrs.lrs_analyze(A, leaf_size=16), A.val, 1e-3)
    X1, _, _ = f1.solve(B, restart=30, maxit=300, tol=1e-10)
    assert_close(X, X1, 1e-9)
    srv.evict(t)
    srv.close()
