"""GPU parity of the batched form (lrs_analyze_batch): several independent
convection-diffusion matrices factored together and solved by one GMRES per
instance and right-hand side.  Each instance is checked against the FP64
oracle run on that instance alone, with the tolerances of the single-matrix
parity tests: ranks equal except at ties, singular values >= 1e-3 sigma_0 to
1e-6 sigma_0 + 1e-9 max|a_ij| (noise-level compressions excepted), one
apply to 1e-9, GMRES to 1e-10 with iteration counts within +-1 and solutions
within 1e-9 (in norm and in every column's largest entry); and against the
same instance factored alone on the GPU (the same result alone and in the
batch, to 1e-9)."""
import numpy as np
import pytest

import oracle
import paper_1510_07363_gb300 as lrs
import workloads as w
from batch_util import Layout, instances, records
from test_gpu_parity import assert_close, rank_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_07363_gb300 import build
    build.build()
    lrs.load()


SIDES = [9, 16, 12, 20, 7, 13, 24]
LEAF = 8


def _split(X, As):
    off = np.concatenate([[0], np.cumsum([A.n for A in As])])
    return [X[off[k]:off[k + 1]] for k in range(len(As))]


@pytest.mark.parametrize("eps", [1e-2, 1e-4])
def test_batched_form_against_oracle(eps):
    As = instances(SIDES)
    plan = lrs.lrs_analyze_batch(As, leaf_size=LEAF)
    f = lrs.lrs_factor(plan, np.concatenate([A.val for A in As]), eps)
    assert f.stats()["symmetric"] == 0
    inst = plan.export(lrs.EXPORT_INSTANCES).reshape(-1, 4)
    L = int(np.log2(len(plan.export(lrs.EXPORT_LEAF_OFF)) - 1))
    lay = Layout(inst, L)
    recs = records(plan.export(lrs.EXPORT_COMPRESS))
    ranks = f.ranks()
    assert len(ranks) == len(recs)
    per = [[] for _ in As]
    for idx, (node, _) in enumerate(recs):
        k, _ = lay.local(node)
        if k is None:
            assert ranks[idx] == 0
        else:
            per[k].append(idx)
    singles = []
    tied = set()
    for k, A in enumerate(As):
        o = oracle.Oracle(A, leaf_size=LEAF)
        o.factor(eps)
        singles.append(o)
        comps = o.compressions()
        assert len(comps) == len(per[k])
        amax = np.abs(A.val).max()
        if rank_parity(f, comps, eps, amax, idx=per[k]):
            tied.add(k)
    Bs = [w.rhs_uniform(A.n, [k + 1, k + 101]) for k, A in enumerate(As)]
    B = np.vstack(Bs)
    for k, (Yk, o) in enumerate(zip(_split(f.apply(B), As), singles)):
        if k not in tied:
            assert_close(Yk, o.apply(Bs[k]), 1e-9)
    X, info, its = f.solve(B, restart=30, maxit=300, tol=1e-10)
    assert info.status == 0
    its = np.asarray(its).reshape(B.shape[1], len(As))     # group c * count + k
    for k, (A, Xk, o) in enumerate(zip(As, _split(X, As), singles)):
        for c in range(B.shape[1]):
            r = np.linalg.norm(w.spmv(A, Xk[:, c]) - Bs[k][:, c]) / np.linalg.norm(Bs[k][:, c])
            assert r <= 1e-10, (k, c)
        Xo, its_o, _, st = o.gmres(Bs[k], restart=30, maxit=300, tol=1e-10)
        assert st == 0
        if k not in tied:
            assert np.all(np.abs(its[:, k].astype(int) - np.asarray(its_o).astype(int)) <= 1), k
        assert_close(Xk, Xo, 1e-9)
        # the same instance factored and solved alone on the GPU
        f1 = lrs.lrs_factor(lrs.lrs_analyze(A, leaf_size=LEAF), A.val, eps)
        X1, info1, its1 = f1.solve(Bs[k], restart=30, maxit=300, tol=1e-10)
        assert info1.status == 0
        assert np.array_equal(np.asarray(its1), its[:, k]), k
        assert_close(Xk, X1, 1e-9)


def test_batched_form_solve_on_device_and_zero_rhs():
    # device pointers give the host-pointer result; an all-zero instance
    # column converges at once with x = 0 while the others iterate
    torch = pytest.importorskip("torch")
    As = instances([10, 17, 6], seed=9)
    plan = lrs.lrs_analyze_batch(As, leaf_size=LEAF)
    f = lrs.lrs_factor(plan, np.concatenate([A.val for A in As]), 1e-3)
    B = np.vstack([w.rhs_uniform(A.n, [5 + k]) for k, A in enumerate(As)])
    B[As[0].n:As[0].n + As[1].n] = 0.0
    X, info, its = f.solve(B, restart=30, maxit=300, tol=1e-10)
    assert info.status == 0
    assert np.all(X[As[0].n:As[0].n + As[1].n] == 0.0)
    assert its[1] == 0 and its[0] > 0 and its[2] > 0
    Xd, info_d, its_d = f.solve(torch.from_numpy(B).cuda(), restart=30, maxit=300, tol=1e-10)
    assert info_d.status == 0 and np.array_equal(its_d, its)
    assert np.array_equal(Xd.cpu().numpy(), X)


def test_rounding_level_gram_columns_and_oversize_blocks():
    # an upwind instance (side 325, flow along -y, Peclet 61) whose compression
    # Gram matrices hand the tridiagonal reduction columns with subnormal
    # squared norms: the reflectors must stay finite and GMRES converge
    A = w.convdiff2d_upwind(325, 4.758394351771332, 61.070309033874075)
    plan = lrs.lrs_analyze(A, leaf_size=64)
    f = lrs.lrs_factor(plan, A.val, 1e-2)
    B = w.rhs_uniform(A.n, [1])
    X, info, _ = f.solve(B, restart=30, maxit=300, tol=1e-10)
    assert info.status == 0
    assert np.linalg.norm(w.spmv(A, X[:, 0]) - B[:, 0]) / np.linalg.norm(B) <= 1e-10


def test_oversize_pivot_block_is_refused_before_launch():
    # depth 2 on 140 x 140 gives pivot blocks of 9800 unknowns, more than the
    # inverse kernels keep in shared memory (9682): refused before any launch
    A = w.poisson2d(140, 140)
    with pytest.raises(lrs.LrsError) as e:
        lrs.lrs_factor(lrs.lrs_analyze(A, depth=2), A.val, 1e-2)
    assert e.value.code == lrs.LRS_ERR_INVALID_ARG
