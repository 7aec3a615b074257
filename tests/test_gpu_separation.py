"""The numeric factorization with the distance-3 separation variant (Sec. 7:
well-separated means cluster distance at least 3) against the oracle run
with the same rule.  Tolerances are those of the single-matrix parity tests:
ranks equal except at ties, singular values >= 1e-3 sigma_0 to 1e-6 sigma_0
+ 1e-9 max|a|, one apply to 1e-9, GMRES to 1e-10 with iterations within +-1
and solutions within 1e-9."""
import numpy as np
import pytest

import oracle
import paper_1510_07363_gb300 as lrs
import workloads as w
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


@pytest.mark.parametrize("make,leaf,eps", [
    (lambda: w.poisson2d(32, 32), 8, 1e-2),
    (lambda: w.poisson3d(10, 10, 10), 16, 1e-4),
    (lambda: w.convdiff2d_upwind(24, 1.3, 50.0), 8, 1e-2),
], ids=["poisson2d_32", "poisson3d_10", "convdiff_24"])
def test_separation3_factorization_against_oracle(make, leaf, eps):
    A = make()
    o = oracle.Oracle(A, leaf_size=leaf, separation=3)
    o.factor(eps)
    f = lrs.lrs_factor(lrs.lrs_analyze(A, leaf_size=leaf, separation=3), A.val, eps)
    comps = o.compressions()
    assert len(f.ranks()) == len(comps)
    ties = rank_parity(f, comps, eps, np.abs(A.val).max())
    B = w.rhs_uniform(A.n, [1, 2])
    if not ties:
        assert_close(f.apply(B), o.apply(B), 1e-9)
    X, info, its = f.solve(B, restart=30, maxit=300, tol=1e-10)
    Xo, its_o, _, st = o.gmres(B, restart=30, maxit=300, tol=1e-10)
    assert info.status == 0 and st == 0
    assert_close(X, Xo, 1e-9)
    if not ties:
        assert np.all(np.abs(its.astype(int) - its_o.astype(int)) <= 1)
