"""The resident dense kernels' CTAs wait on one another through flags in
global memory; every such wait is bounded.  This makes a wait run out on the
GPU (a flag that nothing sets) and checks that it gives up after its limit,
reports the timeout through the kernel status, and leaves the context usable."""
import numpy as np
import pytest

import paper_1510_07363_gb300 as lrs
import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_07363_gb300 import build
    build.build()
    lrs.load()


def test_wait_on_an_unset_flag_times_out_and_the_context_survives():
    code, ms = lrs.lrs_selftest_bounded_wait()
    assert code == lrs.LRS_ERR_TIMEOUT
    assert 1900.0 <= ms <= 10000.0          # the 2 s limit, not an endless spin
    # the device is still usable: a small factorization and solve succeed
    A = w.poisson2d(16, 16)
    f = lrs.lrs_factor(lrs.lrs_analyze(A, leaf_size=16), A.val, 1e-4)
    x, info, its = f.solve(w.rhs_uniform(A.n, [1])[:, 0], tol=1e-10)
    assert info.status == 0
    assert np.linalg.norm(w.spmv(A, x) - w.rhs_uniform(A.n, [1])[:, 0]) <= 1e-9 * np.sqrt(A.n)
