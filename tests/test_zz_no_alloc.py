"""lrs_apply_static, the apply that allocates no device memory (for callers
that cannot call cudaMalloc at apply time), must return what lrs_apply
returns on the same factor and input -- on two calls in a row, since the
static scratch it reuses keeps the previous call's contents.  This file is
collected last so that a failure here comes after every other test ran."""
import ctypes

import numpy as np
import pytest

import paper_1510_07363_gb300 as lrs
import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ready():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_07363_gb300 import build
    build.build()
    lrs.load()
    return torch


def test_apply_static_matches_apply_twice(ready):
    torch = ready
    A = w.poisson3d(12, 12, 12)
    f = lrs.lrs_factor(lrs.lrs_analyze(A, leaf_size=32), A.val, 1e-3)
    for seeds in ([1, 2, 3], [7]):                      # two calls in a row, different shapes
        B = torch.tensor(w.rhs_uniform(A.n, seeds), device="cuda")
        ref = f.apply(B).cpu().numpy()                  # the allocating entry point
        got = lrs.lrs_apply_static(f, B).cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_apply_static_allocates_nothing(ready):
    """After a first call (which looks up the array's address), a call with
    a caller-provided output leaves the caching allocator's allocation count
    and the device's free memory unchanged.  The vectors here (ext_n * 4
    doubles, over 2 MiB each) would show up in either if they were allocated."""
    torch = ready
    A = w.poisson3d(40, 40, 40)
    f = lrs.lrs_factor(lrs.lrs_analyze(A, leaf_size=64), A.val, 1e-2)
    assert f.stats()["ext_n"] * 4 * 8 > (2 << 20)
    B = torch.tensor(w.rhs_uniform(A.n, [1, 2, 3, 4]), device="cuda")
    X = torch.empty_like(B)
    lrs.lrs_apply_static(f, B, out=X)                  # warm-up: address lookup, module load
    torch.cuda.synchronize()
    count0 = torch.cuda.memory_stats()["allocation.all.allocated"]
    free0 = torch.cuda.mem_get_info()[0]
    lrs.lrs_apply_static(f, B, out=X)
    torch.cuda.synchronize()
    assert torch.cuda.memory_stats()["allocation.all.allocated"] == count0
    assert torch.cuda.mem_get_info()[0] >= free0 - (1 << 20)
    ref = f.apply(B).cpu().numpy()
    assert np.linalg.norm(X.cpu().numpy() - ref) <= 1e-12 * np.linalg.norm(ref)


def test_apply_static_rejects_oversize_request(ready):
    torch = ready
    A = w.poisson2d(16, 16)
    f = lrs.lrs_factor(lrs.lrs_analyze(A, leaf_size=16), A.val, 1e-3)
    ext = f.stats()["ext_n"]
    nrhs = (1 << 21) // ext + 1                         # beyond the static array
    B = torch.zeros((nrhs, A.n), dtype=torch.float64, device="cuda")
    X = torch.zeros_like(B)
    code = lrs.load().lrs_apply_static(f._h, ctypes.c_void_p(B.data_ptr()), ctypes.c_void_p(X.data_ptr()), nrhs)
    assert code == lrs.LRS_ERR_INVALID_ARG
