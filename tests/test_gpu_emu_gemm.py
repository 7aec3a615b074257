"""The FP64 block product emulated on the tensor cores (LRS_GEMM_EMU) against
an exact reference, through lrs_block_gemm.

Bound (per output, from the emulation's arithmetic): every group of 512
values of k (eight K chunks of 64, one exponent per row and column) contributes
at most 2^-41.5 max_k |a_ik| max_k |b_kj| (the maxima over the group) of
error; the running sum of an output is kept at the largest row exponent R_i
and the largest column exponent R_j seen so far, so a group is added (and an
earlier sum shifted) at that scale, losing at most one unit of 2^cut there,
2^(cut + R_i + R_j - 2105), twice per group (cut = 5 + ceil(log2 chunks));
and the final conversion rounds once to FP64.  With some margin
|C - C_exact| <= 2^-41 sum_groups(max |a_ik| max |b_kj|)
                 + 2 G 2^(cut + R_i + R_j - 2105) + 2^-52 |C_exact|.
The middle term is at most 2 G 2^(cut - 59) max_k |a_ik| max_k |b_kj| over
the whole contraction; it is zero when every group holds its row's and its
column's largest exponent (one group, or evenly scaled operands) and large
against the first one only when a row peaks in other groups than a column
(test_running_scale_of_rows_and_columns).
The reference is the product in extended precision (numpy longdouble: 64 or
113 significand bits), whose own error is far below the bound.
"""
import numpy as np
import pytest

import paper_1510_07363_gb300 as lrs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_07363_gb300 import build
    build.build()
    lrs.load()


def dev_cm(X):
    """A column-major CUDA copy of the host matrix X."""
    import torch
    return torch.tensor(np.asfortranarray(X)).t().contiguous().t().cuda() if X.ndim == 2 else None


def group_bound(opA, opB):
    """sum over groups of 512 values of k of max_k |a_ik| max_k |b_kj|, per output."""
    k = opA.shape[1]
    tot = np.zeros((opA.shape[0], opB.shape[1]))
    for c0 in range(0, k, 512):
        ma = np.abs(opA[:, c0:c0 + 512]).max(axis=1)
        mb = np.abs(opB[c0:c0 + 512, :]).max(axis=0)
        tot += np.outer(ma, mb)
    return tot


def biased_exponent(x):
    """the exponent the emulation gives a row or column whose largest |entry|
    is x: 1023 + floor(log2 x) for normal x, 1 for subnormals, 0 for zero"""
    x = np.asarray(x, dtype=np.float64)
    _, e = np.frexp(x)
    return np.where(x == 0, 0, np.where(x < np.finfo(np.float64).tiny, 1, e + 1022))


def running_scale_term(opA, opB):
    """2 G 2^(cut + R_i + R_j - 2105), per output: the rounding of each group's
    sum and of the running sum at the largest row and column exponents."""
    k = opA.shape[1]
    groups = (k + 511) // 512
    chunks = (k + 63) // 64
    cut = 5 + (int(np.ceil(np.log2(chunks))) if chunks > 1 else 0)
    Ri = biased_exponent(np.abs(opA).max(axis=1)) if k else np.zeros(opA.shape[0], dtype=int)
    Rj = biased_exponent(np.abs(opB).max(axis=0)) if k else np.zeros(opB.shape[1], dtype=int)
    return 2.0 * groups * np.ldexp(1.0, cut + Ri[:, None] + Rj[None, :] - 2105)


def run(engine, A, B, C0, transa=False, transb=False, accumulate=False, subtract=False):
    C = dev_cm(C0)
    lrs.lrs_block_gemm(engine, dev_cm(A), dev_cm(B), C, transa, transb, accumulate, subtract)
    return C.cpu().numpy()


def exact(opA, opB):
    return (opA.astype(np.longdouble) @ opB.astype(np.longdouble))


def check_bound(got, opA, opB, init=None, sign=1.0):
    ref = exact(opA, opB)
    full = ref * sign + (0 if init is None else init.astype(np.longdouble))
    err = np.abs(got.astype(np.longdouble) - full).astype(np.float64)
    bound = 2.0 ** -41 * group_bound(opA, opB) + running_scale_term(opA, opB) \
        + 2.0 ** -52 * np.abs(full).astype(np.float64) + (0 if init is None else 2.0 ** -52 * np.abs(init))
    assert np.all(err <= bound), float((err / np.maximum(bound, 1e-300)).max())
    return err, bound


def test_running_scale_of_rows_and_columns():
    """Rows of op(A) large in the first group of 512 values of k and small in
    the second, columns of op(B) the other way round: each group's product is
    ~2^-30 of max_k |a_ik| max_k |b_kj|, but the running sum is kept at the
    largest row and column exponents, so both groups lose ~30 bits to its
    rounding.  The error stays within the bound's running-scale term and far
    above the per-group term -- the case the middle term is there for (in the
    factorization's products it is a small entry's relative accuracy, not the
    block's normwise error)."""
    rng = np.random.default_rng(17)
    rows, cols, k = 40, 24, 1024
    opA = rng.standard_normal((rows, k))
    opB = rng.standard_normal((k, cols))
    opA[:, 512:] *= 2.0 ** -30
    opB[:512, :] *= 2.0 ** -30
    got = run(lrs.GEMM_EMU, opA, opB, np.zeros((rows, cols)))
    err, bound = check_bound(got, opA, opB)
    per_group = 2.0 ** -41 * group_bound(opA, opB)
    assert err.max() > 16 * per_group.max()       # the running scale, not the groups, sets the error
    ref = exact(opA, opB).astype(np.float64)
    assert np.abs(got - ref).max() <= 2.0 ** -40 * np.abs(ref).max() * 2.0 ** 22   # ~21 bits kept


SHAPES = [(1, 1, 1), (128, 64, 64), (200, 100, 150), (130, 70, 1000), (64, 300, 17), (257, 129, 3)]


@pytest.mark.parametrize("rows,cols,k", SHAPES)
@pytest.mark.parametrize("transa,transb", [(False, False), (True, False), (False, True), (True, True)])
def test_emulated_product_within_bound(rows, cols, k, transa, transb):
    rng = np.random.default_rng(rows * 7919 + cols * 31 + k + 2 * transa + transb)
    opA = rng.standard_normal((rows, k))
    opB = rng.standard_normal((k, cols))
    A = opA.T.copy() if transa else opA
    B = opB.T.copy() if transb else opB
    got = run(lrs.GEMM_EMU, A, B, np.zeros((rows, cols)), transa, transb)
    check_bound(got, opA, opB)


def test_wide_dynamic_range_and_zero_rows():
    """Entries spread over 2^-40..2^40 within rows and columns, zero rows and
    columns, subnormal entries: the bound holds entry by entry."""
    rng = np.random.default_rng(5)
    rows, cols, k = 150, 90, 300
    opA = rng.standard_normal((rows, k)) * 2.0 ** rng.integers(-40, 41, (rows, k))
    opB = rng.standard_normal((k, cols)) * 2.0 ** rng.integers(-40, 41, (k, cols))
    opA[7, :] = 0.0
    opB[:, 11] = 0.0
    opA[20, :5] = 5e-320                      # subnormal
    opA[21, :] *= 1e-300
    got = run(lrs.GEMM_EMU, opA, opB, np.zeros((rows, cols)))
    check_bound(got, opA, opB)
    assert np.all(got[7, :] == 0.0) and np.all(got[:, 11] == 0.0)


def test_small_integers_are_exact():
    """Integer operands whose products sum to below 2^53 are multiplied
    exactly (the tensor cores' FP32 sums of digit products are exact)."""
    rng = np.random.default_rng(9)
    opA = rng.integers(-2 ** 20, 2 ** 20, (128, 256)).astype(np.float64)
    opB = rng.integers(-2 ** 20, 2 ** 20, (256, 64)).astype(np.float64)
    got = run(lrs.GEMM_EMU, opA, opB, np.zeros((128, 64)))
    assert np.array_equal(got, opA @ opB)      # every partial sum is an integer below 2^53


def test_accumulate_subtract_and_long_contraction():
    rng = np.random.default_rng(11)
    rows, cols, k = 190, 80, 5000             # 79 chunks in the running integer sums
    opA = rng.standard_normal((rows, k))
    opB = rng.standard_normal((k, cols))
    C0 = rng.standard_normal((rows, cols)) * 100.0
    got = run(lrs.GEMM_EMU, opA, opB, C0, accumulate=True, subtract=True)
    check_bound(got, opA, opB, init=C0, sign=-1.0)


def test_not_finite_rows_and_columns_become_nan():
    rng = np.random.default_rng(13)
    opA = rng.standard_normal((100, 70))
    opB = rng.standard_normal((70, 40))
    opA[3, 10] = np.nan
    opB[5, 7] = np.inf
    got = run(lrs.GEMM_EMU, opA, opB, np.zeros((100, 40)))
    assert np.all(np.isnan(got[3, :])) and np.all(np.isnan(got[:, 7]))
    mask = np.ones_like(got, dtype=bool)
    mask[3, :] = False
    mask[:, 7] = False
    A2, B2 = opA.copy(), opB.copy()
    A2[3, :] = 0.0
    B2[:, 7] = 0.0
    err, bound = check_bound(np.where(mask, got, 0.0), A2, B2)


def test_engines_agree():
    """The three engines on the same product: FP64 and the emulation within
    their bounds, the TF32 split within its ~1e-6 relative error."""
    rng = np.random.default_rng(17)
    opA = rng.standard_normal((300, 200))
    opB = rng.standard_normal((200, 150))
    ref = (opA.astype(np.longdouble) @ opB.astype(np.longdouble)).astype(np.float64)
    e64 = run(lrs.GEMM_FP64, opA, opB, np.zeros((300, 150)))
    emu = run(lrs.GEMM_EMU, opA, opB, np.zeros((300, 150)))
    t32 = run(lrs.GEMM_TF32, opA, opB, np.zeros((300, 150)))
    scale = np.abs(opA).max() * np.abs(opB).max() * 200
    assert np.abs(e64 - ref).max() <= 200 * 2.0 ** -53 * scale
    check_bound(emu, opA, opB)
    assert np.abs(t32 - ref).max() <= 1e-5 * scale
