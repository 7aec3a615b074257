"""CPU tests of the serving form's request loop (lrs_server_*): admission by
the HBM budget, continuous batching of the solves against one factor, work
on different factors running at once, eviction and error propagation.  The
device is replaced by the executor hooks: a fake whose 'factor' of a plan at
accuracy eps is the scalar s = 1 + eps and whose solve writes x = s b after a
short sleep, recording what ran when.  No GPU call is made here."""
import ctypes
import threading
import time

import numpy as np
import pytest

import paper_1510_07363_gb300 as lrs
import workloads as w
from paper_1510_07363_gb300 import build as lrs_build


@pytest.fixture(scope="module", autouse=True)
def built():
    lrs_build.build()
    lrs.load()


class FakeExecutor:
    def __init__(self, n_of_plan, bytes_of_eps, factor_s=0.05, solve_s=0.05, fail_eps=None):
        self.n_of_plan = n_of_plan
        self.bytes_of_eps = bytes_of_eps
        self.factor_s, self.solve_s = factor_s, solve_s
        self.fail_eps = fail_eps
        self.lock = threading.Lock()
        self.handles, self.next = {}, 1
        self.running = self.max_running = 0
        self.held = self.max_held = 0
        self.solve_cols = []
        self.events = []

    def _enter(self):
        with self.lock:
            self.running += 1
            self.max_running = max(self.max_running, self.running)

    def _leave(self):
        with self.lock:
            self.running -= 1

    def factor(self, plan, val, eps, prec):
        self._enter()
        time.sleep(self.factor_s)
        self._leave()
        if self.fail_eps is not None and eps == self.fail_eps:
            return lrs.LRS_ERR_SINGULAR_PIVOT, None, 0
        with self.lock:
            h = self.next
            self.next += 1
            nb = self.bytes_of_eps(eps)
            self.handles[h] = (self.n_of_plan[plan], 1.0 + eps, nb)
            self.held += nb
            self.max_held = max(self.max_held, self.held)
            self.events.append(("built", h, time.monotonic()))
        return 0, h, nb

    def solve(self, h, b, x, nrhs, restart, maxit, tol):
        n, s, _ = self.handles[h]
        B = np.ctypeslib.as_array(ctypes.cast(b, ctypes.POINTER(ctypes.c_double)), shape=(n * nrhs,))
        X = np.ctypeslib.as_array(ctypes.cast(x, ctypes.POINTER(ctypes.c_double)), shape=(n * nrhs,))
        self._enter()
        time.sleep(self.solve_s)
        X[:] = s * B
        self._leave()
        with self.lock:
            self.solve_cols.append(nrhs)
        return 0, 3, 1e-12

    def release(self, h):
        with self.lock:
            self.held -= self.handles.pop(h)[2]
            self.events.append(("released", h, time.monotonic()))


def _plans(sides):
    As = [w.poisson2d(N, N) for N in sides]
    plans = [lrs.lrs_analyze(A, leaf_size=16) for A in As]
    return As, plans


def _n_of(plans, As):
    return {plan._h.value: A.n for plan, A in zip(plans, As)}


def test_admission_waits_for_the_budget():
    As, plans = _plans([12, 12])
    fake = FakeExecutor(_n_of(plans, As), lambda eps: 60)
    srv = lrs.Server(hbm_budget=100, workers=2, executor=fake)
    a = srv.factor(plans[0], As[0].val, 1e-2, reserve_bytes=60)
    b = srv.factor(plans[1], As[1].val, 1e-3, reserve_bytes=60)
    _, ia = srv.wait(a)
    assert ia.status == 0 and ia.bytes == 60
    time.sleep(0.3)
    st = srv.stats()
    assert st["resident"] == 1 and st["queued"] == 1 and st["held_bytes"] == 60
    t_evict = time.monotonic()
    srv.evict(a)
    _, ib = srv.wait(b)
    assert ib.status == 0
    assert ib.queue_ms >= 300.0                     # admitted only after the eviction
    built_b = [t for e, h, t in fake.events if e == "built"][-1]
    assert built_b >= t_evict
    assert fake.max_held <= 100
    with pytest.raises(lrs.LrsError) as e:
        srv.factor(plans[0], As[0].val, 1e-2, reserve_bytes=101)
    assert e.value.code == lrs.LRS_ERR_OOM
    srv.close()


def test_solves_against_one_factor_are_merged():
    As, plans = _plans([10])
    A, plan = As[0], plans[0]
    fake = FakeExecutor(_n_of(plans, As), lambda eps: 1, solve_s=0.15)
    srv = lrs.Server(hbm_budget=1 << 40, workers=2, max_batch_rhs=8, executor=fake)
    f = srv.factor(plan, A.val, 0.25)
    srv.wait(f)
    rng = np.random.default_rng(0)
    reqs = []
    for k in range(12):
        B = rng.standard_normal((A.n, 1 + k % 3))
        reqs.append((srv.solve(f, B), B))
    merged = 0
    for t, B in reqs:
        X, info = srv.wait(t)
        assert info.status == 0
        assert np.array_equal(X, 1.25 * B)          # each request gets its own columns back
        assert info.batch_rhs >= B.shape[1]
        merged += info.batch_rhs > B.shape[1]
    assert merged > 0
    assert max(fake.solve_cols) <= 8 and sum(fake.solve_cols) == sum(B.shape[1] for _, B in reqs)
    assert len(fake.solve_cols) < len(reqs)
    assert fake.max_running == 1                    # one factor: one solve at a time
    srv.close()


def test_work_on_different_factors_overlaps():
    As, plans = _plans([8, 9])
    fake = FakeExecutor(_n_of(plans, As), lambda eps: 1, solve_s=0.2)
    srv = lrs.Server(hbm_budget=1 << 40, workers=2, executor=fake)
    fs = [srv.factor(p, A.val, 1e-2) for p, A in zip(plans, As)]
    for f in fs:
        srv.wait(f)
    ts = [srv.solve(f, np.ones(A.n)) for f, A in zip(fs, As)]
    for t, A in zip(ts, As):
        X, info = srv.wait(t)
        assert info.status == 0 and X.shape == (A.n,)
    assert fake.max_running == 2
    srv.close()


def test_failures_eviction_and_bad_tickets():
    As, plans = _plans([8, 8])
    fake = FakeExecutor(_n_of(plans, As), lambda eps: 50, factor_s=0.2, fail_eps=0.5)
    srv = lrs.Server(hbm_budget=100, workers=1, executor=fake)
    bad = srv.factor(plans[0], As[0].val, 0.5, reserve_bytes=50)   # the fake fails this one
    s1 = srv.solve(bad, np.ones(As[0].n))          # queued before the failure is known
    _, info = srv.wait(bad)
    assert info.status == lrs.LRS_ERR_SINGULAR_PIVOT
    _, info = srv.wait(s1)
    assert info.status == lrs.LRS_ERR_SINGULAR_PIVOT
    with pytest.raises(lrs.LrsError) as e:          # known failure: refused at once
        srv.solve(bad, np.ones(As[0].n))
    assert e.value.code == lrs.LRS_ERR_SINGULAR_PIVOT
    good = srv.factor(plans[1], As[1].val, 1e-2, reserve_bytes=50)
    srv.wait(good)
    srv.evict(good)
    with pytest.raises(lrs.LrsError) as e:
        srv.solve(good, np.ones(As[1].n))
    assert e.value.code in (lrs.LRS_ERR_STATE, lrs.LRS_ERR_INVALID_ARG)
    with pytest.raises(lrs.LrsError) as e:
        srv.wait(123456)
    assert e.value.code == lrs.LRS_ERR_INVALID_ARG
    with pytest.raises(lrs.LrsError) as e:
        srv.solve(987654, np.ones(4))
    assert e.value.code == lrs.LRS_ERR_INVALID_ARG
    assert fake.held == 0
    srv.close()


def test_evicting_a_queued_factorization():
    As, plans = _plans([8, 8])
    fake = FakeExecutor(_n_of(plans, As), lambda eps: 60)
    srv = lrs.Server(hbm_budget=100, workers=1, executor=fake)
    a = srv.factor(plans[0], As[0].val, 1e-2, reserve_bytes=60)
    srv.wait(a)
    b = srv.factor(plans[1], As[1].val, 1e-2, reserve_bytes=60)   # waits for the budget
    sb = srv.solve(b, np.ones(As[1].n))
    srv.evict(b)
    _, info = srv.wait(b)
    assert info.status == lrs.LRS_ERR_STATE
    _, info = srv.wait(sb)
    assert info.status == lrs.LRS_ERR_STATE
    assert srv.stats()["queued"] == 0
    srv.close()
    assert fake.held == 0                           # destroy released the resident factor


def test_server_options_are_checked():
    with pytest.raises(lrs.LrsError):
        lrs.Server(hbm_budget=0, executor=FakeExecutor({}, lambda e: 1))
    with pytest.raises(lrs.LrsError):
        lrs.Server(hbm_budget=10, workers=0, executor=FakeExecutor({}, lambda e: 1))


class _PlanSizedFake(FakeExecutor):
    """The fake, sized from the plan itself (its instance export gives the rows)."""

    def __init__(self, **kw):
        super().__init__({}, lambda eps: 1 << 20, **kw)

    def factor(self, plan, val, eps, prec):
        if plan not in self.n_of_plan:
            lib = lrs.load()
            cnt = ctypes.c_int64()
            lib.lrs_plan_export(plan, lrs.EXPORT_INSTANCES, None, ctypes.byref(cnt))
            out = np.zeros(cnt.value, dtype=np.int32)
            lib.lrs_plan_export(plan, lrs.EXPORT_INSTANCES, out.ctypes.data, ctypes.byref(cnt))
            self.n_of_plan[plan] = int(out.reshape(-1, 4)[:, 1].sum())
        return super().factor(plan, val, eps, prec)


def test_serving_request_stream_driver():
    # the benchmark's serving driver end to end on small operators: every
    # request is answered, new tenants leave once built, percentiles ordered
    import bench
    args = bench.parse(["--serving", "--serving-requests", "80", "--serving-rate", "400",
                        "--serving-sides", "6,8,10", "--leaf", "8", "--serving-budget-gib", "1"])
    fake = _PlanSizedFake(factor_s=0.01, solve_s=0.005)
    out = bench.run_serving(args, executor=fake)
    assert out["requests"] == 80
    assert out["solves"] + out["factorizations"] + out["refused_no_room"] == 80
    assert out["failed"] == 0 and out["solves"] > 50
    assert out["solve_ms_p50"] <= out["solve_ms_p99"]
    assert out["solves_per_s"] > 0 and out["unknowns_per_s"] > 0
    assert fake.held == 0                          # every factor released by the end
    kinds = [k for k, *_ in bench.serving_requests(1000, 100.0, 5, 11)]
    assert 0.85 < kinds.count("solve") / 1000 < 0.95



class _RaisingFake(FakeExecutor):
    def solve(self, h, b, x, nrhs, restart, maxit, tol):
        if nrhs == 2:
            raise RuntimeError("executor failure")
        return super().solve(h, b, x, nrhs, restart, maxit, tol)


def test_executor_exceptions_fail_only_their_request():
    As, plans = _plans([8])
    fake = _RaisingFake(_n_of(plans, As), lambda eps: 1)
    srv = lrs.Server(hbm_budget=1 << 30, workers=1, max_batch_rhs=1, executor=fake)
    f = srv.factor(plans[0], As[0].val, 1e-2)
    srv.wait(f)
    bad = srv.solve(f, np.ones((As[0].n, 2)))
    good = srv.solve(f, np.ones(As[0].n))
    _, info = srv.wait(bad)
    assert info.status == lrs.LRS_ERR_STATE
    X, info = srv.wait(good)
    assert info.status == 0 and np.array_equal(X, 1.01 * np.ones(As[0].n))
    srv.close()
