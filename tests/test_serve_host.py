"""Scheduling logic of the serving form, run without a GPU (simulate mode: a
job takes params.i_max microseconds and does no device work)."""
import time

import numpy as np
import pytest


@pytest.fixture(scope="module")
def mc():
    from paper_1810_06860_gb300 import build

    build.build()
    import paper_1810_06860_gb300 as mc

    return mc


def _tiny(m=4, n=3):
    rp = np.arange(m + 1, dtype=np.int64)
    ci = (np.arange(m) % n).astype(np.int32)
    return m, n, rp, ci, np.ones(m, np.float32)


def test_fifo_admission_and_completion(mc):
    with mc.Server(budget_bytes=1 << 40, max_active=3, simulate=True) as s:
        ids = [s.submit(*_tiny(), mc.params(i_max=3000)) for _ in range(10)]
        for j in ids:
            r = s.wait(j, 30)
            assert r["status"] == 0 and r["iters"] == 3000
            assert r["latency_s"] >= r["queue_s"] >= 0
        assert s.admit_order() == ids
        st = s.stats()
        assert st["completed"] == 10 and st["admitted"] == 10 and st["queued"] == 0 and st["active"] == 0
        assert 1 <= st["peak_active"] <= 3 and st["in_use_bytes"] == 0


def test_budget_limits_concurrency(mc):
    """With a budget that holds two footprints at a time, no more than two
    jobs are ever active, although four slots exist."""
    with mc.Server(budget_bytes=1 << 40, max_active=4, simulate=True) as probe:
        j = probe.submit(*_tiny(), mc.params(i_max=1))
        fp = probe.wait(j, 30)["footprint_bytes"]
    with mc.Server(budget_bytes=2 * fp + fp // 2, max_active=4, simulate=True) as s:
        ids = [s.submit(*_tiny(), mc.params(i_max=20000)) for _ in range(8)]
        for j in ids:
            s.wait(j, 30)
        st = s.stats()
        assert st["peak_active"] == 2 and st["peak_in_use_bytes"] <= 2 * fp + fp // 2


def test_oversize_job_runs_alone(mc):
    with mc.Server(budget_bytes=1024, max_active=4, simulate=True) as s:
        ids = [s.submit(*_tiny(), mc.params(i_max=5000)) for _ in range(3)]
        for j in ids:
            assert s.wait(j, 30)["status"] == 0
        assert s.stats()["peak_active"] == 1


def test_arrivals_join_running_jobs(mc):
    """Continuous batching: a job submitted while others run is admitted as
    soon as a slot frees, before the earlier jobs have all finished."""
    with mc.Server(budget_bytes=1 << 40, max_active=2, simulate=True) as s:
        long1 = s.submit(*_tiny(), mc.params(i_max=400000))
        short = s.submit(*_tiny(), mc.params(i_max=1000))
        s.wait(short, 30)
        late = s.submit(*_tiny(), mc.params(i_max=1000))
        r_late = s.wait(late, 30)
        assert s.poll(long1) is None  # the long job is still running
        assert r_late["status"] == 0
        assert s.admit_order() == [long1, short, late]
        s.wait(long1, 30)


def test_cancel_queued_and_running(mc):
    with mc.Server(budget_bytes=1 << 40, max_active=1, simulate=True) as s:
        a = s.submit(*_tiny(), mc.params(i_max=300000))
        b = s.submit(*_tiny(), mc.params(i_max=1000))
        s.cancel(b)
        rb = s.wait(b, 30)
        assert rb["status"] == 8
        s.cancel(a)
        ra = s.wait(a, 30)
        assert ra["status"] in (0, 8)
        assert b not in s.admit_order()


def test_release_and_errors(mc):
    with mc.Server(budget_bytes=1 << 40, max_active=1, simulate=True) as s:
        a = s.submit(*_tiny(), mc.params(i_max=200000))
        with pytest.raises(mc.McError) as e:
            s.release(a)
        assert e.value.status == 5  # MC_EBUSY while running
        s.wait(a, 30)
        s.release(a)
        with pytest.raises(mc.McError):
            s.poll(a)
        with pytest.raises(mc.McError):
            s.submit(0, 3, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32), mc.params())
        with pytest.raises(mc.McError):
            s.wait(12345, 0.01)


def test_wait_times_out_while_pending(mc):
    with mc.Server(budget_bytes=1 << 40, max_active=1, simulate=True) as s:
        a = s.submit(*_tiny(), mc.params(i_max=300000))
        t0 = time.perf_counter()
        with pytest.raises(mc.McError) as e:
            s.wait(a, 0.02)
        assert e.value.status == 7 and time.perf_counter() - t0 < 5
        s.cancel(a)


def test_destroy_with_jobs_in_flight(mc):
    s = mc.Server(budget_bytes=1 << 40, max_active=2, simulate=True)
    for _ in range(6):
        s.submit(*_tiny(), mc.params(i_max=100000))
    s.close()  # cancels, joins the workers, frees; must not hang
