"""Host logic of the serving loop, on the CPU: the server runs with a fake
device (every launch 'runs' for a fixed time on a host timer, no CUDA call),
so admission, the HBM budget, batching, slots and the failure paths (stalled
producer, full queue, oversized job, timeouts, unknown tickets, destroying a
busy server) are exercised without a GPU."""
import threading
import time

import pytest


@pytest.fixture(scope="module")
def bf():
    from paper_1810_11451_gb300 import build
    build.build()
    import paper_1810_11451_gb300 as m
    m.lib()
    return m


FAKE_S, FAKE_R = 0x100000, 0x200000
R_BLOCK = 30720


def job_groups(n_blocks):
    return [(0, n_blocks, 0, 0)]


def test_jobs_complete_in_order_with_latency(bf):
    srv = bf.bf_serve_create(None, n_slots=1, max_batch_jobs=1, hbm_budget_bytes=1 << 30, fake_device_us=300)
    try:
        t0 = bf.bf_now_ns()
        arrivals, tickets = [], []
        for i in range(5):
            a = bf.bf_now_ns()  # explicit arrival stamps: latency = completion - arrival exactly
            arrivals.append(a)
            tickets.append(bf.bf_submit(srv, job_groups(2), bf.BF_FP32, FAKE_S, FAKE_R, cell=i, arrival_ns=a))
        lats = [bf.bf_wait(srv, t, 5_000_000) for t in tickets]
        assert all(l >= 300 for l in lats)
        done_us = [a * 1e-3 + l for a, l in zip(arrivals, lats)]
        # one slot, FIFO: each job completes at least one device time after the
        # one before it, whatever the gaps between the submissions
        assert all(d1 - d0 >= 0.99 * 300 for d0, d1 in zip(done_us, done_us[1:]))
        assert done_us[-1] - t0 * 1e-3 >= 0.99 * 5 * 300
        st = bf.bf_serve_get_stats(srv)
        assert st["submitted"] == 5 and st["completed"] == 5 and st["launches"] == 5
        assert bf.bf_now_ns() - t0 >= 5 * 300_000
    finally:
        bf.bf_serve_destroy(srv)


def test_budget_limits_inflight_bytes(bf):
    per_job = 3 * R_BLOCK
    srv = bf.bf_serve_create(None, n_slots=4, max_batch_jobs=1, hbm_budget_bytes=2 * per_job, fake_device_us=500)
    try:
        ts = [bf.bf_submit(srv, job_groups(3), bf.BF_FP32, FAKE_S, FAKE_R) for _ in range(8)]
        for t in ts:
            bf.bf_wait(srv, t, 10_000_000)
        st = bf.bf_serve_get_stats(srv)
        assert st["max_inflight_bytes"] <= 2 * per_job
        assert st["max_busy_slots"] <= 2
        assert st["budget_waits"] >= 1
        with pytest.raises(bf.BfError) as ei:
            bf.bf_submit(srv, job_groups(3 * 3), bf.BF_FP32, FAKE_S, FAKE_R)
        assert ei.value.status == bf.BF_EBUDGET
        assert bf.bf_serve_get_stats(srv)["rejected_budget"] == 1
    finally:
        bf.bf_serve_destroy(srv)


def test_budget_can_change_at_run_time(bf):
    per_job = 3 * R_BLOCK
    srv = bf.bf_serve_create(None, n_slots=4, max_batch_jobs=1, hbm_budget_bytes=per_job, fake_device_us=20000)
    try:
        bf.bf_serve_pause(srv, True)
        ts = [bf.bf_submit(srv, job_groups(3), bf.BF_FP32, FAKE_S, FAKE_R) for _ in range(4)]
        with pytest.raises(bf.BfError) as ei:  # a queued job could never be admitted
            bf.bf_serve_set_budget(srv, per_job - 1)
        assert ei.value.status == bf.BF_EBUSY
        with pytest.raises(bf.BfError) as ei:
            bf.bf_serve_set_budget(srv, 0)
        assert ei.value.status == bf.BF_EINVAL
        bf.bf_serve_set_budget(srv, 4 * per_job)  # room for all four at once
        bf.bf_serve_pause(srv, False)
        for t in ts:
            bf.bf_wait(srv, t, 10_000_000)
        st = bf.bf_serve_get_stats(srv)
        assert st["max_busy_slots"] == 4 and st["max_inflight_bytes"] == 4 * per_job
    finally:
        bf.bf_serve_destroy(srv)


def test_continuous_batching_merges_and_overlaps(bf):
    srv = bf.bf_serve_create(None, n_slots=2, max_batch_jobs=8, hbm_budget_bytes=1 << 34, fake_device_us=50000)
    try:
        first = bf.bf_submit(srv, job_groups(1), bf.BF_BF16X3, FAKE_S, FAKE_R)
        time.sleep(0.005)
        # these arrive while the first launch runs: they start at once on the
        # second slot, merged into one launch
        rest = [bf.bf_submit(srv, job_groups(1), bf.BF_BF16X3, FAKE_S, FAKE_R) for _ in range(6)]
        for t in [first] + rest:
            bf.bf_wait(srv, t, 10_000_000)
        st = bf.bf_serve_get_stats(srv)
        assert st["max_jobs_per_launch"] >= 2
        assert st["max_busy_slots"] == 2
        assert st["launches"] < 7
    finally:
        bf.bf_serve_destroy(srv)


def test_precisions_are_not_merged(bf):
    srv = bf.bf_serve_create(None, n_slots=1, max_batch_jobs=8, hbm_budget_bytes=1 << 34, fake_device_us=1000)
    try:
        bf.bf_serve_pause(srv, True)
        ts = [bf.bf_submit(srv, job_groups(1), p, FAKE_S, FAKE_R) for p in
              (bf.BF_FP32, bf.BF_FP32, bf.BF_BF16X3, bf.BF_FP32)]
        bf.bf_serve_pause(srv, False)
        for t in ts:
            bf.bf_wait(srv, t, 10_000_000)
        assert bf.bf_serve_get_stats(srv)["launches"] == 3
    finally:
        bf.bf_serve_destroy(srv)


def test_stalled_producer_times_out_then_recovers(bf):
    srv = bf.bf_serve_create(None, n_slots=1, hbm_budget_bytes=1 << 30, fake_device_us=100)
    try:
        bf.bf_serve_pause(srv, True)
        t = bf.bf_submit(srv, job_groups(1), bf.BF_FP32, FAKE_S, FAKE_R)
        with pytest.raises(bf.BfError) as ei:
            bf.bf_wait(srv, t, 20_000)
        assert ei.value.status == bf.BF_ETIMEOUT
        done, _ = bf.bf_poll(srv, t)
        assert not done
        # destroying with queued work held back is refused, the server keeps going
        with pytest.raises(bf.BfError):
            bf.bf_serve_destroy(srv, 20_000)
        bf.bf_serve_pause(srv, False)
        assert bf.bf_wait(srv, t, 5_000_000) >= 20_000
    finally:
        bf.bf_serve_pause(srv, False)
        bf.bf_serve_destroy(srv)


def test_queue_full_and_unknown_tickets(bf):
    srv = bf.bf_serve_create(None, n_slots=1, queue_capacity=3, hbm_budget_bytes=1 << 30, fake_device_us=100)
    try:
        bf.bf_serve_pause(srv, True)
        ts = [bf.bf_submit(srv, job_groups(1), bf.BF_FP32, FAKE_S, FAKE_R) for _ in range(3)]
        with pytest.raises(bf.BfError) as ei:
            bf.bf_submit(srv, job_groups(1), bf.BF_FP32, FAKE_S, FAKE_R)
        assert ei.value.status == bf.BF_EAGAIN
        bf.bf_serve_pause(srv, False)
        for t in ts:
            bf.bf_wait(srv, t, 5_000_000)
        with pytest.raises(bf.BfError) as ei:
            bf.bf_poll(srv, ts[0])  # retired
        assert ei.value.status == bf.BF_ENOTFOUND
        with pytest.raises(bf.BfError) as ei:
            bf.bf_poll(srv, 987654)
        assert ei.value.status == bf.BF_ENOTFOUND
    finally:
        bf.bf_serve_destroy(srv)


def test_bad_arguments(bf):
    with pytest.raises(bf.BfError):
        bf.bf_serve_create(None, n_slots=0, fake_device_us=10)
    with pytest.raises(bf.BfError):
        bf.bf_serve_create(None, n_slots=2)  # real device needs a plan
    srv = bf.bf_serve_create(None, n_slots=1, fake_device_us=10)
    try:
        for S, R, g in [(FAKE_S + 8, FAKE_R, job_groups(1)), (0, FAKE_R, job_groups(1)),
                        (FAKE_S, FAKE_R, [(0, 1, 8, 0)]), (FAKE_S, FAKE_R, [(0, -1, 0, 0)])]:
            with pytest.raises(bf.BfError) as ei:
                bf.bf_submit(srv, g, bf.BF_FP32, S, R)
            assert ei.value.status == bf.BF_EINVAL
    finally:
        bf.bf_serve_destroy(srv)


def test_concurrent_submitters(bf):
    srv = bf.bf_serve_create(None, n_slots=3, max_batch_jobs=4, hbm_budget_bytes=1 << 34, fake_device_us=200)
    tickets, lock = [], threading.Lock()

    def cell(c):
        for _ in range(25):
            t = bf.bf_submit(srv, job_groups(1 + c % 3), bf.BF_FP32, FAKE_S, FAKE_R, cell=c)
            with lock:
                tickets.append(t)
            time.sleep(0.0002)

    th = [threading.Thread(target=cell, args=(c,)) for c in range(4)]
    try:
        for t in th:
            t.start()
        for t in th:
            t.join()
        assert len(set(tickets)) == 100
        for t in tickets:
            bf.bf_wait(srv, t, 10_000_000)
        st = bf.bf_serve_get_stats(srv)
        assert st["completed"] == 100 and st["submitted"] == 100
    finally:
        bf.bf_serve_destroy(srv)


def test_replay_submits_each_job_at_its_arrival(bf):
    """The native load generator submits item i at start + arrival_i (never
    early: latency, counted from the scheduled arrival, is at least the
    device time), applies precoder updates on the way (an update-only item
    gets ticket 0), and counts late submits (a schedule whose start has
    passed is all late)."""
    import ctypes
    srv = bf.bf_serve_create(None, n_slots=4, max_batch_jobs=1, hbm_budget_bytes=1 << 30, fake_device_us=100)
    try:
        n = 12
        ga, ng = bf.make_groups(job_groups(2))
        f_arr = (ctypes.c_int32 * 1)(8)

        def schedule():
            items = (bf.bf_replay_item * (n + 1))()
            items[n].job.arrival_ns = 400_000 * n  # update only
            items[n].W_dev, items[n].f_host, items[n].n_prec, items[n].first_id = FAKE_S, f_arr, 1, 0
            for i in range(n):
                it = items[i]
                it.job.cell, it.job.n_groups, it.job.groups, it.job.prec = i % 3, ng, ga, bf.BF_FP32
                it.job.S_dev, it.job.R_dev, it.job.arrival_ns = FAKE_S, FAKE_R, 400_000 * i  # every 0.4 ms
                if i % 4 == 0:  # a precoder update first (a no-op on the fake device)
                    it.W_dev, it.f_host, it.n_prec, it.first_id = FAKE_S, f_arr, 1, 0
            return items

        start = bf.bf_now_ns() + 2_000_000
        tickets, late = bf.bf_serve_replay(srv, schedule(), start)
        assert bf.bf_now_ns() >= start + 400_000 * n
        assert tickets[n] == 0
        tickets = tickets[:n]
        assert len(set(tickets)) == n and 0 not in tickets and 0 <= late <= n
        lats = [bf.bf_wait(srv, t, 5_000_000) for t in tickets]
        assert all(l >= 100 for l in lats), lats
        tickets, late = bf.bf_serve_replay(srv, schedule(), bf.bf_now_ns() - 10_000_000)
        assert late == n
        for t in tickets[:n]:
            bf.bf_wait(srv, t, 5_000_000)
        assert bf.bf_serve_get_stats(srv)["completed"] == 2 * n
        L = bf._serve_sigs(bf.lib())
        assert L.bf_serve_replay(srv, None, 1, 0, None, None) == bf.BF_EINVAL
        assert bf.bf_serve_replay(srv, (bf.bf_replay_item * 0)(), 0) == ([], 0)
    finally:
        bf.bf_serve_destroy(srv)


def test_deadline_accounting_and_worst_job(bf):
    """Jobs over the deadline are counted by the engine itself, and the worst
    job's latency splits into submit, queue, launch and device time that add
    up to it."""
    srv = bf.bf_serve_create(None, n_slots=1, max_batch_jobs=1, hbm_budget_bytes=1 << 30, fake_device_us=3000,
                             deadline_us=5000)
    try:
        ts = [bf.bf_submit(srv, job_groups(1), bf.BF_FP32, FAKE_S, FAKE_R) for _ in range(4)]
        lats = [bf.bf_wait(srv, t, 5_000_000) for t in ts]
        st = bf.bf_serve_get_stats(srv)
        assert st["deadline_ns"] == 5_000_000 and st["slot_timeout_ns"] == 50_000_000
        # one slot, 3 ms per launch: the first job is within 5 ms, the 3rd and 4th are not
        assert st["over_deadline"] == sum(l > 5000 for l in lats) and st["over_deadline"] >= 2
        assert lats[0] < 5000
        assert abs(st["worst_latency_ns"] * 1e-3 - max(lats)) < 1.0
        parts = st["worst_submit_ns"] + st["worst_queue_ns"] + st["worst_launch_ns"] + st["worst_device_ns"]
        assert parts == st["worst_latency_ns"]
        assert st["worst_queue_ns"] >= 2 * 2_900_000 and st["worst_device_ns"] >= 2_900_000
        assert st["timed_out"] == 0
        # the late jobs waited in the queue behind the single slot longer than their own launch ran
        by = [st[k] for k in ("over_by_submit", "over_by_queue", "over_by_launch", "over_by_device")]
        assert sum(by) == st["over_deadline"] and st["over_by_queue"] >= 1
        # the sums of the four parts add up to the sum of the latencies
        total = sum(st[f"sum_{k}_ns"] for k in ("submit", "queue", "launch", "device"))
        assert abs(total * 1e-3 - sum(lats)) < 4.0 and st["sum_device_ns"] >= 4 * 2_900_000
    finally:
        bf.bf_serve_destroy(srv)
    srv = bf.bf_serve_create(None, n_slots=2, hbm_budget_bytes=1 << 30, fake_device_us=100)
    try:
        t = bf.bf_submit(srv, job_groups(1), bf.BF_FP32, FAKE_S, FAKE_R)
        bf.bf_wait(srv, t, 5_000_000)
        st = bf.bf_serve_get_stats(srv)
        assert st["deadline_ns"] == 500_000  # the 0.5 ms TTI by default
    finally:
        bf.bf_serve_destroy(srv)


def test_watchdog_fails_a_launch_that_does_not_complete(bf):
    """A launch not seen complete within slot_timeout_us fails its jobs with
    BF_ETIMEOUT; its slot and budget stay held until the launch completes, and
    the server then carries on. The fake device's 300 ms launch stands in for
    a launch that hangs."""
    per_job = 2 * R_BLOCK
    srv = bf.bf_serve_create(None, n_slots=1, max_batch_jobs=4, hbm_budget_bytes=4 * per_job,
                             fake_device_us=300_000, slot_timeout_us=20_000)
    try:
        bf.bf_serve_pause(srv, True)  # both jobs go into one launch
        ts = [bf.bf_submit(srv, job_groups(2), bf.BF_FP32, FAKE_S, FAKE_R) for _ in range(2)]
        t0 = time.monotonic()
        bf.bf_serve_pause(srv, False)
        for t in ts:
            with pytest.raises(bf.BfError) as ei:
                bf.bf_wait(srv, t, 2_000_000)
            assert ei.value.status == bf.BF_ETIMEOUT
        waited = time.monotonic() - t0
        assert 0.015 <= waited < 0.25, waited  # given up at the watchdog's limit, not the launch's end
        for t in ts:  # the tickets were retired with their status
            with pytest.raises(bf.BfError) as ei:
                bf.bf_poll(srv, t)
            assert ei.value.status == bf.BF_ENOTFOUND
        st = bf.bf_serve_get_stats(srv)
        assert st["timed_out"] == 2 and st["completed"] == 2 and st["over_deadline"] == 2
        # the budget of the given-up jobs is still held: a job that needs all of it waits
        t_big = bf.bf_submit(srv, job_groups(8), bf.BF_FP32, FAKE_S, FAKE_R)
        done, _ = bf.bf_poll(srv, t_big)
        assert not done
        # the stuck launch completes at 300 ms; the big job then runs (and is
        # itself given up, its launch being as long)
        with pytest.raises(bf.BfError) as ei:
            bf.bf_wait(srv, t_big, 2_000_000)
        assert ei.value.status == bf.BF_ETIMEOUT
        assert time.monotonic() - t0 >= 0.29
        assert bf.bf_serve_get_stats(srv)["timed_out"] == 3
    finally:
        bf.bf_serve_destroy(srv)  # waits for the last launch to complete
    with pytest.raises(bf.BfError) as ei:
        bf.bf_serve_create(None, fake_device_us=10, slot_timeout_us=-1)
    assert ei.value.status == bf.BF_EINVAL
