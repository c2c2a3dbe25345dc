"""The serving loop on the GPU: per-TTI jobs from several cells, admitted under
an HBM budget, merged and overlapped on the device. Each job's R equals its R
computed alone, bit for bit, and matches the FP64 oracle."""
import numpy as np
import pytest

import oracle
import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1810_11451_gb300 as bf  # noqa: E402
from bfrun import to_device_c64  # noqa: E402

N_SYM = 14
MAX_RB = 40


class Cell:
    """One cell: a bank of MAX_RB precoders (64 x f) and a resident S pool."""

    def __init__(self, srv, cell, f, slot_base, seed):
        rng = np.random.default_rng(seed)
        self.cell, self.f, self.slot_base = cell, f, slot_base
        self.W = [wl.precoder_unit_columns(rng, 64, f).astype(np.complex64) for _ in range(MAX_RB)]
        self.S = wl.qam_symbols(rng, 64, (MAX_RB, N_SYM, f, 60)).astype(np.complex64)
        self.Wd = to_device_c64(np.concatenate([w.ravel() for w in self.W]), torch)
        self.Sd = to_device_c64(self.S.ravel(), torch)
        torch.cuda.synchronize()  # the server's streams do not wait for torch's stream
        bf.bf_serve_set_precoders(srv, self.Wd, [f] * MAX_RB, slot_base)

    def groups(self, n_rb):
        blk_s = N_SYM * self.f * 480
        return [(self.slot_base + rb, N_SYM, rb * blk_s, rb * N_SYM * 30720) for rb in range(n_rb)]

    def new_R(self, n_rb):
        return torch.full((n_rb * N_SYM * 64 * 60 * 2,), float("nan"), device="cuda")

    def reference(self, n_rb):
        return [oracle.apply_blocks(self.W[rb], self.S[rb]) for rb in range(n_rb)]


def _R_np(Rt, n_rb):
    torch.cuda.synchronize()
    return Rt.cpu().numpy().view(np.complex64).reshape(n_rb, N_SYM, 64, 60)


@pytest.fixture(scope="module")
def plan():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    p = bf.bf_plan_create(64, 36, 60)
    yield p
    bf.bf_plan_destroy(p)


@pytest.mark.parametrize("prec,tol", [(bf.BF_FP32, 1e-5), (bf.BF_BF16X3, 1e-5), (bf.BF_TF32X3, 1e-5)],
                         ids=["fp32", "bf16x3", "tf32x3"])
def test_alone_equals_in_mix(plan, prec, tol):
    srv = bf.bf_serve_create(plan, n_slots=4, max_batch_jobs=8, hbm_budget_bytes=8 << 30)
    try:
        cells = [Cell(srv, c, f, 1000 + 100 * c, 50 + c) for c, f in enumerate([36, 9, 17, 1])]
        torch.cuda.synchronize()
        probe = cells[0]
        R_alone = probe.new_R(25)
        torch.cuda.synchronize()
        lat = bf.bf_wait(srv, bf.bf_submit(srv, probe.groups(25), prec, probe.Sd, R_alone), 10_000_000)
        assert 0 < lat < 1e6
        alone = _R_np(R_alone, 25)
        # the mix: 32 jobs of uneven size from 4 cells, submitted back to back
        rng = np.random.default_rng(7)
        spec = []
        for k in range(32):
            c, n_rb = cells[k % 4], int(rng.integers(1, MAX_RB + 1))
            if k == 12:
                c, n_rb = probe, 25
            spec.append((c, n_rb, c.new_R(n_rb)))
        torch.cuda.synchronize()
        jobs = [(c, n_rb, Rt, bf.bf_submit(srv, c.groups(n_rb), prec, c.Sd, Rt, cell=c.cell))
                for c, n_rb, Rt in spec]
        lats = [bf.bf_wait(srv, t, 20_000_000) for (_, _, _, t) in jobs]
        st = bf.bf_serve_get_stats(srv)
        assert st["completed"] == 33 and st["max_busy_slots"] >= 2, st
        mixed = _R_np(jobs[12][2], 25)
        assert np.array_equal(mixed.view(np.uint64), alone.view(np.uint64)), "job differs alone vs in the mix"
        for c, n_rb, Rt, _ in jobs[:8]:
            R = _R_np(Rt, n_rb)
            e = oracle.rel_frobenius(list(R), c.reference(n_rb))
            assert e <= tol, e
        assert max(lats) < 1e6
    finally:
        bf.bf_serve_destroy(srv)


def test_budget_serialises_and_precoder_update_is_ordered(plan):
    c_bytes = 10 * N_SYM * (36 * 480 + 30720)
    srv = bf.bf_serve_create(plan, n_slots=4, max_batch_jobs=4, hbm_budget_bytes=int(1.5 * c_bytes))
    try:
        cell = Cell(srv, 0, 36, 5000, 91)
        Rs = [cell.new_R(10) for _ in range(6)]
        torch.cuda.synchronize()
        ts = [bf.bf_submit(srv, cell.groups(10), bf.BF_BF16X3, cell.Sd, R) for R in Rs]
        for t in ts:
            bf.bf_wait(srv, t, 20_000_000)
        st = bf.bf_serve_get_stats(srv)
        assert st["max_inflight_bytes"] <= 1.5 * c_bytes and st["budget_waits"] >= 1, st
        ref = cell.reference(10)
        for R in Rs:
            assert oracle.rel_frobenius(list(_R_np(R, 10)), ref) <= 1e-5
        with pytest.raises(bf.BfError) as ei:
            bf.bf_submit(srv, cell.groups(20), bf.BF_BF16X3, cell.Sd, Rs[0])
        assert ei.value.status == bf.BF_EBUDGET
        # new precoders for the same slots: jobs submitted afterwards use them
        rng = np.random.default_rng(3)
        cell.W = [wl.precoder_unit_columns(rng, 64, 36).astype(np.complex64) for _ in range(MAX_RB)]
        Wd2 = to_device_c64(np.concatenate([w.ravel() for w in cell.W]), torch)
        R2 = cell.new_R(10)
        torch.cuda.synchronize()
        bf.bf_serve_set_precoders(srv, Wd2, [36] * MAX_RB, cell.slot_base)
        bf.bf_wait(srv, bf.bf_submit(srv, cell.groups(10), bf.BF_BF16X3, cell.Sd, R2), 20_000_000)
        assert oracle.rel_frobenius(list(_R_np(R2, 10)), cell.reference(10)) <= 1e-5
        with pytest.raises(bf.BfError) as ei:
            bf.bf_submit(srv, [(99999, 1, 0, 0)], bf.BF_FP32, cell.Sd, R2)
        assert ei.value.status == bf.BF_ENOTFOUND
    finally:
        bf.bf_serve_destroy(srv)


def test_plan_outlives_its_servers():
    """A plan cannot be destroyed while a serving engine uses it."""
    p = bf.bf_plan_create(64, 36, 60)
    srv = bf.bf_serve_create(p, n_slots=2)
    try:
        with pytest.raises(bf.BfError) as ei:
            bf.bf_plan_destroy(p)
        assert ei.value.status == bf.BF_EBUSY
    finally:
        bf.bf_serve_destroy(srv)
    bf.bf_plan_destroy(p)


@pytest.mark.parametrize("prec", [bf.BF_BF16X3, bf.BF_FP32], ids=["bf16x3", "fp32"])
def test_replay_drives_the_device_in_real_time(prec):
    """The serving simulation through the native load generator on the
    device: 8 cells for 200 TTIs (twenty precoder epochs, updated between TTIs
    while other cells' jobs run, an epoch's first jobs sometimes arriving
    early) all complete, each latency counted from its scheduled arrival; one
    random block of every job, copied as the job completes, matches the FP64
    oracle within 1e-5 (a job that read a stale precoder bank would not)."""
    from serving_sim import ServingSim
    p = bf.bf_plan_create(64, 36, 60)
    sim = ServingSim(p, torch, prec=prec)
    try:
        r = sim.run(wl.serving_schedule(n_tti=200), warm_tti=10, sample_every=1, seed=4)
        errs = []
        for smp in r["samples"]:
            W, S = sim.sample_inputs(smp)
            ref = oracle.apply_blocks(W.astype(np.complex128), S[None].astype(np.complex128))[0]
            errs.append(float(np.linalg.norm(smp["R"] - ref) / np.linalg.norm(ref)))
    finally:
        sim.close()
        bf.bf_plan_destroy(p)
    assert r["jobs"] == 8 * 190 and 0 < r["p50_us"] <= r["p99_us"] <= r["max_us"] < 30_000, r
    assert len(errs) == 1600 and max(errs) <= 1e-5, (len(errs), max(errs))
    print("replay, 200 TTIs:", {k: r[k] for k in ("p50_us", "p99_us", "max_us", "late_submits")})


def test_watchdog_on_the_gpu_gives_up_late_launches_and_carries_on(plan):
    """The watchdog on real launches, without a fault. A job of 28,000 blocks
    (the cell's 40 resource blocks x 14 symbols, written 50 times to distinct R
    regions) runs for a few hundred microseconds, and the GPU is kept busy by a
    queue of large matrix products on another stream; with a 1 us limit the
    watchdog gives both jobs up (BF_ETIMEOUT, counted as timed out) while their
    launches still run, and each slot is reused only after its launch really
    completes. Once the server has drained, the given-up jobs' R equal the same
    job served normally, bit for bit, and the first repetition is within 1e-5
    of the oracle."""
    REP = 50
    per_rep = MAX_RB * N_SYM * 30720

    def groups(cell):
        return [(g[0], g[1], g[2], g[3] + rep * per_rep) for rep in range(REP) for g in cell.groups(MAX_RB)]

    def new_R():
        return torch.full((REP * per_rep // 4,), float("nan"), device="cuda")

    srv = bf.bf_serve_create(plan, n_slots=2, max_batch_jobs=1, hbm_budget_bytes=32 << 30, slot_timeout_us=1)
    busy = torch.cuda.Stream()
    try:
        cell = Cell(srv, 0, 36, 3000, 91)
        Rs = [new_R() for _ in range(2)]
        a = torch.randn(8192, 8192, device="cuda", dtype=torch.bfloat16)
        torch.cuda.synchronize()
        with torch.cuda.stream(busy):
            for _ in range(20):  # about 1.1 TFLOP each: milliseconds of queued work
                a = torch.tanh(a @ a)
        ts = [bf.bf_submit(srv, groups(cell), bf.BF_BF16X3, cell.Sd, R) for R in Rs]
        for t in ts:
            with pytest.raises(bf.BfError) as ei:
                bf.bf_wait(srv, t, 10_000_000)
            assert ei.value.status == bf.BF_ETIMEOUT
        st = bf.bf_serve_get_stats(srv)
        assert st["timed_out"] == 2 and st["completed"] == 2 and st["slot_timeout_ns"] == 1000
    finally:
        bf.bf_serve_destroy(srv)  # waits until the given-up launches have completed
    torch.cuda.synchronize()
    srv = bf.bf_serve_create(plan, n_slots=2, max_batch_jobs=1, hbm_budget_bytes=32 << 30)
    try:
        cell = Cell(srv, 0, 36, 3000, 91)  # the same precoders and S
        R2 = new_R()
        torch.cuda.synchronize()
        bf.bf_wait(srv, bf.bf_submit(srv, groups(cell), bf.BF_BF16X3, cell.Sd, R2), 10_000_000)
        assert bf.bf_serve_get_stats(srv)["timed_out"] == 0
    finally:
        bf.bf_serve_destroy(srv)
    torch.cuda.synchronize()
    for R in Rs:
        assert torch.equal(R.view(torch.int32), R2.view(torch.int32))
    first = R2[:per_rep // 4].cpu().numpy().view(np.complex64).reshape(-1, 64, 60)
    e = oracle.rel_frobenius([first], [np.concatenate(cell.reference(MAX_RB)).reshape(-1, 64, 60)])
    assert e < 1e-5
