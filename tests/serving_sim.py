"""Serving simulation: cells emit one beamforming job per 0.5 ms TTI in real
time into a `bf_serve` server; the result is per-job latency (scheduled
arrival to host-observed completion) and throughput.

Workload (the serving recipe of `workloads.serving_schedule`): 8 cells, arrival
t = 0.5 ms * tti + N(0, 50 us); n_rb ~ U{25..273} resource blocks x 14
symbols per job; f ~ U{1..36} per cell per 10-TTI precoder epoch; the
precoders of a cell are re-set every epoch into one of two slot banks.
Device-resident pools stand in for the radio: per cell a seeded S pool of
273 x 14 blocks (read with the epoch's f), a shared seeded pool of unit-column
precoders for every f, and a ring of R buffers. The schedule (with its
precoder updates) is built beforehand and replayed by the library's native
load generator (`bf_serve_replay`), so no interpreter sits in the timing loop.
Every precoder update is scheduled before the earliest job of its epoch (the
arrival jitter can bring a job ahead of the nominal update time).
"""
from __future__ import annotations

import ctypes
import threading
import time

import numpy as np

import paper_1810_11451_gb300 as bf
import workloads as wl

N_RB_MAX, N_SYM = 273, 14


def _c64(arr, torch):
    return torch.from_numpy(np.ascontiguousarray(arr.astype(np.complex64)).view(np.float32)).cuda()


class ServingSim:
    def __init__(self, plan, torch, n_cells=8, seed=5, r_ring=4, prec=bf.BF_BF16X3, budget=8 << 30,
                 n_slots=4, max_batch_jobs=16):
        self.torch, self.plan, self.n_cells, self.prec = torch, plan, n_cells, prec
        rng = np.random.default_rng(seed)
        # shared precoder pool: for every f, 273 unit-column 64 x f precoders
        self.W = {f: _c64(np.concatenate([wl.precoder_unit_columns(rng, 64, f).ravel() for _ in range(N_RB_MAX)]),
                          torch) for f in range(1, 37)}
        # per cell: S pool sized for f = 36 (a prefix is read at smaller f), R ring
        self.S = [_c64(wl.qam_symbols(rng, 64, (N_RB_MAX * N_SYM * 36 * 60,)), torch) for _ in range(n_cells)]
        self.R = [[torch.empty(N_RB_MAX * N_SYM * 64 * 60 * 2, device="cuda") for _ in range(r_ring)]
                  for _ in range(n_cells)]
        torch.cuda.synchronize()
        # every cell's two precoder banks and the largest merged launch,
        # allocated before the server starts
        bf.bf_reserve_precoders(plan, n_cells * 2 * N_RB_MAX)
        bf.bf_reserve_worklists(plan, max_batch_jobs * N_RB_MAX * N_SYM)
        self.srv = bf.bf_serve_create(plan, n_slots=n_slots, max_batch_jobs=max_batch_jobs,
                                      queue_capacity=1 << 16, hbm_budget_bytes=budget)
        self._L = bf._serve_sigs(bf.lib())
        # every cell's full-band group array per (bank, f), built before the
        # real-time loop so that a submit only fills one job struct
        self._groups = {}
        for c in range(n_cells):
            for bank in range(2):
                for f in range(1, 37):
                    self.groups(c, bank, N_RB_MAX, f)

    def slot_base(self, cell, bank):
        return (cell * 2 + bank) * N_RB_MAX

    def groups(self, cell, bank, n_rb, f):
        """The job's groups: the first n_rb entries of the cell's full-band
        group array for (bank, f), built once."""
        key = (cell, bank, f)
        g = self._groups.get(key)
        if g is None:
            base = self.slot_base(cell, bank)
            blk_s = N_SYM * f * 480
            g = bf.make_groups([(base + rb, N_SYM, rb * blk_s, rb * N_SYM * 30720) for rb in range(N_RB_MAX)])[0]
            self._groups[key] = g
        return g, n_rb

    def run(self, jobs, warm_tti=20, tti_ns=500_000, sample_every=0, seed=0):
        """Submit `jobs` (workloads.ServingJob, sorted by arrival) in real time.
        Returns a dict of latency percentiles and throughput. A cell's
        precoders for an epoch are set half a TTI before the epoch starts (or
        20 us before the epoch's earliest job, if the jitter brings one
        earlier), into the bank the previous epoch does not use, spaced 25 us
        apart across cells (update-only items of the schedule). With sample_every = k > 0,
        one seeded random block of every k-th job is copied to the host as
        soon as the job completes (before its R buffer is reused) and returned
        under "samples" with the indices that locate its W and S."""
        srv = self.srv
        f_arrays = {f: (ctypes.c_int32 * N_RB_MAX)(*([f] * N_RB_MAX)) for f in range(1, 37)}
        first = {}  # (cell, epoch) -> (first tti, f, earliest arrival in ns)
        for j in jobs:
            k = (j.cell, j.epoch)
            a = int(j.arrival_s * 1e9)
            if k not in first:
                first[k] = (j.tti, j.f, a)
            else:
                t0_, f0_, a0_ = first[k]
                first[k] = (min(t0_, j.tti), f0_, min(a0_, a))
        # an epoch's precoders are set half a TTI before the epoch (25 us apart
        # across cells), and in any case 20 us before the epoch's earliest job:
        # with the arrival jitter a job can come earlier than the nominal time
        events = [(min(tti * tti_ns - tti_ns // 2 + cell * 25_000, a_min - 20_000), 0, (cell, epoch, f))
                  for (cell, epoch), (tti, f, a_min) in first.items()]
        events += [(int(j.arrival_s * 1e9), 1, j) for j in jobs]
        events.sort(key=lambda e: (e[0], e[1]))
        items = (bf.bf_replay_item * len(events))()
        ring_pos = [0] * self.n_cells
        blocks = flops = 0
        meta = []
        R_of = {}
        for i, (t, kind, x) in enumerate(events):
            it = items[i]
            it.job.arrival_ns = t  # relative to the replay's start
            if kind == 0:
                cell, epoch, f = x
                it.W_dev, it.f_host = self.W[f].data_ptr(), f_arrays[f]
                it.n_prec, it.first_id = N_RB_MAX, self.slot_base(cell, epoch % 2)
                continue
            j = x
            ga, n = self.groups(j.cell, j.epoch % 2, j.n_rb, j.f)
            R = self.R[j.cell][ring_pos[j.cell]]
            R_of[i] = R
            ring_pos[j.cell] = (ring_pos[j.cell] + 1) % len(self.R[j.cell])
            it.job.cell, it.job.n_groups, it.job.groups, it.job.prec = j.cell, n, ga, self.prec
            it.job.S_dev, it.job.R_dev = self.S[j.cell].data_ptr(), R.data_ptr()
            meta.append((i, j))
            if j.tti >= warm_tti:
                blocks += j.n_rb * N_SYM
                flops += j.n_rb * N_SYM * 8 * 64 * 60 * j.f
        # A consumer thread retires each job as it completes, in submission
        # order, while the replay runs (tickets appear in the shared array as
        # the jobs are submitted), as a radio's next stage would.
        tk = (ctypes.c_uint64 * len(events))()
        lat, err, samples = [], [], []
        replay_done = threading.Event()
        rng = np.random.default_rng(seed)
        picks = {n: int(rng.integers(0, j.n_rb * N_SYM)) for n, (_, j) in enumerate(meta)
                 if sample_every and n % sample_every == 0}

        def consume():
            try:
                for n, (i, j) in enumerate(meta):
                    while tk[i] == 0:
                        if replay_done.is_set() and tk[i] == 0:
                            return  # the replay stopped before this job
                        time.sleep(20e-6)
                    v = bf.bf_wait(srv, tk[i], 30_000_000)
                    if j.tti >= warm_tti:
                        lat.append(v)
                    if n in picks:
                        blk = picks[n]
                        R = R_of[i]
                        r = R[blk * 64 * 60 * 2:(blk + 1) * 64 * 60 * 2].cpu().numpy().view(np.complex64)
                        samples.append({"cell": j.cell, "f": j.f, "rb": blk // N_SYM, "sym": blk % N_SYM,
                                        "R": r.reshape(64, 60).copy()})
            except Exception as e:  # reported after the replay
                err.append(e)

        th = threading.Thread(target=consume)
        th.start()
        t0 = bf.bf_now_ns() + 20_000_000  # the schedule starts 20 ms from now
        try:
            _, late = bf.bf_serve_replay(srv, items, t0, tk)
        finally:
            replay_done.set()
            t_last_submit = bf.bf_now_ns()
            th.join()
        if err:
            raise err[0]
        t_end = bf.bf_now_ns()
        stats = bf.bf_serve_get_stats(srv)
        lat = np.array(lat)
        span = (t_last_submit - t0) * 1e-9
        del items, f_arrays
        return {
            "jobs": len(lat), "cells": self.n_cells, "ttis": int(max(j.tti for j in jobs) + 1),
            "p50_us": float(np.percentile(lat, 50)), "p99_us": float(np.percentile(lat, 99)),
            "max_us": float(lat.max()), "mean_us": float(lat.mean()),
            "frac_over_500us": float(np.mean(lat > 500.0)),
            "blocks_per_s": blocks / span, "gflops": flops / span / 1e9,
            "late_submits": late, "drain_ms": (t_end - t_last_submit) * 1e-6,
            "launches": stats["launches"], "max_busy_slots": stats["max_busy_slots"],
            "max_jobs_per_launch": stats["max_jobs_per_launch"], "budget_waits": stats["budget_waits"],
            "max_inflight_bytes": stats["max_inflight_bytes"],
            "engine": {"over_deadline": stats["over_deadline"], "timed_out": stats["timed_out"],
                       "deadline_us": stats["deadline_ns"] * 1e-3, "completed": stats["completed"],
                       "worst_us": {k: stats[f"worst_{k}_ns"] * 1e-3
                                    for k in ("latency", "submit", "queue", "launch", "device")},
                       "over_deadline_by_largest_part": {k: stats[f"over_by_{k}"]
                                                         for k in ("submit", "queue", "launch", "device")},
                       "mean_us": {k: stats[f"sum_{k}_ns"] * 1e-3 / max(1, stats["completed"])
                                   for k in ("submit", "queue", "launch", "device")},
                       "note": "counted by the server over every job, warm-up TTIs included"},
            **({"samples": samples} if sample_every else {}),
        }

    def sample_inputs(self, smp):
        """W (64 x f) and S (f x 60) of a sampled block, as complex64 host arrays."""
        f, rb = smp["f"], smp["rb"]
        W = self.W[f][rb * 64 * f * 2:(rb + 1) * 64 * f * 2].cpu().numpy().view(np.complex64).reshape(64, f)
        o = (rb * N_SYM + smp["sym"]) * f * 60 * 2
        S = self.S[smp["cell"]][o:o + f * 60 * 2].cpu().numpy().view(np.complex64).reshape(f, 60)
        return W, S

    def close(self):
        bf.bf_serve_destroy(self.srv)
