"""Benchmark of batched complex beamforming R = W x S on GB300 (one JSON line).

Workload: the full-band f = 36 case -- 273 resource blocks x 14 OFDM symbols
= 3,822 blocks of S (36 x 60, 64-QAM, complex64), one 64 x 36 unit-column
precoder per resource block shared by its 14 symbols; R is 64 x 60 complex64
per block. A step is one pass of the product over the whole batch: one
persistent kernel launch of a prepared batch in the best form (split-bf16 on
the tensor cores, complex64 in and out). Three buffer sets (S, R) rotate so that the
working set (565 MB) is well above the 129 MB L2 between steps.

Reported beside the headline: blocks/s, the plain FP32 CUDA-core form on the
same GPU, the end-to-end rate through the host-buffer entry point, the
roofline of the dominant kernel, GPU clocks during the timed region, the
accuracy of the timed output against the FP64 oracle, and the oracle's own
CPU rate (the oracle is only run in that CPU-baseline leg).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs the same workload on its own GPU (weak scaling,
no data exchange; rank 0 prints).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

METRIC = "complex GFLOP/s & blocks/s for W×S at f=36 vs FP32 plain; p99 TTI latency"
UNIT = "GFLOP/s"
WORKLOAD = "fullband f=36, 273 RB x 14 symbols = 3,822 blocks, W 64x36 per RB, S 36x60 64-QAM, complex64 in/out"
L2_NOTE = "3 rotating buffer sets of S and R (565 MB > 2x the 129 MB L2)"
FALLBACK_HBM = 6800.0


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM, "fallback"


def traffic_for(kernel_src: str):
    """Per-launch DRAM bytes from the committed ncu summary, if it was taken on
    the current source of the kernel (else None)."""
    path = os.path.join(ROOT, "profiles", "roofline_traffic.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    with open(path) as fh:
        for line in fh:
            if "=" in line and not line.startswith("#"):
                k, v = line.split("=", 1)
                kv[k.strip()] = v.strip()
    src = os.path.join(ROOT, "paper_1810_11451_gb300", "csrc", kernel_src)
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if kv.get("source_sha256_16") != h:
        return None
    try:
        return float(kv["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.out = os.path.join("/tmp", f"bf_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.out, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.15)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.12)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.out):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.out) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = float(parts[2])
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        return dist, dist.get_rank(), world
    return None, 0, 1


def max_over_ranks(dist, x: float) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist):
    if dist is not None:
        dist.barrier()


# ---------------------------------------------------------------- CPU baseline (oracle)
def cpu_baseline(batch, budget_s: float = 12.0):
    """Time the FP64 oracle, as it stands, on the host cores over the whole
    workload, repeated until about budget_s of CPU time; also returns its R."""
    import oracle
    oracle.lib()
    rb = batch.rounded(np.complex64)
    t0 = time.perf_counter()
    reps, ref = 0, None
    while True:
        ref = oracle.apply_batch(rb)
        reps += 1
        if time.perf_counter() - t0 >= budget_s or reps >= 50:
            break
    dt = time.perf_counter() - t0
    gflops = batch.flops() * reps / dt / 1e9
    cores = oracle.num_threads()
    # the same oracle on one core, over the first 20 resource blocks (280 blocks)
    one = type(rb)(rb.W, rb.prec[:20], rb.S[:20], rb.name)
    oracle.set_num_threads(1)
    t1, reps1 = time.perf_counter(), 0
    while time.perf_counter() - t1 < 2.0 or reps1 < 1:
        oracle.apply_batch(one)
        reps1 += 1
    dt1 = time.perf_counter() - t1
    oracle.set_num_threads(cores)
    return {"value": gflops, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"the whole workload ({batch.total_blocks} blocks) x {reps} repetitions, {dt:.1f} s, FP64",
            "single_core": {"value": one.flops() * reps1 / dt1 / 1e9, "unit": UNIT, "cores": 1,
                            "sample": f"first 20 resource blocks ({one.total_blocks} blocks) x {reps1}, {dt1:.1f} s"}}, ref


def cpu_references(done, batches):
    """Part of the CPU-baseline leg: the oracle's R for the other workloads
    (complex64 inputs widened to FP64), flattened in group order."""
    import oracle
    out = {k: np.concatenate([r.reshape(-1) for r in v]) for k, v in done.items()}
    for name, b in batches.items():
        if b is not None:
            out[name] = np.concatenate([r.reshape(-1) for r in oracle.apply_batch(b.rounded(np.complex64))])
    return out


def to_device_ref(torch, ref):
    if ref is None:
        return None
    return torch.from_numpy(np.ascontiguousarray(ref).view(np.float64)).cuda()


def run_reference(args):
    """--impl reference: the oracle timed on the host cores on this workload."""
    dist, rank, world = dist_init()
    if rank != 0:
        return
    import workloads as wl
    import oracle
    batch = wl.config_fullband()
    rb = batch.rounded(np.complex64)
    oracle.lib()
    t0 = time.perf_counter()
    for _ in range(max(1, args.warmup)):
        oracle.apply_blocks(rb.W[0], rb.S[0])
    t_rb = (time.perf_counter() - t0) / max(1, args.warmup)
    # each step: a bounded sample of the workload (its first n_rb resource blocks),
    # sized so that all steps together take about a minute
    n_rb = int(max(1, min(len(rb.S), (60.0 / max(1, args.steps)) / max(t_rb, 1e-6))))
    sample = type(batch)(rb.W, rb.prec[:n_rb], rb.S[:n_rb], rb.name)
    desc = f"first {n_rb} of 273 resource blocks ({n_rb * 14} blocks) per step"
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.apply_batch(sample)
    dt = time.perf_counter() - t0
    v = sample.flops() * args.steps / dt / 1e9
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3 / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": desc},
            "impl": "reference",
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
def time_launches(torch, bf, handles, steps, warmup, stream, graph=False):
    """Launch prepared batches back to back (rotating over `handles`); CUDA
    events on the launching stream bracket the whole timed region. Each step is
    one kernel launch, so the kernel's average launch duration is the region
    divided by the steps (no per-launch events: they would add several
    microseconds each)."""
    launch = bf.bf_batch_launch_graph if graph else bf.bf_batch_launch
    for i in range(warmup):
        launch(handles[i % len(handles)], stream)
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for i in range(steps):
        launch(handles[i % len(handles)], stream)
    stop.record(stream)
    torch.cuda.synchronize()
    return start.elapsed_time(stop)


def end_to_end(torch, bf, plan, Sflat, lay, r_numel, stream, dist, world, flops, steps=20):
    """The same product through bf_apply_batch_host: S copied in from pinned
    host memory and R copied out, every step, inside the timed region.
    Consecutive steps alternate between two streams and two host buffer
    pairs, so a step's copy-in overlaps the previous step's copy-out (as a
    caller keeps both directions of the link busy); the same steps issued on
    one stream, each after the previous one, are reported beside it."""
    S_h = [torch.from_numpy(np.ascontiguousarray(Sflat.astype(np.complex64)).view(np.float32).copy()).pin_memory()
           for _ in range(2)]
    R_h = [torch.empty(r_numel, dtype=torch.float32).pin_memory() for _ in range(2)]
    streams = [stream, torch.cuda.Stream()]
    groups, _ = bf.make_groups(lay.groups)  # marshalled once, outside the timed calls

    def timed(n_streams):
        for i in range(3):
            bf.bf_apply_batch_host(plan, S_h[i % 2], groups, bf.BF_BF16X3, R_h[i % 2], streams[i % n_streams])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(streams[0])
        streams[1].wait_event(e0)
        for i in range(steps):
            k = i % n_streams
            bf.bf_apply_batch_host(plan, S_h[i % 2], groups, bf.BF_BF16X3, R_h[i % 2], streams[k])
        streams[0].wait_stream(streams[1])
        e1.record(streams[0])
        torch.cuda.synchronize()
        return max_over_ranks(dist, e0.elapsed_time(e1) / steps)

    e2e_ms = timed(2)
    serial_ms = timed(1)
    return {"value": world * flops / (e2e_ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": e2e_ms,
            "h2d_bytes_per_step": int(lay.s_bytes), "d2h_bytes_per_step": int(lay.r_blocks * 30720),
            "pipelining": "steps alternate between two streams and two pinned buffer pairs",
            "one_stream_ms_per_step": serial_ms}


def graph_rate(torch, bf, handle, steps, stream, graph=False):
    """Average launch time (ms) of one prepared batch launched back to back."""
    return time_launches(torch, bf, [handle], steps, 5, stream, graph) / steps


def rel_err(torch, bf, plan, R_t, ref_d, n_blocks, stream):
    if ref_d is None:
        return None
    num, den = bf.bf_errnorm(plan, R_t, ref_d, n_blocks, None, stream)
    return float(np.sqrt(num / den)) if den > 0 else 0.0


def uneven_leg(torch, bf, plan, batch, ref_d, stream, steps=200):
    """Uneven batch (16,384 blocks, f ~ U{0..36} per group, geometric groups):
    one persistent graph-captured launch, before and after the autotuner."""
    from bfrun import layout, set_precoders, to_device_c64
    set_precoders(plan, batch, torch)
    lay = layout(batch)
    Sflat, _ = batch.pack_S()
    S = to_device_c64(Sflat, torch)
    R = torch.empty(lay.r_blocks * 64 * 60 * 2, dtype=torch.float32, device="cuda")
    out = {"blocks": batch.total_blocks, "groups": batch.n_groups, "gflop": batch.flops() / 1e9,
           "algorithmic_bytes": batch.algorithmic_bytes()}
    for phase in ("untuned", "tuned"):
        if phase == "tuned":
            t0 = time.perf_counter()
            bf.bf_autotune(plan, bf.BF_BF16X3, stream)
            bf.bf_autotune(plan, bf.BF_FP32, stream)
            bf.bf_autotune(plan, bf.BF_FP32_3M, stream)
            bf.bf_autotune(plan, bf.BF_TF32X3, stream)
            out["autotune_s"] = time.perf_counter() - t0
            names = {v: k for k, v in bf.PRECISIONS.items()}
            form, ns = bf.bf_select_form(plan, bf.BF_TARGET_FP32, lay.groups)
            out["selected_form_fp32_target"] = {"form": names[form], "predicted_marginal_us": ns / 1e3}
            out["tune_table"] = {name: [bf.bf_tune_query(plan, p, f) for f in (0, 8, 16, 24, 36)]
                                 for name, p in (("bf16x3", bf.BF_BF16X3), ("fp32", bf.BF_FP32),
                                                 ("tf32x3", bf.BF_TF32X3))}
        for name, prec in (("bf16x3", bf.BF_BF16X3), ("fp32", bf.BF_FP32), ("tf32x3", bf.BF_TF32X3)):
            h = bf.bf_batch_create(plan, S, None, lay.groups, prec, R)
            bf.bf_batch_set_s_independent(h)  # S is written once, by a copy
            ms = graph_rate(torch, bf, h, steps, stream)
            ms_graph = graph_rate(torch, bf, h, steps, stream, graph=True)
            bf.bf_batch_launch_graph(h, stream)
            err = rel_err(torch, bf, plan, R, ref_d, lay.r_blocks, stream)
            bf.bf_batch_destroy(h)
            out[f"{name}_{phase}"] = {"kernel_ms": ms, "gflops": batch.flops() / ms / 1e6,
                                      "blocks_per_s": batch.total_blocks / ms * 1e3,
                                      "hbm_gbs": batch.algorithmic_bytes() / ms / 1e6,
                                      "graph_launch_ms": ms_graph, "rel_err": err}
    return out


def reduced_leg(torch, bf, plan, batch, ref_d, stream, steps=50):
    """Reduced precision (full band x 8 = 30,576 blocks, 256-QAM + noise): held
    bf16 / fp16 / split images (quantisation timed on its own) and split-bf16
    on complex64."""
    from bfrun import layout, set_precoders, to_device_c64
    set_precoders(plan, batch, torch)
    lay = layout(batch)
    Sflat, _ = batch.pack_S()
    S = to_device_c64(Sflat, torch)
    del Sflat
    R = torch.empty(lay.r_blocks * 64 * 60 * 2, dtype=torch.float32, device="cuda")
    nb = batch.total_blocks
    out = {"blocks": nb, "gflop": batch.flops() / 1e9}
    for name, prec, held in (("bf16_held", bf.BF_BF16, True), ("fp16_held", bf.BF_FP16, True),
                             ("bf16x3_held", bf.BF_BF16X3, True), ("bf16x3_c64", bf.BF_BF16X3, False)):
        r = {}
        if held:
            lh = layout(batch, 0, prec)
            Sq = torch.empty(lh.held_bytes // 4 + 4, dtype=torch.float32, device="cuda")
            sc = torch.empty(nb, dtype=torch.float32, device="cuda")
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            g_c, _ = bf.make_groups(lay.groups)  # marshalled once, outside the timed calls
            q_c = bf.make_offsets(lh.held_off)
            for i in range(6):
                if i == 1:
                    e0.record(stream)
                bf.bf_quantize_symbols(plan, S, g_c, prec, Sq, q_c, sc, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            qms = e0.elapsed_time(e1) / 5
            r["quantize_ms"] = qms
            r["quantize_gbs"] = (lay.s_bytes + lh.held_bytes) / qms / 1e6
            groups = [(g[0], g[1], lh.held_off[i], g[3]) for i, g in enumerate(lay.groups)]
            h = bf.bf_batch_create(plan, Sq, sc, groups, prec, R)
            bf.bf_batch_set_s_independent(h)  # held S is written by the encoder, not a product launch
            s_bytes = lh.held_bytes
        else:
            h = bf.bf_batch_create(plan, S, None, lay.groups, prec, R)
            bf.bf_batch_set_s_independent(h)
            s_bytes = lay.s_bytes
        ms = graph_rate(torch, bf, h, steps, stream)
        bf.bf_batch_launch(h, stream)
        # algorithmic bytes: unpadded S at the operand's type (240 f per block
        # for one bf16/fp16 term, 480 f for two terms or complex64), W at the
        # operand's type (256 f per precoder per 16-bit term, 512 f complex64),
        # R complex64; the padded image bytes (K to a multiple of 16, b to 64)
        # are only traffic
        terms = 2 if prec == bf.BF_BF16X3 else 1
        f = 36
        alg = nb * ((240 * terms if held else 480) * f + 30720) + len(batch.W) * (256 * terms if held else 512) * f
        peak, _ = peaks()
        r.update({"kernel_ms": ms, "gflops": batch.flops() / ms / 1e6, "blocks_per_s": nb / ms * 1e3,
                  "moved_bytes": int(s_bytes + nb * 30720 + len(batch.W) * 64 * 36 * 8),
                  "moved_gbs": (s_bytes + nb * 30720 + len(batch.W) * 64 * 36 * 8) / ms / 1e6,
                  "alg_bytes": int(alg), "alg_gbs": alg / ms / 1e6, "alg_frac": alg / ms / 1e6 / peak,
                  "rel_err": rel_err(torch, bf, plan, R, ref_d, nb, stream)})
        bf.bf_batch_destroy(h)
        if held:
            del Sq, sc
        out[name] = r
    return out


def scaling_leg(torch, bf, plan, batch, ref_d, stream):
    """Signal-level study of per-block scaling: the single-pass fp16 and bf16
    forms on S x 2^e, held (one power-of-two scale per block) against complex64
    S rounded on chip (no per-block scale). Relative error against the oracle's
    R x 2^e; null where R is not finite."""
    from bfrun import layout, set_precoders, to_device_c64
    set_precoders(plan, batch, torch)
    lay = layout(batch)
    Sflat, _ = batch.pack_S()
    nb = batch.total_blocks
    R = torch.empty(lay.r_blocks * 64 * 60 * 2, dtype=torch.float32, device="cuda")
    out = {"blocks": nb, "workload": "256-QAM + noise, f = 36, 6 RB x 14 symbols", "rel_err_by_log2_level": {}}
    for e in (-24, -16, -8, 0, 8, 16, 24):
        S = to_device_c64(Sflat * 2.0 ** e, torch)
        ref_e = ref_d * 2.0 ** e
        row = {}
        for name, prec, held in (("fp16_held", bf.BF_FP16, True), ("fp16_onchip", bf.BF_FP16, False),
                                 ("bf16_held", bf.BF_BF16, True), ("bf16_onchip", bf.BF_BF16, False)):
            if held:
                lh = layout(batch, 0, prec)
                Sq = torch.empty(lh.held_bytes // 4 + 4, dtype=torch.float32, device="cuda")
                sc = torch.empty(nb, dtype=torch.float32, device="cuda")
                bf.bf_quantize_symbols(plan, S, lay.groups, prec, Sq, lh.held_off, sc, stream)
                groups = [(g[0], g[1], lh.held_off[i], g[3]) for i, g in enumerate(lay.groups)]
                bf.bf_apply_batch(plan, Sq, sc, groups, prec, R, stream)
            else:
                bf.bf_apply_batch(plan, S, None, lay.groups, prec, R, stream)
            row[name] = rel_err(torch, bf, plan, R, ref_e, nb, stream)
        out["rel_err_by_log2_level"][str(e)] = row
    return out


def fused_output_leg(torch, bf, plan, batch, ref, stream, steps=2000, n_sets=4):
    """The full-band product writing R straight into the per-antenna layout
    the OFDM stage reads (antenna i's 3,822 x 60 resource elements in one
    row), as complex64 or bf16, from complex64 S or held bf16 S. n_sets
    rotating buffer sets keep the smallest form's working set above L2."""
    from bfrun import decode_r, layout, rl_layout, set_precoders, to_device_c64
    set_precoders(plan, batch, torch)
    lay = layout(batch)
    lh = layout(batch, 0, bf.BF_BF16)
    Sflat, _ = batch.pack_S()
    nb = batch.total_blocks
    S = [to_device_c64(Sflat, torch) for _ in range(n_sets)]
    Sq = [torch.empty(lh.held_bytes // 4 + 4, dtype=torch.float32, device="cuda") for _ in range(n_sets)]
    sc = [torch.empty(nb, dtype=torch.float32, device="cuda") for _ in range(n_sets)]
    g_c, _ = bf.make_groups(lay.groups)
    for s in range(n_sets):
        bf.bf_quantize_symbols(plan, S[s], g_c, bf.BF_BF16, Sq[s], lh.held_off, sc[s], stream)
    ref_blocks = None if ref is None else ref.reshape(nb, 64, 60)
    w_bytes = len(set(batch.prec)) * 64 * 36 * 8
    out = {"blocks": nb, "layout": "antenna-major: row i = antenna i, 60 resource elements per block, blocks in order"}
    for name, prec, held, rtype in (("bf16x3_c64S_c64R", bf.BF_BF16X3, False, bf.BF_R_C64),
                                    ("bf16x3_c64S_bf16R", bf.BF_BF16X3, False, bf.BF_R_BF16),
                                    ("bf16_heldS_bf16R", bf.BF_BF16, True, bf.BF_R_BF16)):
        rl, offs, nbytes = rl_layout(batch, rtype)
        R = [torch.empty(nbytes, dtype=torch.uint8, device="cuda") for _ in range(n_sets)]
        hs = []
        for s in range(n_sets):
            so = lh.held_off if held else [g[2] for g in lay.groups]
            groups = [(g[0], g[1], so[i], offs[i]) for i, g in enumerate(lay.groups)]
            hs.append(bf.bf_batch_create_rl(plan, Sq[s] if held else S[s], sc[s] if held else None, groups, prec,
                                            R[s], rl))
            bf.bf_batch_set_s_independent(hs[-1])  # S sets are written by copies or the encoder only
        ms = time_launches(torch, bf, hs, steps, 20, stream) / steps
        bf.bf_batch_launch(hs[0], stream)
        torch.cuda.synchronize()
        err = None
        if ref_blocks is not None:
            buf = R[0].cpu().numpy()
            if rtype == bf.BF_R_C64:
                got = buf.view(np.complex64).reshape(64, nb, 60).transpose(1, 0, 2).astype(np.complex128)
            else:
                got = decode_r(buf.view(np.uint16).reshape(64, nb, 60, 2), rtype).transpose(1, 0, 2)
            err = float(np.linalg.norm(got - ref_blocks) / np.linalg.norm(ref_blocks))
        moved = (lh.held_bytes if held else lay.s_bytes) + nbytes + w_bytes
        out[name] = {"kernel_ms": ms, "gflops": batch.flops() / ms / 1e6, "blocks_per_s": nb / ms * 1e3,
                     "moved_bytes": int(moved), "moved_gbs": moved / ms / 1e6, "rel_err": err}
        for h in hs:
            bf.bf_batch_destroy(h)
        del R
    del S, Sq, sc
    torch.cuda.empty_cache()
    return out


FILTER_SAMPLE = 16  # blocks of the filter workload checked against the oracle


def filter_cpu_leg(b):
    """Part of the CPU-baseline leg: the oracle's y for FILTER_SAMPLE blocks
    spread over the filter batch, and its rate on those blocks."""
    import oracle
    idx = np.unique(np.linspace(0, b.n_sig - 1, FILTER_SAMPLE).astype(int))
    rb = b.rounded()
    t0 = time.perf_counter()
    ref = oracle.circular_filter(rb.h, rb.s[idx])
    dt = time.perf_counter() - t0
    return idx, ref, {"us_per_block": dt / len(idx) * 1e6, "cores": oracle.num_threads(), "kind": "oracle",
                      "sample": f"{len(idx)} of {b.n_sig} blocks, direct FP64 circular convolution"}


def filter_leg(torch, bf, b, sample, stream, steps=100, variant=None):
    """Fast-convolution filter y = IFFT(MULT(FFT(s))) (Sec. III, Fig. 4, N = 2048)
    over 16 slots x 64 antennas x 14 symbols = 14,336 blocks: 235 MB read and
    235 MB written per launch (inputs larger than L2), one fused kernel."""
    from bfrun import to_device_c64
    f = bf.bf_filter_create(2048)
    h = to_device_c64(b.h, torch)
    bf.bf_filter_set_taps(f, h, len(b.h), stream)
    bf.bf_filter_set_s_independent(f)  # S is filled once, by a copy; the filter never writes it
    # the building block for this size on this GPU (the fastest variant),
    # unless a variant is named
    if variant is None:
        chosen = bf.bf_filter_autotune(f, b.n_sig, stream)
        variants = {bf.FILTER_VARIANTS[v]: bf.bf_filter_tune_query(f, v)[0] for v in range(len(bf.FILTER_VARIANTS))}
    else:
        bf.bf_filter_set_variant(f, variant)
        chosen, variants = variant, None
    S = to_device_c64(b.s, torch)
    Y = torch.empty_like(S)
    for _ in range(5):
        bf.bf_filter_apply(f, S, b.n_sig, Y, stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n0 = bf.bf_filter_launch_count(f)
    e0.record(stream)
    for _ in range(steps):
        bf.bf_filter_apply(f, S, b.n_sig, Y, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = bf.bf_filter_launch_count(f) - n0
    ms = e0.elapsed_time(e1) / steps
    # latency-style figures beside the throughput: one block alone (what the
    # paper timed on one core) and one slot (64 antennas x 14 symbols), each
    # launched back to back
    small = {}
    for name, n_sig in (("one_block", 1), ("one_slot", 896)):
        for _ in range(5):
            bf.bf_filter_apply(f, S, n_sig, Y, stream)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(200):
            bf.bf_filter_apply(f, S, n_sig, Y, stream)
        a1.record(stream)
        torch.cuda.synchronize()
        small[name + "_us"] = a0.elapsed_time(a1) / 200 * 1e3
    moved = b.algorithmic_bytes()
    out = {"blocks": b.n_sig, "n": b.n, "kernel_ms": ms, "blocks_per_s": b.n_sig / ms * 1e3,
           "us_per_block_amortised": ms * 1e3 / b.n_sig, "gflops_conventional": b.flops() / ms / 1e6,
           "moved_bytes": moved, "moved_gbs": moved / ms / 1e6, "gpu_launches": int(launches), **small,
           "variant": {"chosen": bf.FILTER_VARIANTS[chosen], "us_per_launch_tuned": variants},
           "paper_context_us_per_filter": {"original": 27, "intel_fft_library": 19,
                                           "hardware": "Intel Haswell (E9000 blade), one filter"}}
    if sample is not None:
        idx, ref, cpu = sample
        y = Y.cpu().numpy().view(np.complex64).reshape(b.n_sig, b.n)[idx].astype(np.complex128)
        out["rel_err"] = float(np.linalg.norm(y - ref) / np.linalg.norm(ref))
        out["cpu_baseline"] = cpu
    # end to end: pinned host blocks in, filtered blocks out, every call;
    # calls alternate between two streams and two buffer pairs (pipelined),
    # and the same on one stream
    S_h = [S.cpu().pin_memory() for _ in range(2)]
    Y_h = [torch.empty_like(S_h[0]).pin_memory() for _ in range(2)]
    streams = [stream, torch.cuda.Stream()]

    def timed(n_streams, n=6):
        for i in range(2):
            bf.bf_filter_apply_host(f, S_h[i], b.n_sig, Y_h[i], streams[i % n_streams])
        torch.cuda.synchronize()
        e0.record(streams[0])
        streams[1].wait_event(e0)
        for i in range(n):
            bf.bf_filter_apply_host(f, S_h[i % 2], b.n_sig, Y_h[i % 2], streams[i % n_streams])
        streams[0].wait_stream(streams[1])
        e1.record(streams[0])
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    e2e_ms = timed(2)
    out["e2e"] = {"ms": e2e_ms, "blocks_per_s": b.n_sig / e2e_ms * 1e3, "h2d_bytes": moved // 2,
                  "d2h_bytes": moved // 2, "one_stream_ms": timed(1)}
    bf.bf_filter_destroy(f)
    del S, Y, S_h, Y_h
    torch.cuda.empty_cache()
    return out


def finite_json(obj):
    """The JSON line with non-finite numbers (skipped legs) as null."""
    if isinstance(obj, float):
        return obj if np.isfinite(obj) else None
    if isinstance(obj, dict):
        return {k: finite_json(v) for k, v in obj.items()}
    if isinstance(obj, (list, tuple)):
        return [finite_json(v) for v in obj]
    return obj


def run_leg(legs, name, fn, *args):
    """Run one secondary workload; a failure is reported in its entry and the
    headline line is still printed."""
    try:
        legs[name] = fn(*args)
    except Exception as e:  # reported, not hidden: the entry carries the error
        legs[name] = {"error": f"{type(e).__name__}: {e}"}


def serving_leg(torch, bf, ttis, prec):
    """Continuous-batching serving of 8 cells in real time (0.5 ms TTIs)."""
    import workloads as wl
    from serving_sim import ServingSim
    plan = bf.bf_plan_create(64, 36, 60)
    sim = ServingSim(plan, torch, prec=prec)
    try:
        return sim.run(wl.serving_schedule(n_tti=ttis))
    finally:
        sim.close()
        bf.bf_plan_destroy(plan)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg")
    ap.add_argument("--no-plain", action="store_true", help="skip the FP32 plain leg")
    ap.add_argument("--sets", type=int, default=3, help="rotating buffer sets (3 keeps the working set above L2)")
    ap.add_argument("--no-extra", action="store_true", help="skip the uneven, reduced-precision and serving legs")
    ap.add_argument("--serving-ttis", type=int, default=20000, help="TTIs of the split-bf16 serving run")
    ap.add_argument("--filter-variant", type=int, default=None,
                    help="filter building block to time (default: the autotuner's choice)")
    ap.add_argument("--legs", default="fused_output,uneven,reduced,scaling,filter,serving",
                    help="comma-separated secondary workloads to run after the headline")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_1810_11451_gb300 as bf
    import workloads as wl
    from bfrun import layout, set_precoders, to_device_c64

    dist, rank, world = dist_init()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    torch.cuda.init()
    plan = bf.bf_plan_create(64, 36, 60)
    batch = wl.config_fullband()
    set_precoders(plan, batch, torch)
    lay = layout(batch)
    Sflat, _ = batch.pack_S()
    n_sets = max(1, args.sets)
    S_sets = [to_device_c64(Sflat, torch) for _ in range(n_sets)]
    R_sets = [torch.empty(lay.r_blocks * 64 * 60 * 2, dtype=torch.float32, device="cuda") for _ in range(n_sets)]
    stream = torch.cuda.current_stream()
    best = {s: bf.bf_batch_create(plan, S_sets[s], None, lay.groups, bf.BF_BF16X3, R_sets[s]) for s in range(n_sets)}
    plain = {s: bf.bf_batch_create(plan, S_sets[s], None, lay.groups, bf.BF_FP32, R_sets[s]) for s in range(n_sets)}
    plain3 = {s: bf.bf_batch_create(plan, S_sets[s], None, lay.groups, bf.BF_FP32_3M, R_sets[s])
              for s in range(n_sets)}
    tf32 = {s: bf.bf_batch_create(plan, S_sets[s], None, lay.groups, bf.BF_TF32X3, R_sets[s])
            for s in range(n_sets)}
    # No product launch writes any S set (they are filled once, by copies), so
    # each step's kernel may load its S while the previous step's finishes.
    for hs in (best, plain, plain3, tf32):
        for h in hs.values():
            bf.bf_batch_set_s_independent(h)
    handles = [best[s] for s in range(n_sets)]
    flops = batch.flops()
    alg_bytes = batch.algorithmic_bytes()

    # ---- headline: best form, device-resident inputs
    barrier(dist)
    torch.cuda.synchronize()
    launches0 = bf.bf_plan_launch_count(plan)
    with ClockSampler(local) as clk:
        total_ms = time_launches(torch, bf, handles, args.steps, args.warmup, stream)
    launches = bf.bf_plan_launch_count(plan) - launches0 - args.warmup
    barrier(dist)
    total_ms = max_over_ranks(dist, total_ms)
    ms_step = total_ms / args.steps
    kern_ms = total_ms / args.steps  # one kernel launch per step
    value = world * flops * args.steps / (total_ms * 1e-3) / 1e9
    blocks_s = world * batch.total_blocks * args.steps / (total_ms * 1e-3)

    # ---- context for the roofline: a plain device copy moving the launch's
    # algorithmic bytes (half read, half written) over the same number of
    # rotating buffer sets, back to back. At this size the fixed cost of a
    # launch keeps even a copy below the peak measured on large buffers.
    copy_us = float("nan")
    if not args.no_plain:
        half = (alg_bytes // 2) // 16 * 4
        srcs = [torch.zeros(half, dtype=torch.float32, device="cuda") for _ in range(n_sets)]
        dsts = [torch.empty_like(srcs[0]) for _ in range(n_sets)]
        for i in range(max(3, args.warmup)):
            dsts[i % n_sets].copy_(srcs[i % n_sets])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k_copy = 300
        torch.cuda.synchronize()
        e0.record(stream)
        for i in range(k_copy):
            dsts[i % n_sets].copy_(srcs[i % n_sets])
        e1.record(stream)
        torch.cuda.synchronize()
        copy_us = e0.elapsed_time(e1) * 1e3 / k_copy
        copy_bytes = 2 * half * 4
        del srcs, dsts

    # ---- the plain FP32 form on the same GPU
    k2 = max(50, args.steps // 10)
    p_ms = p3_ms = t32_ms = float("nan")
    if not args.no_plain:
        p_total = time_launches(torch, bf, [plain[s] for s in range(n_sets)], k2, args.warmup, stream)
        p_ms = p_total / k2
        p3_ms = time_launches(torch, bf, [plain3[s] for s in range(n_sets)], k2, args.warmup, stream) / k2
        t32_ms = time_launches(torch, bf, [tf32[s] for s in range(n_sets)], k2, args.warmup, stream) / k2

    # ---- the FP32 FMA rate of the CUDA cores: the plain form's roofline
    fma = None
    if not args.no_plain:
        with ClockSampler(local) as fclk:
            fma_tf, fma_ms = bf.bf_measure_fp32_peak(20000, 5, 0, stream)
            fma2_tf, _ = bf.bf_measure_fp32_peak(10000, 5, 1, stream)
            outer_tf, _ = bf.bf_measure_fp32_peak(20000, 5, 2, stream)
        # the peak is the faster of scalar and packed FP32x2 FMAs; the
        # outer-product operand pattern (two new register pairs per FMA, as in
        # any product loop) is reported beside it as the ceiling of such a loop
        fma = {"tflops": max(fma_tf, fma2_tf), "scalar_tflops": fma_tf, "packed_tflops": fma2_tf,
               "outer_product_tflops": outer_tf,
               "ms_per_launch": fma_ms, "clocks": fclk.summary(),
               "how": "bf_measure_fp32_peak: 4 CTAs x 256 threads per SM, 8 independent FMA chains per thread, "
                      "scalar and packed FP32x2 (one register operand per FMA), and packed FP32x2 over a 4 x 4 "
                      "register-blocked outer product (mode 2); best of 5 launches each (CUDA events)"}

    # ---- end to end through the host-buffer entry point
    e2e = None
    if not args.no_e2e:
        e2e = end_to_end(torch, bf, plan, Sflat, lay, R_sets[0].numel(), stream, dist, world, flops)

    # ---- CPU baseline (oracle), which also gives the references for accuracy
    cpu, acc, refs, ref_full = None, None, {}, None
    extra = not args.no_extra and rank == 0
    want = set(x.strip() for x in args.legs.split(",") if x.strip())
    b_uneven = wl.config_uneven() if extra and "uneven" in want else None
    b_reduced = wl.config_reduced() if extra and "reduced" in want else None
    b_filter = wl.config_filter_bench() if extra and "filter" in want else None
    b_scaling = wl.config_reduced(copies=1, n_rb=6, n_sym=14) if extra and "scaling" in want else None
    filter_sample = None
    if rank == 0 and not args.no_cpu:
        cpu, ref = cpu_baseline(batch)
        refs = cpu_references({"fullband": ref}, {"uneven": b_uneven, "reduced": b_reduced, "scaling": b_scaling})
        if b_filter is not None:
            filter_sample = filter_cpu_leg(b_filter)
        ref_full = refs.pop("fullband")
        Rref_d = to_device_ref(torch, ref_full)
        acc = {}
        for name, h in (("bf16x3", best[0]), ("fp32", plain[0]), ("fp32_3m", plain3[0]), ("tf32x3", tf32[0])):
            bf.bf_batch_launch(h, stream)
            num, den = bf.bf_errnorm(plan, R_sets[0], Rref_d, lay.r_blocks, None, stream)
            acc[name] = float(np.sqrt(num / den))
        del Rref_d
    for s in range(n_sets):
        bf.bf_batch_destroy(best[s])
        bf.bf_batch_destroy(plain[s])
        bf.bf_batch_destroy(plain3[s])
        bf.bf_batch_destroy(tf32[s])
    del S_sets, R_sets
    torch.cuda.empty_cache()

    # ---- the other workloads: uneven batching, reduced precision, serving
    legs = {}
    if extra and "fused_output" in want:
        run_leg(legs, "fused_output", fused_output_leg, torch, bf, plan, batch, ref_full, stream)
    ref_full = None
    if b_uneven is not None:
        ref_d = to_device_ref(torch, refs.pop("uneven", None))
        run_leg(legs, "uneven", uneven_leg, torch, bf, plan, b_uneven, ref_d, stream)
        del ref_d
    if b_reduced is not None:
        ref_d = to_device_ref(torch, refs.pop("reduced", None))
        run_leg(legs, "reduced", reduced_leg, torch, bf, plan, b_reduced, ref_d, stream)
        del ref_d
        torch.cuda.empty_cache()
    if b_scaling is not None and "scaling" in refs:
        ref_d = to_device_ref(torch, refs.pop("scaling"))
        run_leg(legs, "scaling", scaling_leg, torch, bf, plan, b_scaling, ref_d, stream)
        del ref_d
    if b_filter is not None:
        run_leg(legs, "filter", filter_leg, torch, bf, b_filter, filter_sample, stream, 100, args.filter_variant)
    if extra and "serving" in want:
        run_leg(legs, "serving_bf16x3", serving_leg, torch, bf, args.serving_ttis, bf.BF_BF16X3)
        run_leg(legs, "serving_fp32", serving_leg, torch, bf, args.serving_ttis, bf.BF_FP32)
    status = bf.bf_device_status(plan)

    peak, peak_kind = peaks()
    achieved = alg_bytes / (kern_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x3", "data": "synthetic",
        "config": {"workload": WORKLOAD, "form": "split-bf16 (hi*hi + hi*lo + lo*hi) tcgen05, FP32 accumulate",
                   "blocks": batch.total_blocks, "l2": L2_NOTE, "launch": "one persistent kernel per step (prepared batch, direct launch; declared S-independent, so a step's S loads while the previous step's kernel finishes)",
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "blocks_per_s": blocks_s,
        "fp32_plain": {"value": world * flops / (p_ms * 1e-3) / 1e9 if p_ms == p_ms else None, "unit": UNIT, "ms_per_step": p_ms,
                       "kernel_ms": p_ms,
                       "blocks_per_s": world * batch.total_blocks / (p_ms * 1e-3),
                       "roofline": None if fma is None or p_ms != p_ms else {
                           "bound": "fma", "achieved_tflops": flops / (p_ms * 1e-3) / 1e12,
                           "peak_tflops": fma["tflops"], "frac": flops / (p_ms * 1e-3) / 1e12 / fma["tflops"],
                           "frac_of_outer_product_rate": flops / (p_ms * 1e-3) / 1e12 / fma["outer_product_tflops"],
                           "peak": fma}},
        "fp32_3m": {"value": world * flops / (p3_ms * 1e-3) / 1e9 if p3_ms == p3_ms else None, "unit": UNIT,
                    "kernel_ms": p3_ms, "form": "FP32 CUDA cores, three real products per complex multiply-add",
                    "frac_of_fma_peak": None if fma is None or p3_ms != p3_ms else
                    flops / (p3_ms * 1e-3) / 1e12 / fma["tflops"],
                    "frac_note": "conventional flops (8 per complex multiply-add) over the measured FMA rate; "
                                 "the form issues 6 of them as FMAs"},
        "tf32x3": {"value": world * flops / (t32_ms * 1e-3) / 1e9 if t32_ms == t32_ms else None, "unit": UNIT,
                   "kernel_ms": t32_ms, "hbm_gbs": alg_bytes / (t32_ms * 1e-3) / 1e9 if t32_ms == t32_ms else None,
                   "form": "split-tf32 (hi*hi + hi*lo + lo*hi) tcgen05 kind::tf32, FP32 accumulate"},
        "speedup_vs_fp32_plain": p_ms / ms_step if p_ms == p_ms else None,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic_for("bf_tc.cu"),
                     "peak_source": f"{peak_kind} hbm_gbs", "kernel": "bf_tc_kernel<3,false,OP_BF16>",
                     "kernel_ms": kern_ms, "algorithmic_bytes_per_launch": alg_bytes,
                     "same_bytes_copy": None if copy_us != copy_us else {
                         "us": copy_us, "gbs": copy_bytes / (copy_us * 1e3),
                         "kernel_time_over_copy_time": kern_ms * 1e3 / copy_us,
                         "how": f"torch copy_ of {copy_bytes / 2e6:.1f} MB into {copy_bytes / 2e6:.1f} MB, "
                                f"{n_sets} rotating sets, back to back (context, not the peak)"}},
        "e2e": e2e,
        "cpu_baseline": cpu,
        "accuracy_rel_frobenius": acc,
        "clocks": clk.summary(),
        "gpu_launches": int(launches),
        "device_status": bf.bf_status_string(status),
    }
    if legs:
        srv = legs.get("serving_bf16x3", {})
        line["p99_tti_latency_ms"] = srv["p99_us"] / 1e3 if "p99_us" in srv else None
        line["legs"] = legs
    bf.bf_plan_destroy(plan)
    if rank == 0:
        print(json.dumps(finite_json(line)), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
