"""CPU checks of the C ABI: the library loads and exports every declared symbol,
argument checks that precede any CUDA call, and the host-side scheduler."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bf():
    from paper_1810_11451_gb300 import build
    build.build()
    import paper_1810_11451_gb300 as m
    m.lib()
    return m


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*?[\s\*]+(bf_[a-z0-9_]+)\s*\(", src, re.M)
    return sorted(set(names))


def test_exports_every_declared_symbol(bf):
    names = declared_functions()
    assert len(names) >= 15
    L = ctypes.CDLL(bf.LIB_PATH)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_binding_names_match_header(bf):
    for n in declared_functions():
        assert hasattr(bf, n), f"binding lacks {n}"


def test_plan_create_rejects_shapes_before_cuda(bf):
    for args in [(32, 36, 60), (64, 37, 60), (64, -1, 60), (64, 36, 64)]:
        with pytest.raises(bf.BfError) as ei:
            bf.bf_plan_create(*args)
        assert ei.value.status == bf.BF_EINVAL
    assert "n_ant" in bf.bf_last_error(None) or "b must" in bf.bf_last_error(None)


def test_status_strings(bf):
    assert bf.bf_status_string(bf.BF_OK) == "BF_OK"
    assert bf.bf_status_string(bf.BF_ETIMEOUT) == "BF_ETIMEOUT"
    assert bf.bf_status_string(99) == "BF_UNKNOWN"


def test_held_block_bytes(bf):
    for f in range(0, 37):
        k = ((2 * f + 15) // 16) * 16
        assert bf.bf_held_block_bytes(f, bf.BF_BF16) == 128 * k
        assert bf.bf_held_block_bytes(f, bf.BF_FP16) == 128 * k
        assert bf.bf_held_block_bytes(f, bf.BF_BF16X3) == 256 * k
        assert bf.bf_held_block_bytes(f, bf.BF_FP32) == 0
    assert bf.bf_held_block_bytes(37, bf.BF_BF16) == 0


def test_missing_library_fails_loudly(bf, monkeypatch):
    monkeypatch.setattr(bf, "LIB_PATH", "/nonexistent/libbf.so")
    monkeypatch.setattr(bf, "_lib", None)
    with pytest.raises(ImportError):
        bf.lib()


class BfTile(ctypes.Structure):
    _fields_ = [("s_off", ctypes.c_int64), ("r_off", ctypes.c_int64), ("prec_id", ctypes.c_int32),
                ("first_block", ctypes.c_int32), ("f", ctypes.c_int16), ("n_blocks", ctypes.c_int16),
                ("flags", ctypes.c_int32)]


def schedule(bf, f_of_slot, groups, prec, held, max_cta):
    L = bf.lib()
    L.bf_schedule.restype = ctypes.c_int32
    fa = (ctypes.c_int32 * len(f_of_slot))(*f_of_slot)
    ga, n = bf.make_groups(groups)
    ncta = ctypes.c_int32()
    nt = L.bf_schedule(fa, len(f_of_slot), ga, n, prec, held, max_cta, None, 0, None, ctypes.byref(ncta))
    assert nt >= 0
    tiles = (BfTile * max(1, nt))()
    begin = (ctypes.c_int32 * (max_cta + 1))()
    nt2 = L.bf_schedule(fa, len(f_of_slot), ga, n, prec, held, max_cta, tiles, nt, begin, ctypes.byref(ncta))
    assert nt2 == nt
    return list(tiles)[:nt], list(begin)[:ncta.value + 1]


@pytest.mark.parametrize("max_cta", [1, 7, 152, 10000])
def test_scheduler_covers_every_block_once(bf, max_cta):
    batch = wl.config_uneven(seed=3, n_blocks=1500)
    from bfrun import layout
    groups = layout(batch).groups
    f_of_slot = batch.f_of_group
    tiles, begin = schedule(bf, f_of_slot, groups, bf.BF_BF16X3, 0, max_cta)
    # every block exactly once, in group order, tiles of <= 2 blocks of one group
    seen = []
    for t in tiles:
        assert 1 <= t.n_blocks <= 2 and t.f == f_of_slot[t.prec_id]
        seen += list(range(t.first_block, t.first_block + t.n_blocks))
    assert seen == list(range(batch.total_blocks))
    # offsets follow the group layout
    blk_group = np.repeat(np.arange(len(groups)), batch.n_blocks)
    first_in_group = np.cumsum([0] + batch.n_blocks[:-1])
    for t in tiles:
        g = blk_group[t.first_block]
        n = t.first_block - first_in_group[g]
        assert t.s_off == groups[g][2] + n * 480 * batch.f_of_group[g]
        assert t.r_off == groups[g][3] + n * 30720
    # contiguous CTA ranges covering all tiles, none empty
    assert begin[0] == 0 and begin[-1] == len(tiles)
    assert all(begin[c] < begin[c + 1] for c in range(len(begin) - 1))
    assert len(begin) - 1 == min(max_cta, batch.total_blocks)
    # cost balance at block granularity: no CTA above the mean by more than one block's cost
    cost = np.array([t.n_blocks * (480 * t.f + 30720) for t in tiles], float)
    per = [cost[begin[c]:begin[c + 1]].sum() for c in range(len(begin) - 1)]
    assert max(per) <= cost.sum() / len(per) + (480 * 36 + 30720)
    # precoder-run flags
    for c in range(len(begin) - 1):
        run = [t for t in tiles[begin[c]:begin[c + 1]] if t.f > 0]
        for i, t in enumerate(run):
            first = i == 0 or run[i - 1].prec_id != t.prec_id
            last = i == len(run) - 1 or run[i + 1].prec_id != t.prec_id
            assert bool(t.flags & 1) == first and bool(t.flags & 2) == last


def test_scheduler_rejects_bad_input(bf):
    L = bf.lib()
    fa = (ctypes.c_int32 * 2)(8, 40)
    ga, n = bf.make_groups([(1, 2, 0, 0)])
    ncta = ctypes.c_int32()
    assert L.bf_schedule(fa, 2, ga, n, bf.BF_FP32, 0, 4, None, 0, None, ctypes.byref(ncta)) == -bf.BF_EINVAL
    ga, n = bf.make_groups([(5, 2, 0, 0)])
    assert L.bf_schedule(fa, 2, ga, n, bf.BF_FP32, 0, 4, None, 0, None, ctypes.byref(ncta)) == -bf.BF_EINVAL
    ga, n = bf.make_groups([(0, 2, 0, 0)])
    assert L.bf_schedule(fa, 2, ga, n, bf.BF_FP32, 1, 4, None, 0, None, ctypes.byref(ncta)) == -bf.BF_EINVAL
    for prec in (bf.BF_FP32_3M, bf.BF_TF32X3):  # no held S for these forms
        assert L.bf_schedule(fa, 2, ga, n, prec, 1, 4, None, 0, None, ctypes.byref(ncta)) == -bf.BF_EINVAL
    assert L.bf_schedule(fa, 2, ga, n, 6, 0, 4, None, 0, None, ctypes.byref(ncta)) == -bf.BF_EINVAL
    assert L.bf_schedule(fa, 2, ga, n, bf.BF_TF32X3, 0, 1, None, 0, None, ctypes.byref(ncta)) == 1
    # two blocks over up to four CTAs: one block (one tile) each; on one CTA, one two-block tile
    assert L.bf_schedule(fa, 2, ga, n, bf.BF_FP32, 0, 4, None, 0, None, ctypes.byref(ncta)) == 2
    assert ncta.value == 2
    assert L.bf_schedule(fa, 2, ga, n, bf.BF_FP32, 0, 1, None, 0, None, ctypes.byref(ncta)) == 1


def test_scheduler_empty_and_zero_f(bf):
    tiles, begin = schedule(bf, [0, 3], [(0, 3, 0, 0), (1, 0, 0, 0)], bf.BF_FP32, 0, 1)
    assert [t.n_blocks for t in tiles] == [2, 1] and all(t.flags == 0 for t in tiles)
    tiles, begin = schedule(bf, [0, 3], [(0, 3, 0, 0), (1, 0, 0, 0)], bf.BF_FP32, 0, 4)
    assert [t.n_blocks for t in tiles] == [1, 1, 1] and begin == [0, 1, 2, 3]
    tiles, begin = schedule(bf, [3], [], bf.BF_FP32, 0, 4)
    assert tiles == [] and begin == [0, 0]


def test_filter_create_rejects_size_before_cuda(bf):
    L = bf._filter_sigs(bf.lib())
    h = ctypes.c_void_p()
    assert L.bf_filter_create(1024, ctypes.byref(h)) == bf.BF_EINVAL and not h.value
    assert "2048" in bf.bf_filter_last_error(None)
    assert L.bf_filter_create(2048, None) == bf.BF_EINVAL
    assert L.bf_filter_destroy(None) == bf.BF_OK


def _table(path, device="NVIDIA GB300", cc=103, sms=152, fmt="libbf-tune-2"):
    prec = ",\n".join(f'    {{"precision": {p}, "tuned": 1, "ns_per_block": [1.0, 2.0, 3.0, 4.0, 5.0], '
                      f'"tile_blocks": [2, 2, 2, 2, 2]}}' for p in range(6))
    with open(path, "w") as fh:
        fh.write(f'{{\n  "format": "{fmt}",\n  "target": {{"device": "{device}", "cc": {cc}, "sm_count": {sms}}},\n'
                 f'  "simt_ctas_per_sm": [2, 2],\n  "f_bucket_upper": [0, 8, 16, 24, 36],\n  "precisions": [\n'
                 f'{prec}\n  ]\n}}\n')


def test_tune_table_is_keyed_by_target(bf, tmp_path):
    """A tune table names the target it was measured on (device name, compute
    capability, SM count); a table from another GPU, or one without a target,
    is refused before anything is loaded."""
    p = str(tmp_path / "t.json")
    _table(p)
    bf.bf_tune_check_target(p, "NVIDIA GB300", 103, 152)
    for other in [("NVIDIA GB300", 103, 148), ("NVIDIA B200", 100, 148), ("NVIDIA GB300", 100, 152),
                  ("NVIDIA GB200", 103, 152)]:
        with pytest.raises(bf.BfError) as ei:
            bf.bf_tune_check_target(p, *other)
        assert ei.value.status == bf.BF_EINVAL and "not on this target" in str(ei.value)
    _table(p, fmt="libbf-tune-1")
    with pytest.raises(bf.BfError) as ei:
        bf.bf_tune_check_target(p, "NVIDIA GB300", 103, 152)
    assert ei.value.status == bf.BF_EINVAL
    with pytest.raises(bf.BfError):
        bf.bf_tune_check_target(str(tmp_path / "missing.json"), "NVIDIA GB300", 103, 152)


def test_new_entry_points_reject_bad_arguments_before_cuda(bf):
    """Argument checks that come before any CUDA call: the FMA probe's ranges,
    the filter calls on a NULL filter, the target check's NULL arguments."""
    L = bf.lib()
    L.bf_measure_fp32_peak.restype = ctypes.c_int
    L.bf_measure_fp32_peak.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                       ctypes.c_void_p]
    t, ms = ctypes.c_double(), ctypes.c_double()
    for iters, reps, mode in [(0, 5, 0), (1 << 25, 5, 0), (10, 0, 0), (10, 1001, 0), (10, 5, 3), (10, 5, -1)]:
        assert L.bf_measure_fp32_peak(iters, reps, mode, ctypes.byref(t), ctypes.byref(ms), None) == bf.BF_EINVAL
    assert L.bf_measure_fp32_peak(10, 5, 0, None, None, None) == bf.BF_EINVAL
    with pytest.raises(bf.BfError) as ei:
        bf.bf_filter_set_variant(None, 0)
    assert ei.value.status == bf.BF_EINVAL
    assert bf.bf_filter_get_variant(None) == -1
    with pytest.raises(bf.BfError) as ei:
        bf.bf_filter_autotune(None, 100)
    assert ei.value.status == bf.BF_EINVAL
    with pytest.raises(bf.BfError) as ei:
        bf.bf_filter_tune_query(None, 0)
    assert ei.value.status == bf.BF_EINVAL
    L.bf_tune_check_target.restype = ctypes.c_int
    L.bf_tune_check_target.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.c_int32, ctypes.c_int32]
    assert L.bf_tune_check_target(None, b"x", 103, 152) == bf.BF_EINVAL
    assert L.bf_tune_check_target(b"/nonexistent/t.json", None, 103, 152) == bf.BF_EINVAL


@pytest.mark.parametrize("max_cta", [1, 2, 3, 5])
def test_scheduler_flags_with_shared_slots_and_empty_flows(bf, max_cta):
    """Consecutive groups on the same precoder slot form one run (no new first
    flag), f = 0 tiles carry no flags and do not break a run, and ranges start
    new runs: the flags equal their definition, worked out in Python."""
    f_of_slot = [36, 0, 8]
    groups = [(0, 5, 0, 0), (0, 3, 0, 0), (1, 2, 0, 0), (0, 2, 0, 0), (2, 4, 0, 0), (2, 1, 0, 0)]
    tiles, begin = schedule(bf, f_of_slot, groups, bf.BF_BF16X3, 0, max_cta)
    for t in tiles:
        if t.f == 0:
            assert t.flags == 0
    for c in range(len(begin) - 1):
        run = [t for t in tiles[begin[c]:begin[c + 1]] if t.f > 0]
        for i, t in enumerate(run):
            first = i == 0 or run[i - 1].prec_id != t.prec_id
            last = i == len(run) - 1 or run[i + 1].prec_id != t.prec_id
            assert bool(t.flags & 1) == first and bool(t.flags & 2) == last, (c, i, t.prec_id, t.flags)
