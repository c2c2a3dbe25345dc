"""The optimizer's per-batch form choice (bf_select_form) on the GPU plan:
from a crafted tune table (exact expected choices worked out by hand) and
from the autotuner's own measurements."""
import json

import pytest

import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1810_11451_gb300 as bf  # noqa: E402
from bfrun import layout, set_precoders  # noqa: E402


@pytest.fixture()
def plan():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    p = bf.bf_plan_create(64, 36, 60)
    yield p
    bf.bf_plan_destroy(p)


def _groups_f(plan, fs_blocks):
    """Set one precoder per (f, n_blocks) pair and return the groups."""
    W = torch.zeros(sum(64 * f for f, _ in fs_blocks) * 2 + 4, device="cuda")
    bf.bf_set_precoders(plan, W, [f for f, _ in fs_blocks], 0)
    torch.cuda.synchronize()
    return [(i, n, 0, 0) for i, (_, n) in enumerate(fs_blocks)]


def test_untuned_defaults(plan):
    g = _groups_f(plan, [(36, 14)])
    assert bf.bf_select_form(plan, bf.BF_TARGET_FP32, g) == (bf.BF_BF16X3, 0.0)
    assert bf.bf_select_form(plan, bf.BF_TARGET_BF16, g) == (bf.BF_BF16, 0.0)


def test_crafted_table(plan, tmp_path):
    path = str(tmp_path / "t.json")
    bf.bf_tune_save(plan, path)
    t = json.load(open(path))
    ns = {bf.BF_BF16X3: [5, 6, 7, 8, 9], bf.BF_FP32: [1, 2, 20, 30, 40], bf.BF_FP16: [1, 1, 1, 1, 1]}
    for e in t["precisions"]:
        if e["precision"] in ns:
            e["tuned"], e["ns_per_block"] = 1, ns[e["precision"]]
    json.dump(t, open(path, "w"))
    bf.bf_tune_load(plan, path)
    # buckets: f = 4 -> 1, f = 36 -> 4
    g_small = _groups_f(plan, [(4, 100)])
    assert bf.bf_select_form(plan, bf.BF_TARGET_FP32, g_small) == (bf.BF_FP32, 200.0)  # 2*100 < 6*100
    g_big = _groups_f(plan, [(36, 100)])
    assert bf.bf_select_form(plan, bf.BF_TARGET_FP32, g_big) == (bf.BF_BF16X3, 900.0)  # 9*100 < 40*100
    # mixed: FP32 10*2 + 10*40 = 420, split 10*6 + 10*9 = 150
    g_mix = _groups_f(plan, [(4, 10), (36, 10)])
    assert bf.bf_select_form(plan, bf.BF_TARGET_FP32, g_mix) == (bf.BF_BF16X3, 150.0)
    # the bf16 target may take the single-pass fp16 form (1 ns everywhere)
    assert bf.bf_select_form(plan, bf.BF_TARGET_BF16, g_mix) == (bf.BF_FP16, 20.0)
    with pytest.raises(bf.BfError) as ei:
        bf.bf_select_form(plan, bf.BF_TARGET_FP32, [(999, 1, 0, 0)])
    assert ei.value.status == bf.BF_ENOTFOUND
    with pytest.raises(bf.BfError) as ei:
        bf.bf_select_form(plan, 7, g_mix)
    assert ei.value.status == bf.BF_EINVAL


def test_measured_choice_full_band(plan):
    """After tuning the four FP32-accurate forms, the full band (f = 36)
    selects the form the measurements make fastest, and its prediction is the
    sum of the tuned per-block costs."""
    batch = wl.config_fullband()
    set_precoders(plan, batch, torch)
    groups = layout(batch).groups
    accurate = (bf.BF_FP32, bf.BF_FP32_3M, bf.BF_BF16X3, bf.BF_TF32X3)
    for p in accurate:
        bf.bf_autotune(plan, p)
    form, ns = bf.bf_select_form(plan, bf.BF_TARGET_FP32, groups)
    costs = {p: bf.bf_tune_query(plan, p, 36)["ns_per_block"] * batch.total_blocks
             for p in accurate}
    assert form == min(costs, key=costs.get) and abs(ns - costs[form]) <= 1e-6 * ns
    print("full band choice:", form, {k: round(v / 1e3, 1) for k, v in costs.items()}, "us")
