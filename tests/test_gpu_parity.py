"""GPU parity of every product form against the FP64 oracle, through the C ABI.

Tolerances (relative Frobenius error over the batch, from the accuracy target
of the method's reduced-precision study): <= 1e-5 for the FP32 forms and the
split bf16 / tf32 forms, <= 2e-2 for single-pass bf16/fp16 (measured against the
unrounded FP64 inputs, so the bound covers the operand rounding). Exact-integer
inputs (odd-integer QAM, Gaussian-integer W in {-2..2}) make every product and
partial sum exact in bf16, fp16, tf32 and fp32, so there every form must match the
oracle bit for bit. R is NaN-poisoned before each run, so unwritten elements
(including f = 0 blocks and ragged tiles) fail.
"""
import numpy as np
import pytest

import oracle
import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1810_11451_gb300 as bf  # noqa: E402
from bfrun import layout, run, set_precoders, to_device_c64  # noqa: E402

TOL_FP32 = 1e-5
TOL_SPLIT = 1e-5
TOL_SINGLE = 2e-2
FORMS = [("fp32", bf.BF_FP32, False), ("bf16x3", bf.BF_BF16X3, False), ("bf16x3_held", bf.BF_BF16X3, True),
         ("bf16", bf.BF_BF16, False), ("bf16_held", bf.BF_BF16, True), ("fp16", bf.BF_FP16, False),
         ("fp16_held", bf.BF_FP16, True), ("fp32_3m", bf.BF_FP32_3M, False), ("tf32x3", bf.BF_TF32X3, False)]


@pytest.fixture(scope="module")
def plan():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    p = bf.bf_plan_create(64, 36, 60)
    yield p
    assert bf.bf_device_status(p) == bf.BF_OK
    bf.bf_plan_destroy(p)


def _ref(batch):
    return oracle.apply_batch(batch.rounded(np.complex64))


# forms checked against the oracle of the complex64-rounded inputs (per-block errors too)
ACCURATE = (bf.BF_FP32, bf.BF_FP32_3M, bf.BF_BF16X3, bf.BF_TF32X3)


def _tol(prec):
    return {bf.BF_FP32: TOL_FP32, bf.BF_FP32_3M: TOL_FP32, bf.BF_BF16X3: TOL_SPLIT,
            bf.BF_TF32X3: TOL_SPLIT}.get(prec, TOL_SINGLE)


def _assert_close(R, ref, tol, what):
    assert all(np.all(np.isfinite(r)) for r in R), f"{what}: unwritten (NaN) outputs"
    e = oracle.rel_frobenius(R, ref)
    assert e <= tol, f"{what}: relative Frobenius error {e:.3e} > {tol:.1e}"
    return e


# the oracle's encoding of each tensor-core form
ENC = {bf.BF_BF16: "bf16", bf.BF_FP16: "fp16", bf.BF_BF16X3: "bf16x3", bf.BF_TF32X3: "tf32x3"}
# what separates a tensor-core result from the FP64 product of the oracle's
# encodings of the same operands: FP32 accumulation rounding only
MECH_BOUND = 2e-6


def _assert_per_block(R, ref, tol, what):
    """Every block within tol of the oracle (relative Frobenius error of the
    block); blocks whose reference is zero (f = 0) must be exactly zero."""
    worst = 0.0
    for g, (a, r) in enumerate(zip(R, ref)):
        if a.size == 0:
            continue
        assert np.all(np.isfinite(a)), f"{what}: group {g}: unwritten (NaN) outputs"
        num, den = oracle.errnorm_blocks(a, r)
        zero = den == 0
        assert np.all(num[zero] == 0), f"{what}: group {g}: nonzero R where the reference is zero"
        if np.any(~zero):
            e = np.sqrt(num[~zero] / den[~zero])
            k = int(np.argmax(e))
            assert e[k] <= tol, f"{what}: group {g} block {k}: error {e[k]:.3e} > {tol:.1e}"
            worst = max(worst, float(e[k]))
    return worst


def _assert_mechanics(R, batch, prec, held, what, bound=MECH_BOUND):
    """Every block against the FP64 product of the oracle's encodings of its
    operands (held S: with its per-block scale; S encoded on chip: unscaled;
    the precoder with its own power-of-two scale). Returns the worst block."""
    name = ENC[prec]
    pairs = [(0, 0), (0, 1), (1, 0)] if name in ("bf16x3", "tf32x3") else [(0, 0)]
    wenc, worst = {}, 0.0
    for g, (p, S) in enumerate(zip(batch.prec, batch.S)):
        if S.shape[0] == 0 or S.shape[1] == 0:
            continue
        if p not in wenc:
            sw, wpl = oracle.quantize_planes(batch.W[p].astype(np.complex64), name)
            wenc[p] = (sw, [a + 1j * b for a, b in wpl])
        sw, Wt = wenc[p]
        ss, spl = oracle.quantize_blocks(S, name, scaled=held)
        exp = oracle.apply_terms(Wt, [a + 1j * b for a, b in spl], pairs, sw) * ss[:, None, None]
        num, den = oracle.errnorm_blocks(R[g], exp)
        e = np.sqrt(num / den)
        k = int(np.argmax(e))
        assert e[k] < bound, f"{what}: group {g} block {k}: mechanics error {e[k]:.2e} >= {bound:.0e}"
        worst = max(worst, float(e[k]))
    return worst


def _check_full(R, batch, prec, held, what, ref_c64, ref_unrounded):
    """The full-size checks of one result: the batch error, every block's
    error against the oracle at the form's tolerance and, for the tensor-core
    forms, every block against the FP64 product of its encoded operands."""
    ref = ref_c64 if prec in ACCURATE else ref_unrounded
    e = _assert_close(R, ref, _tol(prec), what)
    wb = _assert_per_block(R, ref, _tol(prec), what)
    wm = _assert_mechanics(R, batch, prec, held, what) if prec in ENC else None
    print(f"{what}: batch {e:.3e}, worst block {wb:.3e}" + ("" if wm is None else f", worst mechanics {wm:.2e}"))


_REFS = {}


def _full_refs(key, make):
    """A full-size workload and its two oracle results (complex64-rounded
    inputs, and the unrounded inputs), computed once per module."""
    if key not in _REFS:
        _REFS.clear()  # one full-size workload held at a time
        batch = make()
        _REFS[key] = (batch, _ref(batch), oracle.apply_batch(batch))
    return _REFS[key]


@pytest.mark.parametrize("name,prec,held", FORMS, ids=[f[0] for f in FORMS])
def test_exact_integers_bitwise(plan, name, prec, held):
    batch = wl.config_exact_integer()
    R = run(plan, batch, prec, torch, held=held)
    ref = oracle.apply_batch(batch)
    for g, (a, r) in enumerate(zip(R, ref)):
        assert np.array_equal(a.astype(np.complex128), r), \
            f"{name}: group {g} (f={batch.f_of_group[g]}, nb={batch.n_blocks[g]}) differs"


@pytest.mark.parametrize("name,prec,held", FORMS, ids=[f[0] for f in FORMS])
def test_small_config(plan, name, prec, held):
    """One 64x8 precoder, 16-QAM blocks (the small FP32 workload, 300 blocks)."""
    batch = wl.config_small(seed=0, n_blocks=300)
    R = run(plan, batch, prec, torch, held=held)
    ref = _ref(batch) if prec in ACCURATE else oracle.apply_batch(batch)
    _assert_close(R, ref, _tol(prec), name)


@pytest.mark.parametrize("name,prec,held", FORMS, ids=[f[0] for f in FORMS])
def test_fullband_scaled(plan, name, prec, held):
    """f = 36, 13 resource blocks x 14 symbols (odd tile counts per CTA run)."""
    batch = wl.config_fullband(seed=2, n_rb=13, n_sym=14)
    R = run(plan, batch, prec, torch, held=held)
    ref = _ref(batch) if prec in ACCURATE else oracle.apply_batch(batch)
    e = _assert_close(R, ref, _tol(prec), name)
    if prec in ACCURATE:
        for g, (a, r) in enumerate(zip(R, ref)):
            num, den = oracle.errnorm_blocks(a, r)
            assert np.all(np.sqrt(num / den) <= _tol(prec)), f"{name}: group {g} per-block error"
    print(f"{name}: rel err {e:.3e}")


@pytest.mark.parametrize("name,prec,held", [FORMS[0], FORMS[1], FORMS[2], FORMS[4], FORMS[7], FORMS[8]],
                         ids=["fp32", "bf16x3", "bf16x3_held", "bf16_held", "fp32_3m", "tf32x3"])
def test_uneven_scaled(plan, name, prec, held):
    """Uneven f (0..36) per group, geometric group sizes, mixed QAM orders."""
    batch = wl.config_uneven(seed=3, n_blocks=700)
    R = run(plan, batch, prec, torch, held=held)
    ref = _ref(batch) if prec in ACCURATE else oracle.apply_batch(batch)
    for a, f in zip(R, batch.f_of_group):
        if f == 0:
            assert np.all(a == 0)
    _assert_close(R, ref, _tol(prec), name)


@pytest.mark.parametrize("prec,name", [(bf.BF_BF16, "bf16"), (bf.BF_FP16, "fp16"), (bf.BF_BF16X3, "bf16x3")])
def test_quantize_bit_exact(plan, prec, name):
    """Held S is the oracle's encoding, bit for bit (scale, rounding, layout, zero padding)."""
    batch = wl.config_reduced(seed=4, copies=1, n_rb=3, n_sym=3, f=17)
    _, bufs = run(plan, batch, prec, torch, held=True, return_buffers=True)
    lay = layout(batch, 0, prec)
    raw = bufs["S"].cpu().numpy().view(np.uint16)
    scales = bufs["scale"].cpu().numpy()
    f = 17
    kp = ((2 * f + 15) // 16) * 16
    term = 64 * kp
    blk = 0
    for g, S in enumerate(batch.S):
        for n in range(S.shape[0]):
            s, planes = oracle.quantize_planes(S[n].astype(np.complex64), name)
            assert scales[blk] == np.float32(s)
            base = (lay.held_off[g] + n * bf.bf_held_block_bytes(f, prec)) // 2
            for t, (re, im) in enumerate(planes):
                img = np.zeros((64, kp), np.float32)
                img[:60, 0:2 * f:2] = re.T
                img[:60, 1:2 * f:2] = im.T
                bits = (oracle.bf16_bits(img) if name != "fp16"
                        else img.astype(np.float16).view(np.uint16))
                rows, cols = np.meshgrid(np.arange(64), np.arange(kp), indexing="ij")
                off = (rows // 8) * (8 * kp) + (cols // 8) * 64 + (rows % 8) * 8 + (cols % 8)
                got = raw[base + t * term + off]
                assert np.array_equal(got, bits), f"block {blk} term {t} differs"
            blk += 1


@pytest.mark.parametrize("prec,name", [(bf.BF_BF16, "bf16"), (bf.BF_FP16, "fp16"), (bf.BF_BF16X3, "bf16x3")])
def test_reduced_mechanics(plan, prec, name):
    """Held forms against the FP64 product of the encoded operands: only FP32
    accumulation rounding separates them."""
    batch = wl.config_reduced(seed=4, copies=1, n_rb=9, n_sym=5)
    R = run(plan, batch, prec, torch, held=True)
    for g, (p, S) in enumerate(zip(batch.prec, batch.S)):
        W = batch.W[p].astype(np.complex64)
        sw, wpl = oracle.quantize_planes(W, name)
        Wt = [a + 1j * b for a, b in wpl]
        pairs = [(0, 0)] if name != "bf16x3" else [(0, 0), (0, 1), (1, 0)]
        exp = np.empty((S.shape[0], 64, 60), np.complex128)
        for n in range(S.shape[0]):
            ss, spl = oracle.quantize_planes(S[n].astype(np.complex64), name)
            St = [(a + 1j * b)[None] for a, b in spl]
            exp[n] = oracle.apply_terms(Wt, St, pairs, sw * ss)[0]
        e = oracle.rel_frobenius([R[g]], [exp])
        assert e < 2e-6, f"{name}: group {g} mechanics error {e:.2e}"


@pytest.mark.parametrize("prec,name", [(bf.BF_BF16X3, "bf16x3"), (bf.BF_TF32X3, "tf32x3"), (bf.BF_BF16, "bf16"),
                                       (bf.BF_FP16, "fp16")])
def test_onchip_mechanics(plan, prec, name):
    """Complex64 S encoded on chip (no per-block scale; the precoder keeps its
    power-of-two scale) against the FP64 product of the oracle's encodings of
    the same operands: only FP32 accumulation rounding separates them, so a
    wrong rounding, split or dropped term shows up far above the bound."""
    batch = wl.config_reduced(seed=4, copies=1, n_rb=9, n_sym=5)
    R = run(plan, batch, prec, torch)
    split = name in ("bf16x3", "tf32x3")
    for g, (p, S) in enumerate(zip(batch.prec, batch.S)):
        W = batch.W[p].astype(np.complex64)
        sw, wpl = oracle.quantize_planes(W, name)
        Wt = [a + 1j * b for a, b in wpl]
        pairs = [(0, 0), (0, 1), (1, 0)] if split else [(0, 0)]
        exp = np.empty((S.shape[0], 64, 60), np.complex128)
        for n in range(S.shape[0]):
            _, spl = oracle.quantize_planes(S[n].astype(np.complex64), name, scaled=False)
            St = [(a + 1j * b)[None] for a, b in spl]
            exp[n] = oracle.apply_terms(Wt, St, pairs, sw)[0]
        e = oracle.rel_frobenius([R[g]], [exp])
        assert e < 2e-6, f"{name}: group {g} mechanics error {e:.2e}"


def test_reduced_accuracy(plan):
    """The reduced-precision workload (256-QAM + noise, f = 36), scaled down."""
    batch = wl.config_reduced(seed=4, copies=1, n_rb=20, n_sym=14)
    ref64 = oracle.apply_batch(batch)
    ref32 = _ref(batch)
    errs = {}
    for name, prec, held in FORMS[1:]:
        R = run(plan, batch, prec, torch, held=held)
        errs[name] = _assert_close(R, ref32 if prec in ACCURATE else ref64, _tol(prec), name)
    print("reduced-precision errors:", {k: f"{v:.2e}" for k, v in errs.items()})


def test_graph_and_host_paths_bitwise(plan):
    """The graph-captured batch and the host-buffer pipeline give the same bits."""
    batch = wl.config_uneven(seed=9, n_blocks=400)
    for prec in ACCURATE:
        a = run(plan, batch, prec, torch, mode="apply")
        others = [run(plan, batch, prec, torch, mode=m, set_w=False) for m in ("batch", "graph", "host", "apply")]
        for o in others:
            for x, y in zip(a, o):
                assert np.array_equal(x.view(np.uint64), y.view(np.uint64))


def test_host_path_scattered_buffers(plan):
    """bf_apply_batch_host over several chunks with the groups stored in reverse
    order and 16-byte gaps in both host buffers: every group equals the
    device path bit for bit and the gaps keep their fill."""
    batch = wl.config_uneven(seed=21, n_blocks=6000)
    ref = run(plan, batch, bf.BF_BF16X3, torch)
    G, nb, fs = batch.n_groups, batch.n_blocks, batch.f_of_group
    s_offs, r_offs, so, ro = [0] * G, [0] * G, 16, 32
    for g in reversed(range(G)):
        s_offs[g], r_offs[g] = so, ro
        so += nb[g] * fs[g] * 480 + 16
        ro += nb[g] * 30720 + 16
    S_h = torch.zeros(so // 4, dtype=torch.float32).pin_memory()
    R_h = torch.full((ro // 4,), float("nan"), dtype=torch.float32).pin_memory()
    s_np = S_h.numpy().view(np.uint8)
    for g in range(G):
        blk = np.ascontiguousarray(batch.S[g].astype(np.complex64)).view(np.uint8).ravel()
        s_np[s_offs[g]:s_offs[g] + blk.size] = blk
    groups = [(batch.prec[g], nb[g], s_offs[g], r_offs[g]) for g in range(G)]
    bf.bf_apply_batch_host(plan, S_h, groups, bf.BF_BF16X3, R_h)
    torch.cuda.synchronize()
    r_np = R_h.numpy().view(np.uint8)
    written = np.zeros(r_np.size, bool)
    for g in range(G):
        n = nb[g] * 30720
        got = r_np[r_offs[g]:r_offs[g] + n].view(np.uint64)
        assert np.array_equal(got, ref[g].view(np.uint64).ravel()), f"group {g}"
        written[r_offs[g]:r_offs[g] + n] = True
    assert np.all(np.isnan(R_h.numpy()[~written.reshape(-1, 4).all(axis=1)]))


@pytest.mark.parametrize("name,prec,held", FORMS, ids=[f[0] for f in FORMS])
def test_fullband_full_size(plan, name, prec, held):
    """The full-band f = 36 workload at full size (273 x 14 = 3,822 blocks) in
    the launch configuration the bench times, checked in full against the
    oracle, block by block."""
    batch, ref, ref64 = _full_refs("fullband", wl.config_fullband)
    R = run(plan, batch, prec, torch, held=held, mode="batch")
    _check_full(R, batch, prec, held, f"fullband {name}", ref, ref64)


def test_errnorm_matches_numpy(plan):
    rng = np.random.default_rng(5)
    n = 37
    Rref = rng.normal(size=(n, 64, 60)) + 1j * rng.normal(size=(n, 64, 60))
    R = (Rref + 1e-3 * (rng.normal(size=Rref.shape) + 1j * rng.normal(size=Rref.shape))).astype(np.complex64)
    Rd = torch.from_numpy(np.ascontiguousarray(R).view(np.float32)).cuda()
    Rrefd = torch.from_numpy(np.ascontiguousarray(Rref).view(np.float64)).cuda()
    per = torch.zeros(2 * n, dtype=torch.float64, device="cuda")
    num, den = bf.bf_errnorm(plan, Rd, Rrefd, n, per)
    enum, eden = oracle.errnorm_blocks(R, Rref)
    assert np.isclose(num, enum.sum(), rtol=1e-12) and np.isclose(den, eden.sum(), rtol=1e-12)
    p = per.cpu().numpy().reshape(n, 2)
    assert np.allclose(p[:, 0], enum, rtol=1e-12) and np.allclose(p[:, 1], eden, rtol=1e-12)
    assert bf.bf_errnorm(plan, Rd, Rrefd, 0) == (0.0, 0.0)


def test_edge_cases_and_errors(plan):
    batch = wl.config_small(seed=1, n_blocks=3, f=5)
    set_precoders(plan, batch, torch, slot_base=100)
    R_t = torch.zeros(3 * 64 * 60 * 2, device="cuda")
    S_t = torch.zeros(3 * 5 * 60 * 2, device="cuda")
    # empty batch and empty group
    bf.bf_apply_batch(plan, S_t, None, [], bf.BF_FP32, R_t)
    bf.bf_apply_batch(plan, S_t, None, [(100, 0, 0, 0)], bf.BF_FP32, R_t)
    with pytest.raises(bf.BfError) as ei:
        bf.bf_apply_batch(plan, S_t, None, [(4000, 1, 0, 0)], bf.BF_FP32, R_t)  # unset slot
    assert ei.value.status == bf.BF_ENOTFOUND
    with pytest.raises(bf.BfError) as ei:
        bf.bf_apply_batch(plan, S_t, None, [(100, 1, 8, 0)], bf.BF_FP32, R_t)  # misaligned offset
    assert ei.value.status == bf.BF_EINVAL
    with pytest.raises(bf.BfError) as ei:
        bf.bf_apply_batch(plan, S_t.data_ptr() + 4, None, [(100, 1, 0, 0)], bf.BF_FP32, R_t)
    assert ei.value.status == bf.BF_EINVAL
    for prec in (bf.BF_FP32, bf.BF_FP32_3M, bf.BF_TF32X3):
        with pytest.raises(bf.BfError) as ei:
            bf.bf_apply_batch(plan, S_t, R_t, [(100, 1, 0, 0)], prec, R_t)  # no held S for these forms
        assert ei.value.status == bf.BF_EINVAL
    with pytest.raises(bf.BfError) as ei:
        bf.bf_apply_batch(plan, S_t, None, [(100, 1, 0, 0)], 6, R_t)  # unknown precision
    assert ei.value.status == bf.BF_EINVAL
    with pytest.raises(bf.BfError) as ei:
        bf.bf_set_precoders(plan, S_t, [37], 0)  # f > f_max
    assert ei.value.status == bf.BF_EINVAL
    assert bf.bf_device_status(plan) == bf.BF_OK


def test_deterministic(plan):
    batch = wl.config_fullband(seed=6, n_rb=7, n_sym=14)
    for prec in (bf.BF_FP32, bf.BF_BF16X3, bf.BF_BF16, bf.BF_TF32X3):
        a = run(plan, batch, prec, torch)
        b = run(plan, batch, prec, torch, set_w=False)
        assert all(np.array_equal(x.view(np.uint64), y.view(np.uint64)) for x, y in zip(a, b))


def test_autotune_keeps_results_and_round_trips(plan, tmp_path):
    """Tuning changes tile sizes and the CTA split, never a result bit; the
    table survives a save/load round trip."""
    batch = wl.config_uneven(seed=12, n_blocks=900)
    before = {p: run(plan, batch, p, torch) for p in (bf.BF_FP32, bf.BF_BF16X3)}
    for p in (bf.BF_FP32, bf.BF_BF16X3):
        bf.bf_autotune(plan, p)
        q = [bf.bf_tune_query(plan, p, f) for f in (0, 8, 16, 24, 36)]
        assert all(e["tuned"] and e["ns_per_block"] > 0 and e["tile_blocks"] in (1, 2) for e in q), q
        after = run(plan, batch, p, torch)
        for x, y in zip(before[p], after):
            assert np.array_equal(x.view(np.uint64), y.view(np.uint64))
    path = str(tmp_path / "tune.json")
    bf.bf_tune_save(plan, path)
    saved = [bf.bf_tune_query(plan, bf.BF_BF16X3, f) for f in (0, 8, 16, 24, 36)]
    other = bf.bf_plan_create(64, 36, 60)
    try:
        assert not bf.bf_tune_query(other, bf.BF_BF16X3, 36)["tuned"]
        bf.bf_tune_load(other, path)
        got = [bf.bf_tune_query(other, bf.BF_BF16X3, f) for f in (0, 8, 16, 24, 36)]
        assert all(abs(a["ns_per_block"] - b["ns_per_block"]) < 1e-5 and a["tile_blocks"] == b["tile_blocks"]
                   for a, b in zip(saved, got))
        # the same table measured on another target is refused, and the plan keeps its table
        txt = open(path).read()
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        assert f'"sm_count": {sms}' in txt
        with open(path, "w") as fh:
            fh.write(txt.replace(f'"sm_count": {sms}', f'"sm_count": {sms - 4}'))
        with pytest.raises(bf.BfError) as ei:
            bf.bf_tune_load(other, path)
        assert ei.value.status == bf.BF_EINVAL and "not on this target" in str(ei.value)
        assert bf.bf_tune_query(other, bf.BF_BF16X3, 36)["ns_per_block"] == got[-1]["ns_per_block"]
        with open(path, "w") as fh:
            fh.write("{}")
        with pytest.raises(bf.BfError):
            bf.bf_tune_load(other, path)
    finally:
        bf.bf_plan_destroy(other)


@pytest.mark.parametrize("name,prec,held", FORMS, ids=[f[0] for f in FORMS])
def test_uneven_full_size(plan, name, prec, held):
    """The uneven workload at full size (16,384 blocks) in one persistent launch,
    checked in full against the oracle, block by block (f = 0 blocks exactly 0)."""
    batch, ref, ref64 = _full_refs("uneven", wl.config_uneven)
    R = run(plan, batch, prec, torch, held=held, mode="batch")
    _check_full(R, batch, prec, held, f"uneven full size {name}", ref, ref64)


@pytest.mark.parametrize("name,prec", [("bf16x3", bf.BF_BF16X3), ("bf16", bf.BF_BF16), ("fp16", bf.BF_FP16),
                                       ("tf32x3", bf.BF_TF32X3)])
def test_uneven_full_size_repeatable(plan, name, prec):
    """Pipeline races show up as a few wrong blocks that change from run to run:
    the full-size uneven batch (1- and 2-block tiles, f from 0 to 36, many
    precoder switches per CTA) must give the same bits five times over, and the
    first run is checked block by block."""
    batch, ref, ref64 = _full_refs("uneven", wl.config_uneven)
    first = run(plan, batch, prec, torch, mode="batch")
    _assert_per_block(first, ref if prec in ACCURATE else ref64, _tol(prec), name)
    for rep in range(4):
        again = run(plan, batch, prec, torch, mode="batch" if rep % 2 else "apply", set_w=False)
        for g, (x, y) in enumerate(zip(first, again)):
            assert np.array_equal(x.view(np.uint64), y.view(np.uint64)), f"{name}: group {g} differs on repeat {rep}"


@pytest.mark.parametrize("name,prec,held", FORMS, ids=[f[0] for f in FORMS])
def test_reduced_full_size(plan, name, prec, held):
    """The reduced-precision workload at full size (30,576 blocks, 2,184
    precoders), block by block."""
    batch, ref, ref64 = _full_refs("reduced", wl.config_reduced)
    R = run(plan, batch, prec, torch, held=held, mode="batch")
    _check_full(R, batch, prec, held, f"reduced full size {name}", ref, ref64)


def test_bounded_wait_gives_up_and_the_context_stays_usable(plan):
    """Failure detection without a fault: a wait that nothing completes gives
    up at its limit (2 s) and sets the device status; a second role leaves
    through the abort flag before its own limit; the plan then still computes
    correct results."""
    assert bf.bf_device_status(plan) == bf.BF_OK
    r = bf.bf_selftest_wait_timeout(plan)
    assert r["gave_up"] == 1 and 1900 <= r["wait_ms"] <= 4000, r
    assert r["left_on_abort"] == 1 and r["abort_wait_ms"] < 1900, r
    assert bf.bf_device_status(plan) == bf.BF_ETIMEOUT
    assert bf.bf_device_status(plan) == bf.BF_OK  # read and cleared
    batch = wl.config_fullband(seed=6, n_rb=3, n_sym=14)
    _assert_close(run(plan, batch, bf.BF_BF16X3, torch), _ref(batch), TOL_SPLIT, "after the self-test")


def test_reserve_precoders(plan):
    """A reserved precoder store takes slots up to the reservation without
    growing; a reservation below the current size changes nothing."""
    bf.bf_reserve_precoders(plan, 6000)
    bf.bf_reserve_precoders(plan, 10)
    batch = wl.config_small(seed=1, n_blocks=5, f=5)
    _assert_close(run(plan, batch, bf.BF_FP32, torch, slot_base=5999), _ref(batch), TOL_FP32, "slot 5999")
    for bad in (-1, (1 << 24) + 1):
        with pytest.raises(bf.BfError) as ei:
            bf.bf_reserve_precoders(plan, bad)
        assert ei.value.status == bf.BF_EINVAL
    bf.bf_reserve_worklists(plan, 70_000)
    _assert_close(run(plan, batch, bf.BF_BF16X3, torch, slot_base=5999, set_w=False), _ref(batch), TOL_SPLIT,
                  "after the work-list reservation")
    with pytest.raises(bf.BfError) as ei:
        bf.bf_reserve_worklists(plan, -1)
    assert ei.value.status == bf.BF_EINVAL


def test_host_path_pipelines_across_streams(plan):
    """Back-to-back host-buffer calls on two streams with two buffer pairs,
    never synchronised in between (the second call's copy-in overlaps the
    first's copy-out): every call's R equals the device path bit for bit."""
    batch = wl.config_uneven(seed=23, n_blocks=3000)
    ref = run(plan, batch, bf.BF_BF16X3, torch)
    lay = layout(batch)
    Sflat, _ = batch.pack_S()
    S_h = [torch.from_numpy(np.ascontiguousarray(Sflat.astype(np.complex64)).view(np.float32).copy()).pin_memory()
           for _ in range(2)]
    R_h = [torch.full((lay.r_blocks * 64 * 60 * 2,), float("nan"), dtype=torch.float32).pin_memory()
           for _ in range(2)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for rep in range(6):
        k = rep % 2
        if rep >= 2:  # the buffer pair's previous result, checked before it is reused
            streams[k].synchronize()
            got = R_h[k].numpy().view(np.complex64).reshape(-1, 64, 60)
            assert np.array_equal(got.view(np.uint64), np.concatenate(ref).view(np.uint64)), f"call {rep - 2}"
            R_h[k].fill_(float("nan"))
        bf.bf_apply_batch_host(plan, S_h[k], lay.groups, bf.BF_BF16X3, R_h[k], streams[k])
    for k in range(2):
        streams[k].synchronize()
        got = R_h[k].numpy().view(np.complex64).reshape(-1, 64, 60)
        assert np.array_equal(got.view(np.uint64), np.concatenate(ref).view(np.uint64))
    # other chunk sizes move the same bits
    try:
        for first, mx in ((64 << 10, 1 << 20), (8 << 20, 64 << 20)):
            bf.bf_set_host_chunks(plan, first, mx)
            R_h[0].fill_(float("nan"))
            bf.bf_apply_batch_host(plan, S_h[0], lay.groups, bf.BF_BF16X3, R_h[0], streams[0])
            streams[0].synchronize()
            got = R_h[0].numpy().view(np.complex64).reshape(-1, 64, 60)
            assert np.array_equal(got.view(np.uint64), np.concatenate(ref).view(np.uint64)), (first, mx)
        for first, mx in ((1 << 10, 1 << 20), (8 << 20, 4 << 20)):
            with pytest.raises(bf.BfError) as ei:
                bf.bf_set_host_chunks(plan, first, mx)
            assert ei.value.status == bf.BF_EINVAL
    finally:
        bf.bf_set_host_chunks(plan, 4 << 20, 32 << 20)


@pytest.mark.parametrize("prec", [bf.BF_BF16X3, bf.BF_TF32X3, bf.BF_FP32], ids=["bf16x3", "tf32x3", "fp32"])
def test_independent_input_keeps_the_r_side_ordered(plan, prec):
    """A batch declared S-independent loads and multiplies S while the
    previous launch runs, but its R stores still follow that launch: batch B
    writes its R over the S that batch A (launched just before, also
    S-independent: its S comes from a copy) is still reading. Over repeated
    back-to-back pairs A's R and B's R both equal their results computed alone,
    bit for bit, and the setter rejects values other than 0 and 1. (A's S is
    written by B two launches earlier, but the copy in between orders it.)"""
    a = wl.config_fullband(seed=31, n_rb=40, n_sym=14)  # 560 blocks
    b = wl.config_fullband(seed=32, n_rb=30, n_sym=14)  # 420 blocks
    ref_a = run(plan, a, prec, torch)
    ref_b = run(plan, b, prec, torch, slot_base=300)
    set_precoders(plan, a, torch)
    la, lb = layout(a), layout(b, 300)
    Sa = to_device_c64(a.pack_S()[0], torch)
    Sb = to_device_c64(b.pack_S()[0], torch)
    big = torch.zeros(lb.r_blocks * 64 * 60 * 2 + Sa.numel(), dtype=torch.float32, device="cuda")
    Ra = torch.empty(la.r_blocks * 64 * 60 * 2, dtype=torch.float32, device="cuda")
    ha = bf.bf_batch_create(plan, big, None, la.groups, prec, Ra)  # A reads S from the front of `big`
    hb = bf.bf_batch_create(plan, Sb, None, lb.groups, prec, big)  # B writes R over it
    for h in (ha, hb):
        bf.bf_batch_set_s_independent(h, True)
    st = torch.cuda.current_stream()
    try:
        for rep in range(20):
            big[:Sa.numel()].copy_(Sa)  # a copy, not a product launch, writes A's S
            Ra.fill_(float("nan"))
            bf.bf_batch_launch(ha, st)
            bf.bf_batch_launch(hb, st)
            torch.cuda.synchronize()
            got_a = Ra.cpu().numpy().view(np.complex64).reshape(-1, 64, 60)
            got_b = big[:lb.r_blocks * 64 * 60 * 2].cpu().numpy().view(np.complex64).reshape(-1, 64, 60)
            assert np.array_equal(got_a.view(np.uint64), np.concatenate(ref_a).view(np.uint64)), f"A, pair {rep}"
            assert np.array_equal(got_b.view(np.uint64), np.concatenate(ref_b).view(np.uint64)), f"B, pair {rep}"
        assert bf.lib().bf_batch_set_s_independent(ha, 2) == bf.BF_EINVAL
    finally:
        bf.bf_batch_destroy(ha)
        bf.bf_batch_destroy(hb)
