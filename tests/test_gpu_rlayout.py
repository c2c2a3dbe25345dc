"""GPU parity of the strided, reduced-type R output (bf_apply_batch_rl and
bf_batch_create_rl) against the FP64 oracle.

The output is written antenna-major (antenna i's resource elements of every
block in one row, the per-antenna input of the OFDM stage that follows the
product), as complex64 or as bf16 / fp16 pairs rounded to nearest even.

Exact-integer inputs with W in {-32..32} + i{-32..32} and 256-QAM
odd-integer symbols keep every product and partial sum exact in the FP32
accumulator (|R| < 2^24) while most outputs need rounding to bf16 and some to
fp16 (ties included), so the rounded R must equal the oracle's
round-to-nearest-even of the exact result. The comparison is on values
(the sign of an exact zero is not specified by the product). Padding bytes
between rows and blocks must keep their fill.

On real-valued data the bound is the product form's tolerance plus the
output rounding: |x - round(x)| <= u|x| with u = 2^-8 (bf16) or 2^-11 (fp16)
gives a relative Frobenius error of at most u from the rounding alone.
"""
import numpy as np
import pytest

import oracle
import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1810_11451_gb300 as bf  # noqa: E402
from bfrun import decode_r, rl_view, rl_written_mask, run, run_rl  # noqa: E402

FORMS = [("fp32", bf.BF_FP32, False), ("bf16x3", bf.BF_BF16X3, False), ("bf16x3_held", bf.BF_BF16X3, True),
         ("bf16", bf.BF_BF16, False), ("bf16_held", bf.BF_BF16, True), ("fp16", bf.BF_FP16, False),
         ("fp16_held", bf.BF_FP16, True), ("fp32_3m", bf.BF_FP32_3M, False), ("tf32x3", bf.BF_TF32X3, False)]
RTYPES = [("c64", bf.BF_R_C64), ("bf16", bf.BF_R_BF16), ("fp16", bf.BF_R_FP16)]
U_OUT = {bf.BF_R_C64: 0.0, bf.BF_R_BF16: 2.0 ** -8, bf.BF_R_FP16: 2.0 ** -11}
TOL = {bf.BF_FP32: 1e-5, bf.BF_FP32_3M: 1e-5, bf.BF_BF16X3: 1e-5, bf.BF_TF32X3: 1e-5, bf.BF_BF16: 2e-2,
       bf.BF_FP16: 2e-2}


@pytest.fixture(scope="module")
def plan():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    p = bf.bf_plan_create(64, 36, 60)
    yield p
    assert bf.bf_device_status(p) == bf.BF_OK
    bf.bf_plan_destroy(p)


def _round_ref(ref: np.ndarray, rtype: int) -> np.ndarray:
    """The oracle's FP64 result rounded to the output type (exact in FP32 here)."""
    if rtype == bf.BF_R_C64:
        return ref.astype(np.complex64).astype(np.complex128)
    rnd = oracle.bf16_round if rtype == bf.BF_R_BF16 else oracle.fp16_round
    re = rnd(ref.real.astype(np.float32)).astype(np.float64)
    im = rnd(ref.imag.astype(np.float32)).astype(np.float64)
    return re + 1j * im


def _groups(buf, rl, offs, batch):
    return [decode_r(rl_view(buf, rl, o, nb), rl.rtype) for o, nb in zip(offs, batch.n_blocks)]


@pytest.mark.parametrize("rname,rtype", RTYPES, ids=[r[0] for r in RTYPES])
@pytest.mark.parametrize("name,prec,held", FORMS, ids=[f[0] for f in FORMS])
def test_rl_exact_integers_rounded_bitwise(plan, name, prec, held, rname, rtype):
    batch = wl.config_exact_integer(wlim=32, qam=256)
    buf, rl, offs = run_rl(plan, batch, prec, torch, rtype, held=held, pad_block=16, pad_row=32)
    ref = oracle.apply_batch(batch)
    got = _groups(buf, rl, offs, batch)
    for g, (a, r) in enumerate(zip(got, ref)):
        assert np.all(np.isfinite(a)), f"{name}/{rname}: group {g} has unwritten (NaN) elements"
        assert np.array_equal(a, _round_ref(r, rtype)), \
            f"{name}/{rname}: group {g} (f={batch.f_of_group[g]}, nb={batch.n_blocks[g]}) differs"
    mask = rl_written_mask(len(buf), rl, offs, batch.n_blocks)
    assert np.all(buf[~mask[:len(buf)]] == 255), f"{name}/{rname}: bytes outside the layout were written"


@pytest.mark.parametrize("rname,rtype", RTYPES, ids=[r[0] for r in RTYPES])
@pytest.mark.parametrize("name,prec,held", [FORMS[0], FORMS[1], FORMS[4], FORMS[8]],
                         ids=["fp32", "bf16x3", "bf16_held", "tf32x3"])
def test_rl_fullband_scaled_within_tolerance(plan, name, prec, held, rname, rtype):
    """The full-band mix (64x36 precoders, 14 blocks each, 64-QAM) on 40 resource blocks."""
    batch = wl.config_fullband(n_rb=40)
    buf, rl, offs = run_rl(plan, batch, prec, torch, rtype, held=held)
    ref = oracle.apply_batch(batch.rounded(np.complex64))
    got = _groups(buf, rl, offs, batch)
    assert all(np.all(np.isfinite(a)) for a in got)
    e = oracle.rel_frobenius(got, ref)
    bound = TOL[prec] + U_OUT[rtype]
    assert e <= bound, f"{name}/{rname}: relative Frobenius error {e:.3e} > {bound:.2e}"


def test_rl_store_is_a_rounding_of_the_same_accumulator(plan):
    """bf16 / fp16 R are the round-to-nearest-even of the complex64 R of the
    same product on real-valued data (one accumulator, three stores)."""
    batch = wl.config_fullband(n_rb=24)
    c64, rl0, offs = run_rl(plan, batch, bf.BF_BF16X3, torch, bf.BF_R_C64)
    base = [rl_view(c64, rl0, o, nb) for o, nb in zip(offs, batch.n_blocks)]
    for rtype, rnd in ((bf.BF_R_BF16, oracle.bf16_bits), (bf.BF_R_FP16, oracle.fp16_bits)):
        buf, rl, offs2 = run_rl(plan, batch, bf.BF_BF16X3, torch, rtype, set_w=False)
        for b, o, nb in zip(base, offs2, batch.n_blocks):
            v = rl_view(buf, rl, o, nb)
            assert np.array_equal(v[..., 0], rnd(np.ascontiguousarray(b.real)))
            assert np.array_equal(v[..., 1], rnd(np.ascontiguousarray(b.imag)))


def test_rl_default_layout_matches_plain_call(plan):
    """layout = NULL and the explicit packed layout {480, 30720, c64} give the
    same bits as bf_apply_batch."""
    batch = wl.config_uneven(seed=13, n_blocks=2000)
    plain = run(plan, batch, bf.BF_BF16X3, torch)
    out, bufs = run(plan, batch, bf.BF_BF16X3, torch, return_buffers=True, set_w=False)
    for layout in (None, bf.bf_rlayout(480, 30720, bf.BF_R_C64, 0)):
        bufs["R"].fill_(float("nan"))
        bf.bf_apply_batch_rl(plan, bufs["S"], None, bufs["groups"], bf.BF_BF16X3, bufs["R"], layout)
        torch.cuda.synchronize()
        r = bufs["R"].cpu().numpy().view(np.complex64).reshape(-1, 64, 60)
        assert np.array_equal(r.view(np.uint64), np.concatenate(plain).view(np.uint64))


@pytest.mark.parametrize("mode", ["batch", "graph"])
def test_rl_prepared_batch_bitwise(plan, mode):
    batch = wl.config_fullband(n_rb=30)
    a, rl, offs = run_rl(plan, batch, bf.BF_BF16, torch, bf.BF_R_BF16, held=True)
    b, _, _ = run_rl(plan, batch, bf.BF_BF16, torch, bf.BF_R_BF16, held=True, mode=mode, set_w=False)
    assert np.array_equal(a, b)


def test_rl_fullband_full_size_antenna_major_bf16(plan):
    """The full-band batch (3,822 blocks) through the served form: held bf16 S,
    split or single product, bf16 R antenna-major; every block against the oracle."""
    batch = wl.config_fullband()
    ref = oracle.apply_batch(batch.rounded(np.complex64))
    for prec, held in ((bf.BF_BF16X3, False), (bf.BF_BF16, True)):
        buf, rl, offs = run_rl(plan, batch, prec, torch, bf.BF_R_BF16, held=held, set_w=prec == bf.BF_BF16X3)
        got = _groups(buf, rl, offs, batch)
        assert all(np.all(np.isfinite(a)) for a in got)
        e = oracle.rel_frobenius(got, ref)
        assert e <= TOL[prec] + U_OUT[bf.BF_R_BF16], f"prec {prec}: {e:.3e}"
        assert rl.row_stride == batch.total_blocks * 60 * 4 and rl.block_stride == 240


def test_rl_rejects_bad_layouts(plan):
    batch = wl.config_small(n_blocks=4)
    _, bufs = run(plan, batch, bf.BF_FP32, torch, return_buffers=True)
    bad = [bf.bf_rlayout(480, 30720, 3, 0),          # unknown type
           bf.bf_rlayout(480, 30720, bf.BF_R_C64, 1),  # reserved set
           bf.bf_rlayout(472, 30720, bf.BF_R_C64, 0),  # row shorter than 60 elements
           bf.bf_rlayout(240, 30720, bf.BF_R_C64, 0),
           bf.bf_rlayout(488, 30720, bf.BF_R_C64, 0),  # not a multiple of 16
           bf.bf_rlayout(480, 30728, bf.BF_R_C64, 0),
           bf.bf_rlayout(240, 200, bf.BF_R_BF16, 0),   # block stride below 60 elements
           bf.bf_rlayout(-480, 30720, bf.BF_R_C64, 0)]
    for rl in bad:
        with pytest.raises(bf.BfError) as ei:
            bf.bf_apply_batch_rl(plan, bufs["S"], None, bufs["groups"], bf.BF_FP32, bufs["R"], rl)
        assert ei.value.status == bf.BF_EINVAL
        with pytest.raises(bf.BfError) as ei:
            bf.bf_batch_create_rl(plan, bufs["S"], None, bufs["groups"], bf.BF_FP32, bufs["R"], rl)
        assert ei.value.status == bf.BF_EINVAL
    assert bf.bf_device_status(plan) == bf.BF_OK
