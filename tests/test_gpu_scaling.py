"""Per-block power-of-two scaling of held S (the fp16 / bf16 single-pass
forms), measured as a study over signal levels.

The held encoding divides each block by 2^ceil(log2 max|Re|,|Im|) before
rounding and multiplies the FP32 accumulator back in the epilogue. Both steps
are exact powers of two, so scaling S by 2^e changes the encoding not at all
and R by exactly 2^e: the held forms give R(2^e S) = 2^e R(S) bit for bit over
the whole range where the FP32 results stay normal. Without a per-block scale
(complex64 S rounded to fp16 on chip), small signals lose precision in fp16's
subnormal range and large ones overflow it.
"""
import numpy as np
import pytest

import oracle
import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1810_11451_gb300 as bf  # noqa: E402
from bfrun import run  # noqa: E402

LEVELS = (-24, -12, 12, 24)


@pytest.fixture(scope="module")
def plan():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    p = bf.bf_plan_create(64, 36, 60)
    yield p
    assert bf.bf_device_status(p) == bf.BF_OK
    bf.bf_plan_destroy(p)


def scaled(batch, e):
    """The same batch with every S value times 2^e (exact in complex64 here)."""
    return wl.Batch(batch.W, batch.prec, [s * 2.0 ** e for s in batch.S], f"{batch.name}_x2^{e}", batch.seed)


@pytest.mark.parametrize("prec,name", [(bf.BF_FP16, "fp16"), (bf.BF_BF16, "bf16")])
def test_held_forms_are_scale_invariant_bitwise(plan, prec, name):
    base = wl.config_reduced(seed=4, copies=1, n_rb=6, n_sym=14)
    R0 = run(plan, base, prec, torch, held=True)
    for e in LEVELS:
        Re = run(plan, scaled(base, e), prec, torch, held=True, set_w=False)
        for g, (a, b) in enumerate(zip(Re, R0)):
            want = (b * np.float32(2.0 ** e)).astype(np.complex64)
            assert np.array_equal(a.view(np.uint64), want.view(np.uint64)), f"{name} 2^{e}: group {g}"


def test_unscaled_fp16_degrades_outside_its_range(plan):
    """fp16 without a per-block scale: accurate near unit level, far worse at
    2^-24 (subnormal fp16), not finite at 2^24 (above 65504); the held form
    keeps its error at every level."""
    base = wl.config_reduced(seed=4, copies=1, n_rb=6, n_sym=14)
    ref = oracle.apply_batch(base)
    held = oracle.rel_frobenius(run(plan, base, bf.BF_FP16, torch, held=True), ref)
    onchip = oracle.rel_frobenius(run(plan, base, bf.BF_FP16, torch, set_w=False), ref)
    assert held <= 2e-2 and onchip <= 2e-2
    low = run(plan, scaled(base, -24), bf.BF_FP16, torch, set_w=False)
    e_low = oracle.rel_frobenius([r * 2.0 ** 24 for r in low], ref)
    assert e_low > 10 * held, (e_low, held)
    high = run(plan, scaled(base, 24), bf.BF_FP16, torch, set_w=False)
    assert not all(np.all(np.isfinite(r)) for r in high)
    print(f"fp16 rel err: held {held:.2e}; on chip at 2^0 {onchip:.2e}, at 2^-24 {e_low:.2e}, at 2^24 not finite")
