"""Precoder ingest (Sec. III: W is constant, so it is converted once into the
images the kernels read), bit for bit against the oracle's encodings of the
same W: the FP32 planes of the CUDA-core kernels, the power-of-two scale, and
the real-block tensor-core operand B (row 2i = (Re W, -Im W), row 2i + 1 =
(Im W, Re W), divided by the scale) as bf16 hi|lo, fp16 and tf32 hi|lo images
in the documented K-major layout, zero in the K padding."""
import numpy as np
import pytest

import oracle
import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1810_11451_gb300 as bf  # noqa: E402
from bfrun import to_device_c64  # noqa: E402


@pytest.fixture(scope="module")
def plan():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    p = bf.bf_plan_create(64, 36, 60)
    yield p
    bf.bf_plan_destroy(p)


def _layout(vals, kp, esize):
    """Scatter a 128 x kp array into the K-major core-matrix layout: 8 rows x
    16 bytes per core matrix, core matrices 128 bytes apart along K, 8-row
    groups 8*kp*esize bytes apart (offsets here in elements)."""
    per = 16 // esize  # elements per 16-byte row of a core matrix
    r, c = np.meshgrid(np.arange(128), np.arange(kp), indexing="ij")
    off = (r >> 3) * (8 * kp) + (c // per) * (8 * per) + (r & 7) * per + (c % per)
    out = np.zeros(128 * kp, dtype=vals.dtype)
    out[off.ravel()] = vals.ravel()
    return out.view(np.uint8)


def expected_images(W):
    W = np.asarray(W, dtype=np.complex64)
    f = W.shape[1]
    re, im = W.real.astype(np.float32), W.imag.astype(np.float32)
    planes = np.concatenate([re.T.ravel(), im.T.ravel(), (re + im).astype(np.float32).T.ravel()])
    scale = oracle.pow2_scale(oracle.block_maxabs(W))
    inv = np.float32(1.0 / scale)
    kp, kp32 = ((2 * f + 15) // 16) * 16, ((2 * f + 7) // 8) * 8
    B = np.zeros((128, kp), np.float32)
    B[0::2, 0:2 * f:2], B[0::2, 1:2 * f:2] = re, np.negative(im)
    B[1::2, 0:2 * f:2], B[1::2, 1:2 * f:2] = im, re
    xs = (B * inv).astype(np.float32)
    hi, lo = oracle.split_bf16(xs)
    th, tl = oracle.split_tf32(np.ascontiguousarray(xs[:, :kp32]))
    b16 = lambda a: (a.view(np.uint32) >> np.uint32(16)).astype(np.uint16)
    return {
        bf.BF_IMG_FP32: planes.view(np.uint8),
        bf.BF_IMG_SCALE: np.array([scale], np.float32).view(np.uint8),
        bf.BF_IMG_BF16X2: np.concatenate([_layout(b16(hi), kp, 2), _layout(b16(lo), kp, 2)]),
        bf.BF_IMG_FP16: _layout(oracle.fp16_bits(xs), kp, 2),
        bf.BF_IMG_TF32X2: np.concatenate([_layout(th.view(np.uint32), kp32, 4),
                                          _layout(tl.view(np.uint32), kp32, 4)]),
    }


def test_images_match_the_oracle_encodings(plan):
    rng = np.random.default_rng(41)
    Ws = [wl.precoder_unit_columns(rng, 64, f) for f in (1, 7, 8, 9, 17, 36)]
    Ws.append(wl.integer_precoder(rng, 64, 13, 32))            # exact integers, scale 32
    Ws.append(wl.precoder_unit_columns(rng, 64, 5) * 1e-6)     # a small scale
    Ws.append(np.zeros((64, 4), complex))                      # all zero: scale 1
    flat = np.concatenate([np.asarray(W, np.complex64).ravel() for W in Ws])
    Wd = to_device_c64(flat, torch)
    bf.bf_set_precoders(plan, Wd, [W.shape[1] for W in Ws], 200)
    for n, W in enumerate(Ws):
        want = expected_images(W)
        for kind, exp in want.items():
            got = bf.bf_get_precoder_image(plan, 200 + n, kind)
            assert got.size == exp.size, (n, kind, got.size, exp.size)
            assert np.array_equal(got, exp), f"precoder {n} (f = {W.shape[1]}), image kind {kind}"


def test_image_query_errors(plan):
    with pytest.raises(bf.BfError) as ei:
        bf.bf_get_precoder_image(plan, 99999, bf.BF_IMG_FP32)
    assert ei.value.status == bf.BF_ENOTFOUND
    W = to_device_c64(np.ones(64 * 3, np.complex64), torch)
    bf.bf_set_precoders(plan, W, [3], 300)
    with pytest.raises(bf.BfError) as ei:
        bf.bf_get_precoder_image(plan, 300, 9)
    assert ei.value.status == bf.BF_EINVAL
