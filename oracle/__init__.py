"""FP64 CPU oracle for batched complex beamforming -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package. The GPU library (`paper_1810_11451_gb300`)
never imports it, and it never imports the GPU library: the two share no code.

Contents
  * `apply_blocks`, `apply_batch`: the product R = W x S (Sec. III, the
    beamforming equation), computed by the plain C triple loop in
    `bf_oracle.c` in FP64 (the complex multiply-add written out in reals).
  * `rel_frobenius`, `errnorm_blocks`: the accuracy report -- sum |R - Rref|^2
    and sum |Rref|^2 per block and in total, relative Frobenius error.
  * `bf16_round`, `fp16_round`, `tf32_round`, `split_bf16`, `split_tf32`,
    `pow2_scale`, `quantize_planes`, `quantize_blocks`: the reduced-precision
    operand encodings
    (the paper fixes no data type; the readings are: round to nearest even, a
    power-of-two per-block scale taken from the component-wise max-abs, split
    x = hi + lo with hi = round(x) and lo = round(x - hi), all decided in FP32
    as the GPU does).
  * `apply_terms`: the FP64 product of already-encoded operands, used to check
    the tensor-core kernels' mechanics tightly.
  * `circular_filter`, `dft`: the fast-convolution filter y = IFFT(MULT(FFT(s)))
    of Sec. III (filter equation, Fig. 4), N = 2048, evaluated by its
    definition as a circular convolution, and the DFT by its definition, both
    in `bf_filter_oracle.c` (FP64).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import List, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bf_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "bf_filter_oracle.c")]
_LIB_PATH = os.path.join(_HERE, "libbf_oracle.so")
_lib = None


def build(out_path: str = _LIB_PATH, mutant: int = 0, force: bool = False) -> str:
    """Compile bf_oracle.c with gcc (FP64, -O2, no FP contraction, OpenMP).

    `mutant` > 0 plants one of the deliberate mistakes listed in the C source
    (used only by the tests that show the pins catch mistakes)."""
    if not force and os.path.exists(out_path) and \
            os.path.getmtime(out_path) >= max(os.path.getmtime(f) for f in _SRCS):
        return out_path
    tmp = out_path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           f"-DBFO_MUTANT={int(mutant)}"] + _SRCS + ["-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out_path)
    return out_path


def _bind(path: str):
    lib = ctypes.CDLL(path)
    lib.bfo_apply_blocks.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_longlong,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.bfo_apply_blocks.restype = None
    lib.bfo_circular_filter.argtypes = [ctypes.c_int, ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p]
    lib.bfo_circular_filter.restype = None
    lib.bfo_dft.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p]
    lib.bfo_dft.restype = None
    lib.bfo_num_threads.restype = ctypes.c_int
    lib.bfo_set_num_threads.argtypes = [ctypes.c_int]
    lib.bfo_set_num_threads.restype = None
    lib.bfo_mutant_id.restype = ctypes.c_int
    return lib


def lib():
    """The oracle's shared library, built on first use."""
    global _lib
    if _lib is None:
        _lib = _bind(build())
    return _lib


def load_variant(path: str):
    """Bind another build of the oracle (a planted-mistake build in the tests)."""
    return _bind(path)


def num_threads() -> int:
    return int(lib().bfo_num_threads())


def set_num_threads(n: int) -> None:
    """Run the oracle on n threads from now on (timing on one core)."""
    lib().bfo_set_num_threads(int(n))


# --------------------------------------------------------------------------
# The product (Sec. III, beamforming equation)
# --------------------------------------------------------------------------
def apply_blocks(W: np.ndarray, S: np.ndarray, _lib=None) -> np.ndarray:
    """R[n] = W @ S[n] for every block n, in FP64.

    W: (n_ant, f) complex; S: (n_blocks, f, b) complex. Returns complex128
    (n_blocks, n_ant, b). Inputs are widened to complex128 first."""
    L = _lib or lib()
    W = np.ascontiguousarray(W, dtype=np.complex128)
    S = np.ascontiguousarray(S, dtype=np.complex128)
    n_ant, f = W.shape
    if S.ndim != 3 or S.shape[1] != f:
        raise ValueError(f"S must be (n_blocks, {f}, b), got {S.shape}")
    n_blocks, _, b = S.shape
    R = np.empty((n_blocks, n_ant, b), dtype=np.complex128)
    if n_blocks:
        L.bfo_apply_blocks(n_ant, f, b, n_blocks, W.ctypes.data, S.ctypes.data, R.ctypes.data)
    return R


def apply_batch(batch, _lib=None) -> List[np.ndarray]:
    """R of every group of a `workloads.Batch` (list of (n_blocks, n_ant, b) arrays)."""
    return [apply_blocks(batch.W[p], s, _lib) for p, s in zip(batch.prec, batch.S)]


# --------------------------------------------------------------------------
# Accuracy report: relative Frobenius error
# --------------------------------------------------------------------------
def errnorm_blocks(R: np.ndarray, Rref: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Per block: (sum |R - Rref|^2, sum |Rref|^2), summed in FP64."""
    R = np.asarray(R, dtype=np.complex128).reshape(R.shape[0], -1)
    Rref = np.asarray(Rref, dtype=np.complex128).reshape(Rref.shape[0], -1)
    d = R - Rref
    num = np.sum(d.real * d.real + d.imag * d.imag, axis=1)
    den = np.sum(Rref.real * Rref.real + Rref.imag * Rref.imag, axis=1)
    return num, den


def rel_frobenius(R: Sequence[np.ndarray], Rref: Sequence[np.ndarray]) -> float:
    """||R - Rref||_F / ||Rref||_F over all blocks of all groups (0 if both are 0)."""
    num = den = 0.0
    for a, r in zip(R, Rref):
        if a.size == 0:
            continue
        n, d = errnorm_blocks(a, r)
        num += float(n.sum())
        den += float(d.sum())
    if den == 0.0:
        return 0.0 if num == 0.0 else float("inf")
    return float(np.sqrt(num / den))


# --------------------------------------------------------------------------
# Reduced-precision encodings (decided in FP32, round to nearest even)
# --------------------------------------------------------------------------
def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round FP32 values to the nearest bfloat16 (ties to even); returns float32.

    bfloat16 keeps the sign, the 8 exponent bits and the top 7 mantissa bits of
    an FP32; rounding adds half an ulp of the kept part, plus one when the kept
    part is odd (ties to even), then clears the 16 dropped bits. Finite inputs
    whose rounded value stays finite only."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32)


def bf16_bits(x: np.ndarray) -> np.ndarray:
    """The 16-bit patterns of bf16_round(x)."""
    return (bf16_round(x).view(np.uint32) >> np.uint32(16)).astype(np.uint16)


def fp16_round(x: np.ndarray) -> np.ndarray:
    """Round FP32 values to IEEE binary16 (ties to even); returns float32."""
    return np.asarray(x, dtype=np.float32).astype(np.float16).astype(np.float32)


def fp16_bits(x: np.ndarray) -> np.ndarray:
    """The 16-bit patterns of fp16_round(x)."""
    return np.asarray(x, dtype=np.float32).astype(np.float16).view(np.uint16)


def tf32_round(x: np.ndarray) -> np.ndarray:
    """Round FP32 values to the nearest TF32 value (ties to even), kept as
    float32 with the 13 dropped fraction bits zero. TF32 keeps the sign, the 8
    exponent bits and the top 10 fraction bits; the construction is
    bf16_round's with 13 dropped bits instead of 16. Finite inputs whose
    rounded value stays finite only."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(13)) & np.uint64(1)
    u = (u + np.uint64(0xFFF) + lsb) & np.uint64(0xFFFFE000)
    return u.astype(np.uint32).view(np.float32)


def split_tf32(x: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """x ~ hi + lo with hi = tf32(x) and lo = tf32(x - hi); x - hi is exact in FP32."""
    x = np.asarray(x, dtype=np.float32)
    hi = tf32_round(x)
    lo = tf32_round((x - hi).astype(np.float32))
    return hi, lo


def split_bf16(x: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """x ~ hi + lo with hi = bf16(x) and lo = bf16(x - hi); x - hi is exact in FP32."""
    x = np.asarray(x, dtype=np.float32)
    hi = bf16_round(x)
    lo = bf16_round((x - hi).astype(np.float32))
    return hi, lo


def pow2_scales(maxabs: np.ndarray) -> np.ndarray:
    """pow2_scale of every element of an array of FP32 max-abs values."""
    m = np.asarray(maxabs, dtype=np.float32)
    mant, ex = np.frexp(m)          # m = mant * 2^ex, mant in [0.5, 1)
    e = np.where(mant == 0.5, ex - 1, ex)
    s = np.ldexp(np.float32(1.0), e).astype(np.float64)
    return np.where(m == 0, 1.0, s)


def pow2_scale(maxabs: float) -> float:
    """The power of two 2^e with e = ceil(log2(maxabs)), so maxabs / 2^e is in
    (1/2, 1]; 1.0 when maxabs is 0. Decided exactly from the FP32 value."""
    return float(pow2_scales(np.array([maxabs]))[0])


def block_maxabs(x: np.ndarray) -> float:
    """Component-wise max-abs of a complex64 block: max over |re| and |im|."""
    x = np.asarray(x, dtype=np.complex64)
    if x.size == 0:
        return 0.0
    return float(max(np.max(np.abs(x.real)), np.max(np.abs(x.imag))))


def _encode(re: np.ndarray, im: np.ndarray, prec: str):
    """The planes of already scaled FP32 parts (round to nearest even)."""
    if prec == "bf16":
        return [(bf16_round(re), bf16_round(im))]
    if prec == "fp16":
        return [(fp16_round(re), fp16_round(im))]
    if prec == "bf16x3":
        rh, rl = split_bf16(re)
        ih, il = split_bf16(im)
        return [(rh, ih), (rl, il)]
    if prec == "tf32x3":
        rh, rl = split_tf32(re)
        ih, il = split_tf32(im)
        return [(rh, ih), (rl, il)]
    raise ValueError(prec)


def quantize_planes(x: np.ndarray, prec: str, scaled: bool = True):
    """Encode a complex64 block (or precoder) for a tensor-core path.

    prec: "bf16" | "fp16" | "bf16x3" | "tf32x3". Returns (scale, planes) where scale is
    the power of two that multiplies the encoded values back, and planes is a
    list of (re, im) float32 arrays: one pair for single pass, (hi, lo) pairs
    for the split form. With scaled=False the scale is 1."""
    x = np.asarray(x, dtype=np.complex64)
    s = pow2_scale(block_maxabs(x)) if scaled else 1.0
    inv = np.float32(1.0 / s)
    re = (x.real.astype(np.float32) * inv).astype(np.float32)
    im = (x.imag.astype(np.float32) * inv).astype(np.float32)
    return s, _encode(re, im, prec)


def quantize_blocks(S: np.ndarray, prec: str, scaled: bool = True):
    """quantize_planes applied to every block of S (n_blocks, f, b) at once:
    the same steps (component-wise max-abs per block, its power-of-two scale,
    the FP32 product with the scale's inverse, the encoding), vectorised over
    blocks. Returns (scales (n_blocks,) float64, planes as (re, im) pairs of
    (n_blocks, f, b) float32 arrays)."""
    S = np.asarray(S, dtype=np.complex64)
    n = S.shape[0]
    if scaled and S[0].size:
        m = np.maximum(np.abs(S.real).reshape(n, -1).max(axis=1), np.abs(S.imag).reshape(n, -1).max(axis=1))
        s = pow2_scales(m)
    else:
        s = np.ones(n)
    inv = (1.0 / s).astype(np.float32).reshape((n,) + (1,) * (S.ndim - 1))
    re = (S.real.astype(np.float32) * inv).astype(np.float32)
    im = (S.imag.astype(np.float32) * inv).astype(np.float32)
    return s, _encode(re, im, prec)


def apply_terms(W_terms, S_terms, pairs, scale: float = 1.0, _lib=None) -> np.ndarray:
    """FP64 sum over (a, b) in pairs of W_terms[a] @ S_terms[b], times scale.

    W_terms[a]: (n_ant, f) complex; S_terms[b]: (n_blocks, f, b) complex. Used
    with the encoded operands of `quantize_planes` to predict what a
    reduced-precision kernel computes up to FP32 accumulation rounding."""
    R = None
    for a, b_ in pairs:
        t = apply_blocks(W_terms[a], S_terms[b_], _lib)
        R = t if R is None else R + t
    return R * scale


# --------------------------------------------------------------------------
# The fast-convolution filter (Sec. III, filter equation and Fig. 4)
# --------------------------------------------------------------------------
def _c128(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.complex128))


def circular_filter(h: np.ndarray, s: np.ndarray, _lib=None) -> np.ndarray:
    """y = IFFT(FFT(h) * FFT(s)) for every signal, evaluated as the circular
    convolution y[n] = sum_m h[m] s[(n - m) mod N] in FP64.

    h: (N,) or (n_taps <= N,) complex filter sequence (zero-padded to N);
    s: (n_sig, N) complex signals. Returns (n_sig, N) complex128."""
    s = _c128(s)
    if s.ndim == 1:
        s = s[None, :]
    n = s.shape[-1]
    hp = np.zeros(n, np.complex128)
    h = np.asarray(h, dtype=np.complex128).ravel()
    assert h.size <= n
    hp[:h.size] = h
    y = np.empty_like(s)
    L = _lib or lib()
    L.bfo_circular_filter(int(n), int(s.shape[0]), hp.ctypes.data, s.ctypes.data, y.ctypes.data)
    return y


def dft(x: np.ndarray, inverse: bool = False, _lib=None) -> np.ndarray:
    """The DFT by its definition along the last axis: X[k] = sum_j x[j]
    e^{-2 pi i j k / N} (inverse=True: the e^{+...} sum divided by N)."""
    x = _c128(x)
    shp = x.shape
    x2 = x.reshape(-1, shp[-1])
    X = np.empty_like(x2)
    L = _lib or lib()
    L.bfo_dft(int(shp[-1]), 1 if inverse else -1, int(x2.shape[0]), x2.ctypes.data, X.ctypes.data)
    if inverse:
        X /= shp[-1]
    return X.reshape(shp)
