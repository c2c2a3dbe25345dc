"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

The product is R = W x S (Sec. III, beamforming equation). The paper prints
no worked numbers for it, so the oracle is pinned by mathematics: a brute
force in exact integer arithmetic organised differently (a sum of outer
products), a library matmul, the identity precoder, orthonormal columns,
linearity, conjugation, associativity, a closed-form DFT sum, f = 0, and the
paper's printed dimensions. `test_planted_mistakes_are_caught` rebuilds the
oracle with deliberate mistakes and checks that every one of them fails a pin.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_c(rng, shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


# ---------------------------------------------------------------- pins
def pin_outer_product_bruteforce(L):
    """Exact integer brute force, R = sum_k W[:, k] (outer) S[k, :], with Python ints."""
    rng = np.random.default_rng(11)
    for n_ant, f, b in [(1, 1, 1), (3, 2, 4), (4, 3, 5), (2, 5, 3)]:
        W = (rng.integers(-3, 4, (n_ant, f)) + 1j * rng.integers(-3, 4, (n_ant, f)))
        S = (rng.integers(-3, 4, (1, f, b)) + 1j * rng.integers(-3, 4, (1, f, b)))
        acc = [[[0, 0] for _ in range(b)] for _ in range(n_ant)]
        for k in range(f):
            col = [(int(W[i, k].real), int(W[i, k].imag)) for i in range(n_ant)]
            row = [(int(S[0, k, j].real), int(S[0, k, j].imag)) for j in range(b)]
            for i, (a, bb) in enumerate(col):
                for j, (c, d) in enumerate(row):
                    acc[i][j][0] += a * c - bb * d
                    acc[i][j][1] += a * d + bb * c
        R = oracle.apply_blocks(W, S, L)[0]
        for i in range(n_ant):
            for j in range(b):
                if R[i, j].real != acc[i][j][0] or R[i, j].imag != acc[i][j][1]:
                    return False
    return True


def pin_fraction_dyadic(L):
    """Dyadic rationals (k/8) are exact in FP64: compare with Fraction arithmetic."""
    rng = np.random.default_rng(12)
    n_ant, f, b = 3, 4, 2
    Wr, Wi = rng.integers(-16, 17, (n_ant, f)), rng.integers(-16, 17, (n_ant, f))
    Sr, Si = rng.integers(-16, 17, (f, b)), rng.integers(-16, 17, (f, b))
    W = (Wr + 1j * Wi) / 8.0
    S = ((Sr + 1j * Si) / 8.0)[None]
    R = oracle.apply_blocks(W, S, L)[0]
    for i in range(n_ant):
        for j in range(b):
            re = sum(Fraction(int(Wr[i, k]), 8) * Fraction(int(Sr[k, j]), 8)
                     - Fraction(int(Wi[i, k]), 8) * Fraction(int(Si[k, j]), 8) for k in range(f))
            im = sum(Fraction(int(Wr[i, k]), 8) * Fraction(int(Si[k, j]), 8)
                     + Fraction(int(Wi[i, k]), 8) * Fraction(int(Sr[k, j]), 8) for k in range(f))
            if Fraction(R[i, j].real) != re or Fraction(R[i, j].imag) != im:
                return False
    return True


def pin_library_matmul(L):
    """numpy's complex matmul (a library routine) agrees to FP64 rounding."""
    rng = np.random.default_rng(13)
    for n_ant, f, b, nb in [(64, 36, 60, 3), (64, 1, 60, 2), (5, 7, 3, 4), (64, 17, 60, 1)]:
        W = _rand_c(rng, (n_ant, f))
        S = _rand_c(rng, (nb, f, b))
        R = oracle.apply_blocks(W, S, L)
        ref = np.matmul(W[None], S)
        if not np.allclose(R, ref, rtol=1e-13, atol=1e-13 * np.sqrt(f)):
            return False
    return True


def pin_identity(L):
    """W = [I_f; 0] gives R = [S; 0] exactly."""
    rng = np.random.default_rng(14)
    for f in (1, 8, 36):
        W = np.zeros((64, f), complex)
        W[:f, :f] = np.eye(f)
        S = _rand_c(rng, (2, f, 60))
        R = oracle.apply_blocks(W, S, L)
        if not (np.array_equal(R[:, :f, :], S) and np.all(R[:, f:, :] == 0)):
            return False
    return True


def pin_orthonormal_columns(L):
    """W with orthonormal columns (W^H W = I) preserves every column norm of S."""
    rng = np.random.default_rng(15)
    for f in (1, 7, 36):
        Q, _ = np.linalg.qr(_rand_c(rng, (64, f)))
        S = _rand_c(rng, (3, f, 60))
        R = oracle.apply_blocks(Q, S, L)
        if not np.allclose(np.linalg.norm(R, axis=1), np.linalg.norm(S, axis=1), rtol=1e-12):
            return False
    return True


def pin_linearity(L):
    """R(a S1 + b S2) = a R(S1) + b R(S2)."""
    rng = np.random.default_rng(16)
    W = _rand_c(rng, (64, 12))
    S1, S2 = _rand_c(rng, (2, 12, 60)), _rand_c(rng, (2, 12, 60))
    a, b = 0.7 - 1.3j, -2.1 + 0.4j
    lhs = oracle.apply_blocks(W, a * S1 + b * S2, L)
    rhs = a * oracle.apply_blocks(W, S1, L) + b * oracle.apply_blocks(W, S2, L)
    return np.allclose(lhs, rhs, rtol=1e-12, atol=1e-12)


def pin_conjugation(L):
    """R(conj W, conj S) = conj R(W, S), bit for bit."""
    rng = np.random.default_rng(17)
    W, S = _rand_c(rng, (64, 9)), _rand_c(rng, (2, 9, 60))
    return np.array_equal(oracle.apply_blocks(W.conj(), S.conj(), L),
                          oracle.apply_blocks(W, S, L).conj())


def pin_associativity(L):
    """(A B) S = A (B S) with every product taken by the oracle."""
    rng = np.random.default_rng(18)
    A, B = _rand_c(rng, (64, 6)), _rand_c(rng, (6, 5))
    S = _rand_c(rng, (2, 5, 60))
    AB = oracle.apply_blocks(A, B[None], L)[0]
    lhs = oracle.apply_blocks(AB, S, L)
    rhs = oracle.apply_blocks(A, oracle.apply_blocks(B, S, L), L)
    return np.allclose(lhs, rhs, rtol=1e-12, atol=1e-12)


def pin_dft_geometric_sum(L):
    """W[i,k] = exp(-2 pi i ik/N), S[k,j] = exp(2 pi i k m_j/N): R[i,j] is the
    geometric sum sum_k q^k with q = exp(-2 pi i (i - m_j)/N), whose closed form
    is f when q = 1 and (1 - q^f)/(1 - q) otherwise."""
    N, f, b = 64, 36, 60
    i = np.arange(N)[:, None]
    k = np.arange(f)[None, :]
    W = np.exp(-2j * np.pi * i * k / N)
    m = (np.arange(b) * 7) % N
    S = np.exp(2j * np.pi * np.arange(f)[:, None] * m[None, :] / N)[None]
    R = oracle.apply_blocks(W, S, L)[0]
    d = (np.arange(N)[:, None] - m[None, :]) % N
    q = np.exp(-2j * np.pi * d / N)
    with np.errstate(invalid="ignore", divide="ignore"):
        closed = np.where(d == 0, f, (1 - q ** f) / (1 - q))
    return np.allclose(R, closed, atol=1e-11)


def pin_f_zero(L):
    """f = 0: the empty sum, R = 0 everywhere."""
    R = oracle.apply_blocks(np.zeros((64, 0), complex), np.zeros((3, 0, 60), complex), L)
    return R.shape == (3, 64, 60) and np.all(R == 0)


def pin_integer_matmul(L):
    """Exact integer batch: the real-block product with int64 matmul (library)."""
    batch = wl.config_exact_integer(f_list=(1, 5, 36), blocks_per_group=(2,))
    for p, S in zip(batch.prec, batch.S):
        W = batch.W[p]
        Wr, Wi = W.real.astype(np.int64), W.imag.astype(np.int64)
        Sr, Si = S.real.astype(np.int64), S.imag.astype(np.int64)
        Rr = np.matmul(Wr[None], Sr) - np.matmul(Wi[None], Si)
        Ri = np.matmul(Wr[None], Si) + np.matmul(Wi[None], Sr)
        R = oracle.apply_blocks(W, S, L)
        if not (np.array_equal(R.real, Rr) and np.array_equal(R.imag, Ri)):
            return False
    return True


PINS = [pin_outer_product_bruteforce, pin_fraction_dyadic, pin_library_matmul, pin_identity,
        pin_orthonormal_columns, pin_linearity, pin_conjugation, pin_associativity,
        pin_dft_geometric_sum, pin_f_zero, pin_integer_matmul]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_oracle_pin(pin, oracle_lib):
    assert pin(oracle_lib)


def test_paper_dimensions_fixture():
    vals = {}
    with open(os.path.join(GOLDEN, "paper_dimensions.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                vals[k] = int(v)
    assert vals == {"n_ant": wl.N_ANT, "b": wl.B_RE, "f_min": 0, "f_max": wl.F_MAX}


# One mistake per planted build (see BFO_MUTANT in bf_oracle.c): sign of the
# cross term, last flow dropped, S transposed, W conjugated, W column-major,
# accumulators not reset, re/im swapped.
MUTANTS = [1, 2, 3, 4, 5, 6, 7]


@pytest.mark.parametrize("mutant", MUTANTS)
def test_planted_mistakes_are_caught(mutant, tmp_path):
    path = oracle.build(str(tmp_path / f"libbf_oracle_m{mutant}.so"), mutant=mutant, force=True)
    L = oracle.load_variant(path)
    assert L.bfo_mutant_id() == mutant
    failed = [p.__name__ for p in PINS if not p(L)]
    assert failed, f"mutant {mutant} passed every pin"


# ---------------------------------------------------------------- filter pins
# The filter y = IFFT(MULT(FFT(s))) (Sec. III, filter equation, Fig. 4) with
# the unnormalised forward DFT and 1/N in the inverse is the circular
# convolution of the filter sequence h with s. The pins below fix the oracle
# by facts that do not come from it: a hand-worked N = 4 case, the identity
# and shifted-impulse closed forms, the convolution theorem through numpy's
# FFT, linearity, and the DFT's closed forms (impulse, constant, pure tone),
# Parseval's identity and numpy's FFT for the definition-based DFT.
def pin_filter_hand_example(L):
    """N = 4, h = [1, i, 0, 0], s = [1, 0, 0, 1]: y[0] = h0 s0 + h1 s3 = 1 + i,
    y[1] = h1 s0 = i, y[2] = 0, y[3] = h0 s3 = 1 (worked by hand)."""
    y = oracle.circular_filter(np.array([1, 1j, 0, 0]), np.array([[1, 0, 0, 1]]), L)[0]
    return np.array_equal(y, np.array([1 + 1j, 1j, 0, 1]))


def pin_filter_identity(L):
    """h = delta: y = s exactly."""
    rng = np.random.default_rng(40)
    s = _rand_c(rng, (3, 64))
    h = np.zeros(64, complex)
    h[0] = 1
    return np.array_equal(oracle.circular_filter(h, s, L), s)


def pin_filter_shifted_impulse(L):
    """s = delta[n - n0]: y[n] = h[(n - n0) mod N] exactly (the wrap included)."""
    rng = np.random.default_rng(41)
    n = 128
    h = _rand_c(rng, 100)
    hp = np.zeros(n, complex)
    hp[:100] = h
    for n0 in (0, 1, 37, 127):
        s = np.zeros((1, n), complex)
        s[0, n0] = 1
        if not np.array_equal(oracle.circular_filter(h, s, L)[0], np.roll(hp, n0)):
            return False
    return True


def pin_filter_convolution_theorem(L):
    """y = ifft(fft(h) * fft(s)) through numpy's FFT, at N = 2048, to 1e-12."""
    rng = np.random.default_rng(42)
    b = wl.config_filter_small(n_sig=4)
    hp = np.zeros(b.n, complex)
    hp[:b.h.size] = b.h
    ref = np.fft.ifft(np.fft.fft(hp)[None, :] * np.fft.fft(b.s, axis=1), axis=1)
    y = oracle.circular_filter(b.h, b.s, L)
    return np.max(np.abs(y - ref)) <= 1e-12 * np.max(np.abs(ref))


def pin_filter_linearity(L):
    rng = np.random.default_rng(43)
    h = _rand_c(rng, 50)
    s1, s2 = _rand_c(rng, (2, 256)), _rand_c(rng, (2, 256))
    a, c = 0.75 - 0.5j, -1.25 + 2j
    lhs = oracle.circular_filter(h, a * s1 + c * s2, L)
    rhs = a * oracle.circular_filter(h, s1, L) + c * oracle.circular_filter(h, s2, L)
    return np.max(np.abs(lhs - rhs)) <= 1e-12 * np.max(np.abs(rhs))


def pin_dft_closed_forms(L):
    """DFT(delta) = 1, DFT(1) = N delta, DFT(e^{2 pi i k0 n / N}) = N delta[k - k0]."""
    n = 64
    d = np.zeros(n, complex)
    d[0] = 1
    if np.max(np.abs(oracle.dft(d, _lib=L) - 1)) > 1e-13:
        return False
    e = np.zeros(n, complex)
    e[0] = n
    if np.max(np.abs(oracle.dft(np.ones(n, complex), _lib=L) - e)) > 1e-11:
        return False
    k0 = 5
    tone = np.exp(2j * np.pi * k0 * np.arange(n) / n)
    e = np.zeros(n, complex)
    e[k0] = n
    return np.max(np.abs(oracle.dft(tone, _lib=L) - e)) <= 1e-10


def pin_dft_parseval_and_library(L):
    rng = np.random.default_rng(44)
    x = _rand_c(rng, (2, 2048))
    X = oracle.dft(x, _lib=L)
    if abs(np.sum(np.abs(X) ** 2) - 2048 * np.sum(np.abs(x) ** 2)) > 1e-10 * np.sum(np.abs(X) ** 2):
        return False
    if np.max(np.abs(X - np.fft.fft(x, axis=1))) > 1e-10 * np.max(np.abs(X)):
        return False
    return np.max(np.abs(oracle.dft(X, inverse=True, _lib=L) - x)) <= 1e-12 * np.max(np.abs(x))


FILTER_PINS = [pin_filter_hand_example, pin_filter_identity, pin_filter_shifted_impulse,
               pin_filter_convolution_theorem, pin_filter_linearity, pin_dft_closed_forms,
               pin_dft_parseval_and_library]


@pytest.mark.parametrize("pin", FILTER_PINS, ids=[p.__name__ for p in FILTER_PINS])
def test_filter_oracle_pin(pin, oracle_lib):
    assert pin(oracle_lib)


def test_filter_dimensions_fixture():
    with open(os.path.join(GOLDEN, "filter_dimensions.txt")) as fh:
        vals = dict(line.split() for line in fh if line.strip() and not line.startswith("#"))
    assert int(vals["n"]) == wl.FILTER_N


# Filter mistakes (BFO_MUTANT 8..10 in bf_filter_oracle.c): correlation instead
# of convolution, no circular wrap, conjugated taps.
@pytest.mark.parametrize("mutant", [8, 9, 10])
def test_planted_filter_mistakes_are_caught(mutant, tmp_path):
    path = oracle.build(str(tmp_path / f"libbf_oracle_m{mutant}.so"), mutant=mutant, force=True)
    L = oracle.load_variant(path)
    assert L.bfo_mutant_id() == mutant
    failed = [p.__name__ for p in FILTER_PINS if not p(L)]
    assert failed, f"mutant {mutant} passed every filter pin"


# ---------------------------------------------------------------- accuracy report
def test_errnorm_closed_form():
    rng = np.random.default_rng(20)
    Rref = _rand_c(rng, (4, 64, 60))
    delta = 1e-3 * (1 + 2j)
    num, den = oracle.errnorm_blocks(Rref + delta, Rref)
    assert np.allclose(num, 64 * 60 * abs(delta) ** 2, rtol=1e-12)
    assert np.allclose(den, np.linalg.norm(Rref.reshape(4, -1), axis=1) ** 2, rtol=1e-12)
    e = oracle.rel_frobenius([Rref + delta], [Rref])
    assert np.isclose(e, np.linalg.norm(delta * np.ones(Rref.size)) / np.linalg.norm(Rref.ravel()),
                      rtol=1e-12)
    assert oracle.rel_frobenius([np.zeros((1, 2, 2))], [np.zeros((1, 2, 2))]) == 0.0


# ---------------------------------------------------------------- encodings
# Round-to-nearest-even facts of IEEE 754 applied to the bfloat16 format
# (8 exponent bits, 7 stored mantissa bits): FP32 bit pattern -> bf16 pattern.
RNE_CASES = [
    (0x3F800000, 0x3F80),  # 1.0 exact
    (0x3F808000, 0x3F80),  # halfway 1.0 / 1.0078125 -> even (1.0)
    (0x3F818000, 0x3F82),  # halfway, odd kept part -> rounds up to even
    (0x3F808001, 0x3F81),  # just above halfway -> up
    (0x3F807FFF, 0x3F80),  # just below halfway -> down
    (0xBF808000, 0xBF80),  # sign is kept
    (0x3F7FFFFF, 0x3F80),  # carry into the exponent: 0.99999994 -> 1.0
    (0x00000000, 0x0000),
    (0x80000000, 0x8000),
]


def test_bf16_round_to_nearest_even_cases():
    x = np.array([c[0] for c in RNE_CASES], dtype=np.uint32).view(np.float32)
    got = oracle.bf16_bits(x)
    assert [int(g) for g in got] == [c[1] for c in RNE_CASES]


def test_bf16_round_matches_library():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(21)
    x = np.concatenate([rng.normal(size=20000), rng.normal(size=2000) * 1e-30,
                        rng.normal(size=2000) * 1e30]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(oracle.bf16_round(x).view(np.uint32), ref.view(np.uint32))


def test_fp16_round_matches_library():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(22)
    x = (rng.normal(size=20000) * 4).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.float16).to(torch.float32).numpy()
    assert np.array_equal(oracle.fp16_round(x).view(np.uint32), ref.view(np.uint32))


# binary16: 1 sign, 5 exponent (bias 15), 10 fraction bits
FP16_CASES = [
    (1.0, 0x3C00),
    (-2.0, 0xC000),
    (65504.0, 0x7BFF),     # largest finite
    (2049.0, 0x6800),      # tie between 2048 and 2050: even mantissa (2048)
    (2051.0, 0x6802),      # tie between 2050 and 2052: even mantissa (2052)
    (2050.0, 0x6801),      # exact
    (0.0, 0x0000),
    (-0.0, 0x8000),
    (2.0 ** -24, 0x0001),  # smallest subnormal
]


def test_fp16_bits_cases():
    x = np.array([c[0] for c in FP16_CASES], dtype=np.float32)
    assert [int(g) for g in oracle.fp16_bits(x)] == [c[1] for c in FP16_CASES]


# TF32 (8 exponent bits, 10 stored fraction bits): FP32 pattern -> rounded FP32 pattern
TF32_CASES = [
    (0x3F800000, 0x3F800000),  # 1.0 exact
    (0x3F801000, 0x3F800000),  # 1 + 2^-11, halfway 1.0 / 1 + 2^-10 -> even (1.0)
    (0x3F803000, 0x3F804000),  # 1 + 3*2^-11, halfway, odd kept part -> up to even
    (0x3F801001, 0x3F802000),  # just above halfway -> up
    (0x3F800FFF, 0x3F800000),  # just below halfway -> down
    (0xBF801000, 0xBF800000),  # sign is kept
    (0x3FFFF000, 0x40000000),  # 2 - 2^-11: halfway, odd -> carry into the exponent (2.0)
    (0x00000000, 0x00000000),
    (0x80000000, 0x80000000),
]


def test_tf32_round_to_nearest_even_cases():
    x = np.array([c[0] for c in TF32_CASES], dtype=np.uint32).view(np.float32)
    got = oracle.tf32_round(x).view(np.uint32)
    assert [int(g) for g in got] == [c[1] for c in TF32_CASES]


def test_tf32_round_is_the_nearest_tf32_value():
    """Against the definition, in FP64: of the two TF32 values around x (x with
    the 13 low bits cleared, and that plus one TF32 ulp), the nearer one, the
    one with an even last kept bit on a tie."""
    rng = np.random.default_rng(24)
    x = np.concatenate([rng.normal(size=20000), rng.normal(size=2000) * 1e-30,
                        rng.normal(size=2000) * 1e30, np.ldexp(1.0 + np.arange(64) * 2.0 ** -11, 3)])
    x = x.astype(np.float32)
    bits = x.view(np.uint32)
    lo = (bits & np.uint32(0xFFFFE000)).view(np.float32).astype(np.float64)  # toward zero
    hi = ((bits & np.uint32(0xFFFFE000)) + np.uint32(0x2000)).view(np.float32).astype(np.float64)  # away
    xd = x.astype(np.float64)
    dlo, dhi = np.abs(xd - lo), np.abs(hi - xd)
    even_lo = ((bits >> np.uint32(13)) & np.uint32(1)) == 0
    want = np.where(dlo < dhi, lo, np.where(dhi < dlo, hi, np.where(even_lo, lo, hi)))
    assert np.array_equal(oracle.tf32_round(x).astype(np.float64), want)


def test_split_tf32_bound():
    """hi + lo reproduces x to 2^-22 relative; both parts are TF32 values."""
    rng = np.random.default_rng(25)
    x = rng.normal(size=50000).astype(np.float32)
    hi, lo = oracle.split_tf32(x)
    assert np.array_equal(oracle.tf32_round(hi), hi) and np.array_equal(oracle.tf32_round(lo), lo)
    err = np.abs(x.astype(np.float64) - hi.astype(np.float64) - lo.astype(np.float64))
    assert np.all(err <= 2.0 ** -22 * np.abs(x.astype(np.float64)))


def test_split_bf16_bound():
    """hi + lo reproduces x to 2^-16 relative; both parts are bf16 values."""
    rng = np.random.default_rng(23)
    x = rng.normal(size=50000).astype(np.float32)
    hi, lo = oracle.split_bf16(x)
    assert np.array_equal(oracle.bf16_round(hi), hi) and np.array_equal(oracle.bf16_round(lo), lo)
    err = np.abs(x.astype(np.float64) - hi.astype(np.float64) - lo.astype(np.float64))
    assert np.all(err <= 2.0 ** -16 * np.abs(x.astype(np.float64)))
    y = oracle.bf16_round(x)
    h2, l2 = oracle.split_bf16(y)
    assert np.array_equal(h2, y) and np.all(l2 == 0)


@pytest.mark.parametrize("m,s", [(1.0, 1.0), (0.75, 1.0), (1.5, 2.0), (0.5, 0.5), (0.0, 1.0),
                                 (2.0 ** -10, 2.0 ** -10), (3 * 2.0 ** -11, 2.0 ** -9),
                                 (100.0, 128.0), (0.2, 0.25)])
def test_pow2_scale(m, s):
    assert oracle.pow2_scale(m) == s
    if m:
        assert 0.5 < m / s <= 1.0


def test_split_product_within_bound(oracle_lib):
    """The 3-term split product (hi*hi + hi*lo + lo*hi) of unit-power inputs stays
    within the first-order bound of the split: a relative error of a few 2^-16."""
    batch = wl.config_fullband(seed=30, n_rb=2, n_sym=3, f=36)
    W, S = batch.W[0].astype(np.complex64), batch.S[0].astype(np.complex64)
    sw, (wh, wl_) = oracle.quantize_planes(W, "bf16x3")
    ss, (sh, sl) = oracle.quantize_planes(S, "bf16x3")
    Wt = [wh[0] + 1j * wh[1], wl_[0] + 1j * wl_[1]]
    St = [sh[0] + 1j * sh[1], sl[0] + 1j * sl[1]]
    R3 = oracle.apply_terms(Wt, St, [(0, 0), (0, 1), (1, 0)], sw * ss, oracle_lib)
    ref = oracle.apply_blocks(W, S, oracle_lib)
    e = oracle.rel_frobenius([R3], [ref])
    assert 0 < e < 3 * 2.0 ** -16
    R1 = oracle.apply_terms(Wt, St, [(0, 0)], sw * ss, oracle_lib)
    e1 = oracle.rel_frobenius([R1], [ref])
    assert 2.0 ** -12 < e1 < 2.0 ** -7  # single pass: bf16 rounding of both operands


@pytest.mark.parametrize("prec", ["bf16", "fp16", "bf16x3", "tf32x3"])
def test_quantize_planes_scale_hand_worked(prec):
    """The per-block scale is 2^ceil(log2 m) with m the largest of |Re| and |Im|
    over the block (component-wise, not the complex modulus), and the planes are
    the block divided by it. Each case below is worked by hand; every encoded
    value is exactly representable, so the planes are checked exactly too.
      * the largest component is imaginary: [0.25 + 2.5j, -0.5 + 0.125j]:
        m = 2.5 -> 4 (Re alone would give 0.5);
      * |z| crosses a power of two that no component reaches: [0.75 + 0.75j]:
        m = 0.75 -> 1 (the modulus 1.06 would give 2);
      * exact powers of two: m = 1 -> 1, m = 4 (a negative real part) -> 4,
        m = 2^-3 -> 2^-3; one step above a power of two: m = 2 + 2^-21 -> 4;
      * an all-zero block keeps the scale 1."""
    cases = [
        (np.array([0.25 + 2.5j, -0.5 + 0.125j]), 4.0, [0.0625, -0.125], [0.625, 0.03125]),
        (np.array([0.75 + 0.75j]), 1.0, [0.75], [0.75]),
        (np.array([1.0 + 0.5j, 0.25 - 1.0j]), 1.0, [1.0, 0.25], [0.5, -1.0]),
        (np.array([-4.0 + 1.0j, 2.0 - 0.5j]), 4.0, [-1.0, 0.5], [0.25, -0.125]),
        (np.array([0.125 - 0.0625j]), 0.125, [1.0], [-0.5]),
        (np.array([0.5 + (2.0 + 2.0 ** -21) * 1j]), 4.0, [0.125], [None]),
        (np.zeros(3, complex), 1.0, [0.0] * 3, [0.0] * 3),
    ]
    for x, s_want, re_want, im_want in cases:
        blk = x.astype(np.complex64).reshape(1, -1)
        s, planes = oracle.quantize_planes(blk, prec)
        assert s == s_want, (x, s, s_want)
        re, im = planes[0]
        for got, want in ((re.ravel(), re_want), (im.ravel(), im_want)):
            for g, w in zip(got, want):
                if w is not None:
                    assert g == np.float32(w), (x, prec, g, w)
        if len(planes) > 1:  # split forms: exactly representable values leave no lo term
            lo_re, lo_im = planes[1]
            exact = [w is not None for w in im_want]
            assert np.all(lo_re == 0) and np.all(lo_im.ravel()[exact] == 0)
        s1, _ = oracle.quantize_planes(blk, prec, scaled=False)
        assert s1 == 1.0


def test_quantize_planes_scale_is_per_block_component_maximum():
    """Brute force over random blocks: the scale equals the smallest power of two
    that is >= every |Re| and |Im| of the block (found by doubling from 2^-40),
    and a block multiplied by 2^k gets 2^k times the scale and the same planes."""
    rng = np.random.default_rng(41)
    for _ in range(200):
        amp = 2.0 ** rng.integers(-20, 20)
        x = (amp * (rng.normal(size=(7, 9)) + 1j * rng.normal(size=(7, 9)) * rng.uniform(0, 3))).astype(np.complex64)
        m = max(float(np.max(np.abs(x.real))), float(np.max(np.abs(x.imag))))
        p = 2.0 ** -40
        while p < m:
            p *= 2.0
        s, planes = oracle.quantize_planes(x, "bf16")
        assert s == p
        s2, planes2 = oracle.quantize_planes((x * np.float32(8.0)).astype(np.complex64), "bf16")
        assert s2 == 8.0 * s
        assert all(np.array_equal(a, b) for pa, pb in zip(planes, planes2) for a, b in zip(pa, pb))


@pytest.mark.parametrize("prec", ["bf16", "fp16", "bf16x3", "tf32x3"])
def test_quantize_blocks_is_quantize_planes_per_block(prec):
    """The vectorised encoding equals the pinned per-block one, bit for bit,
    on blocks of very different levels (one of them all zero), scaled and not."""
    rng = np.random.default_rng(43)
    S = (rng.normal(size=(12, 5, 7)) + 1j * rng.normal(size=(12, 5, 7))) * \
        (2.0 ** rng.integers(-12, 12, size=12))[:, None, None]
    S[4] = 0
    S = S.astype(np.complex64)
    for scaled in (True, False):
        s, planes = oracle.quantize_blocks(S, prec, scaled)
        for n in range(S.shape[0]):
            s1, p1 = oracle.quantize_planes(S[n], prec, scaled)
            assert s[n] == s1
            for (re, im), (re1, im1) in zip(planes, p1):
                assert np.array_equal(re[n], re1) and np.array_equal(im[n], im1)
