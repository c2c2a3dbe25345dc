"""Seeded synthetic inputs for batched beamforming R = W x S.

Shared by the tests, the bench and the oracle's callers. This module only
draws inputs and lays them out in memory; it contains none of the product's
arithmetic (no W x S, no quantisation, no error norms).

Problem dimensions (Sec. III, beamforming equation): W is n_ant x f with one
row per antenna (64 antennas, Sec. II: 4 x 8 x 2 transceivers), S is f x b with
one row per parallel flow and one column per resource element, b = 60, and
0 <= f <= 36. W is constant while S changes, so many S blocks share one W.

The filter workload (Sec. III, filter equation and Fig. 4) is drawn here too:
blocks of N = 2048 complex time-domain samples and one filter sequence.

Layouts (the readings used throughout the library):
  * complex numbers are interleaved (re, im) pairs;
  * W is row-major n_ant x f (antenna-major), S is row-major f x b (flow-major),
    R is row-major n_ant x b;
  * the blocks of one group (all sharing one precoder) are contiguous.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

N_ANT = 64
B_RE = 60
F_MAX = 36
QAM_ORDERS = (4, 16, 64, 256)

__all__ = [
    "N_ANT", "B_RE", "F_MAX", "QAM_ORDERS", "Batch", "qam_levels",
    "qam_symbols", "qam_integer_symbols", "precoder_unit_columns",
    "integer_precoder", "complex_noise", "geometric_group_sizes",
    "config_small", "config_fullband", "config_uneven", "config_reduced",
    "config_exact_integer", "serving_schedule", "ServingJob",
    "FILTER_N", "FilterBatch", "filter_taps", "filter_signals",
    "config_filter_small", "config_filter_tti", "config_filter_bench",
]

FILTER_N = 2048  # FFT size of the filter (Sec. III: all sizes are 2048)


def qam_levels(order: int) -> np.ndarray:
    """Odd-integer amplitude levels of a square M-QAM: +-1, +-3, ..., +-(sqrt(M)-1)."""
    side = int(round(np.sqrt(order)))
    if side * side != order or side < 2:
        raise ValueError(f"square QAM order expected, got {order}")
    return np.arange(-(side - 1), side, 2, dtype=np.float64)


def qam_integer_symbols(rng: np.random.Generator, order: int, shape) -> np.ndarray:
    """Uniform square-QAM points with odd-integer coordinates (unscaled)."""
    lv = qam_levels(order)
    re = rng.choice(lv, size=shape)
    im = rng.choice(lv, size=shape)
    return re + 1j * im


def qam_symbols(rng: np.random.Generator, order: int, shape) -> np.ndarray:
    """Uniform square-QAM points scaled to unit average power.

    The mean power of the odd-integer constellation is 2(M-1)/3, so the points
    are divided by sqrt(2(M-1)/3) (QPSK 1/sqrt2, 16-QAM 1/sqrt10, 64-QAM
    1/sqrt42, 256-QAM 1/sqrt170).
    """
    return qam_integer_symbols(rng, order, shape) / np.sqrt(2.0 * (order - 1) / 3.0)


def complex_noise(rng: np.random.Generator, variance: float, shape) -> np.ndarray:
    """Circular complex Gaussian CN(0, variance): variance/2 per real component."""
    s = np.sqrt(variance / 2.0)
    return rng.normal(0.0, s, size=shape) + 1j * rng.normal(0.0, s, size=shape)


def precoder_unit_columns(rng: np.random.Generator, n_ant: int, f: int) -> np.ndarray:
    """n_ant x f precoder: i.i.d. CN(0,1) entries, every column scaled to unit 2-norm."""
    w = complex_noise(rng, 1.0, (n_ant, f))
    if f:
        w = w / np.linalg.norm(w, axis=0, keepdims=True)
    return w


def integer_precoder(rng: np.random.Generator, n_ant: int, f: int, lim: int = 2) -> np.ndarray:
    """Precoder with Gaussian-integer entries in {-lim..lim} + i{-lim..lim}."""
    return (rng.integers(-lim, lim + 1, size=(n_ant, f))
            + 1j * rng.integers(-lim, lim + 1, size=(n_ant, f))).astype(np.complex128)


def geometric_group_sizes(rng: np.random.Generator, total: int, mean: float = 14.0,
                          max_size: int = 64) -> List[int]:
    """Group sizes drawn geometric(p = 1/mean) on {1, 2, ...}, redrawn when above
    max_size, the last group truncated so that the sizes sum to total."""
    sizes: List[int] = []
    left = total
    while left > 0:
        g = int(rng.geometric(1.0 / mean))
        while g > max_size:
            g = int(rng.geometric(1.0 / mean))
        g = min(g, left)
        sizes.append(g)
        left -= g
    return sizes


@dataclass
class Batch:
    """A batch of groups; group g multiplies precoder prec[g] with its S blocks.

    W[p]   : complex128 (n_ant, f_p) precoder p
    prec   : precoder index of each group
    S[g]   : complex128 (n_blocks_g, f_{prec[g]}, b) symbol blocks of group g
    The values here are the exact (FP64) draws; the library is given them
    rounded to complex64 (or quantised), and the oracle is given the same
    rounded values widened back to FP64 unless a test says otherwise.
    """
    W: List[np.ndarray]
    prec: List[int]
    S: List[np.ndarray]
    name: str = ""
    seed: int = 0
    n_ant: int = N_ANT
    b: int = B_RE
    meta: dict = field(default_factory=dict)

    @property
    def n_groups(self) -> int:
        return len(self.prec)

    @property
    def f_of_group(self) -> List[int]:
        return [int(self.W[p].shape[1]) for p in self.prec]

    @property
    def n_blocks(self) -> List[int]:
        return [int(s.shape[0]) for s in self.S]

    @property
    def total_blocks(self) -> int:
        return int(sum(self.n_blocks))

    def flops(self) -> int:
        """Algorithmic real flops: 8 per complex multiply-add, n_ant*b*f per block."""
        return int(sum(8 * self.n_ant * self.b * f * n
                       for f, n in zip(self.f_of_group, self.n_blocks)))

    def algorithmic_bytes(self, s_bytes_per_elem: int = 8, w_bytes_per_elem: int = 8,
                          r_bytes_per_elem: int = 8) -> int:
        """Bytes a perfect implementation moves: each S and R once, each used W once."""
        used = sorted(set(self.prec))
        w = sum(self.W[p].size for p in used) * w_bytes_per_elem
        s = sum(s_.size for s_ in self.S) * s_bytes_per_elem
        r = self.total_blocks * self.n_ant * self.b * r_bytes_per_elem
        return int(w + s + r)

    # ---- memory layout (offsets only; no product arithmetic) ----
    def pack_W(self, dtype=np.complex64) -> Tuple[np.ndarray, List[int]]:
        """All precoders packed back to back (row-major n_ant x f each)."""
        flat = np.concatenate([w.astype(dtype).ravel() for w in self.W]) if self.W else np.zeros(0, dtype)
        f = [int(w.shape[1]) for w in self.W]
        return np.ascontiguousarray(flat), f

    def pack_S(self, dtype=np.complex64) -> Tuple[np.ndarray, List[int]]:
        """All S blocks packed in group order; returns (flat, element offset of each group)."""
        offs, pos = [], 0
        for s in self.S:
            offs.append(pos)
            pos += s.size
        flat = (np.concatenate([s.astype(dtype).ravel() for s in self.S])
                if self.S else np.zeros(0, dtype))
        return np.ascontiguousarray(flat), offs

    def r_offsets(self) -> List[int]:
        """Element offset of each group's first R block when R is packed in group order."""
        offs, pos = [], 0
        for n in self.n_blocks:
            offs.append(pos)
            pos += n * self.n_ant * self.b
        return offs

    def rounded(self, dtype=np.complex64) -> "Batch":
        """The same batch with every value rounded to dtype and widened back to complex128."""
        return Batch([w.astype(dtype).astype(np.complex128) for w in self.W], list(self.prec),
                     [s.astype(dtype).astype(np.complex128) for s in self.S], self.name,
                     self.seed, self.n_ant, self.b, dict(self.meta))


def _shared_precoder_batch(rng, n_prec, f, per_group, s_draw, name, seed, n_ant=N_ANT, b=B_RE,
                           w_draw=None) -> Batch:
    w_draw = w_draw or (lambda: precoder_unit_columns(rng, n_ant, f))
    W = [w_draw() for _ in range(n_prec)]
    S = [s_draw((per_group, f, b)) for _ in range(n_prec)]
    return Batch(W, list(range(n_prec)), S, name, seed, n_ant, b)


def config_small(seed: int = 0, n_blocks: int = 1024, f: int = 8) -> Batch:
    """One 64 x f unit-column complex-Gaussian precoder applied to n_blocks 16-QAM
    blocks of f x 60 (unit average power). Defaults: the 64x8, 1,024-block case."""
    rng = np.random.default_rng(seed)
    W = [precoder_unit_columns(rng, N_ANT, f)]
    S = [qam_symbols(rng, 16, (n_blocks, f, B_RE))]
    return Batch(W, [0], S, f"small_f{f}_x{n_blocks}", seed)


def config_fullband(seed: int = 2, n_rb: int = 273, n_sym: int = 14, f: int = 36,
                    qam: int = 64) -> Batch:
    """Full band: one unit-column precoder per resource block, shared by that
    block's n_sym OFDM symbols; S is unit-power M-QAM. Defaults: 273 x 14 = 3,822
    blocks at f = 36, 64-QAM."""
    rng = np.random.default_rng(seed)
    return _shared_precoder_batch(rng, n_rb, f, n_sym, lambda sh: qam_symbols(rng, qam, sh),
                                  f"fullband_f{f}_rb{n_rb}x{n_sym}", seed)


def config_uneven(seed: int = 3, n_blocks: int = 16384, f_max: int = F_MAX,
                  mean_group: float = 14.0, max_group: int = 64) -> Batch:
    """Uneven batch: group sizes geometric(mean 14) capped at 64, f ~ U{0..f_max}
    per group (shared by the group's blocks since they share one 64 x f W),
    QAM order drawn uniformly per group from QPSK/16/64/256."""
    rng = np.random.default_rng(seed)
    sizes = geometric_group_sizes(rng, n_blocks, mean_group, max_group)
    W, S = [], []
    for g in sizes:
        f = int(rng.integers(0, f_max + 1))
        order = int(rng.choice(QAM_ORDERS))
        W.append(precoder_unit_columns(rng, N_ANT, f))
        S.append(qam_symbols(rng, order, (g, f, B_RE)))
    return Batch(W, list(range(len(sizes))), S, f"uneven_x{n_blocks}", seed)


def config_reduced(seed: int = 4, copies: int = 8, n_rb: int = 273, n_sym: int = 14,
                   f: int = 36, noise_var: float = 1e-3) -> Batch:
    """Reduced-precision workload: the full-band f = 36 case repeated `copies`
    times with independent precoders; S is unit-power 256-QAM plus CN(0, 1e-3)
    noise (complex variance 1e-3, 5e-4 per real component)."""
    rng = np.random.default_rng(seed)
    n = copies * n_rb
    return _shared_precoder_batch(
        rng, n, f, n_sym,
        lambda sh: qam_symbols(rng, 256, sh) + complex_noise(rng, noise_var, sh),
        f"reduced_f{f}_x{copies}", seed)


def config_exact_integer(seed: int = 7, f_list: Sequence[int] = (0, 1, 7, 8, 9, 16, 17, 36),
                         blocks_per_group: Sequence[int] = (1, 2, 3), qam: int = 16,
                         wlim: int = 2) -> Batch:
    """Exact-arithmetic batch: Gaussian-integer W in {-2..2}+i{-2..2} and
    unscaled odd-integer QAM symbols. Every product and partial sum is a small
    integer, exact in FP16, BF16, FP32 and FP64."""
    rng = np.random.default_rng(seed)
    W, S, prec = [], [], []
    gi = 0
    for f in f_list:
        for nb in blocks_per_group:
            W.append(integer_precoder(rng, N_ANT, f, wlim))
            S.append(qam_integer_symbols(rng, qam, (nb, f, B_RE)))
            prec.append(gi)
            gi += 1
    return Batch(W, prec, S, "exact_integer", seed)


@dataclass
class ServingJob:
    """One per-TTI beamforming job of a cell."""
    cell: int
    tti: int
    arrival_s: float  # scheduled arrival time, seconds from the start
    n_rb: int         # resource blocks; each has n_sym blocks sharing precoder rb
    f: int            # flows (precoder columns) in the cell's current epoch
    epoch: int        # precoder epoch = tti // epoch_ttis


def serving_schedule(seed: int = 5, n_cells: int = 8, n_tti: int = 20000, tti_s: float = 0.5e-3,
                     jitter_s: float = 50e-6, rb_range=(25, 273), f_range=(1, 36),
                     epoch_ttis: int = 10) -> List[ServingJob]:
    """Job arrivals: every cell emits one job per TTI at tti*0.5 ms plus N(0, 50 us)
    jitter (clipped at 0); n_rb ~ U{25..273} per job; f ~ U{1..36} per cell per
    10-TTI precoder epoch. Sorted by arrival time."""
    rng = np.random.default_rng(seed)
    n_epochs = (n_tti + epoch_ttis - 1) // epoch_ttis
    f_epoch = rng.integers(f_range[0], f_range[1] + 1, size=(n_cells, n_epochs))
    jobs: List[ServingJob] = []
    for t in range(n_tti):
        rbs = rng.integers(rb_range[0], rb_range[1] + 1, size=n_cells)
        jit = rng.normal(0.0, jitter_s, size=n_cells)
        for c in range(n_cells):
            e = t // epoch_ttis
            jobs.append(ServingJob(c, t, max(0.0, t * tti_s + float(jit[c])), int(rbs[c]),
                                   int(f_epoch[c, e]), e))
    jobs.sort(key=lambda j: (j.arrival_s, j.cell))
    return jobs


# --------------------------------------------------------------------------
# Fast-convolution filter inputs (Sec. III, filter equation and Fig. 4)
# --------------------------------------------------------------------------
@dataclass
class FilterBatch:
    """n_sig signal blocks of n complex samples (row-major, signal-major) and
    one filter sequence h of n_taps <= n taps (zero-padded to n by the filter)."""
    h: np.ndarray
    s: np.ndarray
    name: str = ""
    seed: int = 0

    @property
    def n(self) -> int:
        return int(self.s.shape[1])

    @property
    def n_sig(self) -> int:
        return int(self.s.shape[0])

    def algorithmic_bytes(self, elem_bytes: int = 8) -> int:
        """Each signal read once and each output written once (the 2048-point
        spectrum of the filter is read from cache, not counted)."""
        return int(2 * self.n_sig * self.n * elem_bytes)

    def flops(self) -> int:
        """Conventional count: 5 N log2 N real flops per complex FFT, two FFTs
        and one complex multiply (6 flops) per sample per signal."""
        n = self.n
        return int(self.n_sig * (2 * 5 * n * int(np.log2(n)) + 6 * n))

    def rounded(self, dtype=np.complex64) -> "FilterBatch":
        return FilterBatch(self.h.astype(dtype).astype(np.complex128), self.s.astype(dtype).astype(np.complex128),
                           self.name, self.seed)


def filter_taps(rng: np.random.Generator, n_taps: int, decay: float = 64.0) -> np.ndarray:
    """Channel-like FIR: h[m] ~ CN(0, e^{-m/decay}), normalised to unit energy."""
    m = np.arange(n_taps)
    h = complex_noise(rng, 1.0, (n_taps,)) * np.sqrt(np.exp(-m / decay))
    return h / np.sqrt(np.sum(np.abs(h) ** 2))


def filter_signals(rng: np.random.Generator, n_sig: int, n: int = FILTER_N) -> np.ndarray:
    """Time-domain samples CN(0, 1) (the sample statistics of an OFDM signal)."""
    return complex_noise(rng, 1.0, (n_sig, n))


def config_filter_small(seed: int = 10, n_sig: int = 64, n_taps: int = 256) -> FilterBatch:
    """64 blocks of 2048 samples, a 256-tap filter."""
    rng = np.random.default_rng(seed)
    return FilterBatch(filter_taps(rng, n_taps), filter_signals(rng, n_sig), f"filter_x{n_sig}", seed)


def config_filter_tti(seed: int = 11, n_ant: int = N_ANT, n_sym: int = 14, n_taps: int = 256) -> FilterBatch:
    """One slot: one 2048-sample block per antenna and OFDM symbol, 64 x 14 = 896."""
    rng = np.random.default_rng(seed)
    return FilterBatch(filter_taps(rng, n_taps), filter_signals(rng, n_ant * n_sym),
                       f"filter_tti_{n_ant}x{n_sym}", seed)


def config_filter_bench(seed: int = 12, n_ant: int = N_ANT, n_sym: int = 14, n_slots: int = 16,
                        n_taps: int = 256) -> FilterBatch:
    """16 slots of 64 antennas x 14 symbols: 14,336 blocks, 235 MB in and out."""
    rng = np.random.default_rng(seed)
    return FilterBatch(filter_taps(rng, n_taps), filter_signals(rng, n_ant * n_sym * n_slots),
                       f"filter_{n_slots}slots", seed)
