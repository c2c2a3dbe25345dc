"""GPU parity of the fast-convolution filter y = IFFT(MULT(FFT(s))) (Sec. III,
filter equation, Fig. 4; N = 2048) against the FP64 oracle, through the C ABI.

Tolerance: relative Frobenius error <= 1e-5 over the checked signals. An FP32
radix-16/16/8 transform accumulates about log2(N) * 2^-24 ~ 7e-7 of relative
rms error per transform; two transforms, the spectrum product and the FP32
twiddles stay several times below 1e-5, the bound used for every FP32 path.
Outputs are NaN-poisoned before each run, so unwritten samples fail.
"""
import numpy as np
import pytest

import oracle
import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1810_11451_gb300 as bf  # noqa: E402

TOL = 1e-5
N = wl.FILTER_N


@pytest.fixture(scope="module")
def filt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    f = bf.bf_filter_create(N)
    yield f
    bf.bf_filter_destroy(f)


def dev_c64(a):
    flat = np.ascontiguousarray(np.asarray(a, dtype=np.complex64)).view(np.float32)
    return torch.from_numpy(flat.copy()).cuda()


def host_c64(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.complex64)


def run(filt, h, s, set_taps=True):
    if set_taps:
        bf.bf_filter_set_taps(filt, dev_c64(h), len(h))
    s_d = dev_c64(s)
    y_d = torch.full_like(s_d, float("nan"))
    bf.bf_filter_apply(filt, s_d, s.shape[0], y_d)
    return host_c64(y_d).reshape(s.shape)


def rel(y, ref):
    return float(np.linalg.norm(y - ref) / np.linalg.norm(ref))


def test_spectrum_matches_definition_dft(filt):
    b = wl.config_filter_small()
    bf.bf_filter_set_taps(filt, dev_c64(b.h), len(b.h))
    H_d = torch.full((2 * N,), float("nan"), device="cuda")
    bf.bf_filter_spectrum(filt, H_d)
    H = host_c64(H_d)
    hp = np.zeros(N, complex)
    hp[:len(b.h)] = b.h.astype(np.complex64)
    ref = oracle.dft(hp)
    assert np.all(np.isfinite(H)) and rel(H, ref) <= TOL


def test_small_batch(filt):
    b = wl.config_filter_small().rounded()
    y = run(filt, b.h, b.s)
    assert np.all(np.isfinite(y))
    e = rel(y, oracle.circular_filter(b.h, b.s))
    assert e <= TOL, e


def test_closed_forms(filt):
    """h = delta gives y = s; s = delta[n - n0] gives y = h shifted by n0 (with the wrap)."""
    rng = np.random.default_rng(3)
    s = (rng.normal(size=(5, N)) + 1j * rng.normal(size=(5, N))).astype(np.complex64)
    y = run(filt, np.array([1.0 + 0j]), s)
    assert rel(y, s) <= 1e-6
    h = wl.config_filter_small().h.astype(np.complex64)
    imp = np.zeros((4, N), np.complex64)
    shifts = [0, 1, 1000, N - 1]
    for i, n0 in enumerate(shifts):
        imp[i, n0] = 1
    y = run(filt, h, imp)
    hp = np.zeros(N, np.complex64)
    hp[:len(h)] = h
    for i, n0 in enumerate(shifts):
        assert rel(y[i], np.roll(hp, n0)) <= TOL


@pytest.mark.parametrize("n_taps", [1, 2, 2047, 2048])
def test_tap_counts(filt, n_taps):
    """Filter sequences from one tap to the full 2048, against the oracle."""
    rng = np.random.default_rng(n_taps)
    h = (rng.normal(size=n_taps) + 1j * rng.normal(size=n_taps)).astype(np.complex64)
    s = (rng.normal(size=(6, N)) + 1j * rng.normal(size=(6, N))).astype(np.complex64)
    y = run(filt, h, s)
    assert np.all(np.isfinite(y)) and rel(y, oracle.circular_filter(h, s)) <= TOL


def assert_per_block(y, ref, what):
    """Every block within TOL of the oracle (relative error of the block)."""
    assert np.all(np.isfinite(y)), f"{what}: unwritten (NaN) samples"
    d = (y.astype(np.complex128) - ref).reshape(ref.shape[0], -1)
    r = ref.reshape(ref.shape[0], -1)
    e = np.sqrt(np.sum(np.abs(d) ** 2, axis=1) / np.sum(np.abs(r) ** 2, axis=1))
    k = int(np.argmax(e))
    assert e[k] <= TOL, f"{what}: block {k}: error {e[k]:.3e} > {TOL:.0e}"
    return float(e[k])


@pytest.mark.parametrize("n_sig", [1, 3, 607, 1001, 2000])
def test_ragged_counts(filt, n_sig):
    """Counts that leave teams idle, and counts above the number of resident
    teams that make teams loop; every signal is checked."""
    rng = np.random.default_rng(n_sig)
    b = wl.config_filter_small()
    s = (rng.normal(size=(n_sig, N)) + 1j * rng.normal(size=(n_sig, N))).astype(np.complex64)
    y = run(filt, b.h.astype(np.complex64), s)
    ref = oracle.circular_filter(b.h.astype(np.complex64), s)
    assert rel(y, ref) <= TOL
    assert_per_block(y, ref, f"{n_sig} signals")


_RAGGED_REFS = {}  # oracle outputs shared by the variants (same seeded signals)


@pytest.mark.parametrize("variant", range(len(bf.FILTER_VARIANTS)))
def test_ragged_counts_every_variant(filt, variant):
    """Every building block on counts that leave warps, pairs or teams idle
    (1 and 5 signals) and on one that makes them loop with a ragged last
    round (1,001): every signal against the oracle. y starts as NaN, so a
    block a kernel skipped fails too."""
    b = wl.config_filter_small()
    h = b.h.astype(np.complex64)
    try:
        bf.bf_filter_set_variant(filt, variant)
        for n_sig in (1, 5, 1001):
            rng = np.random.default_rng(1000 + n_sig)
            s = (rng.normal(size=(n_sig, N)) + 1j * rng.normal(size=(n_sig, N))).astype(np.complex64)
            if n_sig not in _RAGGED_REFS:
                _RAGGED_REFS[n_sig] = oracle.circular_filter(h, s)
            y = run(filt, h, s)
            assert_per_block(y, _RAGGED_REFS[n_sig], f"variant {variant}, {n_sig} signals")
    finally:
        bf.bf_filter_set_variant(filt, bf.FILTER_DEFAULT_VARIANT)


def test_full_size_every_block(filt):
    """The bench workload (16 slots x 64 antennas x 14 symbols = 14,336 blocks)
    in the bench's launch form (the default building block, 12 warps per CTA),
    every block against the oracle; the same batch through the 8-warp building
    block gives the same bits, and through the three-pass and two-warp ones
    every block is checked against the oracle too."""
    b = wl.config_filter_bench().rounded()
    y = run(filt, b.h, b.s)
    ref = oracle.circular_filter(b.h, b.s)
    e = rel(y, ref)
    assert e <= TOL
    worst = assert_per_block(y, ref, "full size")
    print(f"filter full size: batch {e:.3e}, worst block {worst:.3e}")
    try:
        bf.bf_filter_set_variant(filt, 2)
        y2 = run(filt, b.h, b.s, set_taps=False)
        assert np.array_equal(y2.view(np.uint64), y.view(np.uint64))
        bf.bf_filter_set_variant(filt, 4)
        y4 = run(filt, b.h, b.s, set_taps=False)
        worst4 = assert_per_block(y4, ref, "full size, three-pass")
        print(f"filter full size, three-pass: batch {rel(y4, ref):.3e}, worst block {worst4:.3e}")
        bf.bf_filter_set_variant(filt, 6)
        y6 = run(filt, b.h, b.s, set_taps=False)
        worst6 = assert_per_block(y6, ref, "full size, two warps per block")
        print(f"filter full size, two warps per block: batch {rel(y6, ref):.3e}, worst block {worst6:.3e}")
    finally:
        bf.bf_filter_set_variant(filt, bf.FILTER_DEFAULT_VARIANT)


def test_in_place_host_and_determinism(filt):
    b = wl.config_filter_tti().rounded()
    bf.bf_filter_set_taps(filt, dev_c64(b.h), len(b.h))
    s_d = dev_c64(b.s)
    y1 = torch.empty_like(s_d)
    bf.bf_filter_apply(filt, s_d, b.n_sig, y1)
    y2 = torch.empty_like(s_d)
    bf.bf_filter_apply(filt, s_d, b.n_sig, y2)
    torch.cuda.synchronize()
    assert torch.equal(y1.view(torch.int32), y2.view(torch.int32))
    inplace = s_d.clone()
    bf.bf_filter_apply(filt, inplace, b.n_sig, inplace)
    s_h = torch.from_numpy(np.ascontiguousarray(b.s.astype(np.complex64)).view(np.float32).copy()).pin_memory()
    y_h = torch.full_like(s_h, float("nan")).pin_memory()
    bf.bf_filter_apply_host(filt, s_h, b.n_sig, y_h)
    torch.cuda.synchronize()
    assert torch.equal(inplace.view(torch.int32), y1.view(torch.int32))
    assert torch.equal(y_h.view(torch.int32), y1.cpu().view(torch.int32))


def test_errors(filt):
    with pytest.raises(bf.BfError) as ei:
        bf.bf_filter_create(1024)
    assert ei.value.status == bf.BF_EINVAL
    h = dev_c64(np.ones(4))
    for n_taps in (0, N + 1):
        with pytest.raises(bf.BfError) as ei:
            bf.bf_filter_set_taps(filt, h, n_taps)
        assert ei.value.status == bf.BF_EINVAL
    f2 = bf.bf_filter_create(N)
    try:
        assert bf.bf_filter_get_variant(f2) == bf.FILTER_DEFAULT_VARIANT
        s = dev_c64(np.ones((2, N))).view(-1)  # flat float32 view of two blocks
        with pytest.raises(bf.BfError) as ei:
            bf.bf_filter_apply(f2, s, 2, s)
        assert ei.value.status == bf.BF_ENOTFOUND
        bf.bf_filter_set_taps(f2, h, 4)
        with pytest.raises(bf.BfError) as ei:  # overlapping (16 bytes apart) but not equal
            bf.bf_filter_apply(f2, s, 1, s[4:])
        assert ei.value.status == bf.BF_EINVAL and "overlap" in str(ei.value)
        out = torch.empty_like(s)
        with pytest.raises(bf.BfError) as ei:  # 8-byte aligned only
            bf.bf_filter_apply(f2, s[2:], 1, out)
        assert ei.value.status == bf.BF_EINVAL and "aligned" in str(ei.value)
        bf.bf_filter_apply(f2, s, 0, s)  # no-op
    finally:
        bf.bf_filter_destroy(f2)


def test_host_path_pipelines_across_streams(filt):
    """Host-buffer calls alternating two streams and two buffer pairs, never
    synchronised in between: every call's output equals the device path bit
    for bit."""
    b = wl.config_filter_tti().rounded()
    bf.bf_filter_set_taps(filt, dev_c64(b.h), len(b.h))
    s_d = dev_c64(b.s)
    y_d = torch.empty_like(s_d)
    bf.bf_filter_apply(filt, s_d, b.n_sig, y_d)
    torch.cuda.synchronize()
    want = y_d.cpu().view(torch.int32)
    s_h = [torch.from_numpy(np.ascontiguousarray(b.s.astype(np.complex64)).view(np.float32).copy()).pin_memory()
           for _ in range(2)]
    y_h = [torch.full_like(s_h[0], float("nan")).pin_memory() for _ in range(2)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for rep in range(6):
        k = rep % 2
        if rep >= 2:
            streams[k].synchronize()
            assert torch.equal(y_h[k].view(torch.int32), want), f"call {rep - 2}"
            y_h[k].fill_(float("nan"))
        bf.bf_filter_apply_host(filt, s_h[k], b.n_sig, y_h[k], streams[k])
    for k in range(2):
        streams[k].synchronize()
        assert torch.equal(y_h[k].view(torch.int32), want)


def test_independent_input_keeps_the_y_side_ordered(filt):
    """With s declared independent of pending filter launches, a call reads and
    transforms s while the previous launch finishes but writes y only after
    it: call B writes its y over the s that call A (launched just before) is
    still reading. Over repeated pairs both outputs equal the same calls run
    alone, bit for bit; the setter rejects values other than 0 and 1."""
    b = wl.config_filter_tti().rounded()  # 896 blocks
    bf.bf_filter_set_taps(filt, dev_c64(b.h), len(b.h))
    sa = dev_c64(b.s).view(-1)
    sb = dev_c64(b.s[::-1].copy()).view(-1)
    ya_ref, yb_ref = torch.empty_like(sa), torch.empty_like(sb)
    bf.bf_filter_apply(filt, sa, b.n_sig, ya_ref)
    bf.bf_filter_apply(filt, sb, b.n_sig, yb_ref)
    torch.cuda.synchronize()
    big = torch.empty_like(sa)        # A reads its s here; B writes its y here
    ya = torch.empty_like(sa)
    bf.bf_filter_set_s_independent(filt, True)
    try:
        for rep in range(20):
            big.copy_(sa)             # a copy, not a filter launch, writes A's s
            ya.fill_(float("nan"))
            bf.bf_filter_apply(filt, big, b.n_sig, ya)
            bf.bf_filter_apply(filt, sb, b.n_sig, big)
            torch.cuda.synchronize()
            assert torch.equal(ya.view(torch.int32), ya_ref.view(torch.int32)), f"A, pair {rep}"
            assert torch.equal(big.view(torch.int32), yb_ref.view(torch.int32)), f"B, pair {rep}"
        assert bf.lib().bf_filter_set_s_independent(filt, 2) == bf.BF_EINVAL
    finally:
        bf.bf_filter_set_s_independent(filt, False)


def test_variants_bit_identical_and_accurate(filt):
    """The one-warp two-pass variants (11, 10, 8, 6 and 12 warps per CTA) give
    the same bits; the three-pass and two-warp variants round differently but
    every block stays within the tolerance of the oracle."""
    b = wl.config_filter_tti().rounded()  # 896 blocks
    bf.bf_filter_set_taps(filt, dev_c64(b.h), len(b.h))
    s_d = dev_c64(b.s)
    outs = {}
    try:
        for v in range(7):
            bf.bf_filter_set_variant(filt, v)
            y_d = torch.full_like(s_d, float("nan"))
            bf.bf_filter_apply(filt, s_d, b.n_sig, y_d)
            outs[v] = host_c64(y_d).reshape(b.n_sig, N)
        for v in (1, 2, 3, 5):
            assert np.array_equal(outs[v].view(np.uint64), outs[0].view(np.uint64)), f"variant {v}"
        assert bf.FILTER_DEFAULT_VARIANT in (0, 1, 2, 3, 5)
        ref = oracle.circular_filter(b.h, b.s)
        for v in (0, 4, 6):
            assert_per_block(outs[v], ref, f"variant {v}")
        with pytest.raises(bf.BfError) as ei:
            bf.bf_filter_set_variant(filt, 7)
        assert ei.value.status == bf.BF_EINVAL
    finally:
        bf.bf_filter_set_variant(filt, bf.FILTER_DEFAULT_VARIANT)


def test_autotune_picks_fastest_accurate_and_round_trips(filt, tmp_path):
    """Tuning picks the fastest variant: the pick is the minimum of the timed
    variants and no slower than the default, the tuned filter gives that
    variant's bits and every block stays within the tolerance of the oracle,
    and the choice saves and loads on this GPU; a table from another target or
    of the product kind is refused and leaves the filter unchanged."""
    b = wl.config_filter_tti().rounded()
    bf.bf_filter_set_taps(filt, dev_c64(b.h), len(b.h))
    s_d = dev_c64(b.s)
    try:
        for indep, n_tune in ((True, 112), (False, 112), (False, 4096)):
            bf.bf_filter_set_s_independent(filt, indep)  # tuning times the launch form in use
            v = bf.bf_filter_autotune(filt, n_tune)
            times = {k: bf.bf_filter_tune_query(filt, k) for k in range(len(bf.FILTER_VARIANTS))}
            assert all(t > 0 and n == n_tune for t, n in times.values()), times
            assert times[v][0] == min(t for t, _ in times.values())
            assert times[v][0] <= times[bf.FILTER_DEFAULT_VARIANT][0]  # no slower than the default
            print(f"filter autotune on {n_tune} blocks ({'s independent' if indep else 'dependent'}): "
                  f"variant {v} ({bf.FILTER_VARIANTS[v]}), "
                  + ", ".join(f"{k}: {t:.2f}" for k, (t, _) in times.items()) + " us")
        y1 = torch.full_like(s_d, float("nan"))
        bf.bf_filter_apply(filt, s_d, b.n_sig, y1)
        torch.cuda.synchronize()
        bf.bf_filter_set_variant(filt, v)
        y0 = torch.empty_like(s_d)
        bf.bf_filter_apply(filt, s_d, b.n_sig, y0)
        torch.cuda.synchronize()
        assert torch.equal(y1.view(torch.int32), y0.view(torch.int32))
        assert_per_block(host_c64(y1).reshape(b.n_sig, N), oracle.circular_filter(b.h, b.s), f"tuned variant {v}")
        bf.bf_filter_set_s_independent(filt, False)
        path = str(tmp_path / "filter_tune.json")
        bf.bf_filter_tune_save(filt, path)
        other = bf.bf_filter_create(N)
        try:
            bf.bf_filter_set_variant(other, 4)
            bf.bf_filter_tune_load(other, path)
            assert bf.bf_filter_get_variant(other) == v
            assert abs(bf.bf_filter_tune_query(other, 4)[0] - times[4][0]) < 1e-3
            txt = open(path).read()
            sms = torch.cuda.get_device_properties(0).multi_processor_count
            bad = str(tmp_path / "other_gpu.json")
            with open(bad, "w") as fh:
                fh.write(txt.replace(f'"sm_count": {sms}', f'"sm_count": {sms + 8}'))
            bf.bf_filter_set_variant(other, 4)
            with pytest.raises(bf.BfError) as ei:
                bf.bf_filter_tune_load(other, bad)
            assert ei.value.status == bf.BF_EINVAL and "not on this target" in str(ei.value)
            assert bf.bf_filter_get_variant(other) == 4
            with open(bad, "w") as fh:
                fh.write(txt.replace('"kind": "filter"', '"kind": "product"'))
            with pytest.raises(bf.BfError) as ei:
                bf.bf_filter_tune_load(other, bad)
            assert ei.value.status == bf.BF_EINVAL
        finally:
            bf.bf_filter_destroy(other)
    finally:
        bf.bf_filter_set_s_independent(filt, False)
        bf.bf_filter_set_variant(filt, bf.FILTER_DEFAULT_VARIANT)
