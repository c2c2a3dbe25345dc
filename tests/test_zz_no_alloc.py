"""bf_errnorm_noalloc: the accuracy report for callers that cannot allocate.

A real-time per-TTI loop (0.5 ms slots) must not call cudaMalloc/cudaFree,
which can synchronise the device and stall for an unbounded time, and some
callers have no plan or run where another allocator owns all device memory.
bf_errnorm_noalloc serves them: no plan, no allocation, a fixed scratch array
inside the library. This file checks, through the C ABI, that it returns what
the plan-based bf_errnorm and the oracle's FP64 sums return, on two calls in a row (the second call must
not see the first call's scratch), that a call leaves the device's free
memory unchanged (after a first call, which may load the library's device
code), and that it refuses batches larger than its scratch. The file is named
so that pytest collects it last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_1810_11451_gb300 as bf  # noqa: E402

RTOL = 1e-12  # the tolerance the other error-norm tests use (FP64 sums in a different order)


def _pair(rng, n, noise):
    Rref = rng.normal(size=(n, 64, 60)) + 1j * rng.normal(size=(n, 64, 60))
    R = (Rref + noise * (rng.normal(size=Rref.shape) + 1j * rng.normal(size=Rref.shape))).astype(np.complex64)
    Rd = torch.from_numpy(np.ascontiguousarray(R).view(np.float32)).cuda()
    Rrefd = torch.from_numpy(np.ascontiguousarray(Rref).view(np.float64)).cuda()
    return Rd, Rrefd


def test_noalloc_matches_plan_errnorm_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    plan = bf.bf_plan_create(64, 36, 60)
    try:
        rng = np.random.default_rng(77)
        # two calls in a row with different sizes and values: the second must
        # not pick up anything the first left in the shared scratch
        for n, noise in [(300, 1e-3), (41, 3e-2)]:
            Rd, Rrefd = _pair(rng, n, noise)
            want = bf.bf_errnorm(plan, Rd, Rrefd, n)
            got = bf.bf_errnorm_noalloc(Rd, Rrefd, n)
            assert np.allclose(got, want, rtol=RTOL, atol=0), (got, want)
            # and against the oracle's FP64 sums of the same arrays
            R = Rd.cpu().numpy().view(np.complex64).reshape(n, 64, 60)
            Rref = Rrefd.cpu().numpy().view(np.complex128).reshape(n, 64, 60)
            onum, oden = oracle.errnorm_blocks(R, Rref)
            assert np.allclose(got, (onum.sum(), oden.sum()), rtol=RTOL, atol=0), (got, onum.sum(), oden.sum())
        assert bf.bf_errnorm_noalloc(Rd, Rrefd, 0) == (0.0, 0.0)
        # the promise itself: with the module loaded, a call takes no device memory
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        got = bf.bf_errnorm_noalloc(Rd, Rrefd, 41)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, f"free device memory changed by {free0 - free1} bytes"
        assert np.allclose(got, want, rtol=RTOL, atol=0)
        with pytest.raises(bf.BfError) as ei:
            bf.bf_errnorm_noalloc(Rd, Rrefd, bf.BF_ERRNORM_NOALLOC_MAX_BLOCKS + 1)
        assert ei.value.status == bf.BF_EINVAL
        assert "65536" in bf.bf_last_error(None)
    finally:
        bf.bf_plan_destroy(plan)
