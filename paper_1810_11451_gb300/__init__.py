"""Python binding of libbf: batched complex beamforming R = W x S on GB300.

A thin ctypes layer over the C ABI in `include/bf.h`: every function here has
the C function's name and only marshals arguments (tensors become device or
host pointers via `data_ptr()`, streams become `cudaStream_t` handles). All
arithmetic runs in the library's CUDA kernels; there is no Python or CPU
fallback, and importing a function that needs the library raises when
`libbf.so` has not been built (`python -m paper_1810_11451_gb300.build`).

Statuses other than BF_OK raise `BfError` carrying the status and the plan's
`bf_last_error` text.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_int32, c_int64, c_void_p
from typing import Iterable, Optional, Sequence, Tuple

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbf.so")

# bf_status
BF_OK, BF_EINVAL, BF_ENOMEM, BF_EBUDGET, BF_ECUDA, BF_ETIMEOUT, BF_EAGAIN, BF_EBUSY, \
    BF_ENOTREADY, BF_ENOTFOUND = range(10)
# bf_precision
BF_FP32, BF_BF16, BF_FP16, BF_BF16X3, BF_FP32_3M, BF_TF32X3 = range(6)
PRECISIONS = {"fp32": BF_FP32, "bf16": BF_BF16, "fp16": BF_FP16, "bf16x3": BF_BF16X3, "fp32_3m": BF_FP32_3M,
              "tf32x3": BF_TF32X3}

N_ANT, B_RE, F_LIMIT = 64, 60, 36
S_BYTES_PER_F = B_RE * 8      # one flow row of a complex64 S block
R_BLOCK_BYTES = N_ANT * B_RE * 8
# bf_rtype: element type of R
BF_R_C64, BF_R_BF16, BF_R_FP16 = range(3)
R_ESIZE = {BF_R_C64: 8, BF_R_BF16: 4, BF_R_FP16: 4}


class bf_group(ctypes.Structure):
    """One group of blocks sharing precoder `prec_id` (byte offsets)."""
    _fields_ = [("prec_id", c_int32), ("n_blocks", c_int32), ("s_off", c_int64), ("r_off", c_int64)]


class bf_rlayout(ctypes.Structure):
    """Output layout of R: element (block n, antenna i, RE j) of a group at byte
    r_off + n*block_stride + i*row_stride + j*esize, in type `rtype`."""
    _fields_ = [("row_stride", c_int64), ("block_stride", c_int64), ("rtype", c_int32), ("reserved", c_int32)]


def antenna_major_layout(total_blocks: int, rtype: int = BF_R_C64) -> bf_rlayout:
    """The layout in which antenna i's total_blocks*60 resource elements form
    one contiguous row (block n of the batch at column n*60); a group whose
    first block has batch index n0 takes r_off = n0*60*esize."""
    e = R_ESIZE[int(rtype)]
    return bf_rlayout(int(total_blocks) * B_RE * e, B_RE * e, int(rtype), 0)


class BfError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{status_name(status)}: {message}")
        self.status = status


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded libbf.so (raises ImportError when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libbf.so is not built at {LIB_PATH}; run `python -m paper_1810_11451_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "bf_plan_create": (c_int, [c_int, c_int, c_int, POINTER(c_void_p)]),
            "bf_plan_destroy": (c_int, [c_void_p]),
            "bf_last_error": (c_char_p, [c_void_p]),
            "bf_status_string": (c_char_p, [c_int]),
            "bf_device_status": (c_int, [c_void_p]),
            "bf_selftest_wait_timeout": (c_int, [c_void_p, POINTER(c_int32)]),
            "bf_set_precoders": (c_int, [c_void_p, c_void_p, POINTER(c_int32), c_int32, c_int32, c_void_p]),
            "bf_reserve_precoders": (c_int, [c_void_p, c_int32]),
            "bf_reserve_worklists": (c_int, [c_void_p, c_int64]),
            "bf_set_host_chunks": (c_int, [c_void_p, c_int64, c_int64]),
            "bf_get_precoder_image": (c_int, [c_void_p, c_int32, c_int, c_void_p, c_int64, POINTER(c_int64)]),
            "bf_held_block_bytes": (c_int64, [c_int, c_int]),
            "bf_quantize_symbols": (c_int, [c_void_p, c_void_p, POINTER(bf_group), c_int32, c_int, c_void_p,
                                            POINTER(c_int64), c_void_p, c_void_p]),
            "bf_apply_batch": (c_int, [c_void_p, c_void_p, c_void_p, POINTER(bf_group), c_int32, c_int, c_void_p,
                                       c_void_p]),
            "bf_apply_batch_host": (c_int, [c_void_p, c_void_p, POINTER(bf_group), c_int32, c_int, c_void_p,
                                            c_void_p]),
            "bf_batch_create": (c_int, [c_void_p, c_void_p, c_void_p, POINTER(bf_group), c_int32, c_int, c_void_p,
                                        POINTER(c_void_p)]),
            "bf_apply_batch_rl": (c_int, [c_void_p, c_void_p, c_void_p, POINTER(bf_group), c_int32, c_int, c_void_p,
                                          POINTER(bf_rlayout), c_void_p]),
            "bf_batch_create_rl": (c_int, [c_void_p, c_void_p, c_void_p, POINTER(bf_group), c_int32, c_int,
                                           c_void_p, POINTER(bf_rlayout), POINTER(c_void_p)]),
            "bf_batch_launch": (c_int, [c_void_p, c_void_p]),
            "bf_batch_set_s_independent": (c_int, [c_void_p, c_int32]),
            "bf_batch_destroy": (c_int, [c_void_p]),
            "bf_errnorm": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_void_p, POINTER(c_double), c_void_p]),
            "bf_plan_launch_count": (c_int64, [c_void_p]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def status_name(s: int) -> str:
    try:
        return lib().bf_status_string(int(s)).decode()
    except Exception:
        return f"status {s}"


# ---------------------------------------------------------------- marshalling
def _ptr(x) -> Optional[int]:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if hasattr(x, "ctypes"):  # numpy array (host memory)
        return int(x.ctypes.data)
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream(s) -> Optional[int]:
    if s is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return int(torch.cuda.current_stream().cuda_stream) or None
        except Exception:
            pass
        return None
    if isinstance(s, int):
        return s or None
    return int(s.cuda_stream) or None


_GROUP_DTYPE = None


def make_groups(groups) -> Tuple[ctypes.Array, int]:
    """ctypes array of bf_group from (prec_id, n_blocks, s_off, r_off) rows: a
    list of tuples, an (n, 4) integer array, or an existing ctypes bf_group
    array (passed through). Built through numpy, so large lists are cheap."""
    global _GROUP_DTYPE
    if isinstance(groups, ctypes.Array) and groups._type_ is bf_group:
        return groups, len(groups)
    import numpy as np
    if _GROUP_DTYPE is None:
        _GROUP_DTYPE = np.dtype([("prec_id", "<i4"), ("n_blocks", "<i4"), ("s_off", "<i8"), ("r_off", "<i8")])
        assert _GROUP_DTYPE.itemsize == ctypes.sizeof(bf_group)
    rows = np.asarray(groups if not isinstance(groups, (list, tuple)) or len(groups) else np.zeros((0, 4)),
                      dtype=np.int64).reshape(-1, 4)
    st = np.zeros(max(1, len(rows)), dtype=_GROUP_DTYPE)
    if len(rows):
        st["prec_id"][:len(rows)] = rows[:, 0]
        st["n_blocks"][:len(rows)] = rows[:, 1]
        st["s_off"][:len(rows)] = rows[:, 2]
        st["r_off"][:len(rows)] = rows[:, 3]
    arr = (bf_group * len(st)).from_buffer(st)
    return arr, len(rows)


def _check(status: int, plan=None):
    if status != BF_OK:
        raise BfError(status, bf_last_error(plan))


# ---------------------------------------------------------------- C ABI, same names
def bf_plan_create(n_ant: int = N_ANT, f_max: int = F_LIMIT, b: int = B_RE) -> int:
    h = c_void_p()
    _check(lib().bf_plan_create(n_ant, f_max, b, ctypes.byref(h)))
    return h.value


def bf_plan_destroy(plan) -> None:
    _check(lib().bf_plan_destroy(plan))


def bf_last_error(plan=None) -> str:
    return (lib().bf_last_error(plan) or b"").decode()


def bf_status_string(s: int) -> str:
    return lib().bf_status_string(int(s)).decode()


def bf_device_status(plan) -> int:
    """BF_OK, or BF_ETIMEOUT if a kernel gave up on a bounded wait (cleared)."""
    return int(lib().bf_device_status(plan))


def bf_selftest_wait_timeout(plan) -> dict:
    """Run the bounded-wait self-test kernel (about 2 s); the plan's status
    word is left set (read it with bf_device_status)."""
    out = (c_int32 * 4)()
    _check(lib().bf_selftest_wait_timeout(plan, out), plan)
    return {"gave_up": int(out[0]), "wait_ms": int(out[1]), "left_on_abort": int(out[2]),
            "abort_wait_ms": int(out[3])}


def bf_reserve_precoders(plan, n_slots: int) -> None:
    _check(lib().bf_reserve_precoders(plan, int(n_slots)), plan)


BF_IMG_FP32, BF_IMG_BF16X2, BF_IMG_FP16, BF_IMG_TF32X2, BF_IMG_SCALE = range(5)


def bf_get_precoder_image(plan, slot: int, kind: int):
    """The slot's image of the given kind as a numpy uint8 array (host copy)."""
    import numpy as np
    n = c_int64()
    _check(lib().bf_get_precoder_image(plan, int(slot), int(kind), None, 0, ctypes.byref(n)), plan)
    out = np.zeros(max(1, n.value), dtype=np.uint8)
    _check(lib().bf_get_precoder_image(plan, int(slot), int(kind), out.ctypes.data, n.value, ctypes.byref(n)), plan)
    return out[:n.value]


def bf_set_host_chunks(plan, first_bytes: int, max_bytes: int) -> None:
    _check(lib().bf_set_host_chunks(plan, int(first_bytes), int(max_bytes)), plan)


def bf_reserve_worklists(plan, max_blocks: int) -> None:
    _check(lib().bf_reserve_worklists(plan, int(max_blocks)), plan)


def bf_set_precoders(plan, W_dev, f_list: Sequence[int], first_id: int = 0, stream=None) -> None:
    fa = (c_int32 * max(1, len(f_list)))(*[int(f) for f in f_list])
    _check(lib().bf_set_precoders(plan, _ptr(W_dev), fa, len(f_list), first_id, _stream(stream)), plan)


def bf_held_block_bytes(f: int, prec: int) -> int:
    return int(lib().bf_held_block_bytes(int(f), int(prec)))


def make_offsets(q_off) -> ctypes.Array:
    """ctypes int64 array of per-group byte offsets (built through numpy; an
    existing c_int64 array passes through)."""
    if isinstance(q_off, ctypes.Array) and q_off._type_ is c_int64:
        return q_off
    import numpy as np
    a = np.ascontiguousarray(np.asarray(q_off, dtype=np.int64).reshape(-1))
    if a.size == 0:
        a = np.zeros(1, np.int64)
    return (c_int64 * a.size).from_buffer(a.copy())


def bf_quantize_symbols(plan, S_dev, groups, prec: int, Sq_dev, q_off: Sequence[int], scale_dev,
                        stream=None) -> None:
    ga, n = make_groups(groups)
    qa = make_offsets(q_off)
    _check(lib().bf_quantize_symbols(plan, _ptr(S_dev), ga, n, int(prec), _ptr(Sq_dev), qa, _ptr(scale_dev),
                                     _stream(stream)), plan)


def bf_apply_batch(plan, S_dev, scale_dev, groups, prec: int, R_dev, stream=None) -> None:
    ga, n = make_groups(groups)
    _check(lib().bf_apply_batch(plan, _ptr(S_dev), _ptr(scale_dev), ga, n, int(prec), _ptr(R_dev),
                                _stream(stream)), plan)


def bf_apply_batch_rl(plan, S_dev, scale_dev, groups, prec: int, R_dev, layout: Optional[bf_rlayout],
                      stream=None) -> None:
    ga, n = make_groups(groups)
    lp = ctypes.byref(layout) if layout is not None else None
    _check(lib().bf_apply_batch_rl(plan, _ptr(S_dev), _ptr(scale_dev), ga, n, int(prec), _ptr(R_dev), lp,
                                   _stream(stream)), plan)


def bf_apply_batch_host(plan, S_host, groups, prec: int, R_host, stream=None) -> None:
    ga, n = make_groups(groups)
    _check(lib().bf_apply_batch_host(plan, _ptr(S_host), ga, n, int(prec), _ptr(R_host), _stream(stream)), plan)


def bf_batch_create(plan, S_dev, scale_dev, groups, prec: int, R_dev) -> int:
    ga, n = make_groups(groups)
    h = c_void_p()
    _check(lib().bf_batch_create(plan, _ptr(S_dev), _ptr(scale_dev), ga, n, int(prec), _ptr(R_dev),
                                 ctypes.byref(h)), plan)
    return h.value


def bf_batch_create_rl(plan, S_dev, scale_dev, groups, prec: int, R_dev, layout: Optional[bf_rlayout]) -> int:
    ga, n = make_groups(groups)
    h = c_void_p()
    lp = ctypes.byref(layout) if layout is not None else None
    _check(lib().bf_batch_create_rl(plan, _ptr(S_dev), _ptr(scale_dev), ga, n, int(prec), _ptr(R_dev), lp,
                                    ctypes.byref(h)), plan)
    return h.value


def bf_batch_launch(batch, stream=None) -> None:
    """Launch a prepared batch directly (one persistent kernel)."""
    st = lib().bf_batch_launch(batch, _stream(stream))
    if st != BF_OK:
        raise BfError(st, "bf_batch_launch failed")


def bf_batch_set_s_independent(batch, independent: bool = True) -> None:
    """Declare that no product launch writes the batch's S (see bf.h)."""
    st = lib().bf_batch_set_s_independent(batch, 1 if independent else 0)
    if st != BF_OK:
        raise BfError(st, "bf_batch_set_s_independent failed")


def bf_batch_launch_graph(batch, stream=None) -> None:
    """Replay the prepared batch's captured CUDA graph."""
    L = lib()
    L.bf_batch_launch_graph.restype = c_int
    L.bf_batch_launch_graph.argtypes = [c_void_p, c_void_p]
    st = L.bf_batch_launch_graph(batch, _stream(stream))
    if st != BF_OK:
        raise BfError(st, "bf_batch_launch_graph failed")


def bf_batch_destroy(batch) -> None:
    lib().bf_batch_destroy(batch)


def bf_errnorm(plan, R_dev, Rref_dev, n_blocks: int, per_block_dev=None, stream=None) -> Tuple[float, float]:
    """(sum |R - Rref|^2, sum |Rref|^2) over n_blocks blocks, in FP64."""
    tot = (c_double * 2)()
    _check(lib().bf_errnorm(plan, _ptr(R_dev), _ptr(Rref_dev), int(n_blocks), _ptr(per_block_dev), tot,
                            _stream(stream)), plan)
    return float(tot[0]), float(tot[1])


# ---------------------------------------------------------------- the filter (bf_filter.h)
FILTER_N = 2048


def _filter_sigs(L):
    if not getattr(L, "_filter_sigs", False):
        sig = {
            "bf_filter_create": (c_int, [c_int, POINTER(c_void_p)]),
            "bf_filter_destroy": (c_int, [c_void_p]),
            "bf_filter_last_error": (c_char_p, [c_void_p]),
            "bf_filter_set_taps": (c_int, [c_void_p, c_void_p, c_int, c_void_p]),
            "bf_filter_spectrum": (c_int, [c_void_p, c_void_p, c_void_p]),
            "bf_filter_apply": (c_int, [c_void_p, c_void_p, c_int64, c_void_p, c_void_p]),
            "bf_filter_apply_host": (c_int, [c_void_p, c_void_p, c_int64, c_void_p, c_void_p]),
            "bf_filter_launch_count": (c_int64, [c_void_p]),
            "bf_filter_set_s_independent": (c_int, [c_void_p, c_int32]),
            "bf_filter_set_variant": (c_int, [c_void_p, c_int32]),
            "bf_filter_get_variant": (c_int32, [c_void_p]),
            "bf_filter_autotune": (c_int, [c_void_p, c_int64, c_void_p]),
            "bf_filter_tune_query": (c_int, [c_void_p, c_int32, POINTER(c_double), POINTER(c_int64)]),
            "bf_filter_tune_save": (c_int, [c_void_p, c_char_p]),
            "bf_filter_tune_load": (c_int, [c_void_p, c_char_p]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        L._filter_sigs = True
    return L


def bf_filter_last_error(filt=None) -> str:
    return (_filter_sigs(lib()).bf_filter_last_error(filt) or b"").decode()


def _fcheck(status: int, filt=None):
    if status != BF_OK:
        raise BfError(status, bf_filter_last_error(filt))


def bf_filter_create(n: int = FILTER_N) -> int:
    h = c_void_p()
    _fcheck(_filter_sigs(lib()).bf_filter_create(int(n), ctypes.byref(h)))
    return h.value


def bf_filter_destroy(filt) -> None:
    _filter_sigs(lib()).bf_filter_destroy(filt)


def bf_filter_set_taps(filt, h_dev, n_taps: int, stream=None) -> None:
    _fcheck(_filter_sigs(lib()).bf_filter_set_taps(filt, _ptr(h_dev), int(n_taps), _stream(stream)), filt)


def bf_filter_spectrum(filt, H_dev, stream=None) -> None:
    _fcheck(_filter_sigs(lib()).bf_filter_spectrum(filt, _ptr(H_dev), _stream(stream)), filt)


def bf_filter_apply(filt, s_dev, n_sig: int, y_dev, stream=None) -> None:
    _fcheck(_filter_sigs(lib()).bf_filter_apply(filt, _ptr(s_dev), int(n_sig), _ptr(y_dev), _stream(stream)), filt)


def bf_filter_apply_host(filt, s_host, n_sig: int, y_host, stream=None) -> None:
    _fcheck(_filter_sigs(lib()).bf_filter_apply_host(filt, _ptr(s_host), int(n_sig), _ptr(y_host), _stream(stream)),
            filt)


def bf_filter_set_s_independent(filt, independent: bool = True) -> None:
    """Declare that no pending launch of the library writes the s of later calls (see bf_filter.h)."""
    _fcheck(_filter_sigs(lib()).bf_filter_set_s_independent(filt, 1 if independent else 0), filt)


FILTER_DEFAULT_VARIANT = 5  # two-pass, 12 warps per CTA, spectrum through L1
FILTER_VARIANTS = {0: "two-pass, 11 warps per CTA, spectrum through L1",
                   1: "two-pass, 10 warps per CTA, spectrum through L1", 2: "two-pass, 8 warps per CTA",
                   3: "two-pass, 6 warps per CTA", 4: "three-pass, 4 teams of 128 threads per CTA",
                   5: "two-pass, 12 warps per CTA, spectrum through L1",
                   6: "two-pass, two warps per block, 8 blocks per CTA"}


def bf_filter_set_variant(filt, variant: int) -> None:
    _fcheck(_filter_sigs(lib()).bf_filter_set_variant(filt, int(variant)), filt)


def bf_filter_get_variant(filt) -> int:
    return int(_filter_sigs(lib()).bf_filter_get_variant(filt))


def bf_filter_autotune(filt, n_sig: int, stream=None) -> int:
    """Time every variant on n_sig blocks (in the launch form the filter uses), select the fastest; returns it."""
    _fcheck(_filter_sigs(lib()).bf_filter_autotune(filt, int(n_sig), _stream(stream)), filt)
    return bf_filter_get_variant(filt)


def bf_filter_tune_query(filt, variant: int) -> Tuple[float, int]:
    """(microseconds per launch, n_sig timed) of one variant (0.0 if not timed)."""
    us, n = c_double(), c_int64()
    _fcheck(_filter_sigs(lib()).bf_filter_tune_query(filt, int(variant), ctypes.byref(us), ctypes.byref(n)), filt)
    return float(us.value), int(n.value)


def bf_filter_tune_save(filt, path: str) -> None:
    _fcheck(_filter_sigs(lib()).bf_filter_tune_save(filt, path.encode()), filt)


def bf_filter_tune_load(filt, path: str) -> None:
    _fcheck(_filter_sigs(lib()).bf_filter_tune_load(filt, path.encode()), filt)


def bf_filter_launch_count(filt) -> int:
    return int(_filter_sigs(lib()).bf_filter_launch_count(filt))


def bf_plan_launch_count(plan) -> int:
    return int(lib().bf_plan_launch_count(plan))


def _tune_sigs(L):
    if not getattr(L, "_tune_sigs", False):
        L.bf_autotune.restype = c_int
        L.bf_autotune.argtypes = [c_void_p, c_int, c_void_p]
        L.bf_tune_query.restype = c_int
        L.bf_tune_query.argtypes = [c_void_p, c_int, c_int32, POINTER(c_double), POINTER(c_int32),
                                    POINTER(c_int32)]
        L.bf_tune_save.restype = c_int
        L.bf_tune_save.argtypes = [c_void_p, c_char_p]
        L.bf_tune_load.restype = c_int
        L.bf_tune_load.argtypes = [c_void_p, c_char_p]
        L._tune_sigs = True
    return L


def bf_autotune(plan, prec: int, stream=None) -> None:
    _check(_tune_sigs(lib()).bf_autotune(plan, int(prec), _stream(stream)), plan)


BF_TARGET_FP32, BF_TARGET_BF16 = 0, 1


def bf_select_form(plan, target: int, groups) -> Tuple[int, float]:
    """(form, predicted marginal ns) chosen from the tuned table for these groups."""
    L = lib()
    L.bf_select_form.restype = c_int
    L.bf_select_form.argtypes = [c_void_p, c_int, POINTER(bf_group), c_int32, POINTER(c_int), POINTER(c_double)]
    ga, n = make_groups(groups)
    p, ns = c_int(), c_double()
    _check(L.bf_select_form(plan, int(target), ga, n, ctypes.byref(p), ctypes.byref(ns)), plan)
    return p.value, ns.value


def bf_tune_query(plan, prec: int, f: int) -> dict:
    ns, tb, tuned = c_double(), c_int32(), c_int32()
    _check(_tune_sigs(lib()).bf_tune_query(plan, int(prec), int(f), ctypes.byref(ns), ctypes.byref(tb),
                                           ctypes.byref(tuned)), plan)
    return {"ns_per_block": ns.value, "tile_blocks": tb.value, "tuned": bool(tuned.value)}


def bf_tune_save(plan, path: str) -> None:
    _check(_tune_sigs(lib()).bf_tune_save(plan, path.encode()), plan)


def bf_tune_load(plan, path: str) -> None:
    _check(_tune_sigs(lib()).bf_tune_load(plan, path.encode()), plan)


def bf_tune_check_target(path: str, device_name: str, cc: int, sm_count: int) -> None:
    """Raises BfError (BF_EINVAL) unless the table at path was measured on this target."""
    L = lib()
    L.bf_tune_check_target.restype = c_int
    L.bf_tune_check_target.argtypes = [ctypes.c_char_p, ctypes.c_char_p, c_int32, c_int32]
    _check(L.bf_tune_check_target(path.encode(), device_name.encode(), int(cc), int(sm_count)))


BF_ERRNORM_NOALLOC_MAX_BLOCKS = 65536


def bf_errnorm_noalloc(R_dev, Rref_dev, n_blocks: int, stream=None) -> Tuple[float, float]:
    """bf_errnorm without a plan and without any device allocation (fixed
    in-library scratch, at most BF_ERRNORM_NOALLOC_MAX_BLOCKS blocks)."""
    L = lib()
    L.bf_errnorm_noalloc.restype = c_int
    L.bf_errnorm_noalloc.argtypes = [c_void_p, c_void_p, c_int64, POINTER(c_double), c_void_p]
    tot = (c_double * 2)()
    st = L.bf_errnorm_noalloc(_ptr(R_dev), _ptr(Rref_dev), int(n_blocks), tot, _stream(stream))
    if st != BF_OK:
        raise BfError(st, bf_last_error(None))
    return float(tot[0]), float(tot[1])


def bf_measure_fp32_peak(iters: int = 20000, reps: int = 5, mode: int = 0, stream=None) -> Tuple[float, float]:
    """(TFLOP/s, ms per launch) of the CUDA cores' FP32 FMA probe: mode 0 scalar, 1 packed FP32x2,
    2 packed FP32x2 in a register-blocked outer-product operand pattern."""
    L = lib()
    L.bf_measure_fp32_peak.restype = c_int
    L.bf_measure_fp32_peak.argtypes = [c_int32, c_int32, c_int32, POINTER(c_double), POINTER(c_double), c_void_p]
    t, ms = c_double(), c_double()
    st = L.bf_measure_fp32_peak(int(iters), int(reps), int(mode), ctypes.byref(t), ctypes.byref(ms),
                                _stream(stream))
    if st != BF_OK:
        raise BfError(st, bf_last_error(None))
    return float(t.value), float(ms.value)


# ---------------------------------------------------------------- serving (bf_serve.h)
class bf_serve_config(ctypes.Structure):
    _fields_ = [("n_slots", c_int32), ("max_batch_jobs", c_int32), ("queue_capacity", c_int32),
                ("fake_device_us", c_int32), ("hbm_budget_bytes", c_int64), ("deadline_us", c_int32),
                ("slot_timeout_us", c_int32)]


class bf_job(ctypes.Structure):
    _fields_ = [("cell", c_int32), ("n_groups", c_int32), ("groups", POINTER(bf_group)), ("prec", c_int32),
                ("pad", c_int32), ("S_dev", c_void_p), ("R_dev", c_void_p), ("arrival_ns", c_int64)]


class bf_replay_item(ctypes.Structure):
    """One entry of an arrival schedule for bf_serve_replay."""
    _fields_ = [("job", bf_job), ("W_dev", c_void_p), ("f_host", POINTER(c_int32)), ("n_prec", c_int32),
                ("first_id", c_int32)]


class bf_serve_stats(ctypes.Structure):
    _fields_ = [("submitted", c_int64), ("completed", c_int64), ("launches", c_int64),
                ("rejected_budget", c_int64), ("rejected_full", c_int64), ("budget_waits", c_int64),
                ("max_inflight_bytes", c_int64), ("max_busy_slots", c_int32), ("max_jobs_per_launch", c_int32),
                ("over_deadline", c_int64), ("timed_out", c_int64), ("deadline_ns", c_int64),
                ("slot_timeout_ns", c_int64), ("worst_latency_ns", c_int64), ("worst_submit_ns", c_int64),
                ("worst_queue_ns", c_int64), ("worst_launch_ns", c_int64), ("worst_device_ns", c_int64),
                ("over_by_submit", c_int64), ("over_by_queue", c_int64), ("over_by_launch", c_int64),
                ("over_by_device", c_int64), ("sum_submit_ns", c_int64), ("sum_queue_ns", c_int64),
                ("sum_launch_ns", c_int64), ("sum_device_ns", c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _serve_sigs(L):
    if getattr(L, "_serve_sigs", False):
        return L
    for name, res, args in [
        ("bf_now_ns", c_int64, []),
        ("bf_serve_create", c_int, [c_void_p, POINTER(bf_serve_config), POINTER(c_void_p)]),
        ("bf_serve_destroy", c_int, [c_void_p, c_int64]),
        ("bf_serve_set_precoders", c_int, [c_void_p, c_void_p, POINTER(c_int32), c_int32, c_int32]),
        ("bf_submit", c_int, [c_void_p, POINTER(bf_job), POINTER(ctypes.c_uint64)]),
        ("bf_poll", c_int, [c_void_p, ctypes.c_uint64, POINTER(c_int), POINTER(c_double)]),
        ("bf_wait", c_int, [c_void_p, ctypes.c_uint64, c_int64, POINTER(c_double)]),
        ("bf_serve_pause", c_int, [c_void_p, c_int32]),
        ("bf_serve_set_budget", c_int, [c_void_p, c_int64]),
        ("bf_serve_get_stats", c_int, [c_void_p, POINTER(bf_serve_stats)]),
        ("bf_serve_replay", c_int, [c_void_p, POINTER(bf_replay_item), c_int32, c_int64,
                                    POINTER(ctypes.c_uint64), POINTER(c_int64)]),
    ]:
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    L._serve_sigs = True
    return L


def bf_now_ns() -> int:
    return int(_serve_sigs(lib()).bf_now_ns())


def bf_serve_create(plan, n_slots: int = 4, max_batch_jobs: int = 16, queue_capacity: int = 4096,
                    hbm_budget_bytes: int = 8 << 30, fake_device_us: int = 0, deadline_us: int = 0,
                    slot_timeout_us: int = 0) -> int:
    L = _serve_sigs(lib())
    cfg = bf_serve_config(n_slots, max_batch_jobs, queue_capacity, fake_device_us, hbm_budget_bytes,
                          deadline_us, slot_timeout_us)
    h = c_void_p()
    _check(L.bf_serve_create(plan, ctypes.byref(cfg), ctypes.byref(h)), plan)
    return h.value


def bf_serve_destroy(srv, timeout_us: int = 10_000_000) -> None:
    st = _serve_sigs(lib()).bf_serve_destroy(srv, int(timeout_us))
    if st != BF_OK:
        raise BfError(st, "bf_serve_destroy: jobs still queued or running")


def bf_serve_set_precoders(srv, W_dev, f_list: Sequence[int], first_id: int = 0) -> None:
    fa = (c_int32 * max(1, len(f_list)))(*[int(f) for f in f_list])
    st = _serve_sigs(lib()).bf_serve_set_precoders(srv, _ptr(W_dev), fa, len(f_list), int(first_id))
    if st != BF_OK:
        raise BfError(st, "bf_serve_set_precoders failed")


def bf_submit(srv, groups, prec: int, S_dev, R_dev, cell: int = 0, arrival_ns: int = 0) -> int:
    """Queue a job; returns its ticket. Raises BfError (status BF_EBUDGET,
    BF_EAGAIN, BF_ENOTFOUND, BF_EINVAL) when it is refused."""
    ga, n = make_groups(groups)
    job = bf_job(int(cell), n, ga, int(prec), 0, _ptr(S_dev), _ptr(R_dev), int(arrival_ns))
    t = ctypes.c_uint64()
    st = _serve_sigs(lib()).bf_submit(srv, ctypes.byref(job), ctypes.byref(t))
    if st != BF_OK:
        raise BfError(st, bf_last_error(None))
    return int(t.value)


def bf_poll(srv, ticket: int) -> Tuple[bool, Optional[float]]:
    """(done, latency_us); the ticket is retired once done is returned True.
    A job that finished with an error (BF_ETIMEOUT from the watchdog, BF_ECUDA)
    raises BfError with that status; its ticket is retired too."""
    d, lat = c_int(), c_double()
    st = _serve_sigs(lib()).bf_poll(srv, ctypes.c_uint64(ticket), ctypes.byref(d), ctypes.byref(lat))
    if st != BF_OK:
        raise BfError(st, "bf_poll")
    return bool(d.value), (float(lat.value) if d.value else None)


def bf_wait(srv, ticket: int, timeout_us: int) -> float:
    lat = c_double()
    st = _serve_sigs(lib()).bf_wait(srv, ctypes.c_uint64(ticket), int(timeout_us), ctypes.byref(lat))
    if st != BF_OK:
        raise BfError(st, "bf_wait")
    return float(lat.value)


def bf_serve_pause(srv, paused: bool) -> None:
    _serve_sigs(lib()).bf_serve_pause(srv, int(bool(paused)))


def bf_serve_set_budget(srv, hbm_budget_bytes: int) -> None:
    _check(_serve_sigs(lib()).bf_serve_set_budget(srv, int(hbm_budget_bytes)))


def bf_serve_get_stats(srv) -> dict:
    s = bf_serve_stats()
    _check(_serve_sigs(lib()).bf_serve_get_stats(srv, ctypes.byref(s)))
    return s.as_dict()


def bf_serve_replay(srv, items, start_ns: int, tickets=None) -> Tuple[list, int]:
    """Replay a schedule (a ctypes array of bf_replay_item, arrivals relative
    to start_ns) in native code; returns (tickets, late submits). The GIL is
    released during the call. `tickets` (optional, a ctypes c_uint64 array
    of len(items), zeroed) receives each ticket as its job is submitted, so
    another thread can retire jobs while the replay runs."""
    n = len(items)
    if tickets is None:
        tickets = (ctypes.c_uint64 * max(1, n))()
    late = c_int64()
    _check(_serve_sigs(lib()).bf_serve_replay(srv, items, n, int(start_ns), tickets, ctypes.byref(late)))
    return [int(tickets[i]) for i in range(n)], int(late.value)


class bf_tile(ctypes.Structure):
    """One scheduled work item (see bf_schedule in bf.h)."""
    _fields_ = [("s_off", c_int64), ("r_off", c_int64), ("prec_id", c_int32), ("first_block", c_int32),
                ("f", ctypes.c_int16), ("n_blocks", ctypes.c_int16), ("flags", c_int32)]


def bf_schedule(f_of_slot: Sequence[int], groups, prec: int, held: bool, max_cta: int):
    """The host scheduler: returns (list of bf_tile, cta_begin list)."""
    L = lib()
    L.bf_schedule.restype = c_int32
    fa = (c_int32 * max(1, len(f_of_slot)))(*[int(f) for f in f_of_slot])
    ga, n = make_groups(groups)
    ncta = c_int32()
    nt = L.bf_schedule(fa, len(f_of_slot), ga, n, int(prec), int(bool(held)), int(max_cta), None, 0, None,
                       ctypes.byref(ncta))
    if nt < 0:
        raise BfError(-nt, "bf_schedule rejected its arguments")
    tiles = (bf_tile * max(1, nt))()
    begin = (c_int32 * (int(max_cta) + 1))()
    nt = L.bf_schedule(fa, len(f_of_slot), ga, n, int(prec), int(bool(held)), int(max_cta), tiles, nt, begin,
                       ctypes.byref(ncta))
    if nt < 0:
        raise BfError(-nt, "bf_schedule rejected its arguments")
    return list(tiles)[:nt], list(begin)[:ncta.value + 1]
