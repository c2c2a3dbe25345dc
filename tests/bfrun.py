"""Run a `workloads.Batch` through the C ABI on the GPU (test and bench helper).

Only memory layout and marshalling happens here: the batch is packed into
device buffers (complex64 interleaved, groups back to back), the precoders
are set, and `bf_apply_batch` (or the graph-captured or host-buffer entry
points) computes R. R is poisoned with NaN first so that an element a kernel
fails to write shows up.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional

import numpy as np

import paper_1810_11451_gb300 as bf

N_ANT, B_RE = bf.N_ANT, bf.B_RE
R_ELEMS = N_ANT * B_RE


@dataclass
class Layout:
    groups: list          # (prec_id, n_blocks, s_off, r_off) with byte offsets
    s_bytes: int
    r_blocks: int
    held_off: Optional[list] = None
    held_bytes: int = 0


def layout(batch, slot_base: int = 0, prec: int = bf.BF_FP32) -> Layout:
    groups, s_off, r_off = [], 0, 0
    held_off, h = [], 0
    for p, S in zip(batch.prec, batch.S):
        nb, f = S.shape[0], S.shape[1]
        groups.append((slot_base + p, nb, s_off, r_off))
        s_off += nb * f * B_RE * 8
        r_off += nb * R_ELEMS * 8
        held_off.append(h)
        if prec != bf.BF_FP32:
            h += nb * bf.bf_held_block_bytes(f, prec)
    return Layout(groups, s_off, r_off // (R_ELEMS * 8), held_off, h)


def to_device_c64(arr: np.ndarray, torch, device="cuda"):
    flat = np.ascontiguousarray(arr.astype(np.complex64)).view(np.float32)
    if flat.size == 0:
        flat = np.zeros(4, np.float32)
    return torch.from_numpy(flat).to(device)


def set_precoders(plan, batch, torch, slot_base: int = 0, stream=None):
    Wflat, fs = batch.pack_W()
    Wd = to_device_c64(Wflat, torch)
    bf.bf_set_precoders(plan, Wd, fs, slot_base, stream)
    torch.cuda.synchronize()
    return Wd


def split_R(R_t, batch, torch) -> List[np.ndarray]:
    torch.cuda.synchronize()
    r = R_t.cpu().numpy().view(np.complex64).reshape(-1, N_ANT, B_RE)
    out, pos = [], 0
    for nb in batch.n_blocks:
        out.append(r[pos:pos + nb])
        pos += nb
    return out


def run(plan, batch, prec: int, torch, held: bool = False, mode: str = "apply", slot_base: int = 0,
        set_w: bool = True, return_buffers: bool = False):
    """Compute R for every group; returns a list of complex64 (n_blocks, 64, 60) arrays."""
    if set_w:
        set_precoders(plan, batch, torch, slot_base)
    lay = layout(batch, slot_base, prec)
    Sflat, _ = batch.pack_S()
    R_t = torch.full((max(1, lay.r_blocks) * R_ELEMS * 2,), float("nan"), dtype=torch.float32, device="cuda")
    if mode == "host":
        S_h = torch.from_numpy(np.ascontiguousarray(Sflat.astype(np.complex64)).view(np.float32).copy()).pin_memory() \
            if Sflat.size else torch.zeros(4).pin_memory()
        R_h = torch.full(R_t.shape, float("nan"), dtype=torch.float32).pin_memory()
        bf.bf_apply_batch_host(plan, S_h, lay.groups, prec, R_h)
        torch.cuda.synchronize()
        R_t.copy_(R_h)
        return split_R(R_t, batch, torch)
    S_d = to_device_c64(Sflat, torch)
    scale = None
    S_use, groups = S_d, lay.groups
    if held:
        Sq = torch.zeros(max(16, lay.held_bytes) // 4 + 4, dtype=torch.float32, device="cuda")
        scale = torch.zeros(max(1, batch.total_blocks), dtype=torch.float32, device="cuda")
        bf.bf_quantize_symbols(plan, S_d, lay.groups, prec, Sq, lay.held_off, scale)
        S_use = Sq
        groups = [(g[0], g[1], lay.held_off[i], g[3]) for i, g in enumerate(lay.groups)]
    if mode == "apply":
        bf.bf_apply_batch(plan, S_use, scale, groups, prec, R_t)
    elif mode in ("batch", "graph"):
        h = bf.bf_batch_create(plan, S_use, scale, groups, prec, R_t)
        (bf.bf_batch_launch if mode == "batch" else bf.bf_batch_launch_graph)(h)
        torch.cuda.synchronize()
        bf.bf_batch_destroy(h)
    else:
        raise ValueError(mode)
    out = split_R(R_t, batch, torch)
    if return_buffers:
        return out, dict(S=S_use, scale=scale, R=R_t, groups=groups, S_c64=S_d)
    return out


def rl_layout(batch, rtype: int, pad_block: int = 0, pad_row: int = 0):
    """An antenna-major R layout over the whole batch (antenna i's resource
    elements of every block in one row), with optional padding bytes after
    each block's row segment and after each antenna row. Returns
    (bf_rlayout, group r_off list, total bytes)."""
    e = bf.R_ESIZE[rtype]
    bs = B_RE * e + pad_block
    T = batch.total_blocks
    rs = max(1, T) * bs + pad_row
    offs, n0 = [], 0
    for nb in batch.n_blocks:
        offs.append(n0 * bs)
        n0 += nb
    return bf.bf_rlayout(rs, bs, rtype, 0), offs, N_ANT * rs


def run_rl(plan, batch, prec: int, torch, rtype: int, held: bool = False, pad_block: int = 0, pad_row: int = 0,
           mode: str = "apply", set_w: bool = True):
    """bf_apply_batch_rl (or a prepared batch) into an antenna-major R.
    Returns (R bytes as a numpy uint8 array, bf_rlayout, group r_off list).
    The R buffer is filled with 0xFF bytes first (NaN in every R type)."""
    if set_w:
        set_precoders(plan, batch, torch)
    lay = layout(batch, 0, prec)
    rl, offs, nbytes = rl_layout(batch, rtype, pad_block, pad_row)
    Sflat, _ = batch.pack_S()
    S_d = to_device_c64(Sflat, torch)
    scale, S_use = None, S_d
    s_offs = [g[2] for g in lay.groups]
    if held:
        Sq = torch.zeros(max(16, lay.held_bytes) // 4 + 4, dtype=torch.float32, device="cuda")
        scale = torch.zeros(max(1, batch.total_blocks), dtype=torch.float32, device="cuda")
        bf.bf_quantize_symbols(plan, S_d, lay.groups, prec, Sq, lay.held_off, scale)
        S_use, s_offs = Sq, lay.held_off
    groups = [(g[0], g[1], s_offs[i], offs[i]) for i, g in enumerate(lay.groups)]
    R_t = torch.full((max(16, nbytes),), 255, dtype=torch.uint8, device="cuda")
    if mode == "apply":
        bf.bf_apply_batch_rl(plan, S_use, scale, groups, prec, R_t, rl)
    elif mode in ("batch", "graph"):
        h = bf.bf_batch_create_rl(plan, S_use, scale, groups, prec, R_t, rl)
        (bf.bf_batch_launch if mode == "batch" else bf.bf_batch_launch_graph)(h)
        torch.cuda.synchronize()
        bf.bf_batch_destroy(h)
    else:
        raise ValueError(mode)
    torch.cuda.synchronize()
    return R_t.cpu().numpy(), rl, offs


def rl_view(buf: np.ndarray, rl, r_off: int, n_blocks: int) -> np.ndarray:
    """Group view of an R buffer in layout rl: complex64 (n_blocks, 64, 60) for
    BF_R_C64, else uint16 (n_blocks, 64, 60, 2) holding the (re, im) bit patterns."""
    if rl.rtype == bf.BF_R_C64:
        return np.ndarray((n_blocks, N_ANT, B_RE), np.complex64, buf, r_off, (rl.block_stride, rl.row_stride, 8))
    return np.ndarray((n_blocks, N_ANT, B_RE, 2), np.uint16, buf, r_off, (rl.block_stride, rl.row_stride, 4, 2))


def decode_r(v: np.ndarray, rtype: int) -> np.ndarray:
    """Elements read through rl_view (or any (..., 2) uint16 pair array for the
    16-bit types) as complex128 values."""
    if rtype == bf.BF_R_C64:
        return v.astype(np.complex128)
    if rtype == bf.BF_R_BF16:
        f = (v.astype(np.uint32) << np.uint32(16)).view(np.float32)
    else:
        f = np.ascontiguousarray(v).view(np.float16).astype(np.float32)
    return f[..., 0].astype(np.float64) + 1j * f[..., 1].astype(np.float64)


def rl_written_mask(nbytes: int, rl, offs, n_blocks) -> np.ndarray:
    """Bytes of an R buffer that layout rl assigns to some element."""
    m = np.zeros(max(16, nbytes), np.bool_)
    e = bf.R_ESIZE[rl.rtype]
    for o, nb in zip(offs, n_blocks):
        np.ndarray((nb, N_ANT, B_RE, e), np.bool_, m, o, (rl.block_stride, rl.row_stride, e, 1))[...] = True
    return m
