"""Partition of an encode over several processes, and the gather of the
results (one process per GPU).

Root blocks, channels and images are independent problems: Algorithm 1 runs
its loop over the channels, Algorithm 2 runs its FORALL over the root blocks,
and a root's subtree reads only its own pixels.  So a workload of planes
shards into contiguous ranges of (plane, root row): rank r encodes a band of
whole root rows of one or more planes, with no exchange during the encode.
The only collective is the gather of the variable-length leaf and atom
records at the end: an all-gather of the per-rank counts, then a gather of
the records padded to the largest count, rebased on the receiving rank.

Because the ranges follow the canonical order of the output (planes
ascending, roots in raster order, leaves depth first), concatenating the
ranks' results in rank order gives exactly the single-process encode.

Pieces are ``(plane, root_row0, root_rows)``: plane index in the global
workload, first root row and number of root rows (a root row is ``max_block``
pixel rows).  Leaf records are numpy structured arrays with at least the
fields ``plane``, ``y`` and ``atom_off`` (the library's ``aqmp_leaf``).
"""
from __future__ import annotations

import numpy as np


def partition(shapes, max_block: int, world: int):
    """Split the root rows of the planes ``shapes`` ((h, w) each, multiples of
    ``max_block``) into ``world`` contiguous ranges balanced by pixel count.

    Root row u (in canonical order over all planes) goes to rank
    floor(world * P_u / P), where P_u is the number of pixels in the root rows
    before it and P the total: every rank's share is within one root row of
    P / world.  Returns one list of pieces per rank (possibly empty)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    rows = []                                   # (plane, root row, pixels)
    for p, (h, w) in enumerate(shapes):
        if h % max_block or w % max_block:
            raise ValueError(f"plane {p}: {h}x{w} is not a multiple of {max_block}")
        rows.extend((p, r, w * max_block) for r in range(h // max_block))
    total = sum(px for _, _, px in rows)
    out = [[] for _ in range(world)]
    before = 0
    for p, r, px in rows:
        rank = min(world - 1, (before * world) // total) if total else 0
        before += px
        pieces = out[rank]
        if pieces and pieces[-1][0] == p and pieces[-1][1] + pieces[-1][2] == r:
            pieces[-1] = (p, pieces[-1][1], pieces[-1][2] + 1)
        else:
            pieces.append((p, r, 1))
    return out


def piece_shapes(shapes, pieces, max_block: int):
    """(h, w) of each piece's sub-plane."""
    return [(n * max_block, shapes[p][1]) for p, _, n in pieces]


def piece_views(planes, pieces, max_block: int):
    """The sub-planes of ``pieces``: row slices of the planes (numpy arrays or
    torch tensors, row-major), which keep the parent's row pitch."""
    return [planes[p][r0 * max_block:(r0 + n) * max_block] for p, r0, n in pieces]


def globalize(leaves: np.ndarray, pieces, max_block: int) -> np.ndarray:
    """Leaf records of an encode of ``pieces`` (plane = piece index, y within
    the piece) rewritten in the coordinates of the whole workload."""
    out = leaves.copy()
    if len(out) == 0:
        return out
    idx = out["plane"].astype(np.int64)
    plane_of = np.array([p for p, _, _ in pieces], dtype=np.int64)
    y0 = np.array([r0 * max_block for _, r0, _ in pieces], dtype=np.int64)
    out["plane"] = plane_of[idx].astype(out["plane"].dtype)
    out["y"] = (out["y"].astype(np.int64) + y0[idx]).astype(out["y"].dtype)
    return out


def merge(parts):
    """Concatenate per-rank results ``(leaves, atoms, lo)`` in rank order,
    rebasing each rank's ``atom_off`` by the atoms of the ranks before it.
    ``lo`` may be None throughout."""
    leaves, atoms, los = [], [], []
    base = 0
    for lv, at, lo in parts:
        lv = lv.copy()
        if len(lv):
            lv["atom_off"] = (lv["atom_off"].astype(np.int64) + base).astype(lv["atom_off"].dtype)
        base += len(at)
        leaves.append(lv)
        atoms.append(at)
        los.append(lo)
    cat = lambda xs: np.concatenate(xs) if xs else None  # noqa: E731
    lo_all = None if any(x is None for x in los) else cat(los)
    return cat(leaves), cat(atoms), lo_all


def _gather_bytes(arr: np.ndarray, world: int, device, group):
    """All ranks' byte arrays (padded all-gather; every rank receives all)."""
    import torch
    import torch.distributed as dist
    raw = np.ascontiguousarray(arr).view(np.uint8).reshape(-1)
    n = torch.tensor([raw.size], dtype=torch.int64, device=device)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    sizes = [int(s.item()) for s in sizes]
    cap = max(1, max(sizes))
    buf = torch.zeros(cap, dtype=torch.uint8, device=device)
    if raw.size:
        buf[:raw.size] = torch.from_numpy(raw).to(device)
    bufs = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(bufs, buf, group=group)
    return [b[:s].cpu().numpy() for b, s in zip(bufs, sizes)]


def gather(leaves: np.ndarray, atoms: np.ndarray, lo=None, group=None, device="cpu"):
    """Gather every rank's (already globalized) records; all ranks return
    the merged result in canonical order.  ``device`` is where the
    collective's buffers live ("cpu" for gloo, a CUDA device for NCCL)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    lv = _gather_bytes(leaves, world, device, group)
    at = _gather_bytes(atoms, world, device, group)
    los = _gather_bytes(lo, world, device, group) if lo is not None else [None] * world
    parts = [(a.view(leaves.dtype), b.view(atoms.dtype), None if c is None else c.view(lo.dtype))
             for a, b, c in zip(lv, at, los)]
    return merge(parts)
