"""Partition and gather of a sharded encode (the multi-GPU path), on the CPU.

The per-rank encoder here is the FP64 oracle, so these tests check only the
host logic: that the ranks' contiguous (plane, root row) ranges cover the
workload once, in canonical order and balanced by pixels, and that their
results, rewritten in global coordinates and gathered over gloo ranks, are
exactly the single-process encode."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2605_09190_gb300 import shard, synthetic

MB = 16


def _planes():
    return [synthetic.gradient_scene(64, 128, seed=3), synthetic.piecewise_scene(128, 64, seed=4),
            synthetic.gradient_scene(48, 48, seed=5)]


TOLS = [2.0, 3.0, 1.5]


def _encode_pieces(planes, pieces):
    views = shard.piece_views(planes, pieces, MB)
    if not views:
        return np.zeros(0, oracle.LEAF_DTYPE), np.zeros(0, np.int32), np.zeros(0, np.float64)
    enc = oracle.encode(views, [TOLS[p] for p, _, _ in pieces], min_block=4, max_block=MB, threads=1)
    return shard.globalize(enc.leaves, pieces, MB), enc.atom_j, enc.atom_alpha


def _same(a, b):
    la, ja, aa = a
    lb, jb, ab = b
    assert len(la) == len(lb)
    for f in ("plane", "y", "x", "b", "atom_off", "n_atoms", "converged"):
        assert np.array_equal(la[f], lb[f]), f
    assert np.array_equal(ja, jb)
    assert np.array_equal(aa, ab)


@pytest.mark.parametrize("world", [1, 2, 3, 5, 64])
def test_partition_covers_every_root_row_once_in_order_and_balanced(world):
    shapes = [(64, 128), (128, 64), (48, 48), (16, 256)]
    parts = shard.partition(shapes, MB, world)
    assert len(parts) == world
    seq = [(p, r0 + i) for pieces in parts for p, r0, n in pieces for i in range(n)]
    want = [(p, r) for p, (h, w) in enumerate(shapes) for r in range(h // MB)]
    assert seq == want                       # every root row once, canonical order
    px = [sum(n * MB * shapes[p][1] for p, _, n in pieces) for pieces in parts]
    total = sum(h * w for h, w in shapes)
    row_max = max(w * MB for _, w in shapes)
    for v in px:                             # within one root row of the even share
        assert abs(v - total / world) <= row_max
    for pieces in parts:                     # maximal runs: no two adjacent pieces of one plane touch
        for (p0, r0, n0), (p1, r1, _) in zip(pieces, pieces[1:]):
            assert not (p0 == p1 and r0 + n0 == r1)


def test_partition_rejects_shapes_off_the_root_grid():
    with pytest.raises(ValueError):
        shard.partition([(64, 70)], MB, 2)


def test_merged_piece_encodes_equal_the_whole_encode():
    planes = _planes()
    whole = oracle.encode(planes, TOLS, min_block=4, max_block=MB, threads=1)
    for world in (2, 3, 7):
        parts = [_encode_pieces(planes, pieces) for pieces in shard.partition([p.shape for p in planes], MB, world)]
        merged = shard.merge(parts)
        _same(merged, (whole.leaves, whole.atom_j, whole.atom_alpha))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gloo_rank(rank, world, port):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        planes = _planes()
        pieces = shard.partition([p.shape for p in planes], MB, world)[rank]
        lv, aj, aa = _encode_pieces(planes, pieces)
        got = shard.gather(lv, aj, aa)
        whole = oracle.encode(planes, TOLS, min_block=4, max_block=MB, threads=1)
        _same(got, (whole.leaves, whole.atom_j, whole.atom_alpha))
    finally:
        dist.destroy_process_group()


def test_gather_over_two_gloo_ranks_equals_the_single_process_encode():
    mp = pytest.importorskip("torch.multiprocessing")
    mp.spawn(_gloo_rank, args=(2, _free_port()), nprocs=2, join=True)
