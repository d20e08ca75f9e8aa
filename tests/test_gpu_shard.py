"""The sharded encode on the GPU: each rank's contiguous (plane, root row)
range encoded on its own, rewritten in global coordinates and gathered,
equals the single encode of the whole batch byte for byte -- in one process
(ranks one after another) and as two processes on one GPU gathering over
gloo."""
import os
import socket

import numpy as np
import pytest

from paper_2605_09190_gb300 import shard, synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MB = 64


def _planes():
    batch = synthetic.uneven_rgb_batch(3, seed=5, scene=synthetic.piecewise_scene, wmax=768, hmax=512)
    return [c for (_, _, chans) in batch for c in chans]


def _encode(aqmp, planes):
    dev = [torch.from_numpy(np.ascontiguousarray(p)).cuda() for p in planes]
    code = aqmp.aqmp_encode_planes(dev, 2.0, min_block=4, max_block=MB)
    out = code.copy()
    code.free()
    return out


def _rank_part(aqmp, planes, pieces):
    if not pieces:
        from paper_2605_09190_gb300.aqmp import ATOM_DTYPE, LEAF_DTYPE
        return np.zeros(0, LEAF_DTYPE), np.zeros(0, ATOM_DTYPE), np.zeros(0, np.float32)
    lv, at, lo = _encode(aqmp, shard.piece_views(planes, pieces, MB))
    return shard.globalize(lv, pieces, MB), at, lo


def _same(a, b):
    for x, y in zip(a, b):
        assert x.dtype == y.dtype and x.shape == y.shape
        np.testing.assert_array_equal(np.ascontiguousarray(x).view(np.uint8), np.ascontiguousarray(y).view(np.uint8))


def test_ranks_in_one_process_gather_to_the_single_encode():
    from paper_2605_09190_gb300 import aqmp, build_lib
    build_lib.build()
    planes = _planes()
    whole = _encode(aqmp, planes)
    for world in (2, 3):
        parts = [_rank_part(aqmp, planes, pieces)
                 for pieces in shard.partition([p.shape for p in planes], MB, world)]
        _same(shard.merge(parts), whole)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _proc(rank, world, port):
    import torch.distributed as dist
    from paper_2605_09190_gb300 import aqmp
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        planes = _planes()
        pieces = shard.partition([p.shape for p in planes], MB, world)[rank]
        got = shard.gather(*_rank_part(aqmp, planes, pieces))
        if rank == 0:
            _same(got, _encode(aqmp, planes))
    finally:
        dist.destroy_process_group()


def test_two_processes_on_one_gpu_gather_to_the_single_encode():
    from paper_2605_09190_gb300 import build_lib
    build_lib.build()
    mp = torch.multiprocessing
    mp.spawn(_proc, args=(2, _free_port()), nprocs=2, join=True)
