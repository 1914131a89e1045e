"""World-size-2 gloo test (CPU) of the rank split: an auto count sharded by
home rows and summed once across ranks equals the single-process count; a
batch dealt round-robin covers every catalog once."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1210_1833_gb300 import shard, synthetic

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = synthetic.c1_monopole_box(scale=0.1)

        def cross(xs, x):
            c, _, _ = oracle.count("mono", xs, x, edges0=w.edges0, periodic=True, L=w.L,
                                   nthreads=2)
            return c

        def allreduce(a):
            t = torch.from_numpy(a)
            dist.all_reduce(t)
            return t.numpy()

        got = shard.sharded_auto(cross, w.data, rank, world, self_bin=0, allreduce=allreduce)
        mine = shard.batch_share(7, rank, world)
        seen = torch.zeros(7, dtype=torch.int64)
        seen[mine] = 1
        dist.all_reduce(seen)
        if rank == 0:
            np.save(out, np.concatenate([got.ravel().astype(np.int64), seen.numpy()]))
    finally:
        dist.destroy_process_group()


def test_sharded_auto_count_equals_single_process(tmp_path):
    out = str(tmp_path / "res.npy")
    torch.multiprocessing.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    res = np.load(out)
    w = synthetic.c1_monopole_box(scale=0.1)
    ref, _, _ = oracle.count("mono", w.data, edges0=w.edges0, periodic=True, L=w.L)
    nb = len(w.edges0) - 1
    assert res[:nb].tolist() == ref.ravel().astype(np.int64).tolist()
    assert res[nb:].tolist() == [1] * 7


def test_row_ranges_partition():
    for n in (0, 1, 7, 100):
        for world in (1, 2, 3, 8):
            rs = [shard.row_range(n, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
