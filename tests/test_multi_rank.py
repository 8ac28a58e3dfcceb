"""World-size-2 CPU (gloo) checks of the multi-rank host logic: disjoint shards that
cover every walk once, and the accumulator merge equals the single-process sums."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2201_13240_gb300 import multi  # noqa: E402


def test_shards_cover_everything_once():
    for world in (1, 2, 3, 8):
        for n in (0, 1, 7, 1024, 1001):
            seen = []
            for r in range(world):
                s, e = multi.point_range(r, world, n)
                seen.extend(range(s, e))
            assert seen == list(range(n))
            ids = []
            for r in range(world):
                off, cnt = multi.walk_range(r, world, n, walk_offset=5)
                ids.extend(range(off, off + cnt))
            assert ids == list(range(5, 5 + n))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, npts, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(100 + rank)
    # a rank's accumulators after walking its share of walk ids
    s1 = torch.from_numpy(rng.normal(size=npts))
    s2 = torch.from_numpy(rng.uniform(1, 2, size=npts))
    cnt = torch.from_numpy(rng.integers(1, 50, size=npts).astype(np.int64))
    np.save(os.path.join(out_dir, f"in{rank}.npy"), np.stack([s1.numpy(), s2.numpy(), cnt.numpy()]))
    multi.merge_accumulators((s1, s2, cnt))
    np.save(os.path.join(out_dir, f"out{rank}.npy"), np.stack([s1.numpy(), s2.numpy(), cnt.numpy()]))
    dist.barrier()
    dist.destroy_process_group()


def test_merge_two_ranks_gloo(tmp_path):
    world, npts = 2, 37
    mp.start_processes(_worker, args=(world, _free_port(), npts, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    ins = [np.load(tmp_path / f"in{r}.npy") for r in range(world)]
    want = ins[0] + ins[1]
    for r in range(world):
        got = np.load(tmp_path / f"out{r}.npy")
        assert np.allclose(got, want, rtol=0, atol=1e-12)
