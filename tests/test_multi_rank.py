"""World-size-2 CPU (gloo) checks of the multi-rank host logic: disjoint shards that
cover every walk once, the accumulator merge equals the single-process sums, and walks
sharded over ranks -- by disjoint walk-id ranges or by point blocks -- merge into the
estimate of one process running every walk (the oracle walks on each rank)."""
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


def _walk_worker(rank, world, port, mode, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    import workloads as W
    desc = W.cube3d_problem()
    pts = W.cell_centres(3, 64)[:, W.seeded_subset(64 ** 3, 24, 61)]
    npts, walks, seed = pts.shape[1], 96, 17
    sb = oracle.sigma_bar(desc, 64)[0]
    acc = (torch.zeros(npts, dtype=torch.float64), torch.zeros(npts, dtype=torch.float64),
           torch.zeros(npts, dtype=torch.int64))
    if mode == "walks":
        off, cnt = multi.walk_range(rank, world, walks)
        if cnt > 0:
            o, _ = oracle.solve(desc, pts, cnt, seed=seed, eps=1e-4, sigma_bar=sb, walk_offset=off)
            for t, v in zip(acc, o):
                t += torch.from_numpy(np.asarray(v))
    else:
        a, b = multi.point_range(rank, world, npts)
        # the block's points keep their global indices (the Philox counter's point word):
        # per-point walk counts, zero outside the block
        w = np.zeros(npts, dtype=np.int32)
        w[a:b] = walks
        o, _ = oracle.solve(desc, pts, w, seed=seed, eps=1e-4, sigma_bar=sb)
        for t, v in zip(acc, o):
            t += torch.from_numpy(np.asarray(v))
    multi.merge_accumulators(acc)
    if rank == 0:
        np.save(os.path.join(out_dir, f"merged_{mode}.npy"), np.stack([t.numpy().astype(np.float64) for t in acc]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["walks", "points"])
def test_sharded_walks_merge_to_one_process(tmp_path, orc, mode):
    """Two ranks walk disjoint walk-id ranges of every point (or disjoint point blocks);
    after the all-reduce the counts equal one process's exactly and the sums agree to
    summation-order rounding."""
    import workloads as W
    world = 2
    mp.start_processes(_walk_worker, args=(world, _free_port(), mode, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    got = np.load(tmp_path / f"merged_{mode}.npy")
    desc = W.cube3d_problem()
    pts = W.cell_centres(3, 64)[:, W.seeded_subset(64 ** 3, 24, 61)]
    sb = orc.sigma_bar(desc, 64)[0]
    ref, _ = orc.solve(desc, pts, 96, seed=17, eps=1e-4, sigma_bar=sb)
    assert np.array_equal(got[2], np.asarray(ref[2], dtype=np.float64))
    assert np.allclose(got[0], ref[0], rtol=1e-12, atol=1e-12)
    assert np.allclose(got[1], ref[1], rtol=1e-12, atol=1e-12)
