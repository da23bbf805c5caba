"""Multi-rank paths on CPU (no GPU): time-slab sharding of one window and the merge of the slab
labellings, checked against the oracle's labelling of the whole window; the cut exchange and the
replica reductions run as two gloo ranks."""
import os
import socket

import numpy as np
import pytest

from paper_1903_12294_gb300 import replicas, slabs, synth

EDGE_CASES = [7, 3, 6, 2, 5, 4]


@pytest.fixture(scope="module")
def tiny_bins(orc):
    wl = synth.tiny(T=10, P=6000)
    f, p, a = wl.numpy()
    o = orc.bin(f.shape, p, a)
    return wl, f, o


def test_slab_bounds_cover_the_window():
    for t0, t1, w in [(0, 10, 2), (3, 10, 3), (0, 5, 8), (2, 2, 2), (0, 1, 1)]:
        b = slabs.slab_bounds(t0, t1, w)
        assert len(b) == w and b[0][0] == t0 and b[-1][1] == t1
        assert all(x[1] == y[0] for x, y in zip(b[:-1], b[1:]))
        sizes = [y - x for x, y in b]
        assert max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("edges", EDGE_CASES)
@pytest.mark.parametrize("world", [2, 3])
def test_merged_slabs_equal_whole_window(orc, tiny_bins, edges, world):
    """Labelling slabs separately and merging across the cuts gives the canonical labels and
    feature count of the whole window."""
    wl, f, o = tiny_bins
    t0, t1 = 1, 10
    V = int(np.prod(f.shape[1:]))
    whole, n_whole = orc.segment(f, o["count"], o["mean"], o["key"], t0, t1, wl.preds, edges)
    parts = []
    for ta, tb in slabs.slab_bounds(t0, t1, world):
        lab, n = orc.segment(f, o["count"], o["mean"], o["key"], ta, tb, wl.preds, edges)
        parts.append((ta, tb, lab, n))
    merged, n = slabs.merge_slabs(parts, t0, V, edges, keys=o["key"])
    assert n == n_whole
    assert np.array_equal(merged, whole.astype(np.int64))


def test_merge_needs_the_cut_edges(orc, tiny_bins):
    """Without the merge the slabs disagree with the whole window (the test above is not
    vacuous): some component crosses the cut."""
    wl, f, o = tiny_bins
    V = int(np.prod(f.shape[1:]))
    whole, _ = orc.segment(f, o["count"], o["mean"], o["key"], 0, 10, wl.preds, 7)
    parts = [orc.segment(f, o["count"], o["mean"], o["key"], a, b, wl.preds, 7)
             for a, b in slabs.slab_bounds(0, 10, 2)]
    naive = np.concatenate([np.where(l >= 0, l.astype(np.int64) + off, -1)
                            for (l, _), off in zip(parts, (0, 5 * V))])
    assert not np.array_equal(naive, whole)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir, edges):
    import torch.distributed as dist

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = synth.tiny(T=10, P=6000)
        f, p, a = wl.numpy()
        o = oracle.bin(f.shape, p, a)
        t0, t1 = 1, 10
        V = int(np.prod(f.shape[1:]))
        ta, tb = slabs.slab_bounds(t0, t1, world)[rank]
        lab, n = oracle.segment(f, o["count"], o["mean"], o["key"], ta, tb, wl.preds, edges)
        glob, n_all = slabs.merge_slab_collective(lab, n, ta, tb, t0, V, edges,
                                                  o["key"][ta], o["key"][tb - 1])
        # the replica reductions the measurement uses
        mx = replicas.max_over_ranks(10.0 + rank)
        np.save(os.path.join(out_dir, f"r{rank}.npy"), glob)
        np.save(os.path.join(out_dir, f"r{rank}_meta.npy"), np.array([n_all, mx]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("edges", [7, 6])
def test_cut_exchange_over_gloo(orc, tiny_bins, tmp_path, edges):
    """Two gloo ranks each label their slab, exchange the cut planes and keys, and relabel: the
    two halves together are the whole window's canonical labelling."""
    import torch.multiprocessing as mp
    wl, f, o = tiny_bins
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path), edges),
                       nprocs=world, join=True, start_method="spawn")
    whole, n_whole = orc.segment(f, o["count"], o["mean"], o["key"], 1, 10, wl.preds, edges)
    got = np.concatenate([np.load(tmp_path / f"r{r}.npy") for r in range(world)])
    assert np.array_equal(got, whole.astype(np.int64))
    for r in range(world):
        n_all, mx = np.load(tmp_path / f"r{r}_meta.npy")
        assert int(n_all) == n_whole
        assert mx == 10.0 + world - 1


def test_weak_throughput():
    assert replicas.weak_throughput(1e9, 500.0, 4) == pytest.approx(8e9)
