"""Batched queries (msf_segment_batch): every query's labels and feature count equal a separate
msf_segment call on the same data, and equal the CPU oracle."""
import numpy as np
import pytest
import torch

from paper_1903_12294_gb300 import synth

pytestmark = pytest.mark.gpu

F, C, M = 0, 1, 2
GT, GE, LT, LE, BAND = 0, 1, 2, 3, 4


PERSISTENT = 9   # MSF_SCHED_PERSISTENT | MSF_SCHED_FUSED_CRITERION: one persistent launch


def _check_batch(gpu, orc, f, p, a, queries):
    """The batch in one persistent launch (the default) and in one launch per phase."""
    ctx = gpu.Context(0)
    try:
        ctx.load(*(torch.as_tensor(x).cuda().contiguous() for x in (f, p, a)))
        ctx.bin()
        runs = []
        for sched in (PERSISTENT, 1):
            ctx.set_batch_schedule(sched)
            runs.append(ctx.segment_batch(queries))
        singles = [ctx.segment(t0, t1, pr, e) for (t0, t1, pr, e) in queries]
        torch.cuda.synchronize()
    finally:
        ctx.close()
    o = orc.bin(f.shape, p, a)
    for labels, nfs in runs:
        for (t0, t1, pr, e), lb, nf, (ls, ns) in zip(queries, labels, nfs, singles):
            assert nf == ns
            assert torch.equal(lb, ls)
            lab, n_o = orc.segment(f, o["count"], o["mean"], o["key"], t0, t1, pr, e)
            assert nf == n_o and np.array_equal(lb.cpu().numpy(), lab)


def test_batch_mixed_windows_and_criteria(gpu, orc):
    """Windows starting inside a time chunk, single steps, different predicates and edge
    classes in one batch (3D)."""
    wl = synth.mid(n=48, T=11, P=30000, n_blobs=12)
    f, p, a = wl.numpy()
    q = wl.preds
    queries = [(0, 11, q, 7), (1, 4, q, 7), (3, 4, q, 7), (5, 11, [(F, 0, GT, 0.45, 0)], 7),
               (2, 9, [(F, 0, GT, 0.5, 0), (C, 0, GE, 1, 0)], 3), (6, 8, q, 1), (7, 10, q, 6),
               (0, 2, [], 7), (4, 4, q, 7), (9, 11, [(M, 1, BAND, 0.4, 0.9), (F, 0, GE, 0.3, 0),
                                                    (C, 0, LE, 3, 0)], 7)]
    _check_batch(gpu, orc, f, p, a, queries)


def test_batch_2d_time(gpu, orc):
    rng = np.random.default_rng(4)
    T, nz, ny, nx = 20, 1, 70, 96
    f = rng.random((T, nz, ny, nx)).astype(np.float32)
    P = 3000
    pos = (rng.random((T, 3, P)) * np.array([nx, ny, nz])[None, :, None]).astype(np.float32)
    a = rng.normal(size=(T, 2, P)).astype(np.float32)
    queries = [(t0, t0 + tw, [(F, 0, GT, th, 0)], 7)
               for t0, tw, th in ((0, 20, 0.6), (3, 5, 0.5), (15, 5, 0.55), (7, 1, 0.4),
                                  (2, 17, 0.7))]
    _check_batch(gpu, orc, f, pos, a, queries)


def test_batch_graph_replay(gpu, orc):
    """With graphs on, a repeated batch shape runs plainly, is captured, then replays; replays
    pick up new thresholds and new label buffers, and a new shape runs plainly again. Every
    result equals the single queries and the oracle."""
    wl = synth.mid(n=40, T=10, P=20000, n_blobs=8)
    f, p, a = wl.numpy()
    o = orc.bin(f.shape, p, a)
    ctx = gpu.Context(0)
    try:
        ctx.load(*(torch.as_tensor(x).cuda().contiguous() for x in (f, p, a)))
        ctx.bin()
        ctx.set_batch_graphs(True)
        shape = [(0, 10, "q", 7), (2, 6, "f", 7), (5, 9, "c", 3)]

        def queries(th):
            pr = {"q": [(F, 0, GT, th, 0), (M, 0, BAND, 0.3, 0.9)],
                  "f": [(F, 0, GT, th + 0.05, 0)],
                  "c": [(F, 0, GE, th, 0), (C, 0, GE, 1, 0)]}
            return [(t0, t1, pr[k], e) for t0, t1, k, e in shape]

        seen = []
        for it, th in enumerate([0.5, 0.45, 0.55, 0.6]):
            qs = queries(th)
            labels, nfs = ctx.segment_batch(qs)
            singles = [ctx.segment(t0, t1, pr, e) for (t0, t1, pr, e) in qs]
            seen.append((qs, [lb.cpu().numpy() for lb in labels], nfs,
                         [(ls.cpu().numpy(), ns) for ls, ns in singles]))
        replays = ctx.batch_graph_replays()
        # a different shape: plain launch, correct, and no replay
        qs = [(1, 10, [(F, 0, GT, 0.5, 0)], 7)]
        labels, nfs = ctx.segment_batch(qs)
        ls, ns = ctx.segment(*qs[0])
        assert nfs[0] == ns and torch.equal(labels[0], ls)
        assert ctx.batch_graph_replays() == replays
        ctx.set_batch_graphs(False)
    finally:
        ctx.close()
    assert replays == 2                       # runs 3 and 4 (run 2 captures and launches)
    for qs, labs, nfs, singles in seen:
        for (t0, t1, pr, e), lb, nf, (ls, ns) in zip(qs, labs, nfs, singles):
            assert nf == ns and np.array_equal(lb, ls)
            want, n_o = orc.segment(f, o["count"], o["mean"], o["key"], t0, t1, pr, e)
            assert nf == n_o and np.array_equal(lb, want)


def test_batch_tile_shapes_and_autotune(gpu, orc):
    """Every batch tile shape and schedule (one persistent launch; phase launches with the
    criterion fused, or streamed first on whole 32-voxel rows) gives the single queries'
    labels; the batch autotuner keeps a valid choice, and the batch then still gives them."""
    wl = synth.mid(n=64, T=12, P=20000, n_blobs=8)
    f, p, a = wl.numpy()
    q = wl.preds
    queries = [(0, 12, q, 7), (3, 11, [(F, 0, GT, 0.45, 0)], 7), (5, 6, q, 3), (1, 9, q, 6)]
    o = orc.bin(f.shape, p, a)
    want = [orc.segment(f, o["count"], o["mean"], o["key"], t0, t1, pr, e)
            for (t0, t1, pr, e) in queries]
    ctx = gpu.Context(0)
    try:
        ctx.load(*(torch.as_tensor(x).cuda().contiguous() for x in (f, p, a)))
        ctx.bin()
        got = []
        for sched in (PERSISTENT, 1, 0):
            ctx.set_batch_schedule(sched)
            for tile in [(4, 4, 16), (2, 16, 8), (16, 8, 2), (8, 8, 4)]:
                ctx.set_batch_tile(*tile)
                labels, nfs = ctx.segment_batch(queries)
                got.append(((sched, tile), [l.cpu().numpy() for l in labels], nfs))
        ctx.set_batch_tile(0, 0, 0)
        ctx.set_batch_schedule(PERSISTENT)
        r = ctx.autotune_batch(queries, reps=1)
        assert r["by"] * r["bz"] * r["bt"] == 256 and r["n_tried"] > 3
        assert r["sched"] in (0, 1, PERSISTENT)
        assert 0 < r["ms"] <= r["ms_default"]
        labels, nfs = ctx.segment_batch(queries)
        got.append(("tuned", [l.cpu().numpy() for l in labels], nfs))
        with pytest.raises(gpu.MsfError) as e:
            ctx.set_batch_tile(4, 4, 4)
        assert e.value.status == gpu.MSF_ERR_INVALID_ARG
    finally:
        ctx.close()
    for tile, labs, nfs in got:
        for (lab_o, n_o), lb, nf in zip(want, labs, nfs):
            assert nf == n_o and np.array_equal(lb, lab_o), tile
