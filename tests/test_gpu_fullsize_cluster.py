"""Full-size checks of the clustering and the steps after it, on the workload and centre grid
the benchmark times (128^3 x 32 field, 1M points, k = 16 x 16 x 16 x 4). The brute-force
clustering oracle cannot run at this size, so the clustering is checked by properties that hold
at any size: the counts are those of the labels, and every centre with samples is the
fixed-point mean of its samples (the update rule). Merging, summaries and trajectory pieces are
compared with the oracle at full size."""
import numpy as np
import pytest
import torch

from paper_1903_12294_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

K4 = (16, 16, 16, 4)


def _scale(max_abs, n):
    e = np.frexp(max_abs)[1] if max_abs > 0 else 0
    b = 0
    while (1 << b) < n + 1:
        b += 1
    return 62 - e - b


def _fixed_sums(lab, vals, K):
    """Per label, the exact sum of int64 values (sort + reduceat; labels < 0 dropped)."""
    keep = lab >= 0
    lab, vals = lab[keep], vals[keep]
    order = np.argsort(lab, kind="stable")
    lab, vals = lab[order], vals[order]
    out = np.zeros(K, np.int64)
    if lab.size:
        starts = np.flatnonzero(np.r_[True, lab[1:] != lab[:-1]])
        out[lab[starts]] = np.add.reduceat(vals, starts)
    return out


@pytest.fixture(scope="module")
def clustered(gpu):
    wl = synth.mid(device="cuda")
    T = wl.field.shape[0]
    ctx = gpu.Context(0)
    ctx.load(wl.field, wl.pos, wl.attr)
    ctx.bin()
    fl, pl, c, n, it = ctx.cluster(0, T, 0, K4, w_p=1.0, w_f=1.0, w_d=0.05, max_iter=3)
    seg, nseg = ctx.segment(wl.t0, wl.t1, wl.preds, wl.edges)
    torch.cuda.synchronize()
    yield ctx, wl, fl, pl, c, n, seg
    ctx.close()


def test_cluster_counts_and_centres_are_the_labels_means(clustered):
    ctx, wl, fl, pl, c, n, _ = clustered
    f, p, a = (x.cpu().numpy() for x in (wl.field, wl.pos, wl.attr))
    T, nz, ny, nx = f.shape
    K = len(c)
    key = ctx.bins("cpu")[0].numpy()
    flh, plh = fl.cpu().numpy().ravel(), pl.cpu().numpy().ravel()
    # samples taking part: finite field values; points inside the grid with a finite speed
    fv = f.ravel()
    pv = a[:, 0, :].ravel()
    fok = np.isfinite(fv)
    pok = (key.ravel() >= 0) & np.isfinite(pv)
    assert np.array_equal(flh >= 0, fok) and np.array_equal(plh >= 0, pok)
    assert np.array_equal(np.bincount(flh[fok], minlength=K), n[:, 0])
    assert np.array_equal(np.bincount(plh[pok], minlength=K), n[:, 1])
    ntot = int(fok.sum() + pok.sum())
    kpos = _scale(float(max(nx, ny, nz, T + 1)), ntot)
    kf = _scale(float(np.abs(fv[fok]).max()), ntot)
    kp = _scale(float(np.abs(pv[pok]).max()), ntot)

    def q(v, k):
        return np.rint(v.astype(np.float64) * 2.0 ** k).astype(np.int64)

    tt, zz, yy, xx = np.meshgrid(np.arange(T), np.arange(nz), np.arange(ny), np.arange(nx),
                                 indexing="ij")
    floc = [xx.ravel() + 0.5, yy.ravel() + 0.5, zz.ravel() + 0.5, tt.ravel() + 0.5]
    P = p.shape[2]
    ploc = [p[:, 0, :].ravel(), p[:, 1, :].ravel(), p[:, 2, :].ravel(),
            np.repeat(np.arange(T) + 0.5, P)]
    nsum = n[:, 0] + n[:, 1]
    has = nsum > 0
    for d in range(4):
        s = (_fixed_sums(flh, q(np.asarray(floc[d], np.float32), kpos), K) +
             _fixed_sums(plh, q(np.asarray(ploc[d], np.float32), kpos), K))
        want = (s[has].astype(np.float64) / nsum[has] * 2.0 ** -kpos).astype(np.float32)
        assert np.array_equal(c[has, d].view(np.uint32), want.view(np.uint32)), d
    hp = n[:, 1] > 0
    s = _fixed_sums(plh, q(pv, kp), K)
    want = (s[hp].astype(np.float64) / n[hp, 1] * 2.0 ** -kp).astype(np.float32)
    assert np.array_equal(c[hp, 4].view(np.uint32), want.view(np.uint32))
    hf = n[:, 0] > 0
    s = _fixed_sums(flh, q(fv, kf), K)
    want = (s[hf].astype(np.float64) / n[hf, 0] * 2.0 ** -kf).astype(np.float32)
    assert np.array_equal(c[hf, 5].view(np.uint32), want.view(np.uint32))


def test_merge_and_select_full_size(clustered, orc):
    ctx, wl, fl, pl, c, n, _ = clustered
    for eps in (0.02, 0.05, 0.2):
        m, g = ctx.merge_clusters(c, eps)
        om, og = orc.merge_clusters(c, eps)
        assert g == og and np.array_equal(m, om)
    lo = np.array([-np.inf, -np.inf, -np.inf, 8, -np.inf, 0.5], np.float32)
    hi = np.array([64, np.inf, np.inf, 24, np.inf, np.inf], np.float32)
    assert np.array_equal(ctx.select_clusters(c, lo, hi), orc.select_clusters(c, lo, hi))


def test_stats_full_size(clustered, orc):
    ctx, wl, fl, pl, c, n, _ = clustered
    T = wl.field.shape[0]
    K = len(c)
    g = ctx.cluster_stats(0, T, 0, fl, pl, K)
    f, p, a = (x.cpu().numpy() for x in (wl.field, wl.pos, wl.attr))
    key = ctx.bins("cpu")[0].numpy()
    o = orc.cluster_stats(f, p, a, key, 0, T, 0, fl.cpu().numpy(), pl.cpu().numpy(), K)
    assert np.array_equal(g["n_field"], o["n_field"]) and np.array_equal(g["n_point"], o["n_point"])
    assert np.array_equal(g["lo"], o["lo"]) and np.array_equal(g["hi"], o["hi"])
    assert np.array_equal(g["mean_field"], o["mean_field"], equal_nan=True)
    assert np.array_equal(g["mean_point"], o["mean_point"], equal_nan=True)
    for k in ("std_field", "std_point"):
        ok = ~np.isnan(o[k])
        assert np.array_equal(np.isnan(g[k]), ~ok)
        np.testing.assert_allclose(g[k][ok], o[k][ok], rtol=1e-9)


def test_pieces_full_size(clustered, orc):
    ctx, wl, fl, pl, c, n, seg = clustered
    T = wl.field.shape[0]
    got = ctx.split_trajectories(0, T, pl, 0)
    want = orc.split_trajectories(pl.cpu().numpy(), 2)
    assert np.array_equal(got, want)
    key = ctx.bins("cpu")[0].numpy()
    got = ctx.split_trajectories(wl.t0, wl.t1, seg, 1)
    want = orc.split_trajectories(orc.point_labels(key, wl.t0, seg.cpu().numpy()), 2)
    assert len(want) > 1000 and np.array_equal(got, want)
