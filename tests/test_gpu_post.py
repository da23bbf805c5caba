"""GPU parity of the post-clustering steps against the CPU oracle: cluster merging (§3.3) and
the range query (bit-exact indices), relabelling, per-cluster summaries (counts, extents and
means bit-exact; deviations to 1e-9 relative, their fp64 sums having no fixed order) and
trajectory pieces (§3.4, bit-exact, in both label spaces)."""
import numpy as np
import pytest
import torch

from paper_1903_12294_gb300 import synth

pytestmark = pytest.mark.gpu


def _ctx(gpu, f, p, a, binned=True):
    ctx = gpu.Context(0)
    ctx.load(*(torch.as_tensor(x).cuda().contiguous() for x in (f, p, a)))
    if binned:
        ctx.bin()
    return ctx


def _centres(rng, K, levels=6, jitter=0.01):
    c = rng.normal(size=(K, 6)).astype(np.float32)
    c[:, 4] = (rng.integers(1, levels, K) * (1 + rng.normal(0, jitter, K))).astype(np.float32)
    c[:, 5] = (rng.integers(0, levels, K) * 0.5 + rng.normal(0, jitter, K)).astype(np.float32)
    return c


# ---- §3.3 merging ------------------------------------------------------------------------------

@pytest.mark.parametrize("K,eps,terms", [(1, 0.1, 3), (255, 0.02, 3), (1000, 0.05, 3),
                                         (3001, 0.03, 2), (3001, 0.03, 1), (700, 0.0, 3),
                                         (700, 2.5, 3), (12345, 0.01, 3)])
def test_merge_matches_oracle(gpu, orc, K, eps, terms):
    rng = np.random.default_rng(K)
    c = _centres(rng, K)
    c[::97, 4] = np.nan                                   # NaN matches nothing
    ctx = gpu.Context(0)
    try:
        m, g = ctx.merge_clusters(c, eps, terms)                        # host in, host out
        md = torch.empty(K, dtype=torch.int32, device="cuda")
        m2, g2 = ctx.merge_clusters(torch.as_tensor(c).cuda(), eps, terms, out=md)
        torch.cuda.synchronize()
    finally:
        ctx.close()
    om, og = orc.merge_clusters(c, eps, terms)
    assert g == og and g2 == og
    assert np.array_equal(m, om) and np.array_equal(md.cpu().numpy(), om)


def test_merge_everything_and_errors(gpu):
    rng = np.random.default_rng(1)
    c = rng.normal(size=(5000, 6)).astype(np.float32)
    ctx = gpu.Context(0)
    try:
        m, g = ctx.merge_clusters(c, 3.0)
        assert g == 1 and (m == 0).all()
        for bad in [dict(eps=-1.0), dict(eps=float("nan")), dict(terms=0), dict(terms=4)]:
            args = dict(eps=0.1, terms=3)
            args.update(bad)
            with pytest.raises(gpu.MsfError) as e:
                ctx.merge_clusters(c, args["eps"], args["terms"])
            assert e.value.status == gpu.MSF_ERR_INVALID_ARG
        with pytest.raises(gpu.MsfError) as e:
            ctx.merge_clusters(np.zeros(((1 << 18) + 1, 6), np.float32), 0.1)
        assert e.value.status == gpu.MSF_ERR_TOO_LARGE
    finally:
        ctx.close()


def test_relabel(gpu):
    rng = np.random.default_rng(2)
    K = 900
    mapping = np.minimum(rng.integers(0, K, K), np.arange(K)).astype(np.int32)
    lab = rng.integers(-1, K, size=(7, 33, 65)).astype(np.int32)
    ctx = gpu.Context(0)
    try:
        d = torch.as_tensor(lab).cuda()
        ctx.relabel(d, torch.as_tensor(mapping).cuda())
        want = np.where(lab >= 0, mapping[np.maximum(lab, 0)], lab)
        assert np.array_equal(d.cpu().numpy(), want)
        h = lab.copy()
        ctx.relabel(h, mapping)                                          # host buffers
        assert np.array_equal(h, want)
        bad = lab.copy()
        bad[3, 4, 5] = K
        d = torch.as_tensor(bad).cuda()
        with pytest.raises(gpu.MsfError) as e:
            ctx.relabel(d, torch.as_tensor(mapping).cuda())
        assert e.value.status == gpu.MSF_ERR_INVALID_ARG
        assert np.array_equal(d.cpu().numpy(), bad)                     # unchanged
    finally:
        ctx.close()


# ---- §3.4 range query ----------------------------------------------------------------------

@pytest.mark.parametrize("K", [1, 777, 100000])
def test_select_matches_oracle(gpu, orc, K):
    rng = np.random.default_rng(K + 3)
    c = rng.normal(size=(K, 6)).astype(np.float32)
    lo = np.array([-1, -np.inf, -0.5, -2, -np.inf, 0], np.float32)
    hi = np.array([1, 0.5, np.inf, 2, 1, np.inf], np.float32)
    ctx = gpu.Context(0)
    try:
        got = ctx.select_clusters(c, lo, hi)
        got_d = ctx.select_clusters(torch.as_tensor(c).cuda(), lo, hi)
        none = ctx.select_clusters(c, np.full(6, np.inf, np.float32),
                                   np.full(6, -np.inf, np.float32))
        with pytest.raises(gpu.MsfError) as e:
            ctx.select_clusters(c, np.full(6, np.nan, np.float32), hi)
        assert e.value.status == gpu.MSF_ERR_INVALID_ARG
    finally:
        ctx.close()
    want = orc.select_clusters(c, lo, hi)
    assert np.array_equal(got, want) and np.array_equal(got_d, want) and none.size == 0


# ---- §3.4 summaries ------------------------------------------------------------------------

def _check_stats(g, o):
    assert np.array_equal(g["n_field"], o["n_field"])
    assert np.array_equal(g["n_point"], o["n_point"])
    assert np.array_equal(g["lo"], o["lo"]) and np.array_equal(g["hi"], o["hi"])
    for k in ("mean_field", "mean_point"):
        assert np.array_equal(g[k], o[k], equal_nan=True), k
    for k in ("std_field", "std_point"):
        a, b = g[k], o[k]
        assert np.array_equal(np.isnan(a), np.isnan(b)), k
        np.testing.assert_allclose(a[~np.isnan(a)], b[~np.isnan(b)], rtol=1e-9, atol=1e-300)


def test_stats_of_a_clustering(gpu, orc):
    wl = synth.mid(n=40, T=10, P=30000, n_blobs=8)
    f, p, a = wl.numpy()
    ctx = _ctx(gpu, f, p, a)
    try:
        fl, pl, c, n, it = ctx.cluster(2, 10, 1, (4, 3, 3, 2), w_p=1.0, w_f=2.0, w_d=0.2,
                                       max_iter=5)
        K = len(c)
        g = ctx.cluster_stats(2, 10, 1, fl, pl, K)
        gh = ctx.cluster_stats(2, 10, 1, fl.cpu().numpy(), pl.cpu().numpy(), K)  # host labels
        key = ctx.bins("cpu")[0].numpy()
        flh, plh = fl.cpu().numpy(), pl.cpu().numpy()
    finally:
        ctx.close()
    o = orc.cluster_stats(f, p, a, key, 2, 10, 1, flh, plh, K)
    _check_stats(g, o)
    _check_stats(gh, o)
    assert (g["n_field"] == n[:, 0]).all() and (g["n_point"] == n[:, 1]).all()


def test_stats_random_labels_and_invalid_samples(gpu, orc):
    rng = np.random.default_rng(6)
    T, nz, ny, nx, P, K = 5, 6, 7, 9, 800, 7
    f = rng.normal(2.0, 1.5, size=(T, nz, ny, nx)).astype(np.float32)
    f[1, 2, 3, 4] = np.nan
    pos = (rng.random((T, 3, P)) * np.array([nx, ny, nz])[None, :, None]).astype(np.float32)
    pos[2, 0, 5] = -4.0
    pos[3, 1, 9] = -0.0
    a = rng.normal(size=(T, 2, P)).astype(np.float32)
    a[3, 1, 6] = np.inf
    fl = rng.integers(-1, K, size=(4, nz, ny, nx)).astype(np.int32)
    fl[:, :, :2, :] = 3                                      # warp-uniform runs
    pl = rng.integers(-1, K, size=(4, P)).astype(np.int32)
    pl[:, :64] = 5
    ctx = _ctx(gpu, f, pos, a)
    try:
        g = ctx.cluster_stats(1, 5, 1, torch.as_tensor(fl).cuda(), torch.as_tensor(pl).cuda(), K)
        gf = ctx.cluster_stats(1, 5, 1, torch.as_tensor(fl).cuda(), None, K + 2)  # field only
        key = ctx.bins("cpu")[0].numpy()
        bad = fl.copy()
        bad[0, 0, 0, 0] = K
        with pytest.raises(gpu.MsfError) as e:
            ctx.cluster_stats(1, 5, 1, torch.as_tensor(bad).cuda(), None, K)
        assert e.value.status == gpu.MSF_ERR_INVALID_ARG
    finally:
        ctx.close()
    _check_stats(g, orc.cluster_stats(f, pos, a, key, 1, 5, 1, fl, pl, K))
    _check_stats(gf, orc.cluster_stats(f, pos, a, key, 1, 5, 1, fl, None, K + 2))


# ---- §3.4 trajectory pieces -------------------------------------------------------------------

@pytest.mark.parametrize("min_len", [1, 2, 3])
def test_pieces_of_point_labels(gpu, orc, min_len):
    wl = synth.mid(n=40, T=10, P=30000, n_blobs=8)
    f, p, a = wl.numpy()
    ctx = _ctx(gpu, f, p, a)
    try:
        fl, pl, c, n, it = ctx.cluster(0, 10, 1, (4, 4, 2, 2), w_p=1.0, w_f=1.0, w_d=0.1,
                                       max_iter=4)
        got = ctx.split_trajectories(0, 10, pl, gpu.MSF_SPACE_POINTS, min_len)
        plh = pl.cpu().numpy()
        got_h = ctx.split_trajectories(0, 10, plh, gpu.MSF_SPACE_POINTS, min_len)
    finally:
        ctx.close()
    want = orc.split_trajectories(plh, min_len)
    assert len(want) > 0
    assert np.array_equal(got, want) and np.array_equal(got_h, want)


def test_pieces_of_voxel_labels(gpu, orc):
    """Feature labels from msf_segment; each sample takes its binned voxel's label."""
    wl = synth.mid(n=48, T=12, P=40000, n_blobs=10)
    f, p, a = wl.numpy()
    ctx = _ctx(gpu, f, p, a)
    try:
        lab, nfeat = ctx.segment(3, 12, wl.preds, wl.edges)
        got = ctx.split_trajectories(3, 12, lab, gpu.MSF_SPACE_VOXELS, 2)
        out = torch.zeros((len(got) + 5, 4), dtype=torch.int32, device="cuda")
        _, n = ctx.split_trajectories(3, 12, lab, gpu.MSF_SPACE_VOXELS, 2, out=out)
        small = torch.zeros((max(len(got) - 1, 0), 4), dtype=torch.int32, device="cuda")
        with pytest.raises(gpu.MsfError) as e:
            ctx.split_trajectories(3, 12, lab, gpu.MSF_SPACE_VOXELS, 2, out=small)
        assert e.value.status == gpu.MSF_ERR_CAPACITY
        key = ctx.bins("cpu")[0].numpy()
        labh = lab.cpu().numpy()
    finally:
        ctx.close()
    want = orc.split_trajectories(orc.point_labels(key, 3, labh), 2)
    assert len(want) > 100
    assert np.array_equal(got, want)
    assert n == len(want) and np.array_equal(out[:n].cpu().numpy(), want)
    assert (small.cpu().numpy() == 0).all()                   # nothing written


def test_pieces_edge_cases(gpu, orc):
    rng = np.random.default_rng(12)
    T, nz, ny, nx, P = 6, 4, 5, 6, 4099
    f = rng.normal(size=(T, nz, ny, nx)).astype(np.float32)
    pos = (rng.random((T, 3, P)) * np.array([nx, ny, nz])[None, :, None]).astype(np.float32)
    a = rng.normal(size=(T, 1, P)).astype(np.float32)
    ctx = _ctx(gpu, f, pos, a, binned=False)
    try:
        pl = rng.integers(-1, 3, size=(T, P)).astype(np.int32)
        pl[:, 100:200] = 2                                    # whole trajectories in one label
        for t0, t1, ml in [(0, 6, 2), (2, 3, 1), (2, 3, 2), (0, 6, 6), (1, 5, 4)]:
            got = ctx.split_trajectories(t0, t1, pl[: t1 - t0], gpu.MSF_SPACE_POINTS, ml)
            assert np.array_equal(got, orc.split_trajectories(pl[: t1 - t0], ml)), (t0, t1, ml)
        with pytest.raises(gpu.MsfError) as e:                # voxel space needs binning
            ctx.split_trajectories(0, 6, np.zeros((T, nz, ny, nx), np.int32),
                                   gpu.MSF_SPACE_VOXELS, 2)
        assert e.value.status == gpu.MSF_ERR_NOT_BINNED
        for bad in [dict(t0=3, t1=3), dict(t1=7), dict(ml=0), dict(space=5)]:
            args = dict(t0=0, t1=6, ml=2, space=gpu.MSF_SPACE_POINTS)
            args.update(bad)
            with pytest.raises(gpu.MsfError) as e:
                ctx.split_trajectories(args["t0"], args["t1"], pl, args["space"], args["ml"])
            assert e.value.status == gpu.MSF_ERR_INVALID_ARG
    finally:
        ctx.close()


def test_merge_at_the_largest_k(gpu):
    """K = 2^18 (the limit): distinct values at eps_m = 0 give every centre its own group (the
    identity map); eps_m above 2 gives one group. Closed forms, no oracle needed at this size."""
    K = 1 << 18
    c = np.zeros((K, 6), np.float32)
    c[:, 4] = np.arange(K, dtype=np.float32) + 1.0
    c[:, 5] = -(np.arange(K, dtype=np.float32) + 1.0)
    ctx = gpu.Context(0)
    try:
        m, g = ctx.merge_clusters(torch.as_tensor(c).cuda(), 0.0,
                                  out=torch.empty(K, dtype=torch.int32, device="cuda"))
        assert g == K and np.array_equal(m.cpu().numpy(), np.arange(K, dtype=np.int32))
        m, g = ctx.merge_clusters(c, 3.0)
        assert g == 1 and (m == 0).all()
    finally:
        ctx.close()


def test_pieces_without_points(gpu):
    """A dataset without points has no trajectory pieces."""
    rng = np.random.default_rng(0)
    f = rng.normal(size=(4, 3, 5, 8)).astype(np.float32)
    ctx = gpu.Context(0)
    try:
        ctx.load(torch.as_tensor(f).cuda(), None, None)
        got = ctx.split_trajectories(0, 4, np.zeros((4, 0), np.int32), gpu.MSF_SPACE_POINTS)
        assert got.shape == (0, 4)
    finally:
        ctx.close()
