"""Pins of the post-clustering oracle (§3.3 merging, §3.4 summaries, range queries and
trajectory pieces) against closed forms, invariants and independent brute force."""
import itertools

import numpy as np
import pytest

from paper_1903_12294_gb300 import synth


# ---- §3.4 trajectory pieces -------------------------------------------------------------------

def _pieces_by_groupby(pl, min_len):
    """Independent restatement: group each trajectory's labels into runs with itertools."""
    tw, P = pl.shape
    out = []
    for p in range(P):
        t = 0
        for lab, run in itertools.groupby(pl[:, p].tolist()):
            n = len(list(run))
            if lab >= 0 and n >= min_len:
                out.append((p, t, n, lab))
            t += n
    return np.array(out, np.int32).reshape(-1, 4)


@pytest.mark.parametrize("min_len", [1, 2, 3])
def test_pieces_match_groupby(orc, min_len):
    rng = np.random.default_rng(4)
    pl = rng.integers(-1, 3, size=(17, 300)).astype(np.int32)
    pl[:, :40] = np.repeat(rng.integers(-1, 3, size=(17, 1)), 40, axis=1)  # some long runs
    got = orc.split_trajectories(pl, min_len)
    assert np.array_equal(got, _pieces_by_groupby(pl, min_len))


def test_pieces_special_cases(orc):
    tw, P = 9, 50
    const = np.full((tw, P), 7, np.int32)
    got = orc.split_trajectories(const, 2)
    assert np.array_equal(got, np.stack([np.arange(P), np.zeros(P), np.full(P, tw),
                                         np.full(P, 7)], 1).astype(np.int32))
    assert orc.split_trajectories(np.full((tw, P), -1, np.int32), 1).shape == (0, 4)
    alt = np.where(np.arange(tw)[:, None] % 2 == 0, 3, 4).astype(np.int32).repeat(P, 1)
    assert orc.split_trajectories(alt, 2).shape == (0, 4)            # no two steps in a row
    assert orc.split_trajectories(alt, 1).shape == (tw * P, 4)
    # min_len = 1 covers every labelled sample exactly once
    rng = np.random.default_rng(9)
    pl = rng.integers(-2, 5, size=(13, 77)).astype(np.int32)
    got = orc.split_trajectories(pl, 1)
    assert got[:, 2].sum() == (pl >= 0).sum()
    # one timestep: pieces of length 1 only
    assert orc.split_trajectories(pl[:1], 2).shape == (0, 4)


def test_point_labels_from_voxels(orc):
    """Voxel space: a sample takes the label of its binned voxel, -1 outside the grid."""
    wl = synth.tiny(T=6, P=3000)
    f, p, a = wl.numpy()
    o = orc.bin(f.shape, p, a, keep_sumq=False)
    rng = np.random.default_rng(1)
    T, nz, ny, nx = f.shape
    vl = rng.integers(-1, 50, size=(4, nz, ny, nx)).astype(np.int32)
    got = orc.point_labels(o["key"], 2, vl)
    key = o["key"][2:6]
    want = np.where(key >= 0, vl.reshape(4, -1)[np.arange(4)[:, None], np.maximum(key, 0)], -1)
    assert np.array_equal(got, want)


# ---- §3.3 merging -------------------------------------------------------------------------

def _centres(vals_p, vals_f):
    c = np.zeros((len(vals_p), 6), np.float32)
    c[:, 4] = vals_p
    c[:, 5] = vals_f
    return c


def test_merge_zero_threshold_groups_identical_values(orc):
    rng = np.random.default_rng(3)
    vp = rng.integers(0, 4, 200).astype(np.float32)
    vf = rng.integers(0, 3, 200).astype(np.float32) * 0.5
    m, g = orc.merge_clusters(_centres(vp, vf), 0.0)
    pairs = np.stack([vp, vf], 1)
    _, first, inv = np.unique(pairs, axis=0, return_index=True, return_inverse=True)
    assert g == len(first)
    assert np.array_equal(m, first[inv.ravel()].astype(np.int32))


def test_merge_threshold_above_two_merges_everything(orc):
    """The percent difference never exceeds 2, so eps_m > 2 joins every pair."""
    rng = np.random.default_rng(5)
    c = _centres(rng.normal(size=300).astype(np.float32), rng.normal(size=300).astype(np.float32))
    m, g = orc.merge_clusters(c, 2.01)
    assert g == 1 and (m == 0).all()


def test_merge_is_transitive(orc):
    """1.00 ~ 1.04 ~ 1.08 ~ 1.12 pairwise at 5 % (percent difference about 3.9 %), 1.00 vs 1.08
    not (7.7 %): one group all the same; 3.0 stays alone."""
    c = _centres([1.08, 3.0, 1.0, 1.12, 1.04], [2.0] * 5)
    m, g = orc.merge_clusters(c, 0.05)
    assert g == 2 and list(m) == [0, 1, 0, 0, 0]


def test_merge_needs_both_terms(orc):
    """Field values match, point values do not: merged on the field term alone, not on both."""
    c = _centres([0.0, 10.0, 20.0], [5.0, 5.01, 4.99])
    assert orc.merge_clusters(c, 0.01, orc.MERGE_POINT | orc.MERGE_FIELD)[1] == 3
    m, g = orc.merge_clusters(c, 0.01, orc.MERGE_FIELD)
    assert g == 1 and (m == 0).all()
    m, g = orc.merge_clusters(c, 0.01, orc.MERGE_POINT)
    assert g == 3 and list(m) == [0, 1, 2]


def test_merge_groups_are_graph_components(orc):
    """Groups equal the connected components (networkx) of the pairwise match graph; the
    labels are each component's smallest index."""
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(8)
    K = 120
    vp = (rng.integers(1, 6, K) + rng.normal(0, 0.02, K)).astype(np.float32)
    vf = (rng.integers(1, 4, K) + rng.normal(0, 0.02, K)).astype(np.float32)
    eps = np.float32(0.03)
    m, g = orc.merge_clusters(_centres(vp, vf), float(eps))

    def match(a, b):
        return (a == b) | (np.float32(2) * np.abs(a - b) < eps * (np.abs(a) + np.abs(b)))

    G = nx.Graph()
    G.add_nodes_from(range(K))
    ok = match(vp[:, None], vp[None, :]) & match(vf[:, None], vf[None, :])
    G.add_edges_from(zip(*np.nonzero(np.triu(ok, 1))))
    want = np.empty(K, np.int32)
    comps = list(nx.connected_components(G))
    for comp in comps:
        want[list(comp)] = min(comp)
    assert g == len(comps) and np.array_equal(m, want)


# ---- §3.4 range query ----------------------------------------------------------------------

def test_select_is_a_box_filter(orc):
    rng = np.random.default_rng(2)
    c = rng.normal(size=(500, 6)).astype(np.float32)
    lo = np.array([-1, -np.inf, -0.5, -2, -np.inf, 0], np.float32)
    hi = np.array([1, 0.5, np.inf, 2, 1, np.inf], np.float32)
    got = orc.select_clusters(c, lo, hi)
    want = np.nonzero(((c >= lo) & (c <= hi)).all(1))[0]
    assert np.array_equal(got, want)
    assert orc.select_clusters(c, np.full(6, np.inf, np.float32), np.full(6, -np.inf,
                                                                          np.float32)).size == 0


# ---- §3.4 summaries ------------------------------------------------------------------------

def _clustered(seed=6, T=5, K=7):
    rng = np.random.default_rng(seed)
    nz, ny, nx = 6, 7, 9
    P = 800
    f = rng.normal(2.0, 1.5, size=(T, nz, ny, nx)).astype(np.float32)
    f[1, 2, 3, 4] = np.nan
    pos = (rng.random((T, 3, P)) * np.array([nx, ny, nz])[None, :, None]).astype(np.float32)
    pos[2, 0, 5] = -4.0                                     # outside the grid
    a = rng.normal(size=(T, 2, P)).astype(np.float32)
    a[3, 1, 6] = np.inf
    return f, pos, a, rng


def test_stats_match_numpy(orc):
    f, pos, a, rng = _clustered()
    T, nz, ny, nx = f.shape
    P = pos.shape[2]
    K, t0, t1 = 7, 1, 5
    o = orc.bin(f.shape, pos, a, keep_sumq=False)
    fl = rng.integers(-1, K, size=(t1 - t0, nz, ny, nx)).astype(np.int32)
    pl = rng.integers(-1, K, size=(t1 - t0, P)).astype(np.int32)
    r = orc.cluster_stats(f, pos, a, o["key"], t0, t1, 1, fl, pl, K)
    tt, zz, yy, xx = np.meshgrid(np.arange(t0, t1), np.arange(nz), np.arange(ny), np.arange(nx),
                                 indexing="ij")
    fv = f[t0:t1]
    pv = a[t0:t1, 1]
    inside = o["key"][t0:t1] >= 0
    for c in range(K):
        sel = (fl == c) & np.isfinite(fv)
        psel = (pl == c) & inside & np.isfinite(pv)
        assert r["n_field"][c] == sel.sum() and r["n_point"][c] == psel.sum()
        vals = fv[sel].astype(np.float64)
        np.testing.assert_allclose(r["mean_field"][c], vals.mean(), rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(r["std_field"][c], vals.std(), rtol=1e-9)
        pvals = pv[psel].astype(np.float64)
        np.testing.assert_allclose(r["mean_point"][c], pvals.mean(), rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(r["std_point"][c], pvals.std(), rtol=1e-9)
        px = [pos[t0:t1, i][psel] for i in range(3)]
        lo = [min(xx[sel].min() + 0.5, px[0].min()), min(yy[sel].min() + 0.5, px[1].min()),
              min(zz[sel].min() + 0.5, px[2].min()),
              min(tt[sel].min(), np.nonzero(psel)[0].min() + t0) + 0.5]
        hi = [max(xx[sel].max() + 0.5, px[0].max()), max(yy[sel].max() + 0.5, px[1].max()),
              max(zz[sel].max() + 0.5, px[2].max()),
              max(tt[sel].max(), np.nonzero(psel)[0].max() + t0) + 0.5]
        assert np.array_equal(r["lo"][c], np.array(lo, np.float32))
        assert np.array_equal(r["hi"][c], np.array(hi, np.float32))


def test_stats_one_cluster_and_empty_clusters(orc):
    """K = 1 over every sample gives the window's global mean and deviation; a cluster with no
    samples has zero counts, infinite extents and NaN moments; point labels may be left out."""
    f, pos, a, _ = _clustered(T=4)
    o = orc.bin(f.shape, pos, a, keep_sumq=False)
    fl = np.zeros(f.shape, np.int32)
    r = orc.cluster_stats(f, pos, a, o["key"], 0, 4, 0, fl, None, 3)
    vals = f[np.isfinite(f)].astype(np.float64)
    np.testing.assert_allclose(r["mean_field"][0], vals.mean(), rtol=1e-12)
    np.testing.assert_allclose(r["std_field"][0], vals.std(), rtol=1e-9)
    assert (r["n_point"] == 0).all() and (r["n_field"][1:] == 0).all()
    assert np.isinf(r["lo"][1:]).all() and np.isnan(r["mean_field"][1:]).all()
    assert np.isnan(r["std_point"]).all()
    with pytest.raises(RuntimeError):                       # a label >= K
        orc.cluster_stats(f, pos, a, o["key"], 0, 4, 0, fl + 3, None, 3)
