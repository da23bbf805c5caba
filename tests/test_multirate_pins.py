"""Pins of the CPU oracle for point samples on a finer time grid than the field (§3.4: point
and field data need not share a temporal resolution; §4.1: the particles are saved far more
often than the field). Point step j falls in field step fstep[j]. None of these re-uses the
oracle's code path: counts come from numpy, sums from Python integers, connectivity from
scipy's connected components over an explicit edge list built here."""
from fractions import Fraction

import numpy as np
import pytest

F, C, M = 0, 1, 2
GT, GE, LT, LE, BAND = 0, 1, 2, 3, 4


def _inputs(rng, Tp, nz, ny, nx, P, A):
    pos = np.stack([rng.uniform(-0.3, n + 0.3, (Tp, P)) for n in (nx, ny, nz)],
                   1).astype(np.float32)
    attr = rng.normal(size=(Tp, A, P)).astype(np.float32)
    return pos, attr


def test_multirate_bin_counts_and_exact_sums(orc):
    """Counts per (field step, voxel) are numpy's over all samples of the point steps that fall
    in the field step; the fixed-point scale counts every point sample (P * Tp); the int64
    sums equal exact Python-integer sums of the quantised values."""
    rng = np.random.default_rng(7)
    T, nz, ny, nx, P, A = 3, 2, 3, 4, 150, 2
    fstep = np.array([0, 0, 0, 1, 2, 2, 2], np.int32)
    Tp = fstep.size
    pos, attr = _inputs(rng, Tp, nz, ny, nx, P, A)
    b = orc.bin((T, nz, ny, nx), pos, attr, fstep=fstep)
    V = nx * ny * nz
    assert b["key"].shape == (Tp, P) and b["outside"].shape == (Tp,)
    maxabs = np.abs(attr).max(axis=(0, 2))
    for a in range(A):
        assert int(b["kscale"][a]) == orc.scale_exponent(float(maxabs[a]), P * Tp)
    cnt = b["count"].reshape(T, V)
    for t in range(T):
        js = np.nonzero(fstep == t)[0]
        keys = b["key"][js].reshape(-1)
        assert np.array_equal(cnt[t], np.bincount(keys[keys >= 0], minlength=V))
        for a in range(A):
            k = int(b["kscale"][a])
            vals = attr[js, a, :].reshape(-1)
            for v in range(V):
                exact = sum(round(Fraction(float(x)) * Fraction(2) ** k) for x in vals[keys == v])
                assert int(b["sumq"].reshape(A, T, V)[a, t, v]) == exact
    assert np.all(b["count"].reshape(T, V).sum(1) ==
                  [sum(P - b["outside"][j] for j in np.nonzero(fstep == t)[0]) for t in range(T)])


def _mr_labels(active, key, fstep, t0, edges):
    """Canonical labels from scipy connected components over an explicit edge list: spatial
    26-neighbours, same voxel at t and t+1, and (key[j][p], fstep[j])-(key[j+1][p], fstep[j+1])
    for consecutive point steps whose field steps both lie in the window."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    Tw, nz, ny, nx = active.shape
    V = nz * ny * nx
    N = active.size
    flat = active.reshape(-1)
    idx = np.arange(N).reshape(active.shape)
    us, ws = [], []
    offs = []
    if edges & 1:
        offs += [(0, dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
                 if (dz, dy, dx) != (0, 0, 0)]
    if edges & 2:
        offs.append((1, 0, 0, 0))
    for d in offs:
        for t in range(Tw):
            for z in range(nz):
                for y in range(ny):
                    for x in range(nx):
                        T2, Z, Y, X = t + d[0], z + d[1], y + d[2], x + d[3]
                        if 0 <= T2 < Tw and 0 <= Z < nz and 0 <= Y < ny and 0 <= X < nx:
                            if active[t, z, y, x] and active[T2, Z, Y, X]:
                                us.append(idx[t, z, y, x])
                                ws.append(idx[T2, Z, Y, X])
    if edges & 4:
        for j in range(key.shape[0] - 1):
            ta, tb = int(fstep[j]) - t0, int(fstep[j + 1]) - t0
            if ta < 0 or tb >= Tw:
                continue
            for p in range(key.shape[1]):
                a, b = int(key[j, p]), int(key[j + 1, p])
                if a < 0 or b < 0:
                    continue
                u, w = ta * V + a, tb * V + b
                if flat[u] and flat[w]:
                    us.append(u)
                    ws.append(w)
    G = sp.coo_matrix((np.ones(len(us), np.int8), (us, ws)), shape=(N, N)).tocsr()
    _, comp = connected_components(G, directed=False)
    lab = np.full(N, -1, np.int64)
    ids = np.nonzero(flat)[0]
    cmin = {}
    for i in ids:
        cmin.setdefault(comp[i], i)
    lab[ids] = [cmin[comp[i]] for i in ids]
    return lab.reshape(active.shape)


@pytest.mark.parametrize("edges", range(8))
def test_multirate_segment_matches_csgraph(orc, edges):
    """Random field, points on a grid of 3 point steps per field step (plus an uneven tail):
    the oracle's labels of a window equal the canonical components of the explicit graph."""
    rng = np.random.default_rng(100 + edges)
    T, nz, ny, nx, P = 4, 3, 4, 5, 40
    fstep = np.array([0, 0, 0, 1, 1, 1, 2, 2, 2, 3, 3], np.int32)
    Tp = fstep.size
    field = rng.uniform(0, 1, (T, nz, ny, nx)).astype(np.float32)
    pos, attr = _inputs(rng, Tp, nz, ny, nx, P, 1)
    b = orc.bin(field.shape, pos, attr, fstep=fstep)
    t0, t1 = 1, 4
    preds = [(F, 0, GT, 0.72, 0.0)]
    lab, nf = orc.segment(field, b["count"], b["mean"], b["key"], t0, t1, preds, edges, fstep)
    active = field[t0:t1] > np.float32(0.72)
    ref = _mr_labels(active, b["key"], fstep, t0, edges)
    assert np.array_equal(lab, ref)
    assert nf == int(np.count_nonzero(ref.reshape(-1) == np.arange(ref.size)))


def test_multirate_links_within_one_field_step_closed_form(orc):
    """One point visits voxels x = 0, 2, 4, 6 of a row at four point steps that all fall in
    field step 0; the four voxels are active and not adjacent: with trajectory links they form
    one feature of four voxels inside one field step, without them four features; a second field
    step with the point resting in x = 6 joins through the next point step."""
    T, nz, ny, nx = 2, 1, 1, 8
    fstep = np.array([0, 0, 0, 0, 1], np.int32)
    xs = [0.5, 2.5, 4.5, 6.5, 6.5]
    pos = np.array([[[x], [0.5], [0.5]] for x in xs], np.float32)
    attr = np.ones((5, 1, 1), np.float32)
    field = np.zeros((T, nz, ny, nx), np.float32)
    field[0, 0, 0, [0, 2, 4, 6]] = 1.0
    field[1, 0, 0, 6] = 1.0
    b = orc.bin(field.shape, pos, attr, fstep=fstep)
    pr = [(F, 0, GT, 0.5, 0.0)]
    lab, nf = orc.segment(field, b["count"], b["mean"], b["key"], 0, 1, pr, 7, fstep)
    assert nf == 1 and lab[0, 0, 0, [0, 2, 4, 6]].tolist() == [0, 0, 0, 0]
    lab, nf = orc.segment(field, b["count"], b["mean"], b["key"], 0, 1, pr, 3, fstep)
    assert nf == 4
    lab, nf = orc.segment(field, b["count"], b["mean"], b["key"], 0, 2, pr, 5, fstep)
    assert nf == 1 and lab[1, 0, 0, 6] == 0          # spatial + trajectory, no temporal edge
    feat = orc.features(field, b["count"], attr, b["key"], b["kscale"], 0, 2, lab, fstep)
    assert feat["n_vox"].tolist() == [5] and feat["n_pts"].tolist() == [5]
    assert b["count"][0, 0, 0, [0, 2, 4, 6]].tolist() == [1, 1, 1, 1]


def test_multirate_repeated_steps_reduce_to_one_rate(orc):
    """Every field step holding r identical copies of one point step: counts are r times the
    one-rate counts, means, labels and features' means and deviations are the one-rate ones,
    and n_pts is r times (the links between copies join a voxel-timestep to itself)."""
    from paper_1903_12294_gb300 import synth
    wl = synth.tiny(n=16, T=4, P=3000)
    f, p, a = wl.numpy()
    T = f.shape[0]
    r = 3
    fstep = np.repeat(np.arange(T, dtype=np.int32), r)
    p3, a3 = np.repeat(p, r, axis=0), np.repeat(a, r, axis=0)
    b1, lab1, nf1, f1 = orc.run_all(f, p, a, 0, T, wl.preds)
    b3, lab3, nf3, f3 = orc.run_all(f, p3, a3, 0, T, [(F, 0, GT, 0.4, 0.0), (C, 0, GE, 2 * r, 0)],
                                    fstep=fstep)
    assert np.array_equal(b3["count"], r * b1["count"])
    assert np.array_equal(b3["mean"].view(np.uint32), b1["mean"].view(np.uint32)) or \
        np.allclose(b3["mean"], b1["mean"], rtol=2.5e-7, equal_nan=True)
    assert nf3 == nf1 and np.array_equal(lab3, lab1)
    assert np.array_equal(f3["n_pts"], r * f1["n_pts"])
    np.testing.assert_allclose(f3["mean_attr"], f1["mean_attr"], rtol=1e-12)
    np.testing.assert_allclose(f3["std_attr"], f1["std_attr"], rtol=1e-9, atol=1e-12)


def test_multirate_cluster_one_centre_time_is_the_step_mean(orc):
    """§3.2 with points on their own grid, k = 1: the r point steps of field step f sit
    symmetrically about f + 0.5 (at f + (i + 0.5) / r), so after one update the one centre's time
    is the mean over all samples of their field step + 0.5, whatever the map (with every point
    inside the grid); its position is the mean of voxel centres and point positions, and it
    counts every sample of the window."""
    rng = np.random.default_rng(41)
    T, nz, ny, nx, P, A = 4, 3, 5, 6, 40, 2
    fstep = np.array([0, 0, 0, 1, 2, 2, 2, 2, 2, 3, 3], np.int32)
    Tp = fstep.size
    pos, attr = _inputs(rng, Tp, nz, ny, nx, P, A)
    # every point inside the grid: each point step takes part with all P samples (the symmetry
    # about f + 0.5 holds for whole point steps)
    pos = np.stack([rng.uniform(0.05, m - 0.05, (Tp, P)) for m in (nx, ny, nz)],
                   1).astype(np.float32)
    field = rng.random((T, nz, ny, nx)).astype(np.float32)
    b = orc.bin(field.shape, pos, attr, fstep=fstep)
    t0, t1 = 1, 4
    fl, pl, c, n, it = orc.slic(field, pos, attr, b["key"], t0, t1, 1, (1, 1, 1, 1),
                                max_iter=1, fstep=fstep)
    js = np.nonzero((fstep >= t0) & (fstep < t1))[0]
    assert pl.shape == (js.size, P)
    inside = b["key"][js] >= 0
    assert np.array_equal(pl >= 0, inside) and (pl[inside] == 0).all() and (fl == 0).all()
    nvox = nz * ny * nx
    tf = np.repeat(np.arange(t0, t1) + 0.5, nvox)
    tp = np.repeat(fstep[js] + 0.5, P)[inside.ravel()]
    assert n[0, 0] == tf.size and n[0, 1] == tp.size
    np.testing.assert_allclose(float(c[0, 3]), np.concatenate([tf, tp]).mean(), rtol=2e-7)
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    px = pos[js, 0, :].astype(np.float64)[inside]
    fx = np.tile((xx + 0.5).ravel(), t1 - t0)
    np.testing.assert_allclose(float(c[0, 0]), np.concatenate([fx, px]).mean(), rtol=2e-7)
    np.testing.assert_allclose(float(c[0, 4]), attr[js, 1, :].astype(np.float64)[inside].mean(),
                               rtol=2e-6)


@pytest.mark.parametrize("r", [2, 3])
def test_multirate_cluster_point_steps_join_their_time_seed(orc, r):
    """k = (1, 1, 1, r tw) on a map of r point steps per field step: the seeds' times,
    t0 + (m + 0.5) / r, are exactly the point times f + (i + 0.5) / r, and all seeds share one
    position, so the first assignment puts point step jj of the window (and nothing else) on
    seed jj; field samples at f + 0.5 lie between two seeds for even r (the tie goes to the
    lower one) and on seed r (f - t0) + (r - 1) / 2 for odd r."""
    rng = np.random.default_rng(43 + r)
    T, nz, ny, nx, P, A = 3, 2, 3, 4, 30, 1
    fstep = np.repeat(np.arange(T, dtype=np.int32), r)
    pos, attr = _inputs(rng, fstep.size, nz, ny, nx, P, A)
    field = rng.random((T, nz, ny, nx)).astype(np.float32)
    b = orc.bin(field.shape, pos, attr, fstep=fstep)
    t0, t1 = 1, 3
    tw = t1 - t0
    fl, pl, c, n, it = orc.slic(field, pos, attr, b["key"], t0, t1, 0, (1, 1, 1, r * tw),
                                max_iter=1, fstep=fstep)
    inside = b["key"][r * t0:r * t1] >= 0
    want = np.broadcast_to(np.arange(r * tw)[:, None], inside.shape)
    assert np.array_equal(pl[inside], want[inside]) and (pl[~inside] == -1).all()
    fwant = r * np.arange(tw) + (r - 1) // 2
    assert np.array_equal(fl.reshape(tw, -1), np.broadcast_to(fwant[:, None], (tw, nz * ny * nx)))
