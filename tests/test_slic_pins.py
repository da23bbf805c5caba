"""Pins of the clustering oracle (§3.2) against closed forms and invariants independent of it."""
import numpy as np
import pytest

from paper_1903_12294_gb300 import synth


def _data(seed=3, T=6, n=(20, 12, 10), P=1500, A=2):
    rng = np.random.default_rng(seed)
    nx, ny, nz = n
    f = rng.normal(size=(T, nz, ny, nx)).astype(np.float32)
    pos = (rng.random((T, 3, P)) * np.array([nx, ny, nz])[None, :, None]).astype(np.float32)
    a = rng.normal(size=(T, A, P)).astype(np.float32)
    return f, pos, a


def test_one_centre_is_the_global_mean(orc):
    """k = 1: after one update the centre holds the means of all samples (field samples at
    voxel centres, points at their positions, time t + 0.5)."""
    f, p, a = _data()
    T, nz, ny, nx = f.shape
    o = orc.bin(f.shape, p, a, keep_sumq=False)
    fl, pl, c, n, it = orc.slic(f, p, a, o["key"], 1, T, 1, (1, 1, 1, 1), max_iter=1)
    assert it == 1 and (fl == 0).all() and (pl == 0).all()
    tw = T - 1
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    fx = np.broadcast_to(xx + 0.5, (tw, nz, ny, nx)).ravel()
    fy = np.broadcast_to(yy + 0.5, (tw, nz, ny, nx)).ravel()
    fz = np.broadcast_to(zz + 0.5, (tw, nz, ny, nx)).ravel()
    ft = np.broadcast_to((np.arange(1, T) + 0.5)[:, None, None, None], (tw, nz, ny, nx)).ravel()
    P = p.shape[2]
    px, py, pz = (p[1:, i, :].astype(np.float64).ravel() for i in range(3))
    pt = np.repeat(np.arange(1, T) + 0.5, P)
    want = [np.concatenate([fx, px]).mean(), np.concatenate([fy, py]).mean(),
            np.concatenate([fz, pz]).mean(), np.concatenate([ft, pt]).mean(),
            a[1:, 1, :].astype(np.float64).mean(), f[1:].astype(np.float64).mean()]
    np.testing.assert_allclose(c[0].astype(np.float64), want, rtol=2e-7, atol=1e-6)
    assert n[0, 0] == f[1:].size and n[0, 1] == P * tw


@pytest.mark.parametrize("k", [(4, 3, 2, 2), (3, 5, 1, 3), (7, 1, 2, 1)])
def test_first_assignment_is_the_seed_voronoi(orc, k):
    """Before any update every sample belongs to the nearest seed; on a rectilinear grid of
    seeds that is the grid cell holding the sample along each axis independently (samples
    within 1e-3 of a cell border are skipped: there the fp32 distances decide)."""
    f, p, a = _data()
    T, nz, ny, nx = f.shape
    o = orc.bin(f.shape, p, a, keep_sumq=False)
    fl, pl, c, n, it = orc.slic(f, p, a, o["key"], 0, T, 0, k, max_iter=1)
    C = np.array([nx / k[0], ny / k[1], nz / k[2], T / k[3]])

    def cells(x, y, z, t):
        u = np.stack([x / C[0], y / C[1], z / C[2], t / C[3]])
        edge = (np.abs(u - np.round(u)) < 1e-3).any(0)
        i = np.minimum(np.floor(u).astype(np.int64), np.array(k)[:, None] - 1)
        return ((i[3] * k[2] + i[2]) * k[1] + i[1]) * k[0] + i[0], edge

    tt, zz, yy, xx = np.meshgrid(np.arange(T), np.arange(nz), np.arange(ny), np.arange(nx),
                                 indexing="ij")
    want, edge = cells(xx.ravel() + 0.5, yy.ravel() + 0.5, zz.ravel() + 0.5, tt.ravel() + 0.5)
    assert np.array_equal(fl.ravel()[~edge], want[~edge])
    P = p.shape[2]
    ok = o["key"].ravel() >= 0
    want, edge = cells(p[:, 0].ravel(), p[:, 1].ravel(), p[:, 2].ravel(),
                       np.repeat(np.arange(T) + 0.5, P))
    sel = ok & ~edge
    assert np.array_equal(pl.ravel()[sel], want[sel])
    assert (pl.ravel()[~ok] == -1).all()


def test_value_split_is_found(orc):
    """Two centres along x, a field that is 0 left of x = 6 and 10 from there on (not the seeds'
    midpoint 10), value weight high, space weight low: the clusters settle on the value
    boundary and the centres on the halves' means."""
    T, nz, ny, nx = 4, 3, 4, 20
    f = np.zeros((T, nz, ny, nx), np.float32)
    f[..., 6:] = 10.0
    p = np.zeros((T, 3, 0), np.float32)
    a = np.zeros((T, 1, 0), np.float32)
    key = np.zeros((T, 0), np.int32)
    fl, pl, c, n, it = orc.slic(f, p, a, key, 0, T, 0, (2, 1, 1, 1), w_f=10.0, w_d=0.01,
                                eps_c=1e-6, max_iter=20)
    want = np.broadcast_to((np.arange(nx) >= 6).astype(np.int32), f.shape)
    assert np.array_equal(fl, want)
    assert it < 20
    np.testing.assert_allclose(c[:, 5], [0.0, 10.0], atol=1e-6)
    np.testing.assert_allclose(c[:, 0], [3.0, 13.0], rtol=1e-6)        # means of x + 0.5
    assert n[0, 0] == 6 * ny * nz * T and n[1, 0] == 14 * ny * nz * T


def test_large_time_factor_splits_time(orc):
    """Two centres along t, no value terms, c_f large: the clusters are the two halves of the
    window, whatever the values."""
    f, p, a = _data(T=8)
    o = orc.bin(f.shape, p, a, keep_sumq=False)
    fl, pl, c, n, it = orc.slic(f, p, a, o["key"], 0, 8, 0, (1, 1, 1, 2), w_p=0.0, w_f=0.0,
                                w_d=1.0, c_f=100.0, max_iter=6)
    want = (np.arange(8) >= 4).astype(np.int32)
    assert np.array_equal(fl, np.broadcast_to(want[:, None, None, None], fl.shape))
    ok = o["key"] >= 0
    assert np.array_equal(pl[ok], np.broadcast_to(want[:, None], pl.shape)[ok])


def test_point_order_does_not_matter(orc):
    """Reordering the point ids reorders their labels and changes nothing else (the centre sums
    are exact, so their order is irrelevant)."""
    f, p, a = _data(seed=5)
    o = orc.bin(f.shape, p, a, keep_sumq=False)
    args = dict(w_p=2.0, w_f=1.0, w_d=0.3, c_f=0.7, eps_c=1e-4, max_iter=6)
    r1 = orc.slic(f, p, a, o["key"], 0, 6, 1, (3, 2, 2, 2), **args)
    perm = np.random.default_rng(0).permutation(p.shape[2])
    p2, a2 = np.ascontiguousarray(p[:, :, perm]), np.ascontiguousarray(a[:, :, perm])
    o2 = orc.bin(f.shape, p2, a2, keep_sumq=False)
    r2 = orc.slic(f, p2, a2, o2["key"], 0, 6, 1, (3, 2, 2, 2), **args)
    assert np.array_equal(r1[0], r2[0])
    assert np.array_equal(r1[1][:, perm], r2[1])
    assert np.array_equal(r1[2].view(np.uint32), r2[2].view(np.uint32))
    assert np.array_equal(r1[3], r2[3]) and r1[4] == r2[4]


def test_invalid_samples_take_no_part(orc):
    """Non-finite field values and points outside the grid or with a non-finite value get -1
    and count nowhere; every other label is a centre index."""
    f, p, a = _data(seed=7)
    f[2, 1, 3, 4] = np.nan
    f[0, 0, 0, 0] = np.inf
    p[1, 0, 5] = -3.0                       # outside
    a[2, 0, 9] = np.nan                     # non-finite point value
    o = orc.bin(f.shape, p, a, keep_sumq=False)
    fl, pl, c, n, it = orc.slic(f, p, a, o["key"], 0, 6, 0, (2, 2, 2, 2), max_iter=4)
    assert fl[2, 1, 3, 4] == -1 and fl[0, 0, 0, 0] == -1
    assert pl[1, 5] == -1 and pl[2, 9] == -1
    K = 16
    assert ((fl >= 0) & (fl < K)).sum() == f.size - 2
    assert n[:, 0].sum() == f.size - 2
    assert n[:, 1].sum() == (pl >= 0).sum() == (o["key"] >= 0).sum() - 1


def test_search_region_limits_the_candidates(orc):
    """With the value weight dominating, a sample still only joins a centre whose 2C search
    region holds it: every sample lies within C_i of its centre's final-but-one location along
    each axis, checked here as: no sample is farther than 2 C_i from its final centre."""
    wl = synth.tiny(T=6, P=4000)
    f, p, a = wl.numpy()
    o = orc.bin(f.shape, p, a, keep_sumq=False)
    k = (4, 4, 4, 2)
    fl, pl, c, n, it = orc.slic(f, p, a, o["key"], 0, 6, 0, k, w_f=50.0, w_p=50.0, w_d=0.01,
                                max_iter=5)
    T, nz, ny, nx = f.shape
    C = np.array([nx / k[0], ny / k[1], nz / k[2], 6 / k[3]])
    tt, zz, yy, xx = np.meshgrid(np.arange(T), np.arange(nz), np.arange(ny), np.arange(nx),
                                 indexing="ij")
    cc = c[fl.ravel()]
    d = np.abs(np.stack([xx.ravel() + 0.5, yy.ravel() + 0.5, zz.ravel() + 0.5, tt.ravel() + 0.5],
                        1) - cc[:, :4])
    assert (d <= 2 * C[None, :] + 1e-4).all()


def test_point_value_split_is_found(orc):
    """Points valued 0 left of x = 6 and 10 from there on, point-value weight high, no field
    term: the point clusters settle on the value boundary, the centres' p_c on 0 and 10."""
    T, nz, ny, nx = 4, 2, 3, 20
    rng = np.random.default_rng(11)
    P = 400
    f = np.zeros((T, nz, ny, nx), np.float32)
    p = (rng.random((T, 3, P)) * np.array([nx, ny, nz])[None, :, None]).astype(np.float32)
    p[:, 0, :] = np.where(np.abs(p[:, 0, :] - 6.0) < 0.05, 6.1, p[:, 0, :])  # off the border
    a = np.where(p[:, 0:1, :] >= 6.0, 10.0, 0.0).astype(np.float32)
    o = orc.bin(f.shape, p, a, keep_sumq=False)
    fl, pl, c, n, it = orc.slic(f, p, a, o["key"], 0, T, 0, (2, 1, 1, 1), w_p=10.0, w_f=0.0,
                                w_d=0.01, eps_c=1e-6, max_iter=20)
    assert np.array_equal(pl, (p[:, 0, :] >= 6.0).astype(np.int32))
    np.testing.assert_allclose(c[:, 4], [0.0, 10.0], atol=1e-6)
