"""Pins of the CPU oracle against brute force, library special cases, invariants and closed
forms. None of these re-uses the oracle's own code path."""
from fractions import Fraction

import numpy as np
import pytest

from tests import _pins

F, C, M = 0, 1, 2           # predicate sources
GT, GE, LT, LE, BAND = 0, 1, 2, 3, 4


def _bin_inputs(T, nz, ny, nx, P, A, rng, spread=1.0):
    pos = np.stack([rng.uniform(-0.5 * spread, n + 0.5 * spread, (T, P)) for n in (nx, ny, nz)],
                   1).astype(np.float32)
    attr = rng.normal(size=(T, A, P)).astype(np.float32)
    return pos, attr


# ---------------------------------------------------------------------------------------------
# binning (§3.1 preprocessing index)
# ---------------------------------------------------------------------------------------------

def test_bin_voxel_boundaries_closed_form(orc):
    """Cells are [i,i+1): an integer coordinate belongs to the cell it starts; N, NaN, inf and
    anything below 0 fall outside; -0.0 is inside cell 0."""
    nx, ny, nz, T = 4, 3, 2, 1
    cases = [((0.0, 0.0, 0.0), 0), ((3.999999, 2.5, 1.5), (1 * 3 + 2) * 4 + 3),
             ((4.0, 0.0, 0.0), -1), ((-1e-7, 0.0, 0.0), -1), ((-0.0, -0.0, -0.0), 0),
             ((np.nan, 0, 0), -1), ((np.inf, 0, 0), -1), ((0, -np.inf, 0), -1),
             ((1.0, 1.0, 1.0), (1 * 3 + 1) * 4 + 1), ((0.5, 3.0, 0.5), -1), ((0.5, 0.5, 2.0), -1)]
    pos = np.array([[c[0] for c, _ in cases], [c[1] for c, _ in cases],
                    [c[2] for c, _ in cases]], np.float32)[None]
    attr = np.ones((T, 1, len(cases)), np.float32)
    b = orc.bin((T, nz, ny, nx), pos, attr)
    assert b["key"][0].tolist() == [k for _, k in cases]
    assert b["outside"][0] == sum(k < 0 for _, k in cases)


def test_bin_conservation_and_exact_sums(orc):
    """Counts conserve samples; int64 sums equal exact Python-integer sums of the quantised
    values; the fp32 mean lies within two fp32 roundings (2 * 2^-24 relative) of the exact
    rational mean of the raw attributes, plus the quantisation error 2^-(k+1)."""
    rng = np.random.default_rng(1)
    T, nz, ny, nx, P, A = 3, 3, 4, 5, 400, 2
    pos, attr = _bin_inputs(T, nz, ny, nx, P, A, rng)
    attr[0, 1, :5] = [np.nan, np.inf, -np.inf, 1e30, -1e-30]
    b = orc.bin((T, nz, ny, nx), pos, attr)
    V = nx * ny * nz
    assert np.all(b["count"].reshape(T, V).sum(1) + b["outside"] == P)
    for t in range(T):
        for v in range(V):
            members = np.nonzero(b["key"][t] == v)[0]
            assert b["count"].reshape(T, V)[t, v] == members.size
            for a in range(A):
                k = int(b["kscale"][a])
                exact_q = 0
                exact = Fraction(0)
                for p in members:
                    x = float(attr[t, a, p])
                    if not np.isfinite(x):
                        continue
                    exact_q += round(Fraction(x) * Fraction(2) ** k)   # half-even rounding
                    exact += Fraction(x)
                assert int(b["sumq"].reshape(A, T, V)[a, t, v]) == exact_q
                m = b["mean"].reshape(A, T, V)[a, t, v]
                if members.size == 0:
                    assert np.isnan(m)
                else:
                    ref = exact / members.size
                    bound = 2.01 * 2.0 ** -24 * abs(float(ref)) + 2.0 ** (-k - 1) + 1e-45
                    assert abs(float(m) - float(ref)) <= bound


def test_bin_scale_closed_form(orc):
    """max|attr| = 1.0 gives e = 1 (1.0 = 0.5 * 2^1); 20,000 samples x 8 steps = 160,000 and
    2^18 = 262,144 is the first power of two above 160,001, so k = 62 - 1 - 18 = 43."""
    assert orc.scale_exponent(1.0, 160000) == 43
    assert orc.scale_exponent(0.0, 1) == 62 - 0 - 1
    assert orc.scale_exponent(0.75, 1) == 62 - 0 - 1         # 0.75 = 0.75 * 2^0
    assert orc.scale_exponent(2.0 ** 40, (1 << 20) - 1) == 62 - 41 - 20


def test_bin_constant_attribute_mean_exact(orc):
    """Every sample carries the same value c with a short mantissa (at most 12 significant
    bits): the sum count * c * 2^k and its quotient by the count are exact in fp32, so every
    non-empty voxel's mean is exactly c and its sum is count * c * 2^k."""
    rng = np.random.default_rng(2)
    T, nz, ny, nx, P = 2, 4, 4, 4, 300
    pos, _ = _bin_inputs(T, nz, ny, nx, P, 1, rng, spread=0.0)
    for c in (0.375, -1234.5, 1.5 * 2.0 ** 120, 2.0 ** -130):
        attr = np.full((T, 1, P), c, np.float32)
        b = orc.bin((T, nz, ny, nx), pos, attr)
        cnt = b["count"]
        m = b["mean"][0]
        k = int(b["kscale"][0])
        assert np.all(m[cnt > 0] == np.float32(c))
        assert np.all(np.isnan(m[cnt == 0]))
        want = [round(Fraction(float(np.float32(c))) * Fraction(2) ** k) * int(n)
                for n in cnt.reshape(-1)]
        assert b["sumq"][0].reshape(-1).tolist() == want


def test_bin_mean_fp32_sequence(orc):
    """The mean is the fp32 sequence ((float)sum / (float)count) * 2^-(k/2) * 2^-(k-k/2):
    checked with numpy float32 scalars on a case with long mantissas and three samples."""
    T, nz, ny, nx = 1, 1, 1, 2
    pos = np.array([[[0.5, 0.5, 0.5, 1.5], [0.5] * 4, [0.5] * 4]], np.float32)
    attr = np.array([[[0.1, 0.2, 0.7, -3.3]]], np.float32)
    b = orc.bin((T, nz, ny, nx), pos, attr)
    k = int(b["kscale"][0])
    for v, members in ((0, [0, 1, 2]), (1, [3])):
        s = sum(round(Fraction(float(attr[0, 0, p])) * Fraction(2) ** k) for p in members)
        assert int(b["sumq"][0, 0, 0, 0, v]) == s
        m = np.float32(np.float32(s) / np.float32(len(members)))
        m = np.float32(m * np.float32(2.0 ** -(k // 2)))
        m = np.float32(m * np.float32(2.0 ** -(k - k // 2)))
        assert b["mean"][0, 0, 0, 0, v] == m


def test_bin_empty_particles(orc):
    T, nz, ny, nx = 2, 2, 3, 4
    b = orc.bin((T, nz, ny, nx), np.zeros((T, 3, 0), np.float32), np.zeros((T, 2, 0), np.float32))
    assert b["key"].shape == (T, 0)
    assert not b["count"].any()
    assert np.isnan(b["mean"]).all()
    assert np.all(b["outside"] == 0)


# ---------------------------------------------------------------------------------------------
# criterion + 4D connected components
# ---------------------------------------------------------------------------------------------

def _seg_from_active(orc, active, key=None, edges=7, t0=0):
    """Run the oracle with field in {0,1} and criterion field > 0.5."""
    T = active.shape[0]
    field = active.astype(np.float32)
    cnt = np.zeros(active.shape, np.int32)
    mean = np.zeros((0,) + active.shape, np.float32)
    if key is None:
        key = np.zeros((T, 0), np.int32)
    return orc.segment(field, cnt, mean, key, t0, T, [(F, 0, GT, 0.5, 0.0)], edges)


def test_segment_exhaustive_2x2x2x2(orc):
    """All 2^16 activity patterns of a 2x2x2 grid over 2 timesteps, spatial+temporal edges:
    labels equal the dense transitive closure's component minima."""
    shape = (2, 2, 2, 2)
    N = 16
    full = np.ones(shape, bool)
    A = _pins.adjacency_dense(full, None, 3, shape)
    masks = ((np.arange(1 << N)[:, None] >> np.arange(N)[None, :]) & 1).astype(bool)
    # closure of every induced subgraph at once (batched Boolean squaring)
    R = A[None] & masks[:, :, None] & masks[:, None, :]
    R = R | np.eye(N, dtype=bool)[None]
    for _ in range(4):
        R = np.einsum("bij,bjk->bik", R.astype(np.uint8), R.astype(np.uint8)) > 0
    want = np.where(masks, np.argmax(R, axis=2), -1)
    for mi in range(1 << N):
        lab, nf = _seg_from_active(orc, masks[mi].reshape(shape), edges=3)
        assert np.array_equal(lab.reshape(-1), want[mi]), mi
        assert nf == len(np.unique(want[mi][want[mi] >= 0]))


@pytest.mark.parametrize("seed", range(12))
def test_segment_brute_force_with_trajectories(orc, seed):
    """Random tiny windows with random trajectory keys and every combination of edge classes:
    labels equal the dense transitive closure of the pairwise adjacency."""
    rng = np.random.default_rng(100 + seed)
    Tw, nz, ny, nx = 3, int(rng.integers(1, 4)), int(rng.integers(1, 5)), int(rng.integers(1, 5))
    shape = (Tw, nz, ny, nx)
    V = nz * ny * nx
    active = rng.random(shape) < rng.uniform(0.2, 0.7)
    P = int(rng.integers(0, 31))
    key = rng.integers(-1, V, (Tw, P)).astype(np.int32)
    for edges in range(8):
        A = _pins.adjacency_dense(active, key, edges, shape)
        want = _pins.closure_labels(A, active.reshape(-1))
        lab, nf = _seg_from_active(orc, active, key, edges)
        assert np.array_equal(lab.reshape(-1), want), (seed, edges)


def test_segment_matches_ndimage_label(orc):
    """Without trajectory links the partition equals scipy.ndimage.label with a 3^4 structure
    (all 27 offsets at dt=0, only the centre at dt=+-1); with one timestep it equals the plain
    3x3x3 labelling."""
    from scipy import ndimage
    rng = np.random.default_rng(7)
    active = rng.random((5, 9, 10, 11)) < 0.3
    lab, nf = _seg_from_active(orc, active, edges=3)
    ref, n = ndimage.label(active, structure=_pins.structure_4d())
    assert nf == n
    assert _pins.same_partition(lab, ref - 1)
    lab1, nf1 = _seg_from_active(orc, active[:1], edges=3)
    ref1, n1 = ndimage.label(active[0], structure=np.ones((3, 3, 3)))
    assert nf1 == n1 and _pins.same_partition(lab1[0], ref1 - 1)
    # 2D + time (NZ = 1): the 26-neighbourhood degenerates to 8 neighbours
    act2 = rng.random((4, 1, 20, 20)) < 0.35
    lab2, nf2 = _seg_from_active(orc, act2, edges=3)
    S = np.zeros((3, 3, 3), bool)
    S[1] = True
    S[0, 1, 1] = S[2, 1, 1] = True
    ref2, n2 = ndimage.label(act2[:, 0], structure=S)
    assert nf2 == n2 and _pins.same_partition(lab2[:, 0], ref2 - 1)


def test_segment_matches_csgraph_on_tiny_workload(orc):
    """With every edge class on the tiny workload's real criterion, the oracle's labels equal
    scipy.sparse.csgraph.connected_components on the explicit edge list, canonicalised."""
    from paper_1903_12294_gb300 import synth
    wl = synth.tiny()
    f, p, a = wl.numpy()
    b = orc.bin(f.shape, p, a)
    lab, nf = orc.segment(f, b["count"], b["mean"], b["key"], 0, f.shape[0], wl.preds)
    active = (f > np.float32(0.4)) & (b["count"] >= 2)
    want = _pins.csgraph_labels(active, b["key"], 7)
    assert np.array_equal(lab, want)
    _pins.check_label_invariants(lab, active, b["key"], 7)


def test_segment_window_and_predicates(orc):
    """Predicates on count and mean, each op, and a window [t0,t1) that starts late: the active
    set is the stated conjunction and labels are window-relative."""
    rng = np.random.default_rng(9)
    T, nz, ny, nx = 5, 3, 6, 7
    field = rng.random((T, nz, ny, nx)).astype(np.float32)
    cnt = rng.integers(0, 5, (T, nz, ny, nx)).astype(np.int32)
    mean = rng.random((2, T, nz, ny, nx)).astype(np.float32)
    mean[1][cnt == 0] = np.nan
    key = rng.integers(-1, nx * ny * nz, (T, 40)).astype(np.int32)
    preds_list = [
        [(F, 0, GE, 0.3, 0), (C, 0, BAND, 1, 3)],
        [(M, 1, LT, 0.6, 0), (C, 0, GT, 0.0, 0)],
        [(M, 0, LE, 0.5, 0)],
        [(F, 0, BAND, 0.2, 0.8), (M, 1, GT, 0.1, 0), (C, 0, LE, 3.9, 0), (M, 0, GE, 0.05, 0)],
        [],
    ]
    ops = {GT: np.greater, GE: np.greater_equal, LT: np.less, LE: np.less_equal}
    for preds in preds_list:
        t0, t1 = 1, 4
        lab, nf = orc.segment(field, cnt, mean, key, t0, t1, preds)
        act = np.ones((t1 - t0, nz, ny, nx), bool)
        for src, a, op, lo, hi in preds:
            x = (field, cnt, mean[a] if src == M else None)[src][t0:t1]
            if src == C:
                lo, hi = int(lo), int(hi)
            else:
                lo, hi = np.float32(lo), np.float32(hi)
            with np.errstate(invalid="ignore"):
                act &= ((x >= lo) & (x <= hi)) if op == BAND else ops[op](x, lo)
        want = _pins.csgraph_labels(act, key[t0:t1], 7)
        assert np.array_equal(lab, want)


def test_segment_closed_forms(orc):
    """A solid box is one feature whose label is its first voxel; a point moving one voxel per
    step through otherwise isolated active voxels (one per step, never adjacent) joins them into
    one feature only through trajectory links."""
    shape = (4, 6, 7, 8)
    act = np.zeros(shape, bool)
    act[1:3, 2:5, 1:6, 3:7] = True
    lab, nf = _seg_from_active(orc, act)
    first = np.ravel_multi_index((1, 2, 1, 3), shape)
    assert nf == 1 and np.all(lab[act] == first) and np.all(lab[~act] == -1)

    T = 5
    act = np.zeros((T, 4, 4, 16), bool)
    key = np.full((T, 1), -1, np.int32)
    for t in range(T):
        x = 3 * t
        act[t, 1, 1, x] = True                  # 3 voxels apart: not spatial/temporal neighbours
        key[t, 0] = (1 * 4 + 1) * 16 + x
    lab, nf = _seg_from_active(orc, act, key, edges=7)
    assert nf == 1 and np.all(lab[act] == lab[act][0])
    lab, nf = _seg_from_active(orc, act, key, edges=3)
    assert nf == T


def test_segment_empty_and_degenerate(orc):
    act = np.zeros((3, 2, 2, 2), bool)
    lab, nf = _seg_from_active(orc, act)
    assert nf == 0 and np.all(lab == -1)
    lab, nf = _seg_from_active(orc, np.ones((1, 1, 1, 1), bool))
    assert nf == 1 and lab.reshape(-1).tolist() == [0]
    # empty window
    field = np.ones((2, 1, 1, 3), np.float32)
    lab, nf = orc.segment(field, np.zeros(field.shape, np.int32), np.zeros((0,) + field.shape,
                          np.float32), np.zeros((2, 0), np.int32), 1, 1, [])
    assert nf == 0 and lab.size == 0


# ---------------------------------------------------------------------------------------------
# per-feature statistics (§3.2.2 averages, §3.4 extent and deviations)
# ---------------------------------------------------------------------------------------------

@pytest.mark.filterwarnings("ignore::RuntimeWarning")
def test_features_match_ndimage_reductions(orc):
    """Field statistics per feature equal scipy.ndimage's labelled reductions (sum, mean,
    minimum, maximum, standard deviation, centre of mass, object slices)."""
    from scipy import ndimage
    from paper_1903_12294_gb300 import synth
    wl = synth.tiny()
    f, p, a = wl.numpy()
    b, lab, nf, feat = orc.run_all(f, p, a, 0, f.shape[0], wl.preds)
    idx = feat["label"]
    assert nf == idx.size and np.all(np.diff(idx) > 0)
    lab1 = lab + 1                          # ndimage treats 0 as background
    ix = idx + 1
    f64 = f.astype(np.float64)
    assert np.array_equal(feat["n_vox"], ndimage.sum_labels(np.ones_like(f64), lab1, ix))
    assert np.array_equal(feat["n_pts"], ndimage.sum_labels(b["count"].astype(np.float64),
                                                            lab1, ix).astype(np.int64))
    np.testing.assert_allclose(feat["sum_field"], ndimage.sum_labels(f64, lab1, ix), rtol=1e-12)
    np.testing.assert_allclose(feat["mean_field"], ndimage.mean(f64, lab1, ix), rtol=1e-12)
    np.testing.assert_allclose(feat["std_field"], ndimage.standard_deviation(f64, lab1, ix),
                               rtol=1e-7, atol=1e-12)
    assert np.array_equal(feat["min_field"], ndimage.minimum(f, lab1, ix).astype(np.float32))
    assert np.array_equal(feat["max_field"], ndimage.maximum(f, lab1, ix).astype(np.float32))
    com = np.array(ndimage.center_of_mass(np.ones_like(f64), lab1, ix))
    np.testing.assert_allclose(feat["centroid"], com, rtol=1e-12)
    objs = ndimage.find_objects(lab1)
    for i, l in enumerate(ix):
        sl = objs[l - 1]
        assert feat["bbox"][i].tolist() == [s.start for s in sl] + [s.stop - 1 for s in sl]


def test_features_point_part_closed_forms(orc):
    """Point part: a box feature holding exactly one sample per voxel with attribute value
    v_p = 2.5 has n_pts = volume, mean 2.5, std 0 and an exact fixed-point sum; samples outside
    the feature or outside the window do not count."""
    T, nz, ny, nx = 3, 4, 5, 6
    act = np.zeros((T, nz, ny, nx), bool)
    act[:, 1:3, 1:4, 2:5] = True
    field = act.astype(np.float32) * 2.0
    zz, yy, xx = np.meshgrid(np.arange(1, 3), np.arange(1, 4), np.arange(2, 5), indexing="ij")
    inside = np.stack([xx.ravel() + 0.5, yy.ravel() + 0.5, zz.ravel() + 0.5])
    outside = np.array([[0.5], [0.5], [0.5]])           # an inactive voxel
    pts = np.concatenate([inside, outside], 1).astype(np.float32)
    P = pts.shape[1]
    pos = np.repeat(pts[None], T, 0)
    attr = np.full((T, 1, P), 2.5, np.float32)
    attr[:, 0, -1] = 100.0
    b = orc.bin(field.shape, pos, attr)
    lab, nf = orc.segment(field, b["count"], b["mean"], b["key"], 1, 3, [(F, 0, GT, 1.0, 0)])
    feat = orc.features(field, b["count"], attr, b["key"], b["kscale"], 1, 3, lab)
    vol = 2 * 2 * 3 * 3
    k = int(b["kscale"][0])
    assert nf == 1 and feat["n_vox"][0] == vol and feat["n_pts"][0] == vol
    assert feat["mean_attr"][0, 0] == 2.5 and feat["std_attr"][0, 0] == 0.0
    assert feat["sumq"][0, 0] == vol * int(2.5 * 2 ** k)
    assert feat["mean_field"][0] == 2.0 and feat["std_field"][0] == 0.0
    # centroid of the box: t in {0,1} (window-relative), z {1,2}, y {1,2,3}, x {2,3,4}
    assert feat["centroid"][0].tolist() == [0.5, 1.5, 2.0, 3.0]
    assert feat["bbox"][0].tolist() == [0, 1, 1, 2, 1, 2, 3, 4]


def test_features_linear_field_std_closed_form(orc):
    """Field = x along a full row of n voxels: population std = sqrt((n^2-1)/12)."""
    n = 17
    field = np.arange(n, dtype=np.float32)[None, None, None, :] + 1.0
    lab, nf = orc.segment(field, np.zeros(field.shape, np.int32),
                          np.zeros((0,) + field.shape, np.float32), np.zeros((1, 0), np.int32),
                          0, 1, [(F, 0, GT, 0.5, 0)])
    feat = orc.features(field, np.zeros(field.shape, np.int32), np.zeros((1, 0, 0), np.float32),
                        np.zeros((1, 0), np.int32), [], 0, 1, lab)
    assert nf == 1
    np.testing.assert_allclose(feat["std_field"][0], np.sqrt((n * n - 1) / 12.0), rtol=1e-14)
    assert feat["mean_field"][0] == (n + 1) / 2.0
    assert np.isnan(feat["mean_attr"]).all() or feat["mean_attr"].size == 0


def test_features_conservation_on_mid_slice(orc):
    """Sum over features of n_pts equals the count summed over active voxel-timesteps, and of
    n_vox the number of active voxel-timesteps (mid-shaped workload at reduced size)."""
    from paper_1903_12294_gb300 import synth
    wl = synth.mid(n=40, T=6, P=20000, n_blobs=8)
    f, p, a = wl.numpy()
    b, lab, nf, feat = orc.run_all(f, p, a, 1, 5, wl.preds)
    act = lab >= 0
    assert feat["n_vox"].sum() == act.sum()
    assert feat["n_pts"].sum() == b["count"][1:5][act].sum()
    _pins.check_label_invariants(lab, act, b["key"][1:5], 7)
    # features are sorted by label and labels are component minima
    assert np.all(np.diff(feat["label"]) > 0)
    assert np.all(lab.reshape(-1)[feat["label"]] == feat["label"])


# ---------------------------------------------------------------------------------------------
# per-feature point moments (§3.2.2 centre averages, §3.4 deviations of the point samples)
# ---------------------------------------------------------------------------------------------

def _labels_from_ndimage(active):
    """Canonical labels (component minimum window-linear index, -1 inactive) of the spatial +
    temporal graph, from scipy's labelling alone (the oracle's labelling is not used)."""
    from scipy import ndimage
    s = np.zeros((3, 3, 3, 3), bool)
    s[1] = True                       # all 27 offsets within a step
    s[0, 1, 1, 1] = s[2, 1, 1, 1] = True
    comp, n = ndimage.label(active, structure=s)
    flat = comp.reshape(-1)
    out = np.full(flat.size, -1, np.int32)
    for c in range(1, n + 1):
        idx = np.flatnonzero(flat == c)
        out[idx] = idx.min()
    return out.reshape(active.shape)


def _numpy_point_moments(labels, key, attr, t0, V):
    """Per feature label: (n_pts, mean, population std) of every attribute over the point
    samples whose voxel-timestep carries that label, with raw fp32 values widened to fp64 and
    non-finite values taken as 0 (they still count as samples)."""
    tw = labels.shape[0]
    lab = labels.reshape(tw, V)
    out = {}
    for t in range(tw):
        for p in range(key.shape[1]):
            v = key[t0 + t, p]
            if v < 0 or lab[t, v] < 0:
                continue
            vals = attr[t0 + t, :, p].astype(np.float64)
            vals = np.where(np.isfinite(vals), vals, 0.0)
            out.setdefault(int(lab[t, v]), []).append(vals)
    res = {}
    for l, rows in out.items():
        m = np.array(rows)
        res[l] = (m.shape[0], m.mean(0), m.std(0))
    return res


def test_features_point_moments_two_valued_closed_form(orc):
    """One feature of three voxels holding 1, 3 and 0 samples (n_vox = 3, n_pts = 4): attribute
    0 is 1.0 in the lone sample and 3.0 in the other three, so mean = (1 + 9) / 4 = 2.5 and the
    population variance of a two-valued set, n1 n2 (a - b)^2 / n^2 = 3 * 4 / 16 = 0.75;
    attribute 1 is -2, 2, 2, 2: mean 1, variance 3 * 16 / 16 = 3. Dividing by n_vox, or mixing
    the scaled fixed-point mean with unscaled squares, fails here."""
    T, nz, ny, nx = 1, 1, 1, 5
    field = np.zeros((T, nz, ny, nx), np.float32)
    field[0, 0, 0, 1:4] = 1.0
    pts = np.array([[1.5, 2.2, 2.5, 2.8, 0.5, 4.5],        # voxel 1 once, voxel 2 three times,
                    [0.5] * 6, [0.5] * 6], np.float32)    # two samples off the feature
    pos = pts[None]
    attr = np.array([[[1.0, 3.0, 3.0, 3.0, 50.0, -50.0],
                      [-2.0, 2.0, 2.0, 2.0, 9.0, 9.0]]], np.float32)
    b = orc.bin(field.shape, pos, attr)
    lab, nf = orc.segment(field, b["count"], b["mean"], b["key"], 0, 1, [(F, 0, GT, 0.5, 0)])
    feat = orc.features(field, b["count"], attr, b["key"], b["kscale"], 0, 1, lab)
    assert nf == 1 and feat["n_vox"][0] == 3 and feat["n_pts"][0] == 4
    assert feat["mean_attr"][0].tolist() == [2.5, 1.0]
    np.testing.assert_allclose(feat["std_attr"][0], [np.sqrt(0.75), np.sqrt(3.0)], rtol=1e-14)
    k = b["kscale"]
    assert feat["sumq"][0].tolist() == [int(10 * 2 ** int(k[0])), int(4 * 2 ** int(k[1]))]


def test_features_point_moments_match_numpy(orc):
    """Random window: voxels with 0, 1 and many samples (points clustered onto a few voxels),
    three attributes of different scales, some non-finite values. Each feature's n_pts, mean and
    population std of every attribute equal numpy's over the samples in its voxel-timesteps
    (labels from scipy's labelling, not the oracle's)."""
    rng = np.random.default_rng(1903)
    T, nz, ny, nx = 4, 8, 8, 8
    V = nz * ny * nx
    field = rng.uniform(0, 1, (T, nz, ny, nx)).astype(np.float32)
    P = 600
    hot = rng.choice(V, 12, replace=False)                    # a few crowded voxels, members
    field.reshape(T, V)[:, hot] = 1.0
    pos = np.empty((T, 3, P), np.float32)
    for t in range(T):
        crowd = rng.random(P) < 0.5
        v = np.where(crowd, hot[rng.integers(0, hot.size, P)], rng.integers(0, V, P))
        z, y, x = v // (ny * nx), (v // nx) % ny, v % nx
        pos[t] = np.stack([x + rng.random(P), y + rng.random(P), z + rng.random(P)])
    pos[0, 0, :5] = np.nan                                    # a few samples off the grid
    attr = np.stack([rng.normal(5.0, 2.0, (T, P)), rng.uniform(-1e-3, 3e-3, (T, P)),
                     rng.exponential(100.0, (T, P))], 1).astype(np.float32)
    attr[1, 0, 7] = np.nan                                   # non-finite samples inside a
    attr[2, 2, 11] = np.inf                                  # crowded member voxel
    for t, p in ((1, 7), (2, 11)):
        v = int(hot[0])
        pos[t, :, p] = (v % nx + 0.5, (v // nx) % ny + 0.5, v // (ny * nx) + 0.5)
    b = orc.bin(field.shape, pos, attr)
    t0, t1 = 1, 4
    active = field[t0:t1] > 0.95
    lab = _labels_from_ndimage(active)
    feat = orc.features(field, b["count"], attr, b["key"], b["kscale"], t0, t1, lab)
    ref = _numpy_point_moments(lab, b["key"], attr, t0, V)
    counts = b["count"][t0:t1].reshape(t1 - t0, V)
    n_vox = {int(l): int((lab == l).sum()) for l in feat["label"]}
    assert any(feat["n_pts"][i] != n_vox[int(l)] for i, l in enumerate(feat["label"]))
    assert counts[active.reshape(t1 - t0, V)].max() >= 3      # crowded voxels are members
    checked = 0
    for i, l in enumerate(feat["label"]):
        n, m, s = ref.get(int(l), (0, None, None))
        assert feat["n_pts"][i] == n
        if n == 0:
            assert np.isnan(feat["mean_attr"][i]).all()
            continue
        np.testing.assert_allclose(feat["mean_attr"][i], m, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(feat["std_attr"][i], s, rtol=1e-9, atol=1e-12)
        checked += 1
    assert checked >= 5
    hot_label = {int(lab[t - t0].reshape(V)[hot[0]]) for t in (1, 2)}
    assert hot_label <= {int(l) for l in feat["label"]}      # the non-finite samples count
