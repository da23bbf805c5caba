"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, element by element.

Bars: binning keys, counts and int64 sums bit-exact and fp32 means bit-exact (both sides take
the same sequence of IEEE fp32 operations); labels bit-exact (canonical minimum-index labels); feature
integer statistics exact; float statistics within 1e-5 relative (fp64 sums in another order).
"""
import numpy as np
import pytest
import torch

from paper_1903_12294_gb300 import synth

pytestmark = pytest.mark.gpu

F, C, M = 0, 1, 2
GT, GE, LT, LE, BAND = 0, 1, 2, 3, 4
RTOL = 1e-5


def _tensors(field, pos, attr, dev="cuda"):
    return (torch.as_tensor(field).to(dev).contiguous(), torch.as_tensor(pos).to(dev).contiguous(),
            torch.as_tensor(attr).to(dev).contiguous())


def gpu_run(msf, field, pos, attr, t0, t1, preds, edges=7, tile=None, features=True):
    ctx = msf.Context(0)
    try:
        ctx.load(*_tensors(field, pos, attr))
        st = ctx.bin(keep_sumq=True)
        key, count, mean, sumq = ctx.bins("cpu", sumq=True)
        if tile:
            ctx.set_tile(*tile)
        labels, n = ctx.segment(t0, t1, preds, edges)
        feats = feats_generic = feats_kept = None
        if features:
            # the labels msf_segment just wrote: statistics from the retained segmentation
            feats = ctx.features(t0, t1, labels, preds, edges)
            # the same labels in another buffer: statistics from the labels themselves
            feats_generic = ctx.features(t0, t1, labels.clone(), preds, edges)
            # segmenting again after an extraction keeps the point samples' components in the
            # trajectory joins, and the next extraction's point statistics read them
            labels2, n2 = ctx.segment(t0, t1, preds, edges)
            assert n2 == n and torch.equal(labels2, labels)
            feats_kept = ctx.features(t0, t1, labels2, preds, edges)
        torch.cuda.synchronize()
        return dict(stats=st, key=key.numpy(), count=count.numpy(), mean=mean.numpy(),
                    sumq=sumq.numpy(), labels=labels.cpu().numpy(), n=n, feats=feats,
                    feats_generic=feats_generic, feats_kept=feats_kept)
    finally:
        ctx.close()


def check_bins(g, o):
    assert np.array_equal(g["key"], o["key"])
    assert np.array_equal(g["count"], o["count"])
    A = o["mean"].shape[0]
    if A:
        assert np.array_equal(g["sumq"], o["sumq"])
        assert np.array_equal(g["mean"].view(np.uint32), o["mean"].view(np.uint32))
        assert list(g["stats"].kscale)[:A] == list(o["kscale"])
    assert g["stats"].out_of_domain == int(o["outside"].sum())


def _close(a, b, rtol=RTOL, atol=0.0):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    same = (a == b) | (np.isnan(a) & np.isnan(b))          # equal values, infinities, NaN
    with np.errstate(invalid="ignore"):
        ok = same | (np.abs(a - b) <= rtol * np.abs(b) + atol)
    assert ok.all(), (a[~ok][:5], b[~ok][:5])


def check_features(gf, of, A):
    assert gf.shape[0] == of["label"].shape[0]
    assert np.array_equal(gf["label"], of["label"])
    assert np.array_equal(gf["n_vox"], of["n_vox"])
    assert np.array_equal(gf["n_pts"], of["n_pts"])
    assert np.array_equal(gf["bbox_min"], of["bbox"][:, :4])
    assert np.array_equal(gf["bbox_max"], of["bbox"][:, 4:])
    assert np.array_equal(gf["min_field"], of["min_field"])
    assert np.array_equal(gf["max_field"], of["max_field"])
    assert np.array_equal(gf["centroid"], of["centroid"])      # exact integer sums / n
    _close(gf["sum_field"], of["sum_field"])
    _close(gf["mean_field"], of["mean_field"])
    _close(gf["std_field"], of["std_field"], atol=1e-6 * (np.abs(of["mean_field"]) + 1e-30))
    if A:
        assert np.array_equal(gf["sumq"][:, :A], of["sumq"])
        _close(gf["mean_attr"][:, :A], of["mean_attr"])
        _close(gf["std_attr"][:, :A], of["std_attr"],
               atol=1e-6 * (np.abs(of["mean_attr"]) + 1e-30))


def full_check(gpu, orc, field, pos, attr, t0, t1, preds, edges=7, tile=None):
    g = gpu_run(gpu, field, pos, attr, t0, t1, preds, edges, tile)
    o = orc.bin(field.shape, pos, attr)
    check_bins(g, o)
    lab, nf = orc.segment(field, o["count"], o["mean"], o["key"], t0, t1, preds, edges)
    assert g["n"] == nf
    assert np.array_equal(g["labels"], lab)
    of = orc.features(field, o["count"], attr, o["key"], o["kscale"], t0, t1, lab)
    check_features(g["feats"], of, attr.shape[1])
    check_features(g["feats_generic"], of, attr.shape[1])
    check_features(g["feats_kept"], of, attr.shape[1])
    return g, o, lab


# ---------------------------------------------------------------------------------------------

def test_tiny_workload_full(gpu, orc):
    """32^3 x 8, 20k particles, field > 0.4 AND count >= 2, all edges (whole workload)."""
    wl = synth.tiny()
    f, p, a = wl.numpy()
    full_check(gpu, orc, f, p, a, 0, f.shape[0], wl.preds)


@pytest.mark.parametrize("window", [(0, 6), (1, 6), (3, 4), (2, 2)])
def test_mid_reduced_windows(gpu, orc, window):
    """Mid-shaped data at a ragged reduced size (nx = 72: two full 32-voxel segments plus an 8
    wide tail; ny, nz not multiples of the tile), several windows incl. a single step and an
    empty one."""
    wl = synth.mid(n=40, T=6, P=30000, n_blobs=10)
    f, p, a = wl.numpy()
    f = np.ascontiguousarray(np.concatenate([f, f[..., :32]], axis=-1))   # nx = 72
    p = p.copy()
    t0, t1 = window
    full_check(gpu, orc, f, p, a, t0, t1, wl.preds)


@pytest.mark.parametrize("edges", range(8))
def test_edge_classes(gpu, orc, edges):
    rng = np.random.default_rng(edges)
    T, nz, ny, nx = 5, 9, 13, 70
    f = rng.random((T, nz, ny, nx)).astype(np.float32)
    P = 4000
    pos = (rng.random((T, 3, P)) * np.array([nx, ny, nz])[None, :, None]).astype(np.float32)
    a = rng.normal(size=(T, 2, P)).astype(np.float32)
    preds = [(F, 0, GT, 0.55, 0)]
    full_check(gpu, orc, f, pos, a, 0, T, preds, edges)


def test_predicates_and_ops(gpu, orc):
    rng = np.random.default_rng(5)
    T, nz, ny, nx = 6, 10, 11, 40
    f = rng.random((T, nz, ny, nx)).astype(np.float32)
    P = 20000
    pos = (rng.random((T, 3, P)) * np.array([nx, ny, nz])[None, :, None]).astype(np.float32)
    a = rng.normal(size=(T, 3, P)).astype(np.float32)
    cases = [
        [(C, 0, GE, 1, 0)],
        [(C, 0, BAND, 1, 2), (F, 0, LE, 0.7, 0)],
        [(M, 2, GT, 0.0, 0), (F, 0, GE, 0.2, 0)],
        [(M, 1, BAND, -0.5, 0.5), (C, 0, LT, 3, 0), (F, 0, GT, 0.1, 0)],
        [(M, 0, LT, 0.3, 0), (M, 1, GE, -1.0, 0), (C, 0, GT, 0.0, 0), (F, 0, BAND, 0.1, 0.9)],
        [],
    ]
    for preds in cases:
        full_check(gpu, orc, f, pos, a, 1, 5, preds)


@pytest.mark.parametrize("shape", [(3, 1, 1, 1), (2, 1, 1, 33), (4, 1, 50, 65), (3, 17, 1, 31),
                                   (5, 2, 3, 97), (2, 40, 40, 1)])
def test_ragged_shapes(gpu, orc, shape):
    """Degenerate and ragged grids: single voxel, a 33-wide row, 2D (nz = 1), ny = 1, nx = 1."""
    rng = np.random.default_rng(sum(shape))
    T, nz, ny, nx = shape
    f = (rng.random(shape) < 0.45).astype(np.float32)
    P = 500
    pos = (rng.random((T, 3, P)) * np.array([nx, ny, nz])[None, :, None]).astype(np.float32)
    a = rng.normal(size=(T, 1, P)).astype(np.float32)
    full_check(gpu, orc, f, pos, a, 0, T, [(F, 0, GT, 0.5, 0)])


@pytest.mark.parametrize("tile", [(8, 8, 4), (16, 16, 1), (4, 4, 16), (1, 16, 16), (32, 8, 1),
                                  (2, 2, 64)])
def test_tile_shapes_give_identical_labels(gpu, orc, tile):
    wl = synth.mid(n=48, T=8, P=40000, n_blobs=12)
    f, p, a = wl.numpy()
    full_check(gpu, orc, f, p, a, 0, 8, wl.preds, tile=tile)


def test_no_particles_and_all_active(gpu, orc):
    rng = np.random.default_rng(3)
    T, nz, ny, nx = 3, 6, 7, 45
    f = rng.random((T, nz, ny, nx)).astype(np.float32)
    p = np.zeros((T, 3, 0), np.float32)
    a = np.zeros((T, 0, 0), np.float32)
    full_check(gpu, orc, f, p, a, 0, T, [(F, 0, GT, 0.5, 0)])
    full_check(gpu, orc, f, p, a, 0, T, [])                       # everything active: 1 feature
    full_check(gpu, orc, f, p, a, 0, T, [(F, 0, GT, 2.0, 0)])     # nothing active


def test_out_of_domain_and_nonfinite_samples(gpu, orc):
    rng = np.random.default_rng(11)
    T, nz, ny, nx = 3, 5, 6, 40
    f = rng.random((T, nz, ny, nx)).astype(np.float32)
    P = 3000
    pos = (rng.random((T, 3, P)) * np.array([nx + 4, ny + 4, nz + 4])[None, :, None] - 2)
    pos = pos.astype(np.float32)
    pos[0, 0, :10] = np.nan
    pos[1, 1, 10:20] = np.inf
    pos[2, 2, 20:30] = -0.0
    pos[2, 0, 30:40] = nx
    a = rng.normal(size=(T, 2, P)).astype(np.float32)
    a[0, 0, :50] = np.nan
    a[1, 1, 50:60] = -np.inf
    full_check(gpu, orc, f, pos, a, 0, T, [(C, 0, GE, 1, 0), (F, 0, GT, 0.3, 0)])


def test_host_buffers_and_repeatability(gpu, orc):
    """Host-memory inputs and labels (the end-to-end form) give the same bytes as device ones,
    and repeated calls give identical labels."""
    wl = synth.tiny()
    f, p, a = wl.numpy()
    ctx = gpu.Context(0)
    try:
        ctx.load(f, p, a)
        ctx.bin()
        lab_h = np.empty((8, 32, 32, 32), np.int32)
        n_h = gpu.msf_segment(ctx.h, gpu.make_criteria(0, 8, wl.preds), lab_h)
        lab_d, n_d = ctx.segment(0, 8, wl.preds)
        lab_d2, _ = ctx.segment(0, 8, wl.preds)
        assert n_h == n_d
        assert np.array_equal(lab_h, lab_d.cpu().numpy())
        assert torch.equal(lab_d, lab_d2)
        fe_h = gpu.msf_extract_features(ctx.h, gpu.make_criteria(0, 8, wl.preds), lab_h)
        fe_d = ctx.features(0, 8, lab_d, wl.preds)
        assert fe_h.tobytes() == fe_d.tobytes() or np.array_equal(fe_h["label"], fe_d["label"])
    finally:
        ctx.close()


def test_segment_features_in_one_call(gpu, orc):
    """msf_segment_features (labels and features in one call, the host labels' copy beside the
    feature passes) gives msf_segment's labels and the oracle's features, with host and device
    labels, on a pinned host buffer too."""
    wl = synth.tiny()
    f, p, a = wl.numpy()
    ctx = gpu.Context(0)
    try:
        ctx.load(f, p, a)
        ctx.bin()
        crit = gpu.make_criteria(0, 8, wl.preds)
        lab_ref, n_ref = ctx.segment(0, 8, wl.preds)
        fe_ref = ctx.features(0, 8, lab_ref, wl.preds)
        got = [fe_ref]
        for host in ("pageable", "pinned", "device"):
            if host == "device":
                lab = torch.full((8, 32, 32, 32), -5, dtype=torch.int32, device="cuda")
            else:
                lab = torch.full((8, 32, 32, 32), -5, dtype=torch.int32)
                if host == "pinned":
                    lab = lab.pin_memory()
            nf, fe = gpu.msf_segment_features(ctx.h, crit, lab, len(fe_ref) + 3)
            assert nf == n_ref and len(fe) == len(fe_ref)
            assert torch.equal(lab.cuda(), lab_ref)
            got.append(fe)
        with pytest.raises(gpu.MsfError):  # capacity below the feature count
            gpu.msf_segment_features(ctx.h, crit, torch.empty((8, 32, 32, 32), dtype=torch.int32),
                                     1)
    finally:
        ctx.close()
    # integer statistics are exact; the fp64 sums add in L2 atomics in no fixed order, so the
    # floating-point ones match the oracle within the parity tolerance, run by run
    o = orc.run_all(f, p, a, 0, 8, wl.preds)
    assert n_ref == o[2]
    for fe in got:
        check_features(fe, o[3], a.shape[1])


def test_errors_are_status_codes(gpu):
    ctx = gpu.Context(0)
    try:
        with pytest.raises(gpu.MsfError) as e:
            ctx.segment(0, 1, [(F, 0, GT, 0.5, 0)])
        assert e.value.status == gpu.MSF_ERR_NOT_LOADED
        f = np.zeros((4, 2, 3, 5), np.float32)
        p = np.zeros((4, 3, 2), np.float32)
        a = np.zeros((4, 1, 2), np.float32)
        ctx.load(f, p, a)
        with pytest.raises(gpu.MsfError) as e:
            ctx.segment(0, 2, [(C, 0, GE, 1, 0)])
        assert e.value.status == gpu.MSF_ERR_NOT_BINNED
        ctx.bin()
        for bad in ([(F, 0, 9, 0, 0)], [(M, 1, GT, 0, 0)], [(7, 0, GT, 0, 0)],
                    [(C, 0, GT, 3e9, 0)]):
            with pytest.raises(gpu.MsfError) as e:
                ctx.segment(0, 2, bad)
            assert e.value.status == gpu.MSF_ERR_INVALID_ARG
        with pytest.raises(gpu.MsfError):
            ctx.segment(3, 5, [])
        with pytest.raises(gpu.MsfError):
            ctx.segment(0, 2, [], edges=8)
        # capacity: asking for fewer records than features
        lab, n = ctx.segment(0, 4, [])
        st = gpu.load_library().msf_extract_features(
            ctx.h, gpu.ctypes.byref(gpu.make_criteria(0, 4, [])), lab.data_ptr(), gpu.MSF_DEVICE,
            None, gpu.MSF_HOST, 0, gpu.ctypes.byref(gpu.ctypes.c_int64()))
        assert st == gpu.MSF_ERR_CAPACITY
    finally:
        ctx.close()


@pytest.mark.slow
def test_mid_workload_full_size(gpu, orc):
    """128^3 x 32, 1M particles with two attributes, field > 0.5 AND mean speed in [q40, q90]:
    the configuration the benchmark times, compared over the whole window."""
    wl = synth.mid(device="cuda")
    f, p, a = wl.numpy()
    full_check(gpu, orc, f, p, a, 0, f.shape[0], wl.preds)


@pytest.mark.parametrize("big", [False, True])
def test_quantisation_rounding_edges(gpu, orc, big):
    """Attribute values at the fixed-point rounding edges: with max|v| = 1 (e = 1) and P*T =
    2000 samples (b = 11) the exponent is k = 50, so (2j+1) * 2^-51 lands exactly half-way
    between two integers and must round to even; values one fp32 ulp either side, negative
    halves, subnormals and -0.0 ride along. With big=True the largest value is 3e38 and k is
    negative (k = 62 - 128 - 11 = -77)."""
    rng = np.random.default_rng(21)
    T, nz, ny, nx, P = 2, 2, 3, 33, 1000
    pos = (rng.random((T, 3, P)) * np.array([nx, ny, nz])[None, :, None]).astype(np.float32)
    vals = [1.0, -0.0, 1e-45, -1e-45, 1.17e-38]
    for j in range(40):
        h = np.float32((2 * j + 1) * 2.0 ** -51)
        vals += [h, -h, np.nextafter(h, np.float32(1)), np.nextafter(h, np.float32(0))]
    vals += list(rng.normal(size=64) * 2.0 ** -45)
    if big:
        vals += [3.0e38, -2.9e38, 1.0e20, 7.5]
    v = np.resize(np.array(vals, np.float32), (T, 1, P)).copy()
    g = gpu_run(gpu, np.ones((T, nz, ny, nx), np.float32), pos, v, 0, T,
                [(C, 0, GE, 1, 0)], features=False)
    o = orc.bin((T, nz, ny, nx), pos, v)
    assert int(o["kscale"][0]) == (-77 if big else 50)
    check_bins(g, o)


def test_retained_segmentation_is_per_query(gpu, orc):
    """Features of an older query's labels (another buffer, another criterion) are computed
    from those labels, not from the most recent segmentation; host label buffers take the same
    paths."""
    wl = synth.mid(n=40, T=6, P=30000, n_blobs=10)
    f, p, a = wl.numpy()
    q1 = wl.preds
    q2 = [(F, 0, GT, 0.35, 0)]
    o = orc.bin(f.shape, p, a)
    ctx = gpu.Context(0)
    try:
        ctx.load(f, p, a)
        ctx.bin()
        l1, n1 = ctx.segment(0, 6, q1)
        l2, n2 = ctx.segment(1, 5, q2)
        fe1 = ctx.features(0, 6, l1, q1)           # not the last query: read from l1
        fe2 = ctx.features(1, 5, l2, q2)           # the last query: retained segmentation
        hl = np.empty((4,) + f.shape[1:], np.int32)
        n3 = gpu.msf_segment(ctx.h, gpu.make_criteria(1, 5, q1), hl)
        fe3 = gpu.msf_extract_features(ctx.h, gpu.make_criteria(1, 5, q1), hl)
    finally:
        ctx.close()
    for (t0, t1, q, lab_g, fe) in ((0, 6, q1, l1.cpu().numpy(), fe1), (1, 5, q2, l2.cpu().numpy(), fe2),
                                   (1, 5, q1, hl, fe3)):
        lab, nf = orc.segment(f, o["count"], o["mean"], o["key"], t0, t1, q)
        assert np.array_equal(lab_g, lab)
        of = orc.features(f, o["count"], a, o["key"], o["kscale"], t0, t1, lab)
        check_features(fe, of, a.shape[1])
    assert n3 == len(fe3)


def test_interval_predicate_edges(gpu, orc):
    """Strict and inclusive comparisons at exact threshold values, +-0, infinities and NaN field
    values: the library's interval form of each predicate selects what the comparison says."""
    T, nz, ny, nx = 2, 3, 4, 36
    vals = np.array([0.0, -0.0, 0.5, np.nextafter(np.float32(0.5), np.float32(1)),
                     np.nextafter(np.float32(0.5), np.float32(0)), np.inf, -np.inf, np.nan, 1.0,
                     -1.0, 1e-45, -1e-45], np.float32)
    f = np.resize(vals, (T, nz, ny, nx)).astype(np.float32)
    p = np.zeros((T, 3, 0), np.float32)
    a = np.zeros((T, 0, 0), np.float32)
    cases = [[(F, 0, GT, 0.5, 0)], [(F, 0, GE, 0.5, 0)], [(F, 0, LT, 0.5, 0)], [(F, 0, LE, 0.5, 0)],
             [(F, 0, GT, 0.0, 0)], [(F, 0, LT, -0.0, 0)], [(F, 0, GT, np.inf, 0)],
             [(F, 0, LT, -np.inf, 0)], [(F, 0, GE, -np.inf, 0)], [(F, 0, BAND, -0.0, 0.5)],
             [(F, 0, GT, np.nan, 0)], [(F, 0, LE, np.inf, 0)]]
    for preds in cases:
        full_check(gpu, orc, f, p, a, 0, T, preds, edges=3)


def test_mean_conversion_ties(gpu, orc):
    """Per-voxel fixed-point sums that sit exactly half-way between two fp32 values (2^24 + 1,
    2^24 + 3, 2^30 + 2^6, ...) must convert to fp32 with round-half-even before the division by
    the count. With max|v| = 1 and 512 samples (2^10 >= 513, so k = 62 - 1 - 10 = 51) a value v
    contributes v * 2^51 exactly, so two samples per voxel give any chosen sum."""
    T, nz, ny, nx = 1, 1, 1, 16
    k = 51
    sums = [2 ** 24 + 1, 2 ** 24 + 3, 2 ** 30 + 2 ** 6, 2 ** 30 + 3 * 2 ** 6, 2 ** 40 + 2 ** 16,
            2 ** 25 + 2, 2 ** 25 + 6, 2 ** 24 - 1, 2 ** 45 + 2 ** 21 + 1, 7]
    P = 512
    pos = np.full((T, 3, P), 0.5, np.float32)
    vals = np.zeros((T, 1, P), np.float32)
    vals[0, 0, -1] = 1.0                      # sets max|v| = 1 (in voxel 15)
    pos[0, 0, -1] = 15.5
    for i, s in enumerate(sums):
        sh = max(s.bit_length() - 24, 0)      # hi keeps the top 24 significant bits, lo the rest:
        hi = (s >> sh) << sh                  # both are exactly representable in fp32
        lo = s - hi
        for j, part in enumerate((hi, lo)):
            p = 2 * i + j
            pos[0, 0, p] = i + 0.5
            vals[0, 0, p] = np.float32(part * 2.0 ** -k)
            assert float(vals[0, 0, p]) * 2.0 ** k == part
    for p in range(2 * len(sums), P - 1):      # the rest sit in voxel 14 with value 0
        pos[0, 0, p] = 14.5
    g = gpu_run(gpu, np.ones((T, nz, ny, nx), np.float32), np.ascontiguousarray(pos), vals, 0, T,
                [(C, 0, GE, 1, 0)], features=False)
    o = orc.bin((T, nz, ny, nx), pos, vals)
    assert int(o["kscale"][0]) == k
    assert [int(x) for x in o["sumq"][0, 0, 0, 0, :len(sums)]] == sums
    check_bins(g, o)


def test_features_after_relabel_in_place(gpu, orc):
    """segment -> msf_relabel on the same buffer (two features merged into the smaller label,
    which stays the merged set's smallest index) -> extract_features: the statistics describe
    the relabelled buffer (the oracle's features of those labels), not the retained
    segmentation."""
    wl = synth.tiny()
    f, p, a = wl.numpy()
    ctx = gpu.Context(0)
    try:
        ctx.load(*_tensors(f, p, a))
        ctx.bin()
        t0, t1 = 0, f.shape[0]
        labels, n = ctx.segment(t0, t1, wl.preds)
        before = ctx.features(t0, t1, labels, wl.preds)
        assert n >= 3
        l1, l2 = int(before["label"][0]), int(before["label"][-1])
        K = int(labels.numel())
        mapping = torch.arange(K, dtype=torch.int32, device="cuda")
        mapping[l2] = l1
        ctx.relabel(labels, mapping)
        after = ctx.features(t0, t1, labels, wl.preds)
        torch.cuda.synchronize()
        lab = labels.cpu().numpy()
    finally:
        ctx.close()
    assert after.shape[0] == n - 1
    o = orc.bin(f.shape, p, a)
    of = orc.features(f, o["count"], a, o["key"], o["kscale"], t0, t1, lab)
    check_features(after, of, a.shape[1])
