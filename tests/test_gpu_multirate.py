"""GPU parity for point samples on a finer time grid than the field (§3.4: the two data types
need not share a temporal resolution; §4.1: the particles are saved far more often than the
field), through msf_load_timesteps_mr, against the CPU oracle: binning outputs bit-exact (keys
per point step, counts and sums per field step, means bit-exact), labels bit-exact for every
edge class combination, feature statistics within the parity tolerance, and the batched form
identical to single queries and to the oracle."""
import numpy as np
import pytest
import torch

from paper_1903_12294_gb300 import synth
from tests.test_gpu_parity import check_features

pytestmark = pytest.mark.gpu

F, C, M = 0, 1, 2
GT, GE, BAND = 0, 1, 4


def _load(gpu, wl):
    ctx = gpu.Context(0)
    ctx.load(wl.field.cuda(), wl.pos.cuda(), wl.attr.cuda(), field_step=wl.field_step)
    return ctx


@pytest.mark.parametrize("mapping", ["even", "uneven"])
def test_multirate_bins_labels_features(gpu, orc, mapping):
    """4 point steps per field step, or an uneven map with empty field steps (1 and 4) and
    up to 5 point steps in one."""
    fs = None if mapping == "even" else [0, 0, 0, 2, 2, 3, 3, 3, 3, 3, 5, 5, 6, 7]
    wl = synth.multirate(field_step=fs)
    f, p, a = wl.numpy()
    fstep = np.asarray(wl.field_step, np.int32)
    o = orc.bin(f.shape, p, a, fstep=fstep)
    ctx = _load(gpu, wl)
    try:
        st = ctx.bin(keep_sumq=True)
        key, count, mean, sumq = ctx.bins("cpu", sumq=True)
        assert np.array_equal(key.numpy(), o["key"])
        assert np.array_equal(count.numpy(), o["count"])
        assert np.array_equal(sumq.numpy(), o["sumq"])
        assert np.array_equal(mean.numpy().view(np.uint32), o["mean"].view(np.uint32))
        assert list(st.kscale)[:a.shape[1]] == list(o["kscale"])
        assert st.out_of_domain == int(o["outside"].sum())
        preds = [(F, 0, GT, 0.4, 0.0), (M, 0, BAND, 0.05, 0.9)]
        for edges in range(8):
            for t0, t1 in ((0, 8), (2, 7), (4, 5)):
                labels, n = ctx.segment(t0, t1, preds, edges)
                ref, n_ref = orc.segment(f, o["count"], o["mean"], o["key"], t0, t1, preds,
                                         edges, fstep)
                assert n == n_ref, (edges, t0, t1)
                assert np.array_equal(labels.cpu().numpy(), ref), (edges, t0, t1)
        labels, n = ctx.segment(1, 8, preds, 7)
        ref = labels.cpu().numpy()
        of = orc.features(f, o["count"], a, o["key"], o["kscale"], 1, 8, ref, fstep)
        check_features(ctx.features(1, 8, labels, preds, 7), of, a.shape[1])   # retained
        check_features(ctx.features(1, 8, labels.clone(), preds, 7), of, a.shape[1])
        labels2, _ = ctx.segment(1, 8, preds, 7)                  # components kept
        check_features(ctx.features(1, 8, labels2, preds, 7), of, a.shape[1])
        torch.cuda.synchronize()
    finally:
        ctx.close()


def test_multirate_batched_matches_oracle(gpu, orc):
    """Queries of different windows (one step windows included, whose trajectory links all lie
    inside one field step) in one msf_segment_batch call."""
    wl = synth.multirate()
    f, p, a = wl.numpy()
    fstep = np.asarray(wl.field_step, np.int32)
    o = orc.bin(f.shape, p, a, fstep=fstep)
    queries = [(0, 8, [(F, 0, GT, 0.4, 0.0)], 7), (3, 4, [(F, 0, GT, 0.3, 0.0)], 7),
               (2, 6, [(F, 0, GT, 0.45, 0.0), (C, 0, GE, 3, 0)], 5),
               (5, 8, [(F, 0, GT, 0.5, 0.0)], 6), (1, 2, [(F, 0, GT, 0.35, 0.0)], 4)]
    ctx = _load(gpu, wl)
    try:
        ctx.bin()
        labels, nfs = ctx.segment_batch(queries)
        got = [(l.cpu().numpy(), n) for l, n in zip(labels, nfs)]
    finally:
        ctx.close()
    for (t0, t1, pr, e), (lab, n) in zip(queries, got):
        ref, n_ref = orc.segment(f, o["count"], o["mean"], o["key"], t0, t1, pr, e, fstep)
        assert n == n_ref and np.array_equal(lab, ref), (t0, t1, e)


@pytest.mark.parametrize("mapping,k,t0,t1", [("even", (4, 4, 4, 3), 0, 8),
                                             ("uneven", (3, 5, 2, 4), 2, 8),
                                             ("uneven", (5, 3, 3, 1), 5, 6)])
def test_multirate_cluster_matches_oracle(gpu, orc, mapping, k, t0, t1):
    """§3.2 clustering with points on their own grid (the i-th of the r point steps of field
    step f at time f + (i + 0.5) / r): field and point labels, centres (bit-exact), counts and
    updates as the oracle's; point labels cover the window's point steps. The uneven map holds
    field steps with one, several and no point steps."""
    fs = None if mapping == "even" else [0, 0, 1, 1, 1, 1, 1, 3, 3, 4, 5, 5, 5, 6, 7, 7, 7, 7]
    wl = synth.multirate(n=24, T=8, r=3, P=6000, field_step=fs)
    f, p, a = wl.numpy()
    fstep = np.asarray(wl.field_step, np.int32)
    kw = dict(w_p=2.0, w_f=1.0, w_d=0.2, c_f=1.5, eps_c=1e-3, max_iter=7)
    ctx = _load(gpu, wl)
    try:
        ctx.bin()
        fl, pl, c, n, it = ctx.cluster(t0, t1, 0, k, **kw)
        torch.cuda.synchronize()
        key = ctx.bins("cpu")[0].numpy()
        g = (fl.cpu().numpy(), pl.cpu().numpy(), c, n, it)
    finally:
        ctx.close()
    o = orc.slic(f, p, a, key, t0, t1, 0, k, fstep=fstep, **kw)
    nj = int(np.count_nonzero((fstep >= t0) & (fstep < t1)))
    assert g[1].shape == (nj, p.shape[2]) and o[1].shape == g[1].shape
    assert g[4] == o[4]
    assert np.array_equal(g[0], o[0])
    assert np.array_equal(g[1], o[1])
    assert np.array_equal(g[2].view(np.uint32), o[2].view(np.uint32))
    assert np.array_equal(g[3], o[3])
    assert g[3][:, 1].sum() == np.count_nonzero(g[1] >= 0) > 0


def test_multirate_refusals(gpu):
    """The steps that take one point step per field step (point labels of msf_cluster_stats)
    refuse a dataset on its own grid; a map that decreases is refused at load."""
    wl = synth.multirate(n=16, T=4, r=2, P=500)
    ctx = _load(gpu, wl)
    try:
        ctx.bin()
        fl, pl, c, n, it = ctx.cluster(0, 4, 0, (2, 2, 2, 1))
        assert pl.shape == (8, 500)
        with pytest.raises(gpu.MsfError):
            ctx.cluster_stats(0, 4, 0, fl, pl, 8)
        with pytest.raises(gpu.MsfError):
            ctx.load(wl.field.cuda(), wl.pos.cuda(), wl.attr.cuda(),
                     field_step=[0, 1, 0, 2, 2, 3, 3, 3])
    finally:
        ctx.close()
