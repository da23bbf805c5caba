"""Out-of-core labelling (msf_segment_streamed): a window of a host-resident dataset streamed
through the device in time slabs (§3.4, §4.3: data processed in chunks on the GPU), against the
CPU oracle's labelling of the whole window, bit-exact, for windows cut into three or more slabs
(down to one field step per slab), every edge class combination, a criterion with count and
mean predicates (the slabs bin with the whole dataset's fixed-point scale), and points on their
own time grid with empty field steps (trajectory links that cross one or more cuts)."""
import numpy as np
import pytest

from paper_1903_12294_gb300 import synth

pytestmark = pytest.mark.gpu

F, C, M = 0, 1, 2
GT, GE, BAND = 0, 1, 4


def _stream(gpu, f, p, a, t0, t1, preds, edges, slab, fstep=None):
    ctx = gpu.Context(0)
    try:
        lab = np.full((t1 - t0,) + f.shape[1:], -7, np.int32)
        n = gpu.msf_segment_streamed(ctx.h, f, p, a, gpu.make_criteria(t0, t1, preds, edges),
                                     slab, lab, fstep)
        return lab, n
    finally:
        ctx.close()


def _oracle(orc, f, p, a, t0, t1, preds, edges, fstep=None):
    o = orc.bin(f.shape, p, a, fstep=fstep)
    return orc.segment(f, o["count"], o["mean"], o["key"], t0, t1, preds, edges, fstep)


@pytest.mark.parametrize("edges", range(1, 8))
def test_streamed_tiny_every_edge_class(gpu, orc, edges):
    wl = synth.tiny()
    f, p, a = wl.numpy()
    ref, n_ref = _oracle(orc, f, p, a, 0, 8, wl.preds, edges)
    for slab in (3, 1):
        lab, n = _stream(gpu, f, p, a, 0, 8, wl.preds, edges, slab)
        assert n == n_ref and np.array_equal(lab, ref), (edges, slab)


def test_streamed_mean_predicate_and_late_window(gpu, orc):
    """A mean-speed band (the whole dataset's scale decides every mean bit) on a window that
    starts late and ends early, cut into 2-step slabs, against msf_segment on the resident
    dataset and the oracle."""
    wl = synth.mid(n=48, T=10, P=40000, n_blobs=10)
    f, p, a = wl.numpy()
    preds = wl.preds + [(C, 0, GE, 1, 0)]
    t0, t1 = 2, 9
    ref, n_ref = _oracle(orc, f, p, a, t0, t1, preds, 7)
    lab, n = _stream(gpu, f, p, a, t0, t1, preds, 7, 2)
    assert n == n_ref and np.array_equal(lab, ref)
    ctx = gpu.Context(0)
    try:
        ctx.load(f, p, a)
        ctx.bin()
        res, nr = ctx.segment(t0, t1, preds, 7)
        assert nr == n and np.array_equal(res.cpu().numpy(), lab)
    finally:
        ctx.close()


def test_streamed_points_on_their_own_grid(gpu, orc):
    """Points four times as often as the field and an uneven map with empty field steps (a link
    between consecutive point steps may cross several cuts)."""
    for fs in (None, [0, 0, 0, 2, 2, 3, 3, 3, 3, 3, 5, 5, 6, 7]):
        wl = synth.multirate(field_step=fs)
        f, p, a = wl.numpy()
        fstep = np.asarray(wl.field_step, np.int32)
        preds = [(F, 0, GT, 0.4, 0.0), (M, 0, BAND, 0.05, 0.9)]
        for edges in (7, 5, 4):
            ref, n_ref = _oracle(orc, f, p, a, 0, 8, preds, edges, fstep)
            lab, n = _stream(gpu, f, p, a, 0, 8, preds, edges, 3, fstep)
            assert n == n_ref and np.array_equal(lab, ref), (fs, edges)
