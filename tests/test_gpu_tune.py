"""Schedules and autotuning of msf_segment: every tile shape and schedule gives the oracle's
labels (labels are canonical), and msf_autotune keeps a valid, applied choice per shape."""
import numpy as np
import pytest
import torch

from paper_1903_12294_gb300 import synth

pytestmark = pytest.mark.gpu


def _ctx(gpu, wl):
    ctx = gpu.Context(0)
    ctx.load(*(x.cuda().contiguous() for x in (wl.field, wl.pos, wl.attr)))
    ctx.bin()
    return ctx


@pytest.mark.parametrize("nx", [40, 37])       # 16-byte rows and ragged rows
def test_every_schedule_gives_the_oracle_labels(gpu, orc, nx):
    wl = synth.mid(n=nx, T=10, P=20000, n_blobs=6)
    f, p, a = wl.numpy()
    ctx = _ctx(gpu, wl)
    try:
        got = {}
        for sched in range(8):
            ctx.set_schedule(sched)
            for tile in [(0, 0, 0), (8, 8, 4), (4, 32, 2), (32, 8, 1)]:
                ctx.set_tile(*tile)
                lab, n = ctx.segment(1, 10, wl.preds, wl.edges)
                got[(sched, tile)] = (lab.cpu().numpy(), n)
        ctx.set_schedule(-1)
        ctx.set_tile(0, 0, 0)
    finally:
        ctx.close()
    _, labels, nf, _ = orc.run_all(f, p, a, 1, 10, wl.preds, wl.edges)
    for k, (lab, n) in got.items():
        assert n == nf and np.array_equal(lab, labels), k


def test_fused_criterion_field_only_and_2d(gpu, orc):
    """The fused criterion with field predicates only, and on a 2D + time grid."""
    rng = np.random.default_rng(3)
    T, ny, nx = 20, 70, 96
    f = rng.normal(size=(T, 1, ny, nx)).astype(np.float32)
    P = 3000
    pos = (rng.random((T, 3, P)) * np.array([nx, ny, 1])[None, :, None]).astype(np.float32)
    a = rng.normal(size=(T, 1, P)).astype(np.float32)
    preds = [(0, 0, 0, 0.8, 0.0)]
    ctx = gpu.Context(0)
    try:
        ctx.load(*(torch.as_tensor(x).cuda() for x in (f, pos, a)))
        ctx.bin()
        ctx.set_schedule(3)
        lab, n = ctx.segment(2, 20, preds)
        lab = lab.cpu().numpy()
    finally:
        ctx.close()
    o = orc.bin(f.shape, pos, a, keep_sumq=False)
    want, nf = orc.segment(f, o["count"], o["mean"], o["key"], 2, 20, preds)
    assert n == nf and np.array_equal(lab, want)


def test_autotune_keeps_an_applied_choice(gpu):
    wl = synth.mid(n=64, T=12, P=50000, n_blobs=8)
    ctx = _ctx(gpu, wl)
    try:
        ref, nref = ctx.segment(0, 12, wl.preds, wl.edges)
        ref = ref.cpu().numpy()
        rule = ctx.tuning(0, 12, wl.preds, wl.edges)
        assert rule[3] == 0
        r = ctx.autotune(0, 12, wl.preds, wl.edges, reps=2)
        assert r["by"] * r["bz"] * r["bt"] == 256 and 0 <= r["sched"] <= 5
        assert r["n_tried"] > 4 and 0 < r["ms"] <= r["ms_default"]
        chosen = ctx.tuning(0, 12, wl.preds, wl.edges)
        assert chosen == (r["by"], r["bz"], r["bt"], r["sched"])
        lab, n = ctx.segment(0, 12, wl.preds, wl.edges)            # runs the tuned choice
        assert n == nref and np.array_equal(lab.cpu().numpy(), ref)
        # another window length is another shape: still the rule
        assert ctx.tuning(0, 11, wl.preds, wl.edges) == ctx.tuning(0, 11, wl.preds, wl.edges)
        assert ctx.tuning(0, 11, wl.preds, wl.edges)[3] == 0
        # fixed choices win over the tuned one, and clearing restores the rule
        ctx.set_tile(16, 8, 2)
        ctx.set_schedule(1)
        assert ctx.tuning(0, 12, wl.preds, wl.edges) == (16, 8, 2, 1)
        ctx.set_tile(0, 0, 0)
        ctx.set_schedule(-1)
        assert ctx.tuning(0, 12, wl.preds, wl.edges) == chosen
        ctx.tune_clear()
        assert ctx.tuning(0, 12, wl.preds, wl.edges) == rule
        with pytest.raises(gpu.MsfError) as e:
            ctx.set_schedule(8)
        assert e.value.status == gpu.MSF_ERR_INVALID_ARG
        with pytest.raises(gpu.MsfError) as e:
            ctx.autotune(3, 3, wl.preds, wl.edges)
        assert e.value.status == gpu.MSF_ERR_INVALID_ARG
    finally:
        ctx.close()
