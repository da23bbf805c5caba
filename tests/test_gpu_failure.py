"""Failure detection without a device fault: the kernels' bounded waits give up (a limit of 0
cycles makes them give up at once), the call reports MSF_ERR_TIMEOUT, and the context stays
usable: after restoring the limit the same dataset bins and segments exactly as a fresh context
does."""
import pytest
import torch

from paper_1903_12294_gb300 import synth

pytestmark = pytest.mark.gpu


def test_wait_timeout_is_reported_and_recoverable(gpu):
    wl = synth.tiny(T=6, P=8000)
    dev = [x.cuda() for x in (wl.field, wl.pos, wl.attr)]
    ctx = gpu.Context(0)
    try:
        ctx.load(*dev)
        ctx.set_wait_limit(0)
        with pytest.raises(gpu.MsfError) as e:
            ctx.bin()
        assert e.value.status == gpu.MSF_ERR_TIMEOUT
        with pytest.raises(gpu.MsfError) as e:       # the dataset is not binned
            ctx.segment(0, 6, wl.preds, 7)
        assert e.value.status == gpu.MSF_ERR_NOT_BINNED
        ctx.set_wait_limit(-1)
        ctx.bin()
        lab, n = ctx.segment(0, 6, wl.preds, 7)
        torch.cuda.synchronize()
    finally:
        ctx.close()
    ref_ctx = gpu.Context(0)
    try:
        ref_ctx.load(*dev)
        ref_ctx.bin()
        ref, n_ref = ref_ctx.segment(0, 6, wl.preds, 7)
        torch.cuda.synchronize()
    finally:
        ref_ctx.close()
    assert n == n_ref and torch.equal(lab, ref)


def test_fused_batch_wait_timeout_is_reported_and_recoverable(gpu):
    """The persistent batched launch waits (bounded) on its queries' phase counters; with a
    limit of 0 the first wait that is not already met gives up, every block leaves, the batch
    reports MSF_ERR_TIMEOUT, and the same batch then runs normally with the limit restored."""
    wl = synth.mid(n=48, T=10, P=20000, n_blobs=8)
    dev = [x.cuda() for x in (wl.field, wl.pos, wl.attr)]
    queries = [(t0, t0 + 6, wl.preds, 7) for t0 in range(5)]
    ctx = gpu.Context(0)
    try:
        ctx.load(*dev)
        ctx.bin()
        ctx.set_batch_schedule(9)
        want = [ctx.segment(t0, t1, pr, e) for (t0, t1, pr, e) in queries]
        ctx.set_wait_limit(0)
        with pytest.raises(gpu.MsfError) as e:
            ctx.segment_batch(queries)
        assert e.value.status == gpu.MSF_ERR_TIMEOUT
        ctx.set_wait_limit(-1)
        labels, nfs = ctx.segment_batch(queries)
        torch.cuda.synchronize()
        for (lw, nw), lb, nf in zip(want, labels, nfs):
            assert nf == nw and torch.equal(lb, lw)
    finally:
        ctx.close()
