"""Query server (msf_server_*): continuous batching with memory admission.

Each result must equal msf_segment of the same query alone (canonical labels: bit-exact) and,
on a small case, the CPU oracle, whatever batch and slot it ran in; admission must respect the
pool; failures are reported per query, and injected admission faults leave the server usable.
"""
import threading

import numpy as np
import pytest
import torch

from paper_1903_12294_gb300 import synth

pytestmark = pytest.mark.gpu

F, C, M = 0, 1, 2
GT, GE, BAND = 0, 1, 4


def _dataset_2d(seed=7, T=24, n=128, walkers=6000):
    wl = synth.serving(n=n, T=T, walkers=walkers, seed=seed, nq=1)
    return wl


def _loaded(gpu, wl):
    ctx = gpu.Context(0)
    ctx.load(*(torch.as_tensor(x).cuda().contiguous() for x in wl.numpy()))
    ctx.bin()
    return ctx


def _drain(srv, want, timeout_s=60.0, release=False):
    """Poll until `want` results arrived; returns {tag: (status, n_features, labels copy, batch)}."""
    import time
    out = {}
    t_end = time.time() + timeout_s
    while len(out) < want:
        assert time.time() < t_end, f"only {len(out)} of {want} results"
        for r in srv.poll(cap=64, timeout_ms=200):
            if release:
                lab = srv.take_labels(r)
            else:
                lab = srv.labels(r)
                lab = None if lab is None else lab.clone()
                torch.cuda.synchronize()
            out[r.tag] = (r.status, r.n_features, lab, r.batch_size)
    return out


def test_server_results_equal_single_queries(gpu, orc):
    """A burst of mixed queries from several client threads: every result equals msf_segment of
    that query alone; batches really formed and overlapped."""
    wl = _dataset_2d()
    qs = synth.random_queries(wl, 48, seed=11, tw_range=(1, 24), field_q=(0.85, 0.99))
    qs[3] = (qs[3][0], qs[3][1], [(F, 0, GT, 0.05, 0)], 3)            # field only, no trajectory
    qs[5] = (qs[5][0], qs[5][1], [(F, 0, GT, 0.05, 0), (C, 0, GE, 1, 0)], 6)
    qs[7] = (4, 4, qs[7][2], 7)                                        # empty window
    ctx = _loaded(gpu, wl)
    try:
        srv = gpu.Server(ctx, pool_bytes=1 << 30, max_batch=8, slots=3)
        try:
            def client(k):
                for i in range(k, len(qs), 4):
                    t0, t1, pr, e = qs[i]
                    srv.submit(i, t0, t1, pr, e)
            th = [threading.Thread(target=client, args=(k,)) for k in range(4)]
            for t in th:
                t.start()
            for t in th:
                t.join()
            res = _drain(srv, len(qs), release=True)
            st = srv.stats()
        finally:
            srv.close()
        assert st.completed == len(qs) and st.pending == 0 and st.in_flight == 0
        assert st.pool_used == 0 and 0 < st.pool_peak <= st.pool_bytes
        assert st.max_batch_seen > 1 and st.batches < len(qs)
        for i, (t0, t1, pr, e) in enumerate(qs):
            status, nf, lab, _ = res[i]
            assert status == gpu.MSF_OK
            ref, n_ref = ctx.segment(t0, t1, pr, e)
            torch.cuda.synchronize()
            assert nf == n_ref, i
            if t1 == t0:
                assert lab is None
            else:
                assert torch.equal(lab, ref), i
        # the chain to the oracle on a few of them
        f, p, a = wl.numpy()
        o = orc.bin(f.shape, p, a)
        for i in (0, 3, 5, 9):
            t0, t1, pr, e = qs[i]
            lab_o, n_o = orc.segment(f, o["count"], o["mean"], o["key"], t0, t1, pr, e)
            assert res[i][1] == n_o and np.array_equal(res[i][2].cpu().numpy(), lab_o)
    finally:
        ctx.close()


def test_server_admission_waits_for_memory(gpu):
    """A pool that holds about two queries: the rest wait until results are released, and all
    still complete with the right labels. A query larger than the pool is refused."""
    wl = _dataset_2d(seed=8, T=48)
    q = [(F, 0, GT, float(np.quantile(wl.field.numpy(), 0.9)), 0)]
    qs = [(t0, t0 + 4, q, 7) for t0 in range(0, 48, 4)]   # windows inside one 16-step chunk
    ctx = _loaded(gpu, wl)
    try:
        # bytes one such query holds (labels + scratch), measured on a roomy server
        srv = gpu.Server(ctx, pool_bytes=1 << 30)
        srv.submit(0, *qs[0][:2], q, 7)
        _drain(srv, 1, release=True)
        one = srv.stats().pool_peak
        srv.close()
        pool = int(2.5 * one)
        srv = gpu.Server(ctx, pool_bytes=pool, max_batch=8, slots=2)
        try:
            with pytest.raises(gpu.MsfError) as e:
                srv.submit(99, 0, 48, q, 7)   # 12x the labels, 3x the scratch
            assert e.value.status == gpu.MSF_ERR_TOO_LARGE
            for i, (t0, t1, pr, ed) in enumerate(qs):
                srv.submit(i, t0, t1, pr, ed)
            res = _drain(srv, len(qs), release=True)
            st = srv.stats()
        finally:
            srv.close()
        assert st.pool_peak <= pool and st.max_batch_seen <= 2
        for i, (t0, t1, pr, ed) in enumerate(qs):
            ref, n_ref = ctx.segment(t0, t1, pr, ed)
            torch.cuda.synchronize()
            assert res[i][0] == gpu.MSF_OK and res[i][1] == n_ref and torch.equal(res[i][2], ref)
    finally:
        ctx.close()


def test_server_freezes_dataset_and_checks_tags(gpu):
    wl = _dataset_2d(seed=9, T=8, n=64, walkers=500)
    ctx = _loaded(gpu, wl)
    try:
        srv = gpu.Server(ctx, pool_bytes=64 << 20)
        with pytest.raises(gpu.MsfError) as e:
            ctx.bin()
        assert e.value.status == gpu.MSF_ERR_BUSY
        srv.submit(1, 0, 4, [(F, 0, GT, 0.1, 0)], 7)
        with pytest.raises(gpu.MsfError):
            srv.submit(1, 0, 4, [(F, 0, GT, 0.1, 0)], 7)    # tag still in use
        r = _drain(srv, 1)
        assert r[1][0] == gpu.MSF_OK
        with pytest.raises(gpu.MsfError):
            srv.submit(1, 0, 4, [(F, 0, GT, 0.1, 0)], 7)    # labels not yet released
        srv.release(1)
        srv.submit(1, 0, 2, [(F, 0, GT, 0.1, 0)], 7)        # free again
        _drain(srv, 1, release=True)
        with pytest.raises(gpu.MsfError):
            srv.release(1)                                   # nothing held
        srv.close()
        ctx.bin()                                            # unfrozen
    finally:
        ctx.close()


def test_server_injected_admission_fault(gpu, monkeypatch):
    """MSF_FAULT=admit: each query fails with OUT_OF_MEMORY and nothing leaks; a server started
    without it serves normally afterwards."""
    wl = _dataset_2d(seed=10, T=8, n=64, walkers=500)
    ctx = _loaded(gpu, wl)
    try:
        monkeypatch.setenv("MSF_FAULT", "admit")
        srv = gpu.Server(ctx, pool_bytes=64 << 20)
        monkeypatch.delenv("MSF_FAULT")
        for i in range(3):
            srv.submit(i, 0, 4, [(F, 0, GT, 0.1, 0)], 7)
        res = _drain(srv, 3)
        st = srv.stats()
        srv.close()
        assert all(v[0] == gpu.MSF_ERR_OUT_OF_MEMORY and v[2] is None for v in res.values())
        assert st.pool_used == 0
        srv = gpu.Server(ctx, pool_bytes=64 << 20)
        srv.submit(0, 0, 4, [(F, 0, GT, 0.1, 0)], 7)
        res = _drain(srv, 1, release=True)
        srv.close()
        ref, n_ref = ctx.segment(0, 4, [(F, 0, GT, 0.1, 0)], 7)
        torch.cuda.synchronize()
        assert res[0][0] == gpu.MSF_OK and res[0][1] == n_ref and torch.equal(res[0][2], ref)
    finally:
        ctx.close()
