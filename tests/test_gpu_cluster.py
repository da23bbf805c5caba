"""GPU parity of the multifaceted 4D clustering (msf_cluster, §3.2) against the CPU oracle:
field and point labels bit-exact, centres bit-exact (same fp32 decisions, exact fixed-point
sums, the same fp64 means), counts and the number of updates equal."""
import numpy as np
import pytest
import torch

from paper_1903_12294_gb300 import synth

pytestmark = pytest.mark.gpu


def _run(gpu, orc, f, p, a, t0, t1, attr, k, **kw):
    ctx = gpu.Context(0)
    try:
        ctx.load(*(torch.as_tensor(x).cuda().contiguous() for x in (f, p, a)))
        ctx.bin()
        fl, pl, c, n, it = ctx.cluster(t0, t1, attr, k, **kw)
        torch.cuda.synchronize()
        key = ctx.bins("cpu")[0].numpy()
        g = (fl.cpu().numpy(), pl.cpu().numpy(), c, n, it)
    finally:
        ctx.close()
    o = orc.slic(f, p, a, key, t0, t1, attr, k, **kw)
    assert g[4] == o[4], (g[4], o[4])
    assert np.array_equal(g[0], o[0])
    assert np.array_equal(g[1], o[1])
    assert np.array_equal(g[2].view(np.uint32), o[2].view(np.uint32))
    assert np.array_equal(g[3], o[3])
    return g


PARAMS = [
    dict(w_p=1.0, w_f=1.0, w_d=0.05, c_f=1.0, eps_c=1e-3, max_iter=10),
    dict(w_p=5.0, w_f=0.5, w_d=0.5, c_f=2.0, eps_c=1e-4, max_iter=6),
    dict(w_p=0.0, w_f=0.0, w_d=1.0, c_f=0.5, eps_c=1e-2, max_iter=8),
    dict(w_p=20.0, w_f=20.0, w_d=0.01, c_f=1.0, eps_c=0.0, max_iter=4),
]


@pytest.mark.parametrize("prm", range(len(PARAMS)))
def test_tiny_workload(gpu, orc, prm):
    wl = synth.tiny()
    f, p, a = wl.numpy()
    g = _run(gpu, orc, f, p, a, 0, 8, 0, (4, 4, 4, 2), **PARAMS[prm])
    assert g[4] >= 1


@pytest.mark.parametrize("k", [(3, 5, 2, 3), (7, 2, 3, 1), (1, 1, 1, 1), (6, 6, 6, 4)])
def test_ragged_spacing_and_windows(gpu, orc, k):
    """Seed spacings that are not whole voxels, a window that starts late."""
    wl = synth.mid(n=30, T=9, P=20000, n_blobs=8)
    f, p, a = wl.numpy()
    _run(gpu, orc, f, p, a, 2, 9, 1, k, w_p=2.0, w_f=1.0, w_d=0.2, c_f=1.5, eps_c=1e-3,
         max_iter=7)


def test_invalid_samples(gpu, orc):
    rng = np.random.default_rng(2)
    T, nz, ny, nx, P = 5, 9, 10, 12, 3000
    f = rng.normal(size=(T, nz, ny, nx)).astype(np.float32)
    f[1, 2, 3, 4] = np.nan
    f[4, 0, 0, 0] = -np.inf
    pos = (rng.random((T, 3, P)) * np.array([nx, ny, nz])[None, :, None]).astype(np.float32)
    pos[2, 1, 7] = 99.0
    pos[3, 0, 8] = np.nan
    a = rng.normal(size=(T, 2, P)).astype(np.float32)
    a[0, 1, 11] = np.inf
    _run(gpu, orc, f, pos, a, 0, T, 1, (3, 3, 2, 2), w_p=1.0, w_f=1.0, w_d=0.3, max_iter=5)


def test_2d_time_and_no_points(gpu, orc):
    rng = np.random.default_rng(5)
    T, nz, ny, nx = 12, 1, 40, 56
    f = rng.normal(size=(T, nz, ny, nx)).astype(np.float32)
    P = 2500
    pos = (rng.random((T, 3, P)) * np.array([nx, ny, nz])[None, :, None]).astype(np.float32)
    a = rng.normal(size=(T, 1, P)).astype(np.float32)
    _run(gpu, orc, f, pos, a, 0, T, 0, (5, 4, 1, 3), w_p=1.0, w_f=2.0, w_d=0.1, max_iter=8)
    empty_p = np.zeros((T, 3, 0), np.float32)
    empty_a = np.zeros((T, 0, 0), np.float32)
    _run(gpu, orc, f, empty_p, empty_a, 3, T, 0, (4, 4, 1, 2), w_f=2.0, w_d=0.1, max_iter=8)


def test_errors(gpu):
    wl = synth.tiny(T=4, P=2000)
    ctx = gpu.Context(0)
    try:
        ctx.load(*(x.cuda() for x in (wl.field, wl.pos, wl.attr)))
        with pytest.raises(gpu.MsfError) as e:
            ctx.cluster(0, 4, 0, (2, 2, 2, 2))
        assert e.value.status == gpu.MSF_ERR_NOT_BINNED
        ctx.bin()
        for bad in [dict(t0=2, t1=2), dict(attr=5), dict(k=(0, 1, 1, 1)), dict(max_iter=0)]:
            args = dict(t0=0, t1=4, attr=0, k=(2, 2, 2, 2), max_iter=3)
            args.update(bad)
            with pytest.raises(gpu.MsfError) as e:
                ctx.cluster(args["t0"], args["t1"], args["attr"], args["k"],
                            max_iter=args["max_iter"])
            assert e.value.status == gpu.MSF_ERR_INVALID_ARG
        with pytest.raises(gpu.MsfError) as e:
            ctx.cluster(0, 4, 0, (128, 128, 128, 1))
        assert e.value.status == gpu.MSF_ERR_TOO_LARGE
    finally:
        ctx.close()
