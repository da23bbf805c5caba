"""msf_segment_field_noalloc: the allocation-free, field-only labelling entry point.

It serves callers that cannot allocate device memory when they segment: services that reserve
all device memory up front in a pool of their own and forbid cudaMalloc/cudaFree (which can
synchronise the device and fail under memory pressure), real-time loops, plug-ins whose host
program owns the device memory. The test calls it through the C ABI twice in a row, on two
different fields, and checks each result against msf_segment (the context-based entry point) on
the same data; integer labels must be identical. It also checks field and label buffers that
start one element past a 16-byte boundary, and that a window larger than the fixed scratch is
rejected with MSF_ERR_TOO_LARGE.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

F, GT, BAND = 0, 0, 4


def _reference(gpu, field, pred, edges):
    ctx = gpu.Context(0)
    try:
        T = field.shape[0]
        ctx.load(field, torch.zeros((T, 3, 0), device=field.device),
                 torch.zeros((T, 0, 0), device=field.device))
        labels, n = ctx.segment(0, T, [pred] if pred else [], edges)
        torch.cuda.synchronize()
        return labels, n
    finally:
        ctx.close()


def test_noalloc_matches_msf_segment_twice(gpu):
    lib = gpu.load_library()
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    cases = [
        ((6, 20, 24, 64), (F, 0, GT, 0.62, 0.0), 3),      # 3D, spatial + temporal
        ((9, 1, 80, 96), (F, 0, BAND, 0.3, 0.55), 1),     # 2D+time, spatial only
    ]
    stream = torch.cuda.current_stream()
    for shape, pred, edges in cases:                      # two calls in a row
        field = torch.rand(shape, generator=g, device="cuda", dtype=torch.float32)
        labels = torch.full(shape, -7, dtype=torch.int32, device="cuda")
        p = gpu.msf_pred(*pred)
        n = ctypes.c_int64(-1)
        tw, nz, ny, nx = shape
        st = lib.msf_segment_field_noalloc(nx, ny, nz, tw, field.data_ptr(), ctypes.byref(p),
                                           edges, labels.data_ptr(), ctypes.byref(n),
                                           stream.cuda_stream)
        assert st == gpu.MSF_OK, gpu.msf_status_string(st)
        ref, n_ref = _reference(gpu, field, pred, edges)
        assert n.value == n_ref and n_ref > 1
        assert torch.equal(labels, ref)


def test_noalloc_unaligned_buffers(gpu):
    """Field and labels one float past a 16-byte boundary (nx a multiple of four, so aligned
    rows would take 16-byte loads): the labels are still msf_segment's, aligned or not; buffers
    that are not even 4-byte aligned are refused."""
    lib = gpu.load_library()
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    shape = (5, 12, 20, 32)
    tw, nz, ny, nx = shape
    n_el = tw * nz * ny * nx
    stream = torch.cuda.current_stream()
    pred = (F, 0, GT, 0.6, 0.0)
    p = gpu.msf_pred(*pred)
    fbuf = torch.rand(n_el + 4, generator=g, device="cuda", dtype=torch.float32)
    lbuf = torch.full((n_el + 4,), -7, dtype=torch.int32, device="cuda")
    for off in (0, 1):
        field = fbuf[off:off + n_el].view(shape)
        labels = lbuf[off:off + n_el].view(shape)
        assert (field.data_ptr() % 16 != 0) == (off == 1)
        n = ctypes.c_int64(-1)
        st = lib.msf_segment_field_noalloc(nx, ny, nz, tw, field.data_ptr(), ctypes.byref(p), 3,
                                           labels.data_ptr(), ctypes.byref(n), stream.cuda_stream)
        assert st == gpu.MSF_OK, gpu.msf_status_string(st)
        ref, n_ref = _reference(gpu, field.contiguous(), pred, 3)
        assert n.value == n_ref and n_ref > 1
        assert torch.equal(labels, ref)
    n = ctypes.c_int64(0)
    st = lib.msf_segment_field_noalloc(nx, ny, nz, tw, fbuf.data_ptr() + 2, ctypes.byref(p), 3,
                                       lbuf.data_ptr(), ctypes.byref(n), stream.cuda_stream)
    assert st == gpu.MSF_ERR_INVALID_ARG


def test_noalloc_rejects_windows_beyond_its_scratch(gpu):
    lib = gpu.load_library()
    tw, nz, ny, nx = 64, 64, 64, 64                      # 16.8M voxel-timesteps
    n = ctypes.c_int64(0)
    st = lib.msf_segment_field_noalloc(nx, ny, nz, tw, ctypes.c_void_p(16), None, 3,
                                       ctypes.c_void_p(16), ctypes.byref(n), None)
    assert st == gpu.MSF_ERR_TOO_LARGE
    st = lib.msf_segment_field_noalloc(nx, ny, nz, 2, ctypes.c_void_p(16), None, 7,
                                       ctypes.c_void_p(16), ctypes.byref(n), None)
    assert st == gpu.MSF_ERR_INVALID_ARG                   # trajectory edges need points
