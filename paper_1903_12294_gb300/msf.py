"""ctypes binding of libmsf.so (the C ABI in include/msf.h), same names as the C entry points.

Argument marshalling only: every step of binning, criterion, labelling and feature reduction
runs in the library's CUDA kernels. torch tensors are accepted for convenience (device memory
and streams); their ``data_ptr()`` is passed as a plain pointer. If the library has not been
built, loading fails with an error instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmsf.so")

MSF_OK = 0
MSF_ERR_INVALID_ARG, MSF_ERR_NOT_LOADED, MSF_ERR_NOT_BINNED = -1, -2, -3
MSF_ERR_OUT_OF_MEMORY, MSF_ERR_TOO_LARGE, MSF_ERR_TIMEOUT = -4, -5, -6
MSF_ERR_CUDA, MSF_ERR_CAPACITY, MSF_ERR_INTERNAL, MSF_ERR_BUSY = -7, -8, -9, -10
MSF_HOST, MSF_DEVICE = 0, 1
MSF_SRC_FIELD, MSF_SRC_COUNT, MSF_SRC_MEAN = 0, 1, 2
MSF_OP_GT, MSF_OP_GE, MSF_OP_LT, MSF_OP_LE, MSF_OP_BAND = 0, 1, 2, 3, 4
MSF_EDGE_SPATIAL, MSF_EDGE_TEMPORAL, MSF_EDGE_TRAJ, MSF_EDGE_ALL = 1, 2, 4, 7
MSF_BIN_KEEP_SUMQ = 1
MSF_MAX_PRED, MSF_MAX_ATTR = 4, 8

# every entry point the header declares (checked by the CPU test-suite)
EXPORTS = ("msf_create", "msf_destroy", "msf_set_stream", "msf_load_timesteps",
           "msf_load_timesteps_mr", "msf_segment_streamed",
           "msf_bin_particles", "msf_get_bins", "msf_segment", "msf_extract_features",
           "msf_segment_features",
           "msf_set_tile", "msf_set_profiling", "msf_kernel_times", "msf_status_string",
           "msf_segment_field_noalloc", "msf_segment_batch", "msf_server_create",
           "msf_server_submit", "msf_server_poll", "msf_server_release", "msf_server_get_stats",
           "msf_server_destroy", "msf_set_wait_limit", "msf_cluster", "msf_merge_clusters",
           "msf_relabel", "msf_cluster_stats", "msf_select_clusters", "msf_split_trajectories",
           "msf_set_schedule", "msf_autotune", "msf_get_tuning", "msf_tune_clear",
           "msf_set_batch_graphs", "msf_batch_graph_replays", "msf_set_batch_tile",
           "msf_autotune_batch", "msf_set_batch_schedule")
MSF_SCHED_FUSED_CRITERION, MSF_SCHED_SERIAL_JOINS, MSF_SCHED_PIPELINE = 1, 2, 4
MSF_SCHED_PERSISTENT = 8
MSF_MERGE_POINT, MSF_MERGE_FIELD = 1, 2
MSF_SPACE_POINTS, MSF_SPACE_VOXELS = 0, 1


class msf_pred(ctypes.Structure):
    _fields_ = [("src", ctypes.c_int32), ("attr", ctypes.c_int32), ("op", ctypes.c_int32),
                ("lo", ctypes.c_float), ("hi", ctypes.c_float)]


class msf_criteria(ctypes.Structure):
    _fields_ = [("t0", ctypes.c_int32), ("t1", ctypes.c_int32), ("n_pred", ctypes.c_int32),
                ("pred", msf_pred * MSF_MAX_PRED), ("edges", ctypes.c_uint32)]


class msf_bin_stats(ctypes.Structure):
    _fields_ = [("in_domain", ctypes.c_int64), ("out_of_domain", ctypes.c_int64),
                ("kscale", ctypes.c_int32 * MSF_MAX_ATTR),
                ("max_abs", ctypes.c_float * MSF_MAX_ATTR)]


class msf_feature(ctypes.Structure):
    _fields_ = [("label", ctypes.c_int32), ("bbox_min", ctypes.c_int32 * 4),
                ("bbox_max", ctypes.c_int32 * 4), ("n_attr", ctypes.c_int32),
                ("n_vox", ctypes.c_int64), ("n_pts", ctypes.c_int64),
                ("sum_field", ctypes.c_double), ("mean_field", ctypes.c_double),
                ("std_field", ctypes.c_double), ("min_field", ctypes.c_float),
                ("max_field", ctypes.c_float), ("centroid", ctypes.c_double * 4),
                ("sumq", ctypes.c_int64 * MSF_MAX_ATTR),
                ("mean_attr", ctypes.c_double * MSF_MAX_ATTR),
                ("std_attr", ctypes.c_double * MSF_MAX_ATTR)]


FEATURE_DTYPE = np.dtype(msf_feature)


class msf_cluster_stat(ctypes.Structure):
    _fields_ = [("n_field", ctypes.c_int64), ("n_point", ctypes.c_int64),
                ("lo", ctypes.c_float * 4), ("hi", ctypes.c_float * 4),
                ("mean_field", ctypes.c_double), ("std_field", ctypes.c_double),
                ("mean_point", ctypes.c_double), ("std_point", ctypes.c_double)]


class msf_tune_result(ctypes.Structure):
    _fields_ = [("by", ctypes.c_int32), ("bz", ctypes.c_int32), ("bt", ctypes.c_int32),
                ("sched", ctypes.c_int32), ("ms", ctypes.c_float), ("ms_default", ctypes.c_float),
                ("n_tried", ctypes.c_int32)]


class msf_piece(ctypes.Structure):
    _fields_ = [("point", ctypes.c_int32), ("t_start", ctypes.c_int32),
                ("length", ctypes.c_int32), ("label", ctypes.c_int32)]


class msf_cluster_params(ctypes.Structure):
    _fields_ = [("t0", ctypes.c_int32), ("t1", ctypes.c_int32), ("attr", ctypes.c_int32),
                ("k", ctypes.c_int32 * 4), ("w_p", ctypes.c_float), ("w_f", ctypes.c_float),
                ("w_d", ctypes.c_float), ("c_f", ctypes.c_float), ("eps_c", ctypes.c_float),
                ("max_iter", ctypes.c_int32)]


class msf_server_config(ctypes.Structure):
    _fields_ = [("pool_bytes", ctypes.c_uint64), ("max_batch", ctypes.c_int32),
                ("slots", ctypes.c_int32)]


class msf_server_result(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("status", ctypes.c_int32),
                ("batch_size", ctypes.c_int32), ("n_features", ctypes.c_int64),
                ("labels", ctypes.c_void_p), ("n_labels", ctypes.c_int64),
                ("t_submit_ns", ctypes.c_int64), ("t_admit_ns", ctypes.c_int64),
                ("t_done_ns", ctypes.c_int64)]


class msf_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("max_batch_seen", ctypes.c_int64),
                ("max_slots_busy", ctypes.c_int64), ("pending", ctypes.c_int64),
                ("in_flight", ctypes.c_int64), ("pool_bytes", ctypes.c_uint64),
                ("pool_used", ctypes.c_uint64), ("pool_peak", ctypes.c_uint64)]


class MsfError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {msf_status_string(status)} ({status})")


_lib = None
_lock = threading.Lock()


def load_library(path: str = LIB_PATH):
    """Load libmsf.so; raises if it is missing (build it with ``__graft_entry__.build()``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError(f"libmsf.so not built at {path}; run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        P, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint
        lib.msf_create.argtypes = [ctypes.POINTER(P), i32, P]
        lib.msf_destroy.argtypes = [P]
        lib.msf_destroy.restype = None
        lib.msf_set_stream.argtypes = [P, P]
        lib.msf_load_timesteps.argtypes = [P, i32, i32, i32, i32, P, i64, i32, P, P, i32]
        lib.msf_load_timesteps_mr.argtypes = [P, i32, i32, i32, i32, P, i64, i32, i32, P, P, P,
                                              i32]
        lib.msf_segment_streamed.argtypes = [P, i32, i32, i32, i32, P, i64, i32, i32, P, P, P,
                                             ctypes.POINTER(msf_criteria), i32, P,
                                             ctypes.POINTER(ctypes.c_int64)]
        lib.msf_bin_particles.argtypes = [P, u32, ctypes.POINTER(msf_bin_stats)]
        lib.msf_get_bins.argtypes = [P, P, P, P, P, i32]
        lib.msf_segment.argtypes = [P, ctypes.POINTER(msf_criteria), P, i32,
                                    ctypes.POINTER(ctypes.c_int64)]
        lib.msf_extract_features.argtypes = [P, ctypes.POINTER(msf_criteria), P, i32, P, i32,
                                             i64, ctypes.POINTER(ctypes.c_int64)]
        lib.msf_segment_features.argtypes = [P, ctypes.POINTER(msf_criteria), P, i32,
                                             ctypes.POINTER(i64), P, i32, i64, ctypes.POINTER(i64)]
        lib.msf_set_tile.argtypes = [P, i32, i32, i32]
        lib.msf_set_profiling.argtypes = [P, i32]
        lib.msf_kernel_times.argtypes = [P, P, P, P, i32, i32]
        lib.msf_segment_field_noalloc.argtypes = [i32, i32, i32, i32, P, ctypes.POINTER(msf_pred),
                                                  u32, P, ctypes.POINTER(ctypes.c_int64), P]
        lib.msf_segment_batch.argtypes = [P, i32, ctypes.POINTER(msf_criteria),
                                          ctypes.POINTER(ctypes.c_void_p),
                                          ctypes.POINTER(ctypes.c_int64)]
        lib.msf_server_create.argtypes = [P, ctypes.POINTER(msf_server_config), ctypes.POINTER(P)]
        lib.msf_server_submit.argtypes = [P, ctypes.POINTER(msf_criteria), ctypes.c_uint64]
        lib.msf_server_poll.argtypes = [P, ctypes.POINTER(msf_server_result), i32,
                                        ctypes.POINTER(ctypes.c_int), i32]
        lib.msf_server_release.argtypes = [P, ctypes.c_uint64]
        lib.msf_server_get_stats.argtypes = [P, ctypes.POINTER(msf_server_stats)]
        lib.msf_server_destroy.argtypes = [P]
        lib.msf_set_wait_limit.argtypes = [P, ctypes.c_longlong]
        lib.msf_cluster.argtypes = [P, ctypes.POINTER(msf_cluster_params), P, P, i32, P, P,
                                    ctypes.POINTER(ctypes.c_int)]
        lib.msf_merge_clusters.argtypes = [P, P, i32, i32, ctypes.c_float, i32, P, i32,
                                           ctypes.POINTER(ctypes.c_int32)]
        lib.msf_relabel.argtypes = [P, P, i32, i64, P, i32, i32]
        lib.msf_cluster_stats.argtypes = [P, i32, i32, i32, P, P, i32, i32, P, i32]
        lib.msf_select_clusters.argtypes = [P, P, i32, i32, P, P, P, i32, i32,
                                            ctypes.POINTER(ctypes.c_int32)]
        lib.msf_split_trajectories.argtypes = [P, i32, i32, P, i32, i32, i32, P, i32, i64,
                                               ctypes.POINTER(ctypes.c_int64)]
        lib.msf_set_schedule.argtypes = [P, i32]
        lib.msf_set_batch_graphs.argtypes = [P, i32]
        lib.msf_set_batch_tile.argtypes = [P, i32, i32, i32]
        lib.msf_set_batch_schedule.argtypes = [P, i32]
        lib.msf_autotune_batch.argtypes = [P, i32, P, P, i32, ctypes.POINTER(msf_tune_result)]
        lib.msf_batch_graph_replays.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
        lib.msf_autotune.argtypes = [P, ctypes.POINTER(msf_criteria), i32,
                                     ctypes.POINTER(msf_tune_result)]
        lib.msf_get_tuning.argtypes = [P, ctypes.POINTER(msf_criteria), P]
        lib.msf_tune_clear.argtypes = [P]
        lib.msf_status_string.argtypes = [i32]
        lib.msf_status_string.restype = ctypes.c_char_p
        for n in EXPORTS:
            f = getattr(lib, n)
            if n not in ("msf_destroy", "msf_status_string"):
                f.restype = i32
        _lib = lib
    return _lib


def msf_status_string(status: int) -> str:
    return load_library().msf_status_string(int(status)).decode()


def _check(status, where):
    if status < 0:
        raise MsfError(status, where)
    return status


# ---------------------------------------------------------------------------------------------
# pointer helpers
# ---------------------------------------------------------------------------------------------

def _ptr_kind(x):
    """(pointer, kind) for a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None, MSF_HOST
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous")
        return (x.ctypes.data if x.size else None), MSF_HOST
    import torch
    if isinstance(x, torch.Tensor):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        kind = MSF_DEVICE if x.is_cuda else MSF_HOST
        return (x.data_ptr() if x.numel() else None), kind
    raise TypeError(f"unsupported buffer type {type(x)}")


def make_criteria(t0, t1, preds=(), edges=MSF_EDGE_ALL) -> msf_criteria:
    """preds: sequence of (src, attr, op, lo, hi)."""
    if len(preds) > MSF_MAX_PRED:
        raise ValueError("at most 4 predicates")
    c = msf_criteria()
    c.t0, c.t1, c.n_pred, c.edges = int(t0), int(t1), len(preds), int(edges)
    for i, (src, a, op, lo, hi) in enumerate(preds):
        c.pred[i] = msf_pred(int(src), int(a), int(op), float(lo), float(hi))
    return c


# ---------------------------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ---------------------------------------------------------------------------------------------

def msf_create(device: int = 0, stream=None):
    h = ctypes.c_void_p()
    s = stream if stream is None or isinstance(stream, int) else stream.cuda_stream
    _check(load_library().msf_create(ctypes.byref(h), int(device), s), "msf_create")
    return h


def msf_destroy(ctx):
    load_library().msf_destroy(ctx)


def msf_set_stream(ctx, stream):
    s = stream if stream is None or isinstance(stream, int) else stream.cuda_stream
    _check(load_library().msf_set_stream(ctx, s), "msf_set_stream")


def msf_load_timesteps(ctx, field, pos, attr):
    """field [T][nz][ny][nx] fp32, pos [T][3][P] fp32, attr [T][A][P] fp32 (all host or all
    device)."""
    T, nz, ny, nx = field.shape
    P = pos.shape[2] if pos is not None else 0
    A = attr.shape[1] if attr is not None else 0
    fp, k = _ptr_kind(field)
    pp, kp = _ptr_kind(pos)
    ap, ka = _ptr_kind(attr)
    if P and (kp != k or (A and ka != k)):
        raise ValueError("field, pos and attr must all be host or all device")
    _check(load_library().msf_load_timesteps(ctx, nx, ny, nz, T, fp, P, A, pp, ap, k),
           "msf_load_timesteps")


def msf_load_timesteps_mr(ctx, field, pos, attr, field_step):
    """field [T][nz][ny][nx] fp32; pos [Tp][3][P], attr [Tp][A][P] fp32 on their own time grid;
    field_step [Tp] (host sequence) the field step of each point step (non-decreasing)."""
    import numpy as np
    T, nz, ny, nx = field.shape
    P = pos.shape[2] if pos is not None else 0
    Tp = pos.shape[0] if pos is not None else len(field_step)
    A = attr.shape[1] if attr is not None else 0
    fp, k = _ptr_kind(field)
    pp, kp = _ptr_kind(pos)
    ap, ka = _ptr_kind(attr)
    if P and (kp != k or (A and ka != k)):
        raise ValueError("field, pos and attr must all be host or all device")
    fs = np.ascontiguousarray(np.asarray(field_step, dtype=np.int32).reshape(-1))
    _check(load_library().msf_load_timesteps_mr(ctx, nx, ny, nz, T, fp, P, A, int(Tp), pp, ap,
                                                fs.ctypes.data, k), "msf_load_timesteps_mr")


def msf_segment_streamed(ctx, field, pos, attr, crit: msf_criteria, slab_steps, labels,
                         field_step=None) -> int:
    """Out-of-core labelling of crit's window over host arrays (numpy or CPU tensors): field
    [T][nz][ny][nx], pos [Tp][3][P], attr [Tp][A][P] fp32, field_step [Tp] or None; labels a host
    int32 array [t1-t0][nz][ny][nx]. Returns the number of features."""
    import numpy as np
    T, nz, ny, nx = field.shape
    P = pos.shape[2] if pos is not None else 0
    Tp = pos.shape[0] if pos is not None else T
    A = attr.shape[1] if attr is not None else 0
    ptrs = []
    for x in (field, pos, attr, labels):
        p, k = _ptr_kind(x)
        if p and k != MSF_HOST:
            raise ValueError("msf_segment_streamed takes host arrays")
        ptrs.append(p)
    fs = None
    if field_step is not None:
        fs = np.ascontiguousarray(np.asarray(field_step, dtype=np.int32).reshape(-1))
    n = ctypes.c_int64(0)
    _check(load_library().msf_segment_streamed(
        ctx, nx, ny, nz, T, ptrs[0], P, A, int(Tp), ptrs[1], ptrs[2],
        fs.ctypes.data if fs is not None else None, ctypes.byref(crit), int(slab_steps), ptrs[3],
        ctypes.byref(n)), "msf_segment_streamed")
    return int(n.value)


def msf_bin_particles(ctx, flags: int = 0) -> msf_bin_stats:
    st = msf_bin_stats()
    _check(load_library().msf_bin_particles(ctx, int(flags), ctypes.byref(st)),
           "msf_bin_particles")
    return st


def msf_get_bins(ctx, key=None, count=None, mean=None, sumq=None):
    kinds = {_ptr_kind(x)[1] for x in (key, count, mean, sumq) if x is not None}
    if len(kinds) > 1:
        raise ValueError("all outputs must be host or all device")
    kind = kinds.pop() if kinds else MSF_HOST
    _check(load_library().msf_get_bins(ctx, _ptr_kind(key)[0], _ptr_kind(count)[0],
                                       _ptr_kind(mean)[0], _ptr_kind(sumq)[0], kind),
           "msf_get_bins")


def msf_segment(ctx, crit: msf_criteria, labels) -> int:
    lp, lk = _ptr_kind(labels)
    n = ctypes.c_int64(0)
    _check(load_library().msf_segment(ctx, ctypes.byref(crit), lp, lk, ctypes.byref(n)),
           "msf_segment")
    return int(n.value)


def msf_extract_features(ctx, crit: msf_criteria, labels, cap=None):
    """Returns a numpy structured array (dtype FEATURE_DTYPE) of the features."""
    lib = load_library()
    lp, lk = _ptr_kind(labels)
    n = ctypes.c_int64(0)
    if cap is None:
        st = lib.msf_extract_features(ctx, ctypes.byref(crit), lp, lk, None, MSF_HOST, 0,
                                      ctypes.byref(n))
        if st not in (MSF_OK, MSF_ERR_CAPACITY):
            _check(st, "msf_extract_features")
        cap = int(n.value)
    out = np.zeros(max(cap, 1), FEATURE_DTYPE)
    _check(lib.msf_extract_features(ctx, ctypes.byref(crit), lp, lk, out.ctypes.data, MSF_HOST,
                                    cap, ctypes.byref(n)), "msf_extract_features")
    return out[:int(n.value)]


def msf_segment_features(ctx, crit: msf_criteria, labels, cap):
    """msf_segment into `labels` (host or device tensor) and the features of that labelling in
    one call (the host labels' copy overlaps the feature passes). Returns (number of features,
    numpy structured array of the features, dtype FEATURE_DTYPE)."""
    lib = load_library()
    lp, lk = _ptr_kind(labels)
    nf = ctypes.c_int64(0)
    n = ctypes.c_int64(0)
    out = np.zeros(max(int(cap), 1), FEATURE_DTYPE)
    _check(lib.msf_segment_features(ctx, ctypes.byref(crit), lp, lk, ctypes.byref(nf),
                                    out.ctypes.data, MSF_HOST, int(cap), ctypes.byref(n)),
           "msf_segment_features")
    return int(nf.value), out[:int(n.value)]


def msf_segment_field_noalloc(field, labels, pred=None, edges=MSF_EDGE_SPATIAL | MSF_EDGE_TEMPORAL,
                              stream=None) -> int:
    """Field-only labelling without any allocation (see include/msf.h). field and labels are
    device tensors [tw][nz][ny][nx]; pred is (src, attr, op, lo, hi) on the field or None."""
    tw, nz, ny, nx = field.shape
    fp, fk = _ptr_kind(field)
    lp, lk = _ptr_kind(labels)
    if (fp and fk != MSF_DEVICE) or (lp and lk != MSF_DEVICE):
        raise ValueError("field and labels must be device memory")
    pp = None
    if pred is not None:
        src, a, op, lo, hi = pred
        pp = ctypes.byref(msf_pred(int(src), int(a), int(op), float(lo), float(hi)))
    s = stream if stream is None or isinstance(stream, int) else stream.cuda_stream
    n = ctypes.c_int64(0)
    _check(load_library().msf_segment_field_noalloc(nx, ny, nz, tw, fp, pp, int(edges), lp,
                                                    ctypes.byref(n), s),
           "msf_segment_field_noalloc")
    return int(n.value)


def msf_segment_batch(ctx, crits, labels):
    """crits: list of msf_criteria; labels: list of device int32 tensors (or None for empty
    windows). Returns the list of feature counts."""
    nq = len(crits)
    carr = (msf_criteria * max(nq, 1))(*crits)
    larr = (ctypes.c_void_p * max(nq, 1))(*[_ptr_kind(l)[0] if l is not None else None
                                            for l in labels])
    nf = (ctypes.c_int64 * max(nq, 1))()
    _check(load_library().msf_segment_batch(ctx, nq, carr, larr, nf), "msf_segment_batch")
    return [int(nf[i]) for i in range(nq)]


def msf_set_tile(ctx, by, bz, bt):
    _check(load_library().msf_set_tile(ctx, by, bz, bt), "msf_set_tile")


def make_cluster_params(t0, t1, attr, k, w_p=1.0, w_f=1.0, w_d=1.0, c_f=1.0, eps_c=1e-3,
                        max_iter=10) -> msf_cluster_params:
    return msf_cluster_params(int(t0), int(t1), int(attr), (ctypes.c_int32 * 4)(*[int(x) for x in k]),
                              float(w_p), float(w_f), float(w_d), float(c_f), float(eps_c),
                              int(max_iter))


def msf_cluster(ctx, prm: msf_cluster_params, field_labels=None, point_labels=None):
    """Returns (centers [K][6] float32, counts [K][2] int64, iterations); the label buffers (host
    or device, same kind) are filled when given."""
    K = int(np.prod(list(prm.k)))
    centers = np.zeros((K, 6), np.float32)
    counts = np.zeros((K, 2), np.int64)
    fp, fk = _ptr_kind(field_labels)
    pp, pk = _ptr_kind(point_labels)
    if field_labels is not None and point_labels is not None and fk != pk:
        raise ValueError("label buffers must be both host or both device")
    kind = fk if field_labels is not None else pk
    it = ctypes.c_int(0)
    _check(load_library().msf_cluster(ctx, ctypes.byref(prm), fp, pp, kind, centers.ctypes.data,
                                      counts.ctypes.data, ctypes.byref(it)), "msf_cluster")
    return centers, counts, int(it.value)


def msf_set_wait_limit(ctx, cycles: int):
    _check(load_library().msf_set_wait_limit(ctx, int(cycles)), "msf_set_wait_limit")


def msf_set_profiling(ctx, enable: bool):
    _check(load_library().msf_set_profiling(ctx, int(bool(enable))), "msf_set_profiling")


def msf_kernel_times(ctx, reset=False):
    """{kernel name: (total ms, launches)} accumulated while profiling was enabled."""
    cap = 64
    names = (ctypes.c_char * 48 * cap)()
    ms = (ctypes.c_double * cap)()
    nl = (ctypes.c_int64 * cap)()
    n = _check(load_library().msf_kernel_times(ctx, names, ms, nl, cap, int(bool(reset))),
               "msf_kernel_times")
    return {bytes(names[i]).split(b"\0")[0].decode(): (ms[i], nl[i]) for i in range(min(n, cap))}


def msf_server_create(ctx, pool_bytes=0, max_batch=0, slots=0):
    h = ctypes.c_void_p()
    cfg = msf_server_config(int(pool_bytes), int(max_batch), int(slots))
    _check(load_library().msf_server_create(ctx, ctypes.byref(cfg), ctypes.byref(h)),
           "msf_server_create")
    return h


def msf_server_submit(srv, crit: msf_criteria, tag: int):
    _check(load_library().msf_server_submit(srv, ctypes.byref(crit), int(tag)),
           "msf_server_submit")


def msf_server_poll(srv, cap=256, timeout_ms=0):
    """List of msf_server_result (up to cap), waiting up to timeout_ms for the first."""
    out = (msf_server_result * max(cap, 1))()
    n = ctypes.c_int(0)
    _check(load_library().msf_server_poll(srv, out, int(cap), ctypes.byref(n), int(timeout_ms)),
           "msf_server_poll")
    return [out[i] for i in range(n.value)]


def msf_server_release(srv, tag: int):
    _check(load_library().msf_server_release(srv, int(tag)), "msf_server_release")


def msf_server_get_stats(srv) -> msf_server_stats:
    st = msf_server_stats()
    _check(load_library().msf_server_get_stats(srv, ctypes.byref(st)), "msf_server_get_stats")
    return st


def msf_server_destroy(srv):
    _check(load_library().msf_server_destroy(srv), "msf_server_destroy")


class _DeviceInt32:
    """Zero-copy view of server-owned device labels (CUDA array interface)."""

    def __init__(self, ptr, shape):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<i4",
                                         "data": (int(ptr), False), "version": 3,
                                         "strides": None}


# ---------------------------------------------------------------------------------------------
# convenience wrappers
# ---------------------------------------------------------------------------------------------

def msf_set_schedule(ctx, sched: int):
    _check(load_library().msf_set_schedule(ctx, int(sched)), "msf_set_schedule")


def msf_autotune(ctx, crit: msf_criteria, reps: int = 3) -> dict:
    """Tune msf_segment's tile shape and schedule for crit's problem shape; returns the result
    as a dict (by, bz, bt, sched, ms, ms_default, n_tried)."""
    r = msf_tune_result()
    _check(load_library().msf_autotune(ctx, ctypes.byref(crit), int(reps), ctypes.byref(r)),
           "msf_autotune")
    return {f: getattr(r, f) for f, _ in msf_tune_result._fields_}


def msf_autotune_batch(ctx, crits, labels, reps: int = 3) -> dict:
    """Tune the batched form's tile shape on this batch (labels as for msf_segment_batch)."""
    n = len(crits)
    arr = (msf_criteria * n)(*crits)
    ptrs = (ctypes.c_void_p * n)(*[_ptr_kind(l)[0] if l is not None else None for l in labels])
    r = msf_tune_result()
    _check(load_library().msf_autotune_batch(ctx, n, arr, ptrs, int(reps), ctypes.byref(r)),
           "msf_autotune_batch")
    return {f: getattr(r, f) for f, _ in msf_tune_result._fields_}


def msf_get_tuning(ctx, crit: msf_criteria):
    """(by, bz, bt, sched) msf_segment would use for crit now."""
    cfg = (ctypes.c_int32 * 4)()
    _check(load_library().msf_get_tuning(ctx, ctypes.byref(crit), cfg), "msf_get_tuning")
    return tuple(cfg)


def msf_tune_clear(ctx):
    _check(load_library().msf_tune_clear(ctx), "msf_tune_clear")


# numpy views of the record types (field order and offsets as in the C structs)
CLUSTER_STAT_DTYPE = np.dtype({
    "names": [f for f, _ in msf_cluster_stat._fields_],
    "formats": ["<i8", "<i8", ("<f4", 4), ("<f4", 4), "<f8", "<f8", "<f8", "<f8"],
    "offsets": [getattr(msf_cluster_stat, f).offset for f, _ in msf_cluster_stat._fields_],
    "itemsize": ctypes.sizeof(msf_cluster_stat)})


def msf_merge_clusters(ctx, centers, eps_m, terms=MSF_MERGE_POINT | MSF_MERGE_FIELD, out=None):
    """§3.3 merging. centers [K][6] fp32 (host or device). Returns (map, n_groups); the map is
    written to `out` when given (host or device int32 [K]), else to a new numpy array."""
    cp, ck = _ptr_kind(centers)
    K = int(centers.shape[0])
    m = np.empty(K, np.int32) if out is None else out
    mp, mk = _ptr_kind(m)
    g = ctypes.c_int32(0)
    _check(load_library().msf_merge_clusters(ctx, cp, ck, K, float(eps_m), int(terms), mp, mk,
                                             ctypes.byref(g)), "msf_merge_clusters")
    return m, int(g.value)


def msf_relabel(ctx, labels, mapping):
    """labels[i] = map[labels[i]] in place (host or device buffers)."""
    lp, lk = _ptr_kind(labels)
    mp, mk = _ptr_kind(mapping)
    n = int(np.prod(labels.shape))
    _check(load_library().msf_relabel(ctx, lp, lk, n, mp, mk, int(mapping.shape[0])),
           "msf_relabel")


def msf_cluster_stats(ctx, t0, t1, attr, field_labels, point_labels, K):
    """§3.4 per-cluster summaries; returns a numpy record array [K] (CLUSTER_STAT_DTYPE)."""
    fp, fk = _ptr_kind(field_labels)
    pp, pk = _ptr_kind(point_labels)
    if field_labels is not None and point_labels is not None and fk != pk:
        raise ValueError("label buffers must be both host or both device")
    kind = fk if field_labels is not None else pk
    out = np.zeros(int(K), CLUSTER_STAT_DTYPE)
    _check(load_library().msf_cluster_stats(ctx, int(t0), int(t1), int(attr), fp, pp, kind,
                                            int(K), out.ctypes.data, MSF_HOST),
           "msf_cluster_stats")
    return out


def msf_select_clusters(ctx, centers, lo, hi):
    """§3.4 range query over centre properties: ascending int32 indices (numpy)."""
    cp, ck = _ptr_kind(centers)
    K = int(centers.shape[0])
    lo = np.ascontiguousarray(lo, np.float32)
    hi = np.ascontiguousarray(hi, np.float32)
    n = ctypes.c_int32(0)
    lib = load_library()
    st = lib.msf_select_clusters(ctx, cp, ck, K, lo.ctypes.data, hi.ctypes.data, None, MSF_HOST,
                                 0, ctypes.byref(n))
    if st not in (MSF_OK, MSF_ERR_CAPACITY):
        _check(st, "msf_select_clusters")
    out = np.empty(max(n.value, 1), np.int32)
    _check(lib.msf_select_clusters(ctx, cp, ck, K, lo.ctypes.data, hi.ctypes.data,
                                   out.ctypes.data, MSF_HOST, out.size, ctypes.byref(n)),
           "msf_select_clusters")
    return out[:n.value].copy()


def msf_split_trajectories(ctx, t0, t1, labels, space, min_len=2, out=None):
    """§3.4 trajectory pieces. Returns an int32 array [n][4] (point, t_start, length, label);
    `out` (host or device int32 [cap][4]) is filled instead when given and large enough, and
    (out, n) is returned."""
    lp, lk = _ptr_kind(labels)
    n = ctypes.c_int64(0)
    lib = load_library()
    if out is not None:
        op, ok = _ptr_kind(out)
        _check(lib.msf_split_trajectories(ctx, int(t0), int(t1), lp, lk, int(space),
                                          int(min_len), op, ok, int(out.shape[0]),
                                          ctypes.byref(n)), "msf_split_trajectories")
        return out, int(n.value)
    st = lib.msf_split_trajectories(ctx, int(t0), int(t1), lp, lk, int(space), int(min_len),
                                    None, MSF_HOST, 0, ctypes.byref(n))
    if st not in (MSF_OK, MSF_ERR_CAPACITY):
        _check(st, "msf_split_trajectories")
    res = np.empty((max(n.value, 1), 4), np.int32)
    _check(lib.msf_split_trajectories(ctx, int(t0), int(t1), lp, lk, int(space), int(min_len),
                                      res.ctypes.data, MSF_HOST, res.shape[0], ctypes.byref(n)),
           "msf_split_trajectories")
    return res[:n.value].copy()


class Context:
    """Owns one msf_ctx on a device; all calls run on the given (or torch's current) stream."""

    def __init__(self, device: int = 0, stream=None):
        if stream is None:
            import torch
            stream = torch.cuda.current_stream(device)
        self.device = device
        self.h = msf_create(device, stream)
        self.shape = None

    def close(self):
        if self.h:
            msf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_stream(self, stream):
        msf_set_stream(self.h, stream)

    def load(self, field, pos, attr, field_step=None):
        """field_step: the field step of each point step when the points have their own time
        grid (pos [Tp][3][P]); None for one point step per field step."""
        if field_step is None:
            msf_load_timesteps(self.h, field, pos, attr)
        else:
            msf_load_timesteps_mr(self.h, field, pos, attr, field_step)
        self.shape = tuple(field.shape)
        self.P = pos.shape[2] if pos is not None else 0
        self.A = attr.shape[1] if attr is not None else 0
        self.Tp = pos.shape[0] if pos is not None else self.shape[0]
        T = self.shape[0]
        fs = (np.arange(self.Tp) if field_step is None
              else np.asarray(field_step, dtype=np.int64).reshape(-1))
        # first point step of each field step, [T + 1]
        self.pj0 = np.searchsorted(fs, np.arange(T + 1), side="left").astype(np.int64)

    def bin(self, keep_sumq=False):
        return msf_bin_particles(self.h, MSF_BIN_KEEP_SUMQ if keep_sumq else 0)

    def bins(self, device="cpu", sumq=False):
        import torch
        T, nz, ny, nx = self.shape
        key = torch.empty((getattr(self, "Tp", T), self.P), dtype=torch.int32, device=device)
        count = torch.empty((T, nz, ny, nx), dtype=torch.int32, device=device)
        mean = torch.empty((self.A, T, nz, ny, nx), dtype=torch.float32, device=device)
        sq = torch.empty((self.A, T, nz, ny, nx), dtype=torch.int64, device=device) \
            if sumq else None
        msf_get_bins(self.h, key, count, mean if self.A else None, sq if self.A else None)
        return key, count, mean, sq

    def segment(self, t0, t1, preds=(), edges=MSF_EDGE_ALL, labels=None):
        import torch
        if self.shape is None:            # let the library report the missing dataset
            return None, msf_segment(self.h, make_criteria(t0, t1, preds, edges), labels)
        T, nz, ny, nx = self.shape
        if labels is None:
            labels = torch.empty((t1 - t0, nz, ny, nx), dtype=torch.int32,
                                 device=f"cuda:{self.device}")
        n = msf_segment(self.h, make_criteria(t0, t1, preds, edges), labels)
        return labels, n

    def features(self, t0, t1, labels, preds=(), edges=MSF_EDGE_ALL):
        return msf_extract_features(self.h, make_criteria(t0, t1, preds, edges), labels)

    def segment_batch(self, queries, labels=None):
        """queries: list of (t0, t1, preds, edges). Allocates device label tensors unless given."""
        import torch
        T, nz, ny, nx = self.shape
        crits = [make_criteria(t0, t1, p, e) for (t0, t1, p, e) in queries]
        if labels is None:
            labels = [torch.empty((t1 - t0, nz, ny, nx), dtype=torch.int32,
                                  device=f"cuda:{self.device}") for (t0, t1, _, _) in queries]
        return labels, msf_segment_batch(self.h, crits, labels)

    def set_tile(self, by, bz, bt):
        msf_set_tile(self.h, by, bz, bt)

    def cluster(self, t0, t1, attr, k, w_p=1.0, w_f=1.0, w_d=1.0, c_f=1.0, eps_c=1e-3,
                max_iter=10):
        """§3.2 clustering of the window; returns (field labels [t1-t0][nz][ny][nx], point labels
        [nj][P] over the window's point steps) device tensors, centers [K][6], counts [K][2] and
        the number of centre updates."""
        import torch
        T, nz, ny, nx = self.shape
        dev = f"cuda:{self.device}"
        fl = torch.empty((t1 - t0, nz, ny, nx), dtype=torch.int32, device=dev)
        nj = int(self.pj0[t1] - self.pj0[t0])  # the point steps that fall in the window
        pl = torch.empty((nj, max(self.P, 1)), dtype=torch.int32, device=dev)[:, :self.P]
        prm = make_cluster_params(t0, t1, attr, k, w_p, w_f, w_d, c_f, eps_c, max_iter)
        centers, counts, it = msf_cluster(self.h, prm, fl, pl.contiguous() if self.P else None)
        return fl, pl, centers, counts, it

    def set_batch_tile(self, by, bz, bt):
        _check(load_library().msf_set_batch_tile(self.h, int(by), int(bz), int(bt)),
               "msf_set_batch_tile")

    def set_batch_schedule(self, sched):
        _check(load_library().msf_set_batch_schedule(self.h, int(sched)),
               "msf_set_batch_schedule")

    def autotune_batch(self, queries, labels=None, reps=3):
        import torch
        T, nz, ny, nx = self.shape
        crits = [make_criteria(t0, t1, p, e) for (t0, t1, p, e) in queries]
        if labels is None:
            labels = [torch.empty((t1 - t0, nz, ny, nx), dtype=torch.int32,
                                  device=f"cuda:{self.device}") for (t0, t1, _, _) in queries]
        return msf_autotune_batch(self.h, crits, labels, reps)

    def set_batch_graphs(self, enable=True):
        _check(load_library().msf_set_batch_graphs(self.h, int(bool(enable))),
               "msf_set_batch_graphs")

    def batch_graph_replays(self):
        n = ctypes.c_int64(0)
        _check(load_library().msf_batch_graph_replays(self.h, ctypes.byref(n)),
               "msf_batch_graph_replays")
        return int(n.value)

    def set_schedule(self, sched):
        msf_set_schedule(self.h, sched)

    def autotune(self, t0, t1, preds=(), edges=MSF_EDGE_ALL, reps=3):
        return msf_autotune(self.h, make_criteria(t0, t1, preds, edges), reps)

    def tuning(self, t0, t1, preds=(), edges=MSF_EDGE_ALL):
        return msf_get_tuning(self.h, make_criteria(t0, t1, preds, edges))

    def tune_clear(self):
        msf_tune_clear(self.h)

    def merge_clusters(self, centers, eps_m, terms=MSF_MERGE_POINT | MSF_MERGE_FIELD, out=None):
        return msf_merge_clusters(self.h, centers, eps_m, terms, out)

    def relabel(self, labels, mapping):
        msf_relabel(self.h, labels, mapping)

    def cluster_stats(self, t0, t1, attr, field_labels, point_labels, K):
        return msf_cluster_stats(self.h, t0, t1, attr, field_labels, point_labels, K)

    def select_clusters(self, centers, lo, hi):
        return msf_select_clusters(self.h, centers, lo, hi)

    def split_trajectories(self, t0, t1, labels, space, min_len=2, out=None):
        return msf_split_trajectories(self.h, t0, t1, labels, space, min_len, out)

    def set_wait_limit(self, cycles):
        msf_set_wait_limit(self.h, cycles)

    def profiling(self, on=True):
        msf_set_profiling(self.h, on)

    def kernel_times(self, reset=False):
        return msf_kernel_times(self.h, reset)


class Server:
    """A query server over a Context's resident dataset (see include/msf.h, msf_server_*)."""

    def __init__(self, ctx: Context, pool_bytes=0, max_batch=0, slots=0):
        self.ctx = ctx
        self.h = msf_server_create(ctx.h, pool_bytes, max_batch, slots)

    def close(self):
        if self.h:
            msf_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def submit(self, tag, t0, t1, preds=(), edges=MSF_EDGE_ALL):
        msf_server_submit(self.h, make_criteria(t0, t1, preds, edges), tag)

    def poll(self, cap=256, timeout_ms=0):
        return msf_server_poll(self.h, cap, timeout_ms)

    def labels(self, res):
        """torch view (no copy) of a result's labels; valid until release(res.tag). Work that
        reads it on a stream must finish before the release (the pool memory is reused)."""
        import torch
        if not res.labels:
            return None
        T, nz, ny, nx = self.ctx.shape
        tw = res.n_labels // (nz * ny * nx)
        return torch.as_tensor(_DeviceInt32(res.labels, (tw, nz, ny, nx)),
                               device=f"cuda:{self.ctx.device}")

    def release(self, tag):
        msf_server_release(self.h, tag)

    def take_labels(self, res):
        """Copy of a result's labels (None if it has none), then release them to the pool."""
        import torch
        v = self.labels(res)
        if v is None:
            return None
        out = v.clone()
        torch.cuda.current_stream(self.ctx.device).synchronize()
        self.release(res.tag)
        return out

    def stats(self):
        return msf_server_get_stats(self.h)
