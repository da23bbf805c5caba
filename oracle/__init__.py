"""Plain CPU oracle for multifaceted 4D segmentation (Sauer & Ma, arXiv 1903.12294).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()`` and by the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``. The GPU library never imports,
links or runs anything from here, and nothing here uses the GPU library.

The arithmetic lives in ``msf_oracle.c`` (plain C, fp64), built with gcc into
``liborc.so`` beside it; this module only marshals numpy arrays through ctypes.

Functions and the passages they follow:
  ``bin``       - §3.1 preprocessing index (point samples -> field voxels, per-voxel aggregates;
                  point steps may fall several to a field step, §3.4 and §4.1)
  ``segment``   - combined field+point membership (§3.2, choice of variables) and 4D connected
                  components by breadth-first flood fill (connectivity is this library's
                  definition; the paper's clustering imposes none, §3.3)
  ``features``  - per-feature averages (§3.2.2 cluster centre), extent and deviations (§3.4)
  ``slic``      - the paper's multifaceted 4D clustering (§3.2; ``msf_slic.c``)
  ``merge_clusters``, ``select_clusters``, ``cluster_stats``, ``split_trajectories`` - cluster
                  merging (§3.3), range queries, summaries and trajectory pieces (§3.4;
                  ``msf_post.c``)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "msf_oracle.c")
_SRC_SLIC = os.path.join(_HERE, "msf_slic.c")
_SRC_POST = os.path.join(_HERE, "msf_post.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

SRC_FIELD, SRC_COUNT, SRC_MEAN = 0, 1, 2
OP_GT, OP_GE, OP_LT, OP_LE, OP_BAND = 0, 1, 2, 3, 4
EDGE_SPATIAL, EDGE_TEMPORAL, EDGE_TRAJ = 1, 2, 4
EDGE_ALL = EDGE_SPATIAL | EDGE_TEMPORAL | EDGE_TRAJ


def build(force: bool = False) -> str:
    """Compile the oracle sources with gcc (portable flags only: the same source builds on x86
    and Arm; no floating-point contraction, so fp32 expressions round step by step)."""
    srcs = [_SRC, _SRC_SLIC, _SRC_POST]
    newest = max(os.path.getmtime(s) for s in srcs)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(
            ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, *srcs,
             "-lm"],
            check=True,
        )
        os.replace(tmp, _LIB)
    return _LIB


class _Pred(ctypes.Structure):
    _fields_ = [("src", ctypes.c_int32), ("attr", ctypes.c_int32), ("op", ctypes.c_int32),
                ("lo", ctypes.c_float), ("hi", ctypes.c_float)]


class _Criteria(ctypes.Structure):
    _fields_ = [("t0", ctypes.c_int32), ("t1", ctypes.c_int32), ("n_pred", ctypes.c_int32),
                ("pred", _Pred * 4), ("edges", ctypes.c_uint32)]


class _SlicParams(ctypes.Structure):
    _fields_ = [("t0", ctypes.c_int), ("t1", ctypes.c_int), ("attr", ctypes.c_int),
                ("k", ctypes.c_int * 4), ("w_p", ctypes.c_float), ("w_f", ctypes.c_float),
                ("w_d", ctypes.c_float), ("c_f", ctypes.c_float), ("eps_c", ctypes.c_float),
                ("max_iter", ctypes.c_int)]


class _FeatOut(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in (
        "label", "n_vox", "n_pts", "bbox", "sum_field", "mean_field", "std_field", "min_field",
        "max_field", "centroid", "sumq", "mean_attr", "std_attr")]


class _StatsOut(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in (
        "n_field", "n_point", "lo", "hi", "mean_field", "std_field", "mean_point", "std_point")]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64 = ctypes.c_int64
            lib.oracle_bin.argtypes = [ctypes.c_int] * 4 + [i64, ctypes.c_int] + [P] * 8
            lib.oracle_bin.restype = ctypes.c_int
            lib.oracle_bin_mr.argtypes = ([ctypes.c_int] * 5 + [P, i64, ctypes.c_int] + [P] * 8)
            lib.oracle_bin_mr.restype = ctypes.c_int
            lib.oracle_segment_mr.argtypes = ([ctypes.c_int] * 4 + [P, P, P, i64, ctypes.c_int, P, P,
                                              ctypes.POINTER(_Criteria), P, P])
            lib.oracle_segment_mr.restype = ctypes.c_int
            lib.oracle_features_mr.argtypes = ([ctypes.c_int] * 4 + [P, P, i64, ctypes.c_int,
                                               ctypes.c_int, P, P, P, P, ctypes.c_int,
                                               ctypes.c_int, P, i64, ctypes.POINTER(_FeatOut), P])
            lib.oracle_features_mr.restype = ctypes.c_int
            lib.oracle_segment.argtypes = [ctypes.c_int] * 4 + [P, P, P, i64, P,
                                                                ctypes.POINTER(_Criteria), P, P]
            lib.oracle_segment.restype = ctypes.c_int
            lib.oracle_features.argtypes = ([ctypes.c_int] * 4 + [P, P, i64, ctypes.c_int, P, P,
                                            P, ctypes.c_int, ctypes.c_int, P, i64,
                                            ctypes.POINTER(_FeatOut), P])
            lib.oracle_features.restype = ctypes.c_int
            lib.oracle_slic.argtypes = ([ctypes.c_int] * 4 + [P, i64, ctypes.c_int, P, P, P,
                                        ctypes.POINTER(_SlicParams), P, P, P, P,
                                        ctypes.POINTER(ctypes.c_int)])
            lib.oracle_slic.restype = ctypes.c_int
            lib.oracle_slic_mr.argtypes = ([ctypes.c_int] * 4 + [P, i64, ctypes.c_int,
                                           ctypes.c_int, P, P, P, P,
                                           ctypes.POINTER(_SlicParams), P, P, P, P,
                                           ctypes.POINTER(ctypes.c_int)])
            lib.oracle_slic_mr.restype = ctypes.c_int
            lib.oracle_merge_clusters.argtypes = [ctypes.c_int, P, ctypes.c_float, ctypes.c_int, P]
            lib.oracle_merge_clusters.restype = ctypes.c_int
            lib.oracle_select_clusters.argtypes = [ctypes.c_int, P, P, P, P]
            lib.oracle_select_clusters.restype = ctypes.c_int
            lib.oracle_cluster_stats.argtypes = ([ctypes.c_int] * 4 + [P, i64, ctypes.c_int, P, P,
                                                 P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P,
                                                 P, ctypes.c_int, ctypes.POINTER(_StatsOut)])
            lib.oracle_cluster_stats.restype = ctypes.c_int
            lib.oracle_point_labels.argtypes = [i64, i64, ctypes.c_int, ctypes.c_int, P, P, P]
            lib.oracle_point_labels.restype = None
            lib.oracle_split_trajectories.argtypes = [i64, ctypes.c_int, P, ctypes.c_int, P, i64]
            lib.oracle_split_trajectories.restype = i64
            lib.oracle_scale_exponent.argtypes = [ctypes.c_double, i64]
            lib.oracle_scale_exponent.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None and a.size else ctypes.c_void_p(0)


def scale_exponent(max_abs: float, n_samples: int) -> int:
    """k = 62 - e - b of the fixed-point attribute sums (see ``msf_oracle.c``)."""
    return int(_load().oracle_scale_exponent(float(max_abs), int(n_samples)))


def _fstep_array(fstep, Tp):
    if fstep is None:
        return None
    f = np.ascontiguousarray(fstep, dtype=np.int32).reshape(-1)
    if f.size != Tp:
        raise ValueError("fstep must have one entry per point step")
    return f


def bin(field_shape, pos, attr, keep_sumq=True, fstep=None):
    """§3.1 preprocessing index. ``field_shape`` = (T, NZ, NY, NX); ``pos`` [Tp][3][P] fp32;
    ``attr`` [Tp][A][P] fp32; ``fstep`` [Tp] the field step of every point step
    (non-decreasing; None: Tp == T, one point step per field step). Returns dict key [Tp][P],
    count, sumq, mean ([A][T][...]), kscale, outside [Tp]."""
    T, nz, ny, nx = (int(s) for s in field_shape)
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    P = pos.shape[2]
    Tp = pos.shape[0]
    attr = np.ascontiguousarray(attr, dtype=np.float32)
    if attr.ndim != 3 or attr.shape[0] != Tp or attr.shape[2] != P:
        raise ValueError("attr must be [Tp][A][P]")
    fs = _fstep_array(fstep, Tp)
    if fs is None and Tp != T:
        raise ValueError("pos must be [T][3][P] without a step map")
    A = attr.shape[1]
    key = np.empty((Tp, P), np.int32)
    count = np.empty((T, nz, ny, nx), np.int32)
    sumq = np.empty((A, T, nz, ny, nx), np.int64) if keep_sumq else None
    mean = np.empty((A, T, nz, ny, nx), np.float32)
    kscale = np.zeros(max(A, 1), np.int32)
    outside = np.empty(Tp, np.int64)
    rc = _load().oracle_bin_mr(nx, ny, nz, T, Tp, _ptr(fs), P, A, _ptr(pos), _ptr(attr),
                               _ptr(key), _ptr(count), _ptr(sumq), _ptr(mean), _ptr(kscale),
                               _ptr(outside))
    if rc != 0:
        raise RuntimeError(f"oracle_bin failed: {rc}")
    return dict(key=key, count=count, sumq=sumq, mean=mean, kscale=kscale[:A], outside=outside)


def make_criteria(t0, t1, preds=(), edges=EDGE_ALL):
    """preds: sequence of (src, attr, op, lo, hi)."""
    c = _Criteria()
    c.t0, c.t1, c.n_pred, c.edges = int(t0), int(t1), len(preds), int(edges)
    if len(preds) > 4:
        raise ValueError("at most 4 predicates")
    for i, (src, a, op, lo, hi) in enumerate(preds):
        c.pred[i] = _Pred(int(src), int(a), int(op), float(lo), float(hi))
    return c


def segment(field, count, mean, key, t0, t1, preds=(), edges=EDGE_ALL, fstep=None):
    """Criterion + 4D connected components. key [Tp][P]; fstep [Tp] maps point steps to field
    steps (None: one per field step). Returns (labels [Tw][NZ][NY][NX] int32, n_features)."""
    field = np.ascontiguousarray(field, dtype=np.float32)
    T, nz, ny, nx = field.shape
    count = np.ascontiguousarray(count, dtype=np.int32)
    mean = np.ascontiguousarray(mean, dtype=np.float32)
    key = np.ascontiguousarray(key, dtype=np.int32)
    P = key.shape[1] if key.ndim == 2 else 0
    Tp = key.shape[0] if key.ndim == 2 else T
    fs = _fstep_array(fstep, Tp) if P else None
    crit = make_criteria(t0, t1, preds, edges)
    labels = np.empty((max(t1 - t0, 0), nz, ny, nx), np.int32)
    nf = ctypes.c_int64(0)
    rc = _load().oracle_segment_mr(nx, ny, nz, T, _ptr(field), _ptr(count), _ptr(mean), P,
                                   Tp if fs is not None else T, _ptr(fs), _ptr(key),
                                   ctypes.byref(crit), _ptr(labels), ctypes.byref(nf))
    if rc != 0:
        raise RuntimeError(f"oracle_segment failed: {rc}")
    return labels, int(nf.value)


def features(field, count, attr, key, kscale, t0, t1, labels, fstep=None):
    """Per-feature statistics, ascending label order. attr [Tp][A][P], key [Tp][P], fstep as
    in ``segment``. Returns a dict of numpy arrays."""
    field = np.ascontiguousarray(field, dtype=np.float32)
    T, nz, ny, nx = field.shape
    count = np.ascontiguousarray(count, dtype=np.int32)
    key = np.ascontiguousarray(key, dtype=np.int32)
    P = key.shape[1] if key.ndim == 2 else 0
    Tp = key.shape[0] if key.ndim == 2 else T
    fs = _fstep_array(fstep, Tp) if P else None
    attr = np.ascontiguousarray(attr, dtype=np.float32)
    A = attr.shape[1] if attr.ndim == 3 else 0
    kscale = np.ascontiguousarray(np.asarray(kscale, dtype=np.int32).reshape(-1))
    if kscale.size == 0:
        kscale = np.zeros(1, np.int32)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    nf = int(np.count_nonzero(labels.reshape(-1) == np.arange(labels.size, dtype=np.int64)))
    Af = max(A, 1)
    out = dict(
        label=np.empty(nf, np.int32), n_vox=np.empty(nf, np.int64), n_pts=np.empty(nf, np.int64),
        bbox=np.empty((nf, 8), np.int32), sum_field=np.empty(nf, np.float64),
        mean_field=np.empty(nf, np.float64), std_field=np.empty(nf, np.float64),
        min_field=np.empty(nf, np.float32), max_field=np.empty(nf, np.float32),
        centroid=np.empty((nf, 4), np.float64), sumq=np.empty((nf, Af), np.int64),
        mean_attr=np.empty((nf, Af), np.float64), std_attr=np.empty((nf, Af), np.float64))
    fo = _FeatOut(*[_ptr(out[n]) for n, _ in _FeatOut._fields_])
    n_out = ctypes.c_int64(0)
    rc = _load().oracle_features_mr(nx, ny, nz, T, _ptr(field), _ptr(count), P, A,
                                    Tp if fs is not None else T, _ptr(fs), _ptr(attr),
                                    _ptr(key), _ptr(kscale), int(t0), int(t1), _ptr(labels), nf,
                                    ctypes.byref(fo), ctypes.byref(n_out))
    if rc != 0:
        raise RuntimeError(f"oracle_features failed: {rc}")
    for n in ("sumq", "mean_attr", "std_attr"):
        out[n] = out[n][:, :A]
    return out


def run_all(field, pos, attr, t0, t1, preds, edges=EDGE_ALL, fstep=None):
    """bin -> segment -> features in one call (the whole path, CPU)."""
    b = bin(field.shape, pos, attr, keep_sumq=False, fstep=fstep)
    labels, nf = segment(field, b["count"], b["mean"], b["key"], t0, t1, preds, edges, fstep)
    f = features(field, b["count"], attr, b["key"], b["kscale"], t0, t1, labels, fstep)
    return b, labels, nf, f


def slic(field, pos, attr, key, t0, t1, attr_index, k, w_p=1.0, w_f=1.0, w_d=1.0, c_f=1.0,
         eps_c=1e-3, max_iter=10, fstep=None):
    """§3.2 multifaceted 4D clustering (msf_slic.c). k = (kx, ky, kz, kt) seeds per dimension.
    pos/attr/key are per point step ([Tp][...]); fstep [Tp] maps point steps to field steps
    (None: one per field step). Returns (field_label [Tw][NZ][NY][NX] int32, point_label
    [window point steps][P] int32, centers [K][6] fp32 (x, y, z, t, p_c, f_c), counts [K][2]
    int64 (field, point samples), updates made)."""
    field = np.ascontiguousarray(field, dtype=np.float32)
    T, nz, ny, nx = field.shape
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    attr = np.ascontiguousarray(attr, dtype=np.float32)
    key = np.ascontiguousarray(key, dtype=np.int32)
    P = pos.shape[2] if pos.ndim == 3 else 0
    Tp = pos.shape[0] if pos.ndim == 3 else T
    A = attr.shape[1] if attr.ndim == 3 else 0
    fs = _fstep_array(fstep, Tp) if fstep is not None else None
    prm = _SlicParams(int(t0), int(t1), int(attr_index), (ctypes.c_int * 4)(*[int(x) for x in k]),
                      float(w_p), float(w_f), float(w_d), float(c_f), float(eps_c), int(max_iter))
    K = int(np.prod(k))
    tw = t1 - t0
    if fs is None:
        nj = tw
    else:
        nj = int(np.count_nonzero((fs >= t0) & (fs < t1)))
    fl = np.empty((tw, nz, ny, nx), np.int32)
    pl = np.empty((nj, P), np.int32)
    centers = np.empty((K, 6), np.float32)
    counts = np.empty((K, 2), np.int64)
    it = ctypes.c_int(0)
    rc = _load().oracle_slic_mr(nx, ny, nz, T, _ptr(field), P, A, Tp if fs is not None else T,
                                _ptr(fs), _ptr(pos), _ptr(attr), _ptr(key), ctypes.byref(prm),
                                _ptr(fl), _ptr(pl), _ptr(centers), _ptr(counts),
                                ctypes.byref(it))
    if rc != 0:
        raise RuntimeError(f"oracle_slic failed: {rc}")
    return fl, pl, centers, counts, int(it.value)


MERGE_POINT, MERGE_FIELD = 1, 2


def merge_clusters(centers, eps_m, terms=MERGE_POINT | MERGE_FIELD):
    """§3.3 cluster merging (msf_post.c). centers [K][6] fp32. Returns (map [K] int32 with the
    smallest centre index of each centre's group, number of groups)."""
    c = np.ascontiguousarray(centers, dtype=np.float32)
    K = c.shape[0]
    m = np.empty(K, np.int32)
    g = _load().oracle_merge_clusters(K, _ptr(c), float(eps_m), int(terms), _ptr(m))
    if g < 0:
        raise RuntimeError("oracle_merge_clusters failed")
    return m, int(g)


def select_clusters(centers, lo, hi):
    """§3.4 range query: ascending indices i with lo[j] <= centers[i][j] <= hi[j] for all j."""
    c = np.ascontiguousarray(centers, dtype=np.float32)
    lo = np.ascontiguousarray(lo, dtype=np.float32)
    hi = np.ascontiguousarray(hi, dtype=np.float32)
    out = np.empty(max(c.shape[0], 1), np.int32)
    n = _load().oracle_select_clusters(c.shape[0], _ptr(c), _ptr(lo), _ptr(hi), _ptr(out))
    return out[:n].copy()


def cluster_stats(field, pos, attr, key, t0, t1, attr_index, field_labels, point_labels, K):
    """§3.4 per-cluster summaries (msf_post.c). Either label array may be None. Returns a dict
    of n_field, n_point [K] int64; lo, hi [K][4] fp32 (x, y, z, t); mean_field, std_field,
    mean_point, std_point [K] fp64."""
    field = np.ascontiguousarray(field, dtype=np.float32)
    T, nz, ny, nx = field.shape
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    attr = np.ascontiguousarray(attr, dtype=np.float32)
    key = np.ascontiguousarray(key, dtype=np.int32)
    P = pos.shape[2] if pos.ndim == 3 else 0
    A = attr.shape[1] if attr.ndim == 3 else 0
    fl = None if field_labels is None else np.ascontiguousarray(field_labels, dtype=np.int32)
    pl = None if point_labels is None else np.ascontiguousarray(point_labels, dtype=np.int32)
    r = dict(n_field=np.empty(K, np.int64), n_point=np.empty(K, np.int64),
             lo=np.empty((K, 4), np.float32), hi=np.empty((K, 4), np.float32),
             mean_field=np.empty(K), std_field=np.empty(K), mean_point=np.empty(K),
             std_point=np.empty(K))
    o = _StatsOut(*[r[n].ctypes.data for n, _ in _StatsOut._fields_])
    rc = _load().oracle_cluster_stats(nx, ny, nz, T, _ptr(field), P, A, _ptr(pos), _ptr(attr),
                                      _ptr(key), int(t0), int(t1), int(attr_index),
                                      ctypes.c_void_p(0) if fl is None else _ptr(fl),
                                      ctypes.c_void_p(0) if pl is None else _ptr(pl), int(K),
                                      ctypes.byref(o))
    if rc != 0:
        raise RuntimeError(f"oracle_cluster_stats failed: {rc}")
    return r


def point_labels(key, t0, voxel_labels):
    """Labels of the window's point samples from voxel labels [Tw][NZ][NY][NX]: the label of the
    voxel binning placed each sample in, -1 outside the grid."""
    key = np.ascontiguousarray(key, dtype=np.int32)
    vl = np.ascontiguousarray(voxel_labels, dtype=np.int32)
    tw = vl.shape[0]
    V = int(np.prod(vl.shape[1:]))
    P = key.shape[1]
    out = np.empty((tw, P), np.int32)
    _load().oracle_point_labels(V, P, int(t0), tw, _ptr(key), _ptr(vl), _ptr(out))
    return out


def split_trajectories(point_labels, min_len=2):
    """§3.4 trajectory pieces (msf_post.c): [n][4] int32 rows (point, t_start, length, label) in
    (point, t_start) order."""
    pl = np.ascontiguousarray(point_labels, dtype=np.int32)
    tw, P = pl.shape
    lib = _load()
    n = lib.oracle_split_trajectories(P, tw, _ptr(pl), int(min_len), ctypes.c_void_p(0), 0)
    out = np.empty((max(n, 1), 4), np.int32)
    lib.oracle_split_trajectories(P, tw, _ptr(pl), int(min_len), _ptr(out), n)
    return out[:n].copy()
