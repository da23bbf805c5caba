"""Sharding one query's window across ranks by time slabs, and merging the slab labellings.

Time is the fourth dimension of the labelling (§3.2, §3.3), so a contiguous range of timesteps
is itself a window: rank r labels the slab [t_a, t_b) of the query window [t0, t1) on its own
GPU (msf_segment with that window). Labels are canonical per slab: the smallest slab-linear
index of the component. Only two kinds of edges cross a cut at t_b, both between the slab's last
plane (t_b - 1) and the next slab's first plane (t_b):

  * temporal edges: the same voxel member at t_b - 1 and at t_b;
  * trajectory links: a point whose voxel at t_b - 1 and at t_b are both members.

One exchange gathers, per cut, the two label planes and the point keys at both steps. Every rank
then runs the same small union-find over the labels those edges join, in global terms
(slab label + (t_a - t0) * V is the window-linear index), taking the minimum as the root, and
relabels its own slab: the result is exactly the canonical labelling of the whole window.

The labelling of each slab runs in the CUDA library; this module holds only the host logic of
the cut (plain numpy), and `merge_slab_collective` moves the boundary data with
torch.distributed (gloo on CPU, NCCL between GPUs).
"""
from __future__ import annotations

import numpy as np

EDGE_TEMPORAL, EDGE_TRAJ = 2, 4


def slab_bounds(t0: int, t1: int, world: int):
    """Contiguous, near-equal slabs [t_a, t_b) of [t0, t1), one per rank (empty ones last)."""
    n = t1 - t0
    out, a = [], t0
    for r in range(world):
        b = a + n // world + (1 if r < n % world else 0)
        out.append((a, b))
        a = b
    return out


def cut_pairs(left_last, right_first, key_left, key_right, edges, off_left, off_right):
    """Global label pairs joined across one cut.

    left_last, right_first: int32 [V] label planes (slab labels, -1 = not a member) at t_b - 1
    and t_b; key_left, key_right: int32 [P] point voxels at those steps (-1 = outside);
    off_left, off_right: the slabs' offsets (t_a - t0) * V. Returns (a, b) int64 arrays."""
    left_last = np.asarray(left_last).reshape(-1)
    right_first = np.asarray(right_first).reshape(-1)
    a, b = [], []
    if edges & EDGE_TEMPORAL:
        m = (left_last >= 0) & (right_first >= 0)
        a.append(left_last[m].astype(np.int64) + off_left)
        b.append(right_first[m].astype(np.int64) + off_right)
    if (edges & EDGE_TRAJ) and key_left is not None and len(key_left):
        kl = np.asarray(key_left).astype(np.int64)
        kr = np.asarray(key_right).astype(np.int64)
        ok = (kl >= 0) & (kr >= 0)
        la = np.full(kl.shape, -1, np.int64)
        lb = np.full(kr.shape, -1, np.int64)
        la[ok] = left_last[kl[ok]]
        lb[ok] = right_first[kr[ok]]
        m = ok & (la >= 0) & (lb >= 0)
        a.append(la[m] + off_left)
        b.append(lb[m] + off_right)
    if not a:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    return np.concatenate(a), np.concatenate(b)


def merge_map(a, b):
    """Union-find over the joined global labels (root = smallest). Returns (labels, roots) sorted
    by label, covering every label that takes part in a join, and the number of joins that
    merged two different sets."""
    pairs = np.unique(np.stack([np.minimum(a, b), np.maximum(a, b)], 1), axis=0) \
        if len(a) else np.zeros((0, 2), np.int64)
    labels = np.unique(pairs.reshape(-1))
    parent = {int(x): int(x) for x in labels}

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    merges = 0
    for x, y in pairs:
        rx, ry = find(int(x)), find(int(y))
        if rx != ry:
            lo, hi = min(rx, ry), max(rx, ry)
            parent[hi] = lo
            merges += 1
    roots = np.array([find(int(x)) for x in labels], np.int64)
    return labels, roots, merges


def relabel(slab_labels, offset, labels, roots):
    """Global canonical labels of one slab: slab label + offset, replaced by its root where the
    label was joined across a cut; -1 stays -1."""
    g = np.asarray(slab_labels).astype(np.int64)
    out = np.where(g >= 0, g + offset, -1)
    if len(labels):
        idx = np.searchsorted(labels, out)
        idx = np.clip(idx, 0, len(labels) - 1)
        hit = (out >= 0) & (labels[idx] == out)
        out = np.where(hit, roots[idx], out)
    return out


def merge_slabs(slabs, t0, V, edges, keys=None):
    """Merge the labellings of consecutive slabs in one process.

    slabs: list of (t_a, t_b, labels [t_b - t_a][...] int32, n_features); keys: int32 [T][P] point
    voxels of the dataset (needed for trajectory edges). Returns (labels of [t0, t_end) as int64,
    number of features)."""
    a_all, b_all = [], []
    for (ta, tb, lab, _), (tc, td, lab2, _) in zip(slabs[:-1], slabs[1:]):
        if tb == ta or td == tc:
            continue
        kl = keys[tb - 1] if keys is not None else None
        kr = keys[tc] if keys is not None else None
        a, b = cut_pairs(lab[-1], lab2[0], kl, kr, edges, (ta - t0) * V, (tc - t0) * V)
        a_all.append(a)
        b_all.append(b)
    a = np.concatenate(a_all) if a_all else np.zeros(0, np.int64)
    b = np.concatenate(b_all) if b_all else np.zeros(0, np.int64)
    labels, roots, merges = merge_map(a, b)
    out = [relabel(lab, (ta - t0) * V, labels, roots) for (ta, tb, lab, _) in slabs if tb > ta]
    n = sum(s[3] for s in slabs) - merges
    return np.concatenate(out, 0) if out else np.zeros((0,), np.int64), n


def merge_slab_collective(slab_labels, n_features, ta, tb, t0, V, edges, key_first, key_last,
                          group=None):
    """The cut exchange among ranks: every rank passes its slab [ta, tb) labels (numpy int32,
    [tb - ta][...]), its feature count and the point keys at ta and tb - 1; returns this rank's
    slab in global canonical labels and the feature count of the whole window (same on every
    rank). Uses torch.distributed (all_gather_object) on the default or given group."""
    import torch.distributed as dist
    lab = np.asarray(slab_labels)
    mine = {
        "ta": ta, "tb": tb, "n": int(n_features),
        "first": lab[0].reshape(-1).copy() if tb > ta else None,
        "last": lab[-1].reshape(-1).copy() if tb > ta else None,
        "key_first": None if key_first is None else np.asarray(key_first).copy(),
        "key_last": None if key_last is None else np.asarray(key_last).copy(),
    }
    world = dist.get_world_size(group)
    every = [None] * world
    dist.all_gather_object(every, mine, group=group)
    every = sorted([e for e in every if e["tb"] > e["ta"]], key=lambda e: e["ta"])
    a_all, b_all = [], []
    for L, R in zip(every[:-1], every[1:]):
        a, b = cut_pairs(L["last"], R["first"], L["key_last"], R["key_first"], edges,
                         (L["ta"] - t0) * V, (R["ta"] - t0) * V)
        a_all.append(a)
        b_all.append(b)
    a = np.concatenate(a_all) if a_all else np.zeros(0, np.int64)
    b = np.concatenate(b_all) if b_all else np.zeros(0, np.int64)
    labels, roots, merges = merge_map(a, b)
    n = sum(e["n"] for e in every) - merges
    return relabel(lab, (ta - t0) * V, labels, roots), n
