"""Test-side helpers that pin the oracle to something other than itself.

Nothing here follows the oracle's algorithm: connectivity is checked by a dense Boolean
transitive closure of an adjacency matrix built pair by pair, by scipy's ndimage labelling and
by scipy's sparse connected components; partitions are compared up to renaming.
"""
import numpy as np


def adjacency_dense(active, key, edges, V_shape):
    """Dense adjacency over all voxel-timesteps of a tiny window, pair by pair.
    active: [Tw][NZ][NY][NX] bool; key: [Tw][P] int (window-relative rows), -1 = none."""
    Tw, nz, ny, nx = V_shape
    N = Tw * nz * ny * nx
    coords = np.array([(t, z, y, x) for t in range(Tw) for z in range(nz) for y in range(ny)
                       for x in range(nx)])
    act = active.reshape(-1)
    A = np.zeros((N, N), dtype=bool)
    for u in range(N):
        for w in range(N):
            if u == w or not (act[u] and act[w]):
                continue
            d = coords[u] - coords[w]
            if edges & 1 and d[0] == 0 and np.abs(d[1:]).max() == 1:
                A[u, w] = True
            if edges & 2 and abs(d[0]) == 1 and not np.any(d[1:]):
                A[u, w] = True
    if edges & 4 and key is not None and key.size:
        V = nz * ny * nx
        for t in range(Tw - 1):
            for p in range(key.shape[1]):
                a, b = key[t, p], key[t + 1, p]
                if a < 0 or b < 0:
                    continue
                u, w = t * V + a, (t + 1) * V + b
                if act[u] and act[w]:
                    A[u, w] = A[w, u] = True
    return A


def closure_labels(A, active_flat):
    """Canonical labels from the reflexive transitive closure of A (repeated squaring)."""
    N = A.shape[0]
    R = A.copy() | np.eye(N, dtype=bool)
    while True:
        R2 = (R.astype(np.uint8) @ R.astype(np.uint8)) > 0
        if (R2 == R).all():
            break
        R = R2
    lab = np.full(N, -1, np.int64)
    for u in range(N):
        if active_flat[u]:
            lab[u] = int(np.argmax(R[u]))      # first reachable index = component minimum
    return lab


def same_partition(a, b):
    """True when two label arrays induce the same partition (inactive = -1 in both)."""
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    if not np.array_equal(a < 0, b < 0):
        return False
    m = a >= 0
    pa, pb = a[m], b[m]
    if pa.size == 0:
        return True
    pairs = np.unique(np.stack([pa, pb], 1), axis=0)
    return (len(np.unique(pairs[:, 0])) == len(pairs) and
            len(np.unique(pairs[:, 1])) == len(pairs))


def structure_4d():
    """scipy.ndimage structuring element for 26-neighbour space and same-voxel t+-1."""
    S = np.zeros((3, 3, 3, 3), dtype=bool)
    S[1] = True
    S[0, 1, 1, 1] = S[2, 1, 1, 1] = True
    return S


def edge_list(active, key, edges):
    """Explicit undirected edge list (numpy, vectorised over offsets) for csgraph."""
    Tw, nz, ny, nx = active.shape
    idx = np.arange(active.size).reshape(active.shape)
    us, ws = [], []
    offs = []
    if edges & 1:
        offs += [(0, dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
                 if (dz, dy, dx) > (0, 0, 0)]
    if edges & 2:
        offs.append((1, 0, 0, 0))
    for dt, dz, dy, dx in offs:
        src = [slice(max(0, -d), n - max(0, d)) for d, n in zip((dt, dz, dy, dx), active.shape)]
        dst = [slice(s.start + d, s.stop + d) for s, d in zip(src, (dt, dz, dy, dx))]
        a = active[tuple(src)] & active[tuple(dst)]
        us.append(idx[tuple(src)][a])
        ws.append(idx[tuple(dst)][a])
    if edges & 4 and key is not None and key.size and Tw > 1:
        V = nz * ny * nx
        flat = active.reshape(-1)
        for t in range(Tw - 1):
            a, b = key[t], key[t + 1]
            ok = (a >= 0) & (b >= 0)
            u = t * V + a[ok].astype(np.int64)
            w = (t + 1) * V + b[ok].astype(np.int64)
            ok2 = flat[u] & flat[w]
            us.append(u[ok2])
            ws.append(w[ok2])
    if not us:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    return np.concatenate(us), np.concatenate(ws)


def csgraph_labels(active, key, edges):
    """Canonical labels via scipy.sparse.csgraph.connected_components on the explicit edges."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    N = active.size
    u, w = edge_list(active, key, edges)
    G = sp.coo_matrix((np.ones(u.size, np.int8), (u, w)), shape=(N, N)).tocsr()
    _, comp = connected_components(G, directed=False)
    flat = active.reshape(-1)
    # canonical: each component's smallest active index
    big = np.iinfo(np.int64).max
    cmin = np.full(comp.max() + 1, big, np.int64)
    ids = np.nonzero(flat)[0]
    np.minimum.at(cmin, comp[ids], ids)
    lab = np.full(N, -1, np.int64)
    lab[ids] = cmin[comp[ids]]
    return lab.reshape(active.shape)


def check_label_invariants(labels, active, key, edges):
    """Invariants that any correct canonical labelling satisfies."""
    lab = labels.reshape(-1).astype(np.int64)
    act = active.reshape(-1)
    assert np.array_equal(lab >= 0, act), "labelled <=> active"
    ids = np.nonzero(act)[0]
    assert np.all(lab[ids] <= ids), "label is not above its voxel"
    assert np.all(lab[lab[ids]] == lab[ids]), "label points at its own root"
    u, w = edge_list(active, key, edges)
    assert np.array_equal(lab[u], lab[w]), "an edge joins two labels"
