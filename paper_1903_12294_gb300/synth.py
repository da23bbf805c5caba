"""Seeded synthetic inputs shaped like the workloads of Sauer & Ma (arXiv 1903.12294).

This module holds data generation only: none of the method's arithmetic (binning, criterion,
labelling, reduction) appears here. Both the CUDA path and the CPU oracle consume the bytes it
produces. The paper's datasets (the S3D lifted-jet combustion run of §4.1 and the Beijing
taxi/traffic data of §4.2) are not available, so these generators stand in for them with
their shapes: a 3D field plus tracer particles that carry attributes, and a 2D+time traffic
density plus vehicle trajectories (§4.2 treats the city as 2D+time).

Every array is produced with ``torch`` on the requested device from a seed; small random
parameters (blob centres, vortex axes, Fourier modes) come from numpy's PCG64 with the same
seed. Layouts: field ``[T][NZ][NY][NX]`` fp32, positions ``[T][3][P]`` fp32 in grid units
(voxel (x,y,z) covers [x,x+1)x[y,y+1)x[z,z+1)), attributes ``[T][A][P]`` fp32.

Workloads (seed = 190312294 + config number):
  1 tiny        32^3 x 8, 6 drifting Gaussian blobs + N(0,0.05); 20k particles in 3 Lamb-Oseen
                vortices (RK2, dt 0.5), attribute |u|
  2 mid         128^3 x 32, 40 drifting/merging blobs + 0.1*LogNormal(0,0.5); 1M particles on
                curl noise, attributes speed and the field value at the particle
  3 combustion  256^3 x 24, |k|^-5/3 random-phase field folded into flame-like sheets; 8M
                particles, attributes temperature, mixture fraction, speed, age
  4 batched     192^3 x 32, blobs; 4M particles, 3 attributes; plus 64 random queries
  5 serving     1024^2 x 1 x 96 traffic density from ~208k road-lattice walkers; 2 attributes
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field as dc_field

import numpy as np
import torch

SEED_BASE = 190312294

# Predicate encoding shared by every caller of the library (source, op), mirrored from the
# public C header's enums so that query generators can be written without importing the
# binding.
SRC_FIELD, SRC_COUNT, SRC_MEAN = 0, 1, 2
OP_GT, OP_GE, OP_LT, OP_LE, OP_BAND = 0, 1, 2, 3, 4
EDGE_SPATIAL, EDGE_TEMPORAL, EDGE_TRAJ = 1, 2, 4
EDGE_ALL = 7


@dataclass
class Workload:
    """One synthetic dataset plus the query (or queries) run on it."""
    name: str
    field: torch.Tensor              # [T][NZ][NY][NX] fp32
    pos: torch.Tensor                # [T][3][P] fp32
    attr: torch.Tensor               # [T][A][P] fp32
    t0: int = 0
    t1: int = 0
    preds: list = dc_field(default_factory=list)   # [(src, attr, op, lo, hi)]
    edges: int = EDGE_ALL
    queries: list = dc_field(default_factory=list)  # batched / served: [(t0, t1, preds, edges)]
    attr_names: tuple = ()
    # point samples on their own time grid: pos/attr are [Tp][...] and point step j falls in
    # field step field_step[j] (None: one point step per field step)
    field_step: list = None

    @property
    def shape(self):
        return tuple(self.field.shape)

    @property
    def vt(self):
        T, nz, ny, nx = self.field.shape
        return nx * ny * nz * (self.t1 - self.t0)

    def to(self, device):
        return Workload(self.name, self.field.to(device), self.pos.to(device),
                        self.attr.to(device), self.t0, self.t1, list(self.preds), self.edges,
                        list(self.queries), self.attr_names, self.field_step)

    def numpy(self):
        return (self.field.cpu().numpy(), self.pos.cpu().numpy(), self.attr.cpu().numpy())


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _tgen(seed, device):
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def _quantile(x: torch.Tensor, qs, seed, n=1 << 20):
    """Quantiles of a large tensor from a fixed random subsample (torch.quantile caps size)."""
    flat = x.reshape(-1)
    flat = flat[torch.isfinite(flat)]
    if flat.numel() > n:
        idx = torch.randint(0, flat.numel(), (n,), generator=_tgen(seed, flat.device),
                            device=flat.device)
        flat = flat[idx]
    q = torch.quantile(flat.double(), torch.tensor(qs, dtype=torch.float64, device=flat.device))
    return [float(np.float32(v)) for v in q.cpu().tolist()]


# ---------------------------------------------------------------------------------------------
# fields
# ---------------------------------------------------------------------------------------------

def _blob_field(T, nz, ny, nx, centres0, vel, sigma, amp, device):
    """Sum of Gaussian blobs whose centres drift linearly in time (separable, clipped to +-4
    sigma boxes)."""
    f = torch.zeros((T, nz, ny, nx), dtype=torch.float32, device=device)
    dims = (nx, ny, nz)
    for t in range(T):
        for c0, v, s, a in zip(centres0, vel, sigma, amp):
            c = c0 + v * t
            lo = [max(0, int(math.floor(c[d] - 4 * s))) for d in range(3)]
            hi = [min(dims[d], int(math.ceil(c[d] + 4 * s)) + 1) for d in range(3)]
            if any(h <= l for l, h in zip(lo, hi)):
                continue
            g = []
            for d in range(3):
                xs = torch.arange(lo[d], hi[d], device=device, dtype=torch.float32)
                g.append(torch.exp(-((xs - float(c[d])) ** 2) / (2.0 * s * s)))
            blk = (a * g[2][:, None, None] * g[1][None, :, None] * g[0][None, None, :])
            f[t, lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] += blk
    return f


def _spectral_field(T, n, seed, device, slope=-5.0 / 3.0):
    """Random-phase periodic field with energy spectrum ~|k|^slope; phases advance in time with
    frequency ~|k|^(2/3). Normalised to zero mean and unit variance per step."""
    g = _tgen(seed, "cpu")
    k1 = torch.fft.fftfreq(n, d=1.0 / n)
    k3 = torch.fft.rfftfreq(n, d=1.0 / n)
    KZ, KY, KX = torch.meshgrid(k1, k1, k3, indexing="ij")
    kk = torch.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    kk[0, 0, 0] = 1.0
    # E(k) ~ k^slope spread over a shell of area ~k^2 -> amplitude ~ sqrt(k^slope / k^2)
    amp = torch.sqrt(kk ** slope / kk ** 2)
    amp[0, 0, 0] = 0.0
    amp[kk > n / 3] = 0.0
    phase0 = torch.rand(kk.shape, generator=g) * (2 * math.pi)
    omega = 0.15 * kk ** (2.0 / 3.0)
    out = torch.empty((T, n, n, n), dtype=torch.float32, device=device)
    amp, phase0, omega = amp.to(device), phase0.to(device), omega.to(device)
    for t in range(T):
        ph = phase0 + omega * t
        spec = torch.polar(amp, ph)
        f = torch.fft.irfftn(spec, s=(n, n, n))
        f = (f - f.mean()) / f.std()
        out[t] = f.float()
    return out


# ---------------------------------------------------------------------------------------------
# particle velocity fields
# ---------------------------------------------------------------------------------------------

class _CurlNoise:
    """u(x,t) = sum_m cos(k_m.x + phi_m + w_m t) (k_m x a_m): the curl of the vector potential
    sum_m a_m sin(k_m.x + ...), hence divergence-free. Periodic on the box."""

    def __init__(self, rng, box, n_modes=3, speed=0.8, device="cpu"):
        L = np.asarray(box, dtype=np.float64)
        ks, cs = [], []
        for _ in range(n_modes):
            nvec = rng.integers(-3, 4, size=3)
            while not nvec.any():
                nvec = rng.integers(-3, 4, size=3)
            k = 2 * np.pi * nvec / L
            a = rng.normal(size=3)
            c = np.cross(k, a)
            ks.append(k)
            cs.append(c)
        cs = np.asarray(cs)
        cs *= speed / max(np.linalg.norm(cs, axis=1).sum(), 1e-12)
        self.k = torch.tensor(np.asarray(ks), dtype=torch.float32, device=device)
        self.c = torch.tensor(cs, dtype=torch.float32, device=device)
        self.phi = torch.tensor(rng.uniform(0, 2 * np.pi, n_modes), dtype=torch.float32,
                                device=device)
        self.w = torch.tensor(rng.uniform(-0.2, 0.2, n_modes), dtype=torch.float32,
                              device=device)

    def __call__(self, x, t):  # x [3][P]
        ph = self.k @ x + (self.phi + self.w * t)[:, None]       # [M][P]
        return self.c.t() @ torch.cos(ph)                          # [3][P]


class _Vortices:
    """Sum of Lamb-Oseen vortices about random axes; scaled so |u| <= 1."""

    def __init__(self, rng, box, n=3, rc=4.0, device="cpu"):
        L = np.asarray(box, dtype=np.float64)
        self.c = torch.tensor(rng.uniform(0, 1, (n, 3)) * L, dtype=torch.float32, device=device)
        ax = rng.normal(size=(n, 3))
        ax /= np.linalg.norm(ax, axis=1, keepdims=True)
        self.e = torch.tensor(ax, dtype=torch.float32, device=device)
        self.rc = rc
        # peak of (1-exp(-r^2/rc^2))/r is ~0.6382/rc at r ~ 1.1209 rc; cap each at 1/n
        self.gam = (2 * math.pi * rc / 0.6382) / n

    def __call__(self, x, t):
        u = torch.zeros_like(x)
        for j in range(self.c.shape[0]):
            d = x - self.c[j][:, None]
            e = self.e[j][:, None]
            dp = d - (e * d).sum(0, keepdim=True) * e
            r2 = (dp * dp).sum(0, keepdim=True).clamp_min(1e-12)
            r = torch.sqrt(r2)
            ut = self.gam / (2 * math.pi * r) * (1 - torch.exp(-r2 / (self.rc ** 2)))
            u += ut * torch.cross(e.expand_as(dp), dp, dim=0) / r
        return u


def _advect(x0, vel, T, dt, box, device):
    """RK2 (midpoint) trajectories with periodic wrap. Returns positions [T][3][P] and the
    velocity magnitude at each sample."""
    L = torch.tensor(box, dtype=torch.float32, device=device)[:, None]
    P = x0.shape[1]
    pos = torch.empty((T, 3, P), dtype=torch.float32, device=device)
    spd = torch.empty((T, P), dtype=torch.float32, device=device)
    x = x0.clone()
    for t in range(T):
        pos[t] = x
        u = vel(x, float(t))
        spd[t] = torch.linalg.vector_norm(u, dim=0)
        xm = x + 0.5 * dt * u
        x = torch.remainder(x + dt * vel(xm, t + 0.5 * dt), L)
    return pos, spd


def _sample_nearest(field_t, p):
    """Field value in the voxel containing each particle (clamped; data synthesis only)."""
    nz, ny, nx = field_t.shape
    ix = p[0].floor().long().clamp(0, nx - 1)
    iy = p[1].floor().long().clamp(0, ny - 1)
    iz = p[2].floor().long().clamp(0, nz - 1)
    return field_t[iz, iy, ix]


# ---------------------------------------------------------------------------------------------
# the five workloads
# ---------------------------------------------------------------------------------------------

def tiny(device="cpu", n=32, T=8, P=20000, seed=SEED_BASE + 1):
    rng = _rng(seed)
    box = (n, n, n)
    nb = 6
    c0 = rng.uniform(6.0 / 32 * n, 26.0 / 32 * n, (nb, 3))
    d = rng.normal(size=(nb, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    f = _blob_field(T, n, n, n, c0, d * 1.0, [3.0] * nb, [1.0] * nb, device)
    f += 0.05 * torch.randn(f.shape, generator=_tgen(seed, device), device=device)
    x0 = torch.rand((3, P), generator=_tgen(seed + 7, device), device=device) * n
    vel = _Vortices(rng, box, device=device)
    pos, spd = _advect(x0, vel, T, 0.5, box, device)
    attr = spd[:, None, :].contiguous()
    preds = [(SRC_FIELD, 0, OP_GT, 0.4, 0.0), (SRC_COUNT, 0, OP_GE, 2.0, 0.0)]
    return Workload("tiny", f, pos, attr, 0, T, preds, EDGE_ALL, attr_names=("speed",))


def multirate(device="cpu", n=32, T=8, r=4, P=20000, seed=SEED_BASE + 6, field_step=None):
    """Points saved more often than the field (§4.1): the tiny workload's drifting blobs over T
    field steps, and particles in the same vortex flow sampled r times per field step (Tp = r T
    point steps, 2 voxel lengths of time per field step, so a point crosses voxels between the
    point steps of one field step). ``field_step`` overrides the even map (any non-decreasing
    map of len(field_step) point steps into [0, T))."""
    rng = _rng(seed)
    box = (n, n, n)
    nb = 6
    c0 = rng.uniform(6.0 / 32 * n, 26.0 / 32 * n, (nb, 3))
    d = rng.normal(size=(nb, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    f = _blob_field(T, n, n, n, c0, d * 1.0, [3.0] * nb, [1.0] * nb, device)
    f += 0.05 * torch.randn(f.shape, generator=_tgen(seed, device), device=device)
    fs = list(field_step) if field_step is not None else [t for t in range(T) for _ in range(r)]
    Tp = len(fs)
    x0 = torch.rand((3, P), generator=_tgen(seed + 7, device), device=device) * n
    vel = _Vortices(rng, box, device=device)
    pos, spd = _advect(x0, vel, Tp, 2.0 * T / Tp, box, device)
    attr = torch.stack([spd, pos[:, 2] / n], dim=1).contiguous()
    preds = [(SRC_FIELD, 0, OP_GT, 0.4, 0.0), (SRC_COUNT, 0, OP_GE, 2.0, 0.0)]
    return Workload("multirate", f, pos, attr, 0, T, preds, EDGE_ALL,
                    attr_names=("speed", "height"), field_step=fs)


def mid(device="cpu", n=128, T=32, P=1 << 20, seed=SEED_BASE + 2, n_blobs=40):
    rng = _rng(seed)
    box = (n, n, n)
    sig = rng.uniform(3.0, 8.0, n_blobs)
    # pairs of blobs drift toward each other and meet around mid-window
    c0 = np.empty((n_blobs, 3))
    vel = np.empty((n_blobs, 3))
    for i in range(0, n_blobs, 2):
        mid_pt = rng.uniform(0.15 * n, 0.85 * n, 3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        sep = rng.uniform(0.3, 0.6) * T
        c0[i] = mid_pt - d * sep * 0.5
        vel[i] = d * sep / T
        if i + 1 < n_blobs:
            c0[i + 1] = mid_pt + d * sep * 0.5
            vel[i + 1] = -d * sep / T
    amp = rng.uniform(0.7, 1.3, n_blobs)
    f = _blob_field(T, n, n, n, c0, vel, sig, amp, device)
    g = _tgen(seed, device)
    f += 0.1 * torch.exp(0.5 * torch.randn(f.shape, generator=g, device=device))
    x0 = torch.rand((3, P), generator=_tgen(seed + 7, device), device=device) * n
    velf = _CurlNoise(rng, box, n_modes=3, speed=0.9, device=device)
    pos, spd = _advect(x0, velf, T, 1.0, box, device)
    samp = torch.stack([_sample_nearest(f[t], pos[t]) for t in range(T)])
    attr = torch.stack([spd, samp], dim=1).contiguous()
    q40, q90 = _quantile(spd, [0.4, 0.9], seed)
    preds = [(SRC_FIELD, 0, OP_GT, 0.5, 0.0), (SRC_MEAN, 0, OP_BAND, q40, q90)]
    return Workload("mid", f, pos, attr, 0, T, preds, EDGE_ALL, attr_names=("speed", "field"))


def combustion(device="cpu", n=256, T=24, P=8 << 20, seed=SEED_BASE + 3, width=0.15):
    rng = _rng(seed)
    box = (n, n, n)
    g = _spectral_field(T, n, seed, device)
    f = torch.exp(-((g - 0.0) / width) ** 2)
    x0 = torch.rand((3, P), generator=_tgen(seed + 7, device), device=device) * n
    velf = _CurlNoise(rng, box, n_modes=3, speed=1.0, device=device)
    pos, spd = _advect(x0, velf, T, 1.0, box, device)
    age0 = torch.rand(P, generator=_tgen(seed + 11, device), device=device) * 50.0
    temp = torch.stack([300.0 + 1700.0 * _sample_nearest(f[t], pos[t]) for t in range(T)])
    zmix = torch.stack([0.5 + 0.5 * torch.tanh(_sample_nearest(g[t], pos[t])) for t in range(T)])
    age = torch.stack([age0 + t for t in range(T)])
    attr = torch.stack([temp, zmix, spd, age], dim=1).contiguous()
    del g
    qT60, = _quantile(temp, [0.6], seed)
    zlo, zhi = _quantile(zmix, [0.2, 0.8], seed + 1)
    preds = [(SRC_FIELD, 0, OP_GT, 0.5, 0.0), (SRC_MEAN, 0, OP_GT, qT60, 0.0),
             (SRC_MEAN, 1, OP_BAND, zlo, zhi)]
    return Workload("combustion", f, pos, attr, 0, T, preds, EDGE_ALL,
                    attr_names=("temperature", "mixture_fraction", "speed", "age"))


def random_queries(wl: Workload, nq, seed, tw_range, field_q=(0.80, 0.97), ops=(OP_GT, OP_BAND)):
    """Queries with their own thresholds, attribute and window: T_w ~ U{lo..hi},
    t0 ~ U{0..T-T_w}, attribute ~ U{0..A-1}, op ~ U{ops}, thresholds from stored quantiles."""
    rng = _rng(seed)
    T = wl.field.shape[0]
    A = wl.attr.shape[1]
    fq = _quantile(wl.field, list(np.linspace(field_q[0], field_q[1], 8)), seed)
    aq = [_quantile(wl.attr[:, a], [0.1, 0.3, 0.5, 0.7, 0.9], seed + a) for a in range(A)]
    qs = []
    for _ in range(nq):
        tw = int(rng.integers(tw_range[0], min(tw_range[1], T) + 1))
        t0 = int(rng.integers(0, T - tw + 1))
        a = int(rng.integers(0, A))
        op = int(ops[int(rng.integers(0, len(ops)))])
        thr = fq[int(rng.integers(0, len(fq)))]
        preds = [(SRC_FIELD, 0, OP_GT, thr, 0.0)]
        if op == OP_BAND:
            i = int(rng.integers(0, 3))
            preds.append((SRC_MEAN, a, OP_BAND, aq[a][i], aq[a][i + 2]))
        else:
            preds.append((SRC_MEAN, a, op, aq[a][int(rng.integers(0, 4))], 0.0))
        qs.append((t0, t0 + tw, preds, EDGE_ALL))
    return qs


def batched(device="cpu", n=192, T=32, P=4 << 20, seed=SEED_BASE + 4, nq=64, n_blobs=48):
    wl = mid(device=device, n=n, T=T, P=P, seed=seed, n_blobs=n_blobs)
    age0 = torch.rand(P, generator=_tgen(seed + 11, device), device=device) * 20.0
    age = torch.stack([age0 + t for t in range(T)])
    wl.attr = torch.cat([wl.attr, age[:, None, :]], dim=1).contiguous()
    wl.name = "batched"
    wl.attr_names = ("speed", "field", "age")
    wl.queries = random_queries(wl, nq, seed + 100, (2, 32))
    t0, t1, preds, edges = wl.queries[0]
    wl.t0, wl.t1, wl.preds, wl.edges = t0, t1, preds, edges
    return wl


def serving(device="cpu", n=1024, T=96, walkers=208334, seed=SEED_BASE + 5, spacing=16,
            nq=200):
    """2D+time (§4.2): walkers move along a lattice of roads every ``spacing`` px (turning at
    crossings) or along a few diagonal highways, 1-8 px per step; density = smoothed walker count
    + N(0,0.02). Attributes: speed, trip age."""
    rng = _rng(seed)
    g = _tgen(seed, device)
    W = walkers
    hw = int(0.1 * W)                    # walkers on diagonal highways
    # lattice walkers: start on a road crossing, move along x or y
    cx = torch.randint(0, n // spacing, (W,), generator=g, device=device) * spacing
    cy = torch.randint(0, n // spacing, (W,), generator=g, device=device) * spacing
    x = cx.float() + 0.5
    y = cy.float() + 0.5
    dirs = torch.tensor([[1, 0], [-1, 0], [0, 1], [0, -1]], dtype=torch.float32, device=device)
    di = torch.randint(0, 4, (W,), generator=g, device=device)
    spd = torch.randint(1, 9, (W,), generator=g, device=device).float()
    # highway walkers move diagonally
    hsel = torch.zeros(W, dtype=torch.bool, device=device)
    hsel[:hw] = True
    hdir = torch.tensor([[1, 1], [-1, -1], [1, -1], [-1, 1]], dtype=torch.float32,
                        device=device) / math.sqrt(2.0)
    age = torch.zeros(W, device=device)
    pos = torch.empty((T, 3, W), dtype=torch.float32, device=device)
    attr = torch.empty((T, 2, W), dtype=torch.float32, device=device)
    dens = torch.zeros((T, 1, n, n), dtype=torch.float32, device=device)
    for t in range(T):
        pos[t, 0], pos[t, 1], pos[t, 2] = x, y, torch.full_like(x, 0.5)
        attr[t, 0], attr[t, 1] = spd, age
        ix = x.floor().long().clamp(0, n - 1)
        iy = y.floor().long().clamp(0, n - 1)
        dens[t, 0].view(-1).index_add_(0, iy * n + ix, torch.ones_like(x))
        dv = torch.where(hsel[:, None], hdir[di], dirs[di])
        x = torch.remainder(x + dv[:, 0] * spd, float(n))
        y = torch.remainder(y + dv[:, 1] * spd, float(n))
        # lattice walkers snap to the nearest road and may turn
        turn = (torch.rand(W, generator=g, device=device) < 0.2) & ~hsel
        di = torch.where(turn, torch.randint(0, 4, (W,), generator=g, device=device), di)
        onx = (dirs[di][:, 0] != 0) & ~hsel
        ony = (dirs[di][:, 1] != 0) & ~hsel
        y = torch.where(onx, torch.round((y - 0.5) / spacing) * spacing % n + 0.5, y)
        x = torch.where(ony, torch.round((x - 0.5) / spacing) * spacing % n + 0.5, x)
        newtrip = torch.rand(W, generator=g, device=device) < 0.02
        age = torch.where(newtrip, torch.zeros_like(age), age + 1)
        spd = torch.where(torch.rand(W, generator=g, device=device) < 0.1,
                          torch.randint(1, 9, (W,), generator=g, device=device).float(), spd)
    # Gaussian smoothing (sigma 2 px), separable
    r = torch.arange(-6, 7, device=device, dtype=torch.float32)
    k = torch.exp(-r ** 2 / 8.0)
    k = (k / k.sum())
    d = dens.reshape(T, 1, n, n)
    d = torch.nn.functional.conv2d(d, k.view(1, 1, 1, -1), padding=(0, 6))
    d = torch.nn.functional.conv2d(d, k.view(1, 1, -1, 1), padding=(6, 0))
    f = d.reshape(T, 1, n, n) + 0.02 * torch.randn((T, 1, n, n), generator=g, device=device)
    wl = Workload("serving", f.contiguous(), pos, attr.contiguous(), 0, T, [], EDGE_ALL,
                  attr_names=("speed", "age"))
    wl.queries = random_queries(wl, nq, seed + 100, (4, 64), field_q=(0.90, 0.99))
    t0, t1, preds, edges = wl.queries[0]
    wl.t0, wl.t1, wl.preds, wl.edges = t0, t1, preds, edges
    _ = rng
    return wl


CONFIGS = {1: tiny, 2: mid, 3: combustion, 4: batched, 5: serving}


def make(config: int, device="cpu", **kw) -> Workload:
    return CONFIGS[int(config)](device=device, **kw)


def poisson_arrivals(rate_hz, duration_s, seed):
    """Arrival times of a Poisson process (serving workload)."""
    rng = _rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            return out
        out.append(t)
