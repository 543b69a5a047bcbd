"""Seeded synthetic inputs: triangular meshes, bathymetry, Manning fields,
boundary tags and initial states.

This module is the only code shared by the CUDA path's tests and the oracle.
It holds none of the finite-volume arithmetic: it only places nodes, splits
quads into triangles, samples fields at cell centroids and lists boundary
edges.  Everything is deterministic for a given seed (numpy PCG64).

Workloads (stand-ins for the paper's meshes, which are not available):

* ``canal``  -- the dam-break canal of Section 6.3, oriented along x
  (200 m x 10 m), quads split along the (i,j)->(i+1,j+1) diagonal, interior
  nodes jittered uniformly by +-``jitter`` of the spacing.
* ``river``  -- a 20 km x 2 km reach standing in for the Mille Iles river
  meshes (Section 6.4): a meandering channel, a cosine bowl 5 m deep and
  200 m wide below a +2 m floodplain, 500 Gaussian bumps on the floodplain,
  a 1e-4 longitudinal bed slope, per-cell Manning n ~ U[0.02, 0.06],
  inflow on the channel cross-section at x = 0, fixed stage at x = 20 km,
  walls on the banks.  Node and cell numbering are shuffled by the seed so
  that the mesh carries no grid locality (as a mesh file from an
  unstructured mesher would not).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BC_WALL, BC_INFLOW, BC_TRANSMISSIVE, BC_STAGE = 0, 1, 2, 3


@dataclass
class MeshInput:
    nodes: np.ndarray            # [n_nodes, 2] float64, metres
    tris: np.ndarray             # [n_cells, 3] int32, counter-clockwise
    z: np.ndarray                # [n_cells] float64 bed elevation (m)
    manning: np.ndarray          # [n_cells] float64 Manning n (s m^-1/3)
    bcs: list = field(default_factory=list)   # [(node_pairs [k,2] int32, kind, value)]
    h: np.ndarray = None         # initial depth [n_cells]
    hu: np.ndarray = None
    hv: np.ndarray = None
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_cells(self) -> int:
        return int(self.tris.shape[0])

    def centroids(self) -> np.ndarray:
        return self.nodes[self.tris].mean(axis=1)


def _grid(nx, ny, Lx, Ly, jitter, rng):
    xs = np.linspace(0.0, Lx, nx + 1)
    ys = np.linspace(0.0, Ly, ny + 1)
    X, Y = np.meshgrid(xs, ys)                       # [ny+1, nx+1]
    dx, dy = Lx / nx, Ly / ny
    if jitter > 0.0:
        jx = rng.uniform(-jitter * dx, jitter * dx, size=X.shape)
        jy = rng.uniform(-jitter * dy, jitter * dy, size=Y.shape)
        interior = np.zeros(X.shape, bool)
        interior[1:-1, 1:-1] = True
        X = X + np.where(interior, jx, 0.0)
        Y = Y + np.where(interior, jy, 0.0)
    nodes = np.stack([X.ravel(), Y.ravel()], axis=1)
    j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    p00 = (j * (nx + 1) + i).ravel()
    p10 = p00 + 1
    p01 = p00 + (nx + 1)
    p11 = p01 + 1
    # two counter-clockwise triangles per quad, split along p00 -> p11
    tris = np.empty((2 * nx * ny, 3), np.int64)
    tris[0::2] = np.stack([p00, p10, p11], axis=1)
    tris[1::2] = np.stack([p00, p11, p01], axis=1)
    return nodes, tris.astype(np.int32)


def _side_pairs(nx, ny):
    """Boundary node pairs of the grid, by side (before any shuffle)."""
    def nid(i, j):
        return j * (nx + 1) + i
    i = np.arange(nx)
    j = np.arange(ny)
    bottom = np.stack([nid(i, 0), nid(i + 1, 0)], axis=1)
    top = np.stack([nid(i, ny), nid(i + 1, ny)], axis=1)
    left = np.stack([nid(0, j), nid(0, j + 1)], axis=1)
    right = np.stack([nid(nx, j), nid(nx, j + 1)], axis=1)
    return dict(bottom=bottom, top=top, left=left, right=right)


def canal(nx=200, ny=10, Lx=200.0, Ly=10.0, jitter=0.2, seed=1, hL=10.0, hR=1.0,
          x_dam=100.0, manning=0.0, side_bc=BC_WALL) -> MeshInput:
    """Dam-break canal (Section 6.3, oriented along x): h = hL where the cell
    centroid has x < x_dam, else hR; zero velocity; flat bed; uniform Manning
    n; every boundary a wall unless ``side_bc`` says otherwise."""
    rng = np.random.default_rng(seed)
    nodes, tris = _grid(nx, ny, Lx, Ly, jitter, rng)
    n = tris.shape[0]
    cx = nodes[tris][:, :, 0].mean(axis=1)
    h = np.where(cx < x_dam, hL, hR).astype(np.float64)
    mi = MeshInput(nodes=nodes, tris=tris, z=np.zeros(n), manning=np.full(n, float(manning)),
                   h=h, hu=np.zeros(n), hv=np.zeros(n), name=f"canal_{nx}x{ny}",
                   meta=dict(nx=nx, ny=ny, Lx=Lx, Ly=Ly, jitter=jitter, seed=seed, hL=hL,
                             hR=hR, x_dam=x_dam))
    if side_bc != BC_WALL:
        sides = _side_pairs(nx, ny)
        allp = np.concatenate([sides[k] for k in ("bottom", "top", "left", "right")])
        mi.bcs.append((allp.astype(np.int32), side_bc, 0.0))
    return mi


def river_bed(x, y, bumps, Ly=2000.0):
    """Bed elevation of the synthetic reach at points (x, y)."""
    yc = 0.5 * Ly + 400.0 * np.sin(2.0 * np.pi * x / 2000.0)
    d = np.abs(y - yc)
    in_channel = d < 100.0
    z = np.where(in_channel, 2.0 - 5.0 * 0.5 * (1.0 + np.cos(np.pi * d / 100.0)), 2.0)
    return z, in_channel


def river(nx=8064, ny=806, Lx=20000.0, Ly=2000.0, jitter=0.2, seed=1, n_bumps=500,
          Q=2000.0, eta0=1.0, stage=1.0, manning_range=(0.02, 0.06), fully_wet=False,
          shuffle=True) -> MeshInput:
    """Synthetic river reach (stand-in for the Mille Iles meshes, Section 6.4).

    ``fully_wet`` sets eta0 = max(z) + 0.5 and the outflow stage equal to it,
    so every cell starts with at least 0.5 m of water."""
    rng = np.random.default_rng(seed)
    nodes, tris = _grid(nx, ny, Lx, Ly, jitter, rng)
    n = tris.shape[0]
    c = nodes[tris].mean(axis=1)
    cx, cy = c[:, 0], c[:, 1]
    z, in_channel = river_bed(cx, cy, None, Ly)
    # 500 Gaussian bumps on the floodplain, evaluated inside a +-3.5 sigma window
    sig = rng.uniform(50.0, 300.0, n_bumps)
    amp = rng.uniform(0.5, 3.0, n_bumps)
    bx = rng.uniform(0.0, Lx, n_bumps)
    by = rng.uniform(0.0, Ly, n_bumps)
    dx, dy = Lx / nx, Ly / ny
    bump = np.zeros(n)
    for b in range(n_bumps):
        r = 3.5 * sig[b]
        i0, i1 = max(int((bx[b] - r) / dx) - 1, 0), min(int((bx[b] + r) / dx) + 2, nx)
        j0, j1 = max(int((by[b] - r) / dy) - 1, 0), min(int((by[b] + r) / dy) + 2, ny)
        if i0 >= i1 or j0 >= j1:
            continue
        jj, ii = np.meshgrid(np.arange(j0, j1), np.arange(i0, i1), indexing="ij")
        q = (jj * nx + ii).ravel()
        cells = np.concatenate([2 * q, 2 * q + 1])
        r2 = (cx[cells] - bx[b]) ** 2 + (cy[cells] - by[b]) ** 2
        bump[cells] += amp[b] * np.exp(-0.5 * r2 / (sig[b] * sig[b]))
    z = z + np.where(in_channel, 0.0, bump)
    z = z + 1e-4 * (Lx - cx)                       # bed rises upstream: no exact ties
    man = rng.uniform(manning_range[0], manning_range[1], n)
    if fully_wet:
        eta0 = float(z.max()) + 0.5
        stage = eta0
    h = np.maximum(eta0 - z, 0.0)
    sides = _side_pairs(nx, ny)
    # inflow: left-side edges whose midpoint lies within the channel width
    lp = sides["left"]
    ymid = 0.5 * (nodes[lp[:, 0], 1] + nodes[lp[:, 1], 1])
    _, inch = river_bed(np.zeros_like(ymid), ymid, None, Ly)
    inflow_pairs = lp[inch]
    stage_pairs = sides["right"]
    perm_nodes = None
    if shuffle:
        perm_nodes = rng.permutation(nodes.shape[0])      # new id -> old id
        inv = np.empty_like(perm_nodes)
        inv[perm_nodes] = np.arange(perm_nodes.shape[0])
        nodes = nodes[perm_nodes]
        tris = inv[tris].astype(np.int32)
        inflow_pairs = inv[inflow_pairs]
        stage_pairs = inv[stage_pairs]
        perm_cells = rng.permutation(n)
        tris, z, man, h = tris[perm_cells], z[perm_cells], man[perm_cells], h[perm_cells]
        # rotate the vertex order of each triangle too (orientation kept)
        rot = rng.integers(0, 3, n)
        idx = (np.arange(3)[None, :] + rot[:, None]) % 3
        tris = np.take_along_axis(tris, idx, axis=1).astype(np.int32)
    mi = MeshInput(nodes=nodes, tris=np.ascontiguousarray(tris, dtype=np.int32), z=z,
                   manning=man, h=h, hu=np.zeros(n), hv=np.zeros(n),
                   name=f"river_{nx}x{ny}",
                   meta=dict(nx=nx, ny=ny, Lx=Lx, Ly=Ly, seed=seed, Q=Q, eta0=eta0,
                             stage=stage, shuffle=shuffle))
    mi.bcs.append((np.ascontiguousarray(inflow_pairs, dtype=np.int32), BC_INFLOW, float(Q)))
    mi.bcs.append((np.ascontiguousarray(stage_pairs, dtype=np.int32), BC_STAGE, float(stage)))
    return mi


# --------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------

def dam_break_4k(seed=1) -> MeshInput:
    """4,000-cell canal, h = 10 / 1 m, n = 0, walls (500 FP64 steps, CFL 0.9)."""
    return canal(200, 10, 200.0, 10.0, 0.2, seed, 10.0, 1.0, 100.0, 0.0)


def dam_break_dry_1m(seed=1, manning=0.03) -> MeshInput:
    """1,000,000-cell canal (2000 x 250), dry bed downstream, n = 0.03."""
    return canal(2000, 250, 200.0, 10.0, 0.2, seed, 10.0, 0.0, 100.0, manning)


def river_13m(seed=1) -> MeshInput:
    """12,999,168-cell synthetic river, partially dry, Q = 2000 m^3/s."""
    return river(8064, 806, seed=seed)


def river_13m_wet(seed=1) -> MeshInput:
    """The 12,999,168-cell river, fully wet (depth >= 0.5 m): every cell runs
    the flux path in every step."""
    return river(8064, 806, seed=seed, fully_wet=True)


def river_adjoint(nx, ny, seed=1, u0=0.5) -> MeshInput:
    """The adjoint workload's reach: the river generator on the 20 km x 2 km
    domain at nx x ny quads, fully wet, with the free surface inclined from
    eta0 + 1 m at x = 0 to eta0 = max(z) + 0.5 m at the outflow (Section 6.5.1's
    initialisation) and the water moving downstream at u0 m/s, so that it flows
    past the gauges from the first step and the loss depends on the Manning
    coefficients as well as on the bed."""
    mi = river(nx, ny, seed=seed, fully_wet=True)
    eta0 = mi.meta["eta0"]
    mi = inclined_plane(mi, eta_up=eta0 + 1.0, eta_down=eta0)
    mi.hu = u0 * mi.h
    mi.meta.update(u0=u0)
    return mi


def river_adjoint_1m(seed=1) -> MeshInput:
    """1,001,728-cell adjoint reach (river_adjoint at 2236 x 224 quads)."""
    return river_adjoint(2236, 224, seed=seed)


def river_adjoint_20k(seed=1) -> MeshInput:
    """20,224-cell copy of the adjoint reach (316 x 32 quads, the same 20 km x 2 km)."""
    return river_adjoint(316, 32, seed=seed)


def river_cells(n_cells, seed=1, **kw) -> MeshInput:
    """A river reach with about ``n_cells`` cells (aspect 10:1)."""
    ny = max(int(round(math.sqrt(n_cells / 20.0))), 2)
    nx = max(int(round(n_cells / (2.0 * ny))), 2)
    return river(nx, ny, seed=seed, **kw)


def canal_cells(n_cells, seed=1, **kw) -> MeshInput:
    """A dam-break canal with about ``n_cells`` cells (aspect 20:1)."""
    ny = max(int(round(math.sqrt(n_cells / 40.0))), 2)
    nx = max(int(round(n_cells / (2.0 * ny))), 2)
    return canal(nx, ny, 200.0, 10.0, 0.2, seed, **kw)


def ensemble_members(n_members=256, seed=1, lo=2e4, hi=5e5):
    """Members of the uncertainty ensemble: sizes log-uniform in [lo, hi],
    even members canals, odd members rivers; Manning n ~ U[0.015, 0.08] and
    inflow Q ~ U[500, 3000] m^3/s per member.  A canal member receives the
    same discharge per unit width as a 200 m river channel (Q * 10 / 200)
    through its upstream edge, on top of its dam-break initial state."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(math.log(lo), math.log(hi), n_members))
    mans = rng.uniform(0.015, 0.08, n_members)
    Qs = rng.uniform(500.0, 3000.0, n_members)
    out = []
    for k in range(n_members):
        s = int(sizes[k])
        if k % 2 == 0:
            mi = canal_cells(s, seed=seed * 1000 + k, manning=float(mans[k]))
            ny, nx = mi.meta["ny"], mi.meta["nx"]
            left = _side_pairs(nx, ny)["left"].astype(np.int32)
            mi.bcs.append((left, BC_INFLOW, float(Qs[k]) * 10.0 / 200.0))
        else:
            mi = river_cells(s, seed=seed * 1000 + k, Q=float(Qs[k]),
                             manning_range=(float(mans[k]), float(mans[k])))
        mi.meta.update(member=k, manning=float(mans[k]), Q=float(Qs[k]))
        out.append(mi)
    return out


def gauge_cells(n_cells, n_gauges=64, seed=1):
    """Seeded gauge cells for the misfit loss."""
    rng = np.random.default_rng(seed + 7919)
    return np.sort(rng.choice(n_cells, size=n_gauges, replace=False)).astype(np.int32)


def perturbation(n, seed):
    """Seeded standard-normal field xi (used for target runs and directions)."""
    return np.random.default_rng(seed).standard_normal(n)


# --------------------------------------------------------------------------
# Initial conditions of the paper's river experiments, on the synthetic reach
# --------------------------------------------------------------------------

def inclined_plane(mi: MeshInput, eta_up: float, eta_down: float) -> MeshInput:
    """Free surface on an inclined plane from eta_up at x = 0 to eta_down at
    x = Lx, zero velocity (the Montreal initialisation, Section 6.5.1: water
    gains speed downstream sooner than from a horizontal plane)."""
    x = mi.centroids()[:, 0]
    Lx = mi.meta.get("Lx", float(x.max()))
    eta = eta_up + (eta_down - eta_up) * x / Lx
    mi.h = np.maximum(eta - mi.z, 0.0)
    mi.hu = np.zeros_like(mi.h)
    mi.hv = np.zeros_like(mi.h)
    mi.meta.update(init="inclined_plane", eta_up=eta_up, eta_down=eta_down)
    return mi


def dam_failure(mi: MeshInput, x_dam: float, h_up: float = 30.0, h_down: float = 29.0) -> MeshInput:
    """One-dimensional Riemann problem on the reach: water depth h_up upstream
    of x_dam and h_down downstream, zero velocity (the fictitious dam failure,
    Section 6.4.2, 30 m / 29 m)."""
    x = mi.centroids()[:, 0]
    mi.h = np.where(x < x_dam, h_up, h_down).astype(np.float64)
    mi.hu = np.zeros_like(mi.h)
    mi.hv = np.zeros_like(mi.h)
    mi.meta.update(init="dam_failure", x_dam=x_dam, h_up=h_up, h_down=h_down)
    return mi
