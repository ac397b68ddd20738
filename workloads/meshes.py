"""Structured meshes and workload parameters (geometry and configuration only).

2D: a square torso [0, L]^2 split into right triangles along the "/" diagonal of
every cell, with an elliptic heart; an element is a heart element when its
centroid lies inside the ellipse.  3D: a box split into six Kuhn tetrahedra per
hexahedron (all along the main diagonal, so the mesh is conforming); every
element is heart tissue (isolated heart, Sec. 2.2 of the paper).

Fibre frames are per element, stored as a d x d matrix whose columns are the
local axes (fibre, sheet, normal) in the global basis.  The conductivity values
and the Mitchell-Schaeffer parameters are workload inputs, passed unchanged to
both the oracle and the CUDA library.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Mesh:
    dim: int
    coords: np.ndarray          # (n_nodes, dim) float64, cm
    elems: np.ndarray           # (n_elems, dim+1) int32
    region: np.ndarray          # (n_elems,) int32: 1 heart, 0 torso
    fibre: np.ndarray           # (n_elems, dim, dim) float64, columns = local axes
    shape: tuple                # nodes per axis
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.coords.shape[0])

    @property
    def n_elems(self) -> int:
        return int(self.elems.shape[0])


def _rot2(theta: np.ndarray) -> np.ndarray:
    c, s = np.cos(theta), np.sin(theta)
    r = np.empty(theta.shape + (2, 2))
    r[..., 0, 0] = c
    r[..., 1, 0] = s
    r[..., 0, 1] = -s
    r[..., 1, 1] = c
    return r


def torso_square_2d(n: int, length: float = 10.0, centre=(5.0, 5.0),
                    semi_axes=(3.0, 2.0), fibre_deg: float = 30.0) -> Mesh:
    """n x n nodes on [0, length]^2; elliptic heart; uniform fibre angle."""
    h = length / (n - 1)
    xs = np.arange(n) * h
    X, Y = np.meshgrid(xs, xs, indexing="xy")       # node id = j * n + i
    coords = np.stack([X.ravel(), Y.ravel()], axis=1)
    i, j = np.meshgrid(np.arange(n - 1), np.arange(n - 1), indexing="xy")
    v00 = (j * n + i).ravel()
    v10, v01 = v00 + 1, v00 + n
    v11 = v01 + 1
    t1 = np.stack([v00, v10, v11], axis=1)
    t2 = np.stack([v00, v11, v01], axis=1)
    elems = np.empty((2 * v00.size, 3), dtype=np.int64)
    elems[0::2], elems[1::2] = t1, t2
    cen = coords[elems].mean(axis=1)
    a, b = semi_axes
    inside = ((cen[:, 0] - centre[0]) / a) ** 2 + ((cen[:, 1] - centre[1]) / b) ** 2 <= 1.0
    theta = np.full(elems.shape[0], np.deg2rad(fibre_deg))
    return Mesh(dim=2, coords=coords, elems=elems.astype(np.int32),
                region=inside.astype(np.int32), fibre=_rot2(theta), shape=(n, n),
                meta=dict(length=length, centre=tuple(centre), semi_axes=tuple(semi_axes),
                          fibre_deg=fibre_deg, h=h))


_KUHN = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def slab_3d(nx: int, ny: int, nz: int, size=(1.0, 1.0, 0.3),
            theta0_deg: float = -60.0, theta1_deg: float = 60.0) -> Mesh:
    """nx x ny x nz nodes on a box; Kuhn split; fibre angle linear in depth."""
    hx, hy, hz = size[0] / (nx - 1), size[1] / (ny - 1), size[2] / (nz - 1)
    Z, Y, X = np.meshgrid(np.arange(nz) * hz, np.arange(ny) * hy, np.arange(nx) * hx,
                          indexing="ij")                 # node id = (k*ny + j)*nx + i
    coords = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    k, j, i = np.meshgrid(np.arange(nz - 1), np.arange(ny - 1), np.arange(nx - 1), indexing="ij")
    base = ((k * ny + j) * nx + i).ravel()
    step = np.array([1, nx, nx * ny])
    tets = []
    for perm in _KUHN:
        v0 = base
        v1 = v0 + step[perm[0]]
        v2 = v1 + step[perm[1]]
        v3 = v2 + step[perm[2]]
        tets.append(np.stack([v0, v1, v2, v3], axis=1))
    elems = np.stack(tets, axis=1).reshape(-1, 4)
    cz = coords[elems][:, :, 2].mean(axis=1)
    theta = np.deg2rad(theta0_deg + (theta1_deg - theta0_deg) * cz / size[2])
    c, s = np.cos(theta), np.sin(theta)
    fr = np.zeros((elems.shape[0], 3, 3))
    fr[:, 0, 0], fr[:, 1, 0] = c, s          # fibre  a = ( cos, sin, 0)
    fr[:, 0, 1], fr[:, 1, 1] = -s, c         # sheet  t = (-sin, cos, 0)
    fr[:, 2, 2] = 1.0                        # normal n = e_z
    return Mesh(dim=3, coords=coords, elems=elems.astype(np.int32),
                region=np.ones(elems.shape[0], dtype=np.int32), fibre=fr,
                shape=(nx, ny, nz),
                meta=dict(size=tuple(size), theta_deg=(theta0_deg, theta1_deg), h=(hx, hy, hz)))


# Mitchell-Schaeffer model (published defaults) mapped to mV with the rest and
# excited potentials of the paper's 2D test case.
_MS = dict(tau_in=0.3, tau_out=6.0, tau_open=120.0, tau_close=150.0, v_gate=0.13,
           v_rest=-90.0, v_peak=50.0)


def params_2d(dt: float) -> dict:
    """Parameters of the 2D torso workloads (mS/cm, cm^-1, uF/cm^2, ms)."""
    p = dict(sigma_i=(3.0, 0.3, 0.3), sigma_e=(2.0, 1.3, 1.3), sigma_T=2.0,
             chi=1000.0, Cm=1.0, dt=dt, stim_amp=50.0, stim_t=(0.0, 1.0))
    p.update(_MS)
    return p


def params_3d(dt: float) -> dict:
    """Parameters of the orthotropic 3D slab workloads."""
    p = dict(sigma_i=(3.0, 1.0, 0.3), sigma_e=(2.0, 1.65, 1.3), sigma_T=2.0,
             chi=1000.0, Cm=1.0, dt=dt, stim_amp=50.0, stim_t=(0.0, 1.0))
    p.update(_MS)
    return p


def stimulus_left_apex(mesh: Mesh, radius: float = 0.5, amp: float = 50.0) -> np.ndarray:
    """Per-node amplitude: nodes within `radius` of the ellipse's left apex."""
    cx, cy = mesh.meta["centre"]
    a = mesh.meta["semi_axes"][0]
    d = np.hypot(mesh.coords[:, 0] - (cx - a), mesh.coords[:, 1] - cy)
    return np.where(d <= radius, amp, 0.0)


def stimulus_seeded_disc(mesh: Mesh, seed: int, radius: float = 0.25,
                         amp: float = 50.0, margin: float = 0.5) -> np.ndarray:
    """Per-node amplitude on a disc whose centre is drawn uniformly inside the
    ellipse shrunk by `margin` (rejection sampling from a seeded generator)."""
    rng = np.random.default_rng(seed)
    cx, cy = mesh.meta["centre"]
    a, b = mesh.meta["semi_axes"]
    a2, b2 = max(a - margin, 0.1), max(b - margin, 0.1)
    while True:
        px, py = rng.uniform(-a2, a2), rng.uniform(-b2, b2)
        if (px / a2) ** 2 + (py / b2) ** 2 <= 1.0:
            break
    d = np.hypot(mesh.coords[:, 0] - (cx + px), mesh.coords[:, 1] - (cy + py))
    return np.where(d <= radius, amp, 0.0)


def stimulus_centre_ball(mesh: Mesh, radius: float = 0.1, amp: float = 50.0) -> np.ndarray:
    size = mesh.meta["size"]
    c = np.array(size) / 2.0
    d = np.linalg.norm(mesh.coords - c, axis=1)
    return np.where(d <= radius, amp, 0.0)


def batched_slices(count: int = 64, seed: int = 2026, min_k: int = 4, max_k: int = 32,
                   step: int = 32):
    """Seeded uneven 2D torso slices: side 1 + step*k nodes, k ~ U{min_k..max_k},
    ellipse semi-axes ~ U(1.5, 3.5) cm clipped to fit the 10 cm box with a
    0.5 cm margin, fibre angle ~ U(0, 90) deg, stimulus disc seeded per slice."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(count):
        k = int(rng.integers(min_k, max_k + 1))
        n = 1 + step * k
        a = float(min(rng.uniform(1.5, 3.5), 4.5))
        b = float(min(rng.uniform(1.5, 3.5), 4.5))
        fib = float(rng.uniform(0.0, 90.0))
        out.append(dict(n=n, semi_axes=(a, b), fibre_deg=fib, stim_seed=seed + s))
    return out
