"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module generates problem data only: meshes, coefficients and right-hand sides.
It contains none of the finite element method itself (no barycentric maps, no path
walk, no derivative tables, no assembly, no solve), so that the CUDA path and the
oracle can both consume its output without sharing any of the method's arithmetic.

Workloads (the paper measures on a ball mesh it does not publish, Section 3 and
Table 4; these synthetic convex meshes stand in for it):

* ``cube_mesh(n)`` - the unit cube cut into n^3 cells, each cell split into the six
  Kuhn (Freudenthal) tetrahedra that share the cell's main diagonal.  The split is
  conforming across cells.
* ``jitter`` moves every interior vertex by a seeded uniform offset in
  [-jitter*h, jitter*h]^3 (h = 1/n), so the mesh is unstructured but the boundary
  of the cube stays exact and every tetrahedron keeps its orientation for
  jitter < 0.25.
* ``affine`` maps every vertex by x -> M x afterwards (a convex parallelepiped).
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

# The configurations the library is measured and tested on.
CUBE4 = dict(n=4, jitter=0.0, seed=0, affine=None,
             alpha=(1.5, 1.5, 1.5), K=(1.0, 1.0, 1.0))
CUBE16_JITTER = dict(n=16, jitter=0.2, seed=1, affine=None,
                     alpha=(1.3, 1.6, 1.8), K=(1.0, 2.0, 0.5))
PARALLELEPIPED24 = dict(n=24, jitter=0.15, seed=2,
                        affine=((1.0, 0.3, 0.0), (0.0, 1.0, 0.2), (0.0, 0.0, 0.7)),
                        alpha=(1.2, 1.5, 1.9), K=(1.0, 1.0, 1.0))
# the same parallelepiped recipe at 16^3 cells (3,375 dofs, the same 17 right-hand sides):
# kernel profiles that need a few GB on the device at most
PARALLELEPIPED16 = dict(PARALLELEPIPED24, n=16)

WORKLOADS = {
    "cube4": CUBE4,
    "cube16_jitter": CUBE16_JITTER,
    "parallelepiped24": PARALLELEPIPED24,
    "parallelepiped16": PARALLELEPIPED16,
}


@dataclass
class Mesh:
    verts: np.ndarray          # float64 [n_nodes, 3], row-major
    tets: np.ndarray           # int32 [n_tets, 4]
    n: int = 0                 # cells per cube edge (0 if not a cube mesh)
    jitter: float = 0.0
    affine: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.verts.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])


def _node_id(n: int, ix, iy, iz):
    return ix + (n + 1) * (iy + (n + 1) * iz)


def cube_mesh(n: int, jitter: float = 0.0, seed: int = 0, affine=None) -> Mesh:
    """Kuhn-split cube mesh with n^3 cells and 6 n^3 tetrahedra.

    Node (ix, iy, iz) has index ix + (n+1)(iy + (n+1) iz).  For cell (cx, cy, cz) and each
    permutation s of the three axes (in itertools order) the tetrahedron is
    c, c + e_s0, c + e_s0 + e_s1, c + (1,1,1).
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    if not (0.0 <= jitter < 0.25):
        raise ValueError("jitter must lie in [0, 0.25) to keep tetrahedra valid")
    h = 1.0 / n
    g = np.arange(n + 1, dtype=np.float64) * h
    iz, iy, ix = np.meshgrid(np.arange(n + 1), np.arange(n + 1), np.arange(n + 1),
                             indexing="ij")
    verts = np.stack([g[ix.ravel()], g[iy.ravel()], g[iz.ravel()]], axis=1)

    tets = []
    cz, cy, cx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    cx, cy, cz = cx.ravel(), cy.ravel(), cz.ravel()
    unit = np.eye(3, dtype=np.int64)
    # tets ordered cell-major, permutation-minor
    per_cell = []
    for perm in itertools.permutations(range(3)):
        o0 = np.zeros(3, dtype=np.int64)
        o1 = o0 + unit[perm[0]]
        o2 = o1 + unit[perm[1]]
        o3 = np.ones(3, dtype=np.int64)
        per_cell.append([o0, o1, o2, o3])
    for offs in per_cell:
        tets.append(np.stack([_node_id(n, cx + o[0], cy + o[1], cz + o[2]) for o in offs],
                             axis=1))
    tets = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)

    if jitter > 0.0:
        ixr, iyr, izr = ix.ravel(), iy.ravel(), iz.ravel()
        interior = (ixr > 0) & (ixr < n) & (iyr > 0) & (iyr < n) & (izr > 0) & (izr < n)
        rng = np.random.default_rng(seed)
        off = rng.uniform(-jitter * h, jitter * h, size=(int(interior.sum()), 3))
        verts[interior] += off

    aff = None
    if affine is not None:
        aff = np.asarray(affine, dtype=np.float64).reshape(3, 3)
        verts = verts @ aff.T
    return Mesh(verts=np.ascontiguousarray(verts), tets=np.ascontiguousarray(tets), n=n,
                jitter=jitter, affine=aff, meta=dict(seed=seed))


def workload_mesh(name: str) -> Mesh:
    w = WORKLOADS[name]
    return cube_mesh(w["n"], w["jitter"], w["seed"], w["affine"])


# ----------------------------------------------------------------------------------
# Right-hand sides.  The manufactured problem is written for the unit cube (a_i = 0,
# b_i = 1 on every axis-parallel line), u(x) = prod_i g(x_i), g(t) = t^2 (1-t)^2.
# ----------------------------------------------------------------------------------

_G_COEF = {2: 1.0, 3: -2.0, 4: 1.0}      # g(t) = t^2 - 2 t^3 + t^4


def g_profile(t):
    t = np.asarray(t, dtype=np.float64)
    return t * t * (1.0 - t) ** 2


def manufactured_u(x: np.ndarray) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    return g_profile(x[..., 0]) * g_profile(x[..., 1]) * g_profile(x[..., 2])


def _rl_left_g(t, order):
    """Left Riemann-Liouville derivative on [0, t] of g, term by term from the power rule."""
    t = np.asarray(t, dtype=np.float64)
    out = np.zeros_like(t)
    for m, c in _G_COEF.items():
        out += c * math.gamma(m + 1) / math.gamma(m + 1 - order) * np.power(t, m - order)
    return out


def manufactured_f(x: np.ndarray, alpha, K) -> np.ndarray:
    """Source f = sum_i K_i s_i (D_L^{alpha_i} + D_R^{alpha_i}) u with s_i = 1/(2 cos(pi alpha_i/2)).

    This is the right-hand side of -sum_i K_i d^{alpha_i} u / d|x_i|^{alpha_i} = f for the
    Riesz derivative d^a/d|x|^a = -(D_L^a + D_R^a) / (2 cos(pi a / 2)).  Because g is
    symmetric about 1/2, the right derivative at t equals the left derivative at 1 - t.
    """
    x = np.asarray(x, dtype=np.float64)
    gx = [g_profile(x[..., i]) for i in range(3)]
    f = np.zeros(x.shape[:-1])
    for i in range(3):
        a = float(alpha[i])
        s = 1.0 / (2.0 * math.cos(math.pi * a / 2.0))
        t = x[..., i]
        # clip to the closed cube; nodes on the boundary have t in {0, 1}
        with np.errstate(divide="ignore", invalid="ignore"):
            dl = _rl_left_g(np.clip(t, 0.0, 1.0), a)
            dr = _rl_left_g(np.clip(1.0 - t, 0.0, 1.0), a)
        dl = np.where(np.isfinite(dl), dl, 0.0)
        dr = np.where(np.isfinite(dr), dr, 0.0)
        other = np.ones_like(t)
        for k in range(3):
            if k != i:
                other = other * gx[k]
        f += float(K[i]) * s * (dl + dr) * other
    return f


def nodal_source(mesh: Mesh, alpha, K) -> np.ndarray:
    """Manufactured f sampled at the nodes (its P1 interpolant), float64 [n_nodes]."""
    return manufactured_f(mesh.verts, alpha, K)


def workload_rhs(name: str, mesh: Mesh) -> np.ndarray:
    """Nodal right-hand sides of a named workload, float64 [n_nodes] or [n_nodes, nrhs].

    The cubes take the manufactured source of their alpha and K (one column).  The
    parallelepiped (whose chords do not run from 0 to 1, so the manufactured profile does
    not apply) takes f = 1 and 16 seeded N(0, 1) columns (seed 11): 17 columns."""
    w = WORKLOADS[name]
    if w["affine"] is None:
        return nodal_source(mesh, w["alpha"], w["K"])
    return np.concatenate([np.ones((mesh.n_nodes, 1)), random_rhs(mesh.n_nodes, 16, seed=11)],
                          axis=1)


def random_rhs(n_nodes: int, nrhs: int, seed: int) -> np.ndarray:
    """Seeded N(0,1) nodal right-hand sides, float64 column-major [n_nodes, nrhs] (as F-order)."""
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.standard_normal((n_nodes, nrhs)))


def noisy_observation(u: np.ndarray, level: float, seed: int) -> np.ndarray:
    """u_obs = u + level * max|u| * xi, xi ~ N(0,1) seeded."""
    rng = np.random.default_rng(seed)
    u = np.asarray(u, dtype=np.float64)
    return u + level * float(np.max(np.abs(u))) * rng.standard_normal(u.shape)


def batch_specs(n_meshes: int = 64, seed: int = 3, nmin: int = 6, nmax: int = 20):
    """Uneven batch: per mesh a cube side n ~ U{nmin..nmax} and alpha_i ~ U(1.1, 1.9)."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(nmin, nmax + 1, size=n_meshes)
    alphas = rng.uniform(1.1, 1.9, size=(n_meshes, 3))
    return [dict(n=int(ns[m]), alpha=tuple(float(a) for a in alphas[m])) for m in range(n_meshes)]
