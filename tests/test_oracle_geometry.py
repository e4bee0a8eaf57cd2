"""Pins of the oracle's mesh records (Section 2.2 volume coordinates, Section 2.1 quadrature)."""
import os

import numpy as np
import pytest

from paper_1811_03339_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
AFF = ((1.0, 0.3, 0.0), (0.0, 1.0, 0.2), (0.0, 0.0, 0.7))


@pytest.mark.parametrize("n,jit,aff", [(4, 0.0, None), (5, 0.2, None), (4, 0.15, AFF)])
def test_barycentric_map_reproduces_vertices(oracle_for, n, jit, aff):
    mesh, o = oracle_for(n, jit, 7, aff)
    P = np.concatenate([np.ones((mesh.n_tets, 1, 4)),
                        np.transpose(mesh.verts[mesh.tets], (0, 2, 1))], axis=1)
    # lambda(v_k) = e_k  <=>  M_T P_T = I
    err = np.abs(np.einsum("tij,tjk->tik", o.M, P) - np.eye(4)).max()
    assert err < 1e-12
    # gradients of the four volume coordinates sum to zero, constants to one
    assert np.abs(o.M[:, :, 1:].sum(axis=1)).max() < 1e-10
    assert np.abs(o.M[:, :, 0].sum(axis=1) - 1.0).max() < 1e-12


@pytest.mark.parametrize("n,jit,aff", [(4, 0.0, None), (6, 0.2, None), (4, 0.15, AFF)])
def test_volumes_sum_to_domain(oracle_for, n, jit, aff):
    mesh, o = oracle_for(n, jit, 7, aff)
    expect = 1.0 if aff is None else abs(np.linalg.det(np.asarray(aff)))
    assert abs(o.vol.sum() - expect) < 1e-13
    assert np.all(o.vol > 0)
    assert abs(o.gw.sum() - expect) < 1e-13


@pytest.mark.parametrize("n,jit", [(3, 0.0), (5, 0.2)])
def test_face_neighbours(oracle_for, n, jit):
    mesh, o = oracle_for(n, jit, 3)
    T = mesh.n_tets
    # a Kuhn cube has 2 boundary triangles per cell face on the 6 sides
    assert int((o.nbr < 0).sum()) == 12 * n * n
    for t in range(T):
        for k in range(4):
            u = o.nbr[t, k]
            if u < 0:
                continue
            # symmetric, and the shared face is the one opposite vertex k of t
            assert t in o.nbr[u]
            shared = set(mesh.tets[t]) - {mesh.tets[t, k]}
            assert shared <= set(mesh.tets[u])
    # dofs: interior vertices in ascending node order
    ix = np.arange(mesh.n_nodes)
    i = ix % (n + 1)
    j = (ix // (n + 1)) % (n + 1)
    k = ix // (n + 1) ** 2
    interior = (i > 0) & (i < n) & (j > 0) & (j < n) & (k > 0) & (k < n)
    assert np.array_equal(o.dof >= 0, interior)
    assert np.array_equal(o.dof[interior], np.arange(interior.sum()))


def test_quadrature_exact_for_quadratics(oracle_for):
    # the 4-point rule is exact up to degree 2 on every tet, hence on the unit cube
    mesh, o = oracle_for(5, 0.2, 11)
    x, y, z = o.gp.T
    w = o.gw
    assert abs((w * x * x).sum() - 1 / 3) < 1e-13
    assert abs((w * x * y).sum() - 1 / 4) < 1e-13
    assert abs((w * y * z).sum() - 1 / 4) < 1e-13
    assert abs((w * z).sum() - 1 / 2) < 1e-13
    # Gauss points lie strictly inside their tets with barycentric (a,b,b,b)
    a, b = (5 + 3 * 5 ** 0.5) / 20, (5 - 5 ** 0.5) / 20
    lam = np.einsum("tij,tqj->tqi", o.M,
                    np.concatenate([np.ones((mesh.n_tets, 4, 1)), o.gp.reshape(-1, 4, 3)], -1))
    expect = np.full((4, 4), b)
    np.fill_diagonal(expect, a)
    assert np.abs(lam - expect[None]).max() < 1e-12


def _golden_fig_vc():
    rows = []
    with open(os.path.join(HERE, "golden", "volume_coordinates_fig_vc.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            rows.append((parts[0], [int(v) for v in parts[1:5]], int(parts[5])))
    return rows


def test_volume_coordinate_zero_pattern_matches_fig_vc(oracle_for):
    """Points on each vertex/edge/face of a tet have the zero pattern the paper tabulates."""
    mesh, o = oracle_for(3, 0.2, 5)
    rng = np.random.default_rng(0)
    names = "ABCD"
    for t in (0, 17, 100):
        V = mesh.verts[mesh.tets[t]]
        for pos, mask, dim in _golden_fig_vc():
            idx = [names.index(c) for c in pos]
            wts = rng.uniform(0.2, 1.0, size=len(idx))
            wts /= wts.sum()
            x = (wts[:, None] * V[idx]).sum(0)
            lam = o.M[t] @ np.r_[1.0, x]
            zero = (np.abs(lam) < 1e-12).astype(int)
            assert list(zero) == mask, (pos, lam)
            assert 3 - int(zero.sum()) == dim
