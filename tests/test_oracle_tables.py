"""Pins of the oracle's derivative tables (Section 2.1).

* Linear functions are reproduced exactly by P1, so the all-nodes tables applied to the
  nodal values of p(x) = 1, x_i, x_k must equal the closed-form Riemann-Liouville
  derivatives of p on the chord [a_i(x), b_i(x)] (power rule of the fractional calculus).
* One basis function along one line is checked against eq. "def" itself: the fractional
  integral by adaptive quadrature (scipy, algebraic weight) and its x-derivative by a
  finite difference - no use of the closed form.
"""
import math

import numpy as np
import pytest

AFF = ((1.0, 0.3, 0.0), (0.0, 1.0, 0.2), (0.0, 0.0, 0.7))


def _rl_linear(a, b, x, c0, c1, gamma, side):
    """Closed-form RL derivative of order gamma of p(y) = c0 + c1 * y at y = x on [a, b]."""
    if side == "L":
        d = x - a
        # D_L (c0 + c1 a + c1 (y - a))
        val = c1 * d ** (1 - gamma) / math.gamma(2 - gamma)
        if gamma < 1:
            val += (c0 + c1 * a) * d ** (-gamma) / math.gamma(1 - gamma)
        return val
    d = b - x
    # D_R (c0 + c1 b - c1 (b - y))
    val = -c1 * d ** (1 - gamma) / math.gamma(2 - gamma)
    if gamma < 1:
        val += (c0 + c1 * b) * d ** (-gamma) / math.gamma(1 - gamma)
    return val


@pytest.mark.parametrize("gamma", [0.55, 0.75, 0.95, 1.0])
@pytest.mark.parametrize("n,jit,aff", [(3, 0.0, None), (4, 0.2, None), (3, 0.15, AFF)])
def test_tables_reproduce_linear_functions(oracle_for, gamma, n, jit, aff):
    mesh, o = oracle_for(n, jit, 9, aff)
    rng = np.random.default_rng(1)
    z = mesh.verts
    for g in rng.choice(o.n_gp, size=10, replace=False):
        x = o.gp[g]
        for axis in range(3):
            _, _, _, rl, _ = o.walk(g, axis, -1)
            _, _, _, rr, _ = o.walk(g, axis, +1)
            a, b = x[axis] - rl, x[axis] + rr
            L = o.table_row(g, axis, -1, gamma, all_nodes=True)
            R = o.table_row(g, axis, +1, gamma, all_nodes=True)
            other = [k for k in range(3) if k != axis][0]
            tests = [
                (np.ones(mesh.n_nodes), 1.0, 0.0),            # p = 1
                (z[:, axis], 0.0, 1.0),                         # p = x_i
                (z[:, other], x[other], 0.0),                   # p = x_k, const on the line
                (2.0 - 3.0 * z[:, axis] + 0.5 * z[:, other], 2.0 + 0.5 * x[other], -3.0),
            ]
            for nodal, c0, c1 in tests:
                for tab, side in ((L, "L"), (R, "R")):
                    want = _rl_linear(a, b, x[axis], c0, c1, gamma, side)
                    got = float(tab @ nodal)
                    assert abs(got - want) <= 1e-11 * max(1.0, abs(want)), (g, axis, side, got, want)


def test_interior_rows_drop_only_the_boundary_term(oracle_for):
    """Dof rows equal the all-nodes rows restricted to interior vertices minus the
    boundary term, which is zero for interior basis functions (phi_j(a) = 0)."""
    mesh, o = oracle_for(4, 0.2, 3)
    interior = o.dof >= 0
    for g in (0, 101, 777):
        for axis in range(3):
            for d in (-1, 1):
                full = o.table_row(g, axis, d, 0.8, all_nodes=True)
                dofs = o.table_row(g, axis, d, 0.8, all_nodes=False)
                assert np.allclose(full[interior], dofs, rtol=0, atol=1e-13)


def _phi_along_line(mesh, o, node, x, axis, ys):
    """Value of the P1 basis function of `node` at points x + (y - x_axis) e_axis, by
    locating each point in every tet (brute force)."""
    out = np.zeros(len(ys))
    for m, y in enumerate(ys):
        p = x.copy()
        p[axis] = y
        lam = np.einsum("tij,j->ti", o.M, np.r_[1.0, p])
        t = int(np.argmax(lam.min(axis=1)))
        k = np.nonzero(mesh.tets[t] == node)[0]
        out[m] = lam[t, k[0]] if len(k) else 0.0
    return out


def test_left_derivative_against_definition(oracle_for):
    """D_L^gamma phi_j(x) = d/dx I^{1-gamma} phi_j(x) (eq. "def"), integral by quadrature."""
    integrate = pytest.importorskip("scipy.integrate")
    mesh, o = oracle_for(3, 0.2, 5)
    gamma = 0.7
    for g, axis in ((40, 0), (211, 1), (333, 2)):
        L = o.table_row(g, axis, -1, gamma)
        x = o.gp[g].copy()
        _, _, _, rl, _ = o.walk(g, axis, -1)
        a = x[axis] - rl
        nodes = np.nonzero(o.dof >= 0)[0]
        j = int(np.argmax(np.abs(L)))
        node = nodes[j]
        # breakpoints of phi along the line: path segment ends (kinks of the P1 function)
        st, r0, r1, _, _ = o.walk(g, axis, -1)
        kinks = sorted(x[axis] - r1)

        def frac_integral(xx):
            f = lambda y: _phi_along_line(mesh, o, node, x, axis, np.array([y]))[0]
            edges = [a] + [k for k in kinks if a < k < xx] + [xx]
            val = sum(_piece(f, lo, hi, xx, gamma, integrate)
                      for lo, hi in zip(edges[:-1], edges[1:]))
            return val / math.gamma(1 - gamma)

        h = 2e-5
        F = [frac_integral(x[axis] + s * h) for s in (-2, -1, 1, 2)]
        deriv = (F[0] - 8 * F[1] + 8 * F[2] - F[3]) / (12 * h)
        assert abs(deriv - L[j]) < 2e-6 * max(1.0, abs(L[j])), (g, axis, deriv, L[j])


def _piece(f, lo, hi, xx, gamma, integrate):
    """int_lo^hi (xx - y)^(-gamma) f(y) dy; singular weight only on the last piece."""
    if hi == xx:
        return integrate.quad(f, lo, hi, weight="alg", wvar=(0.0, -gamma), limit=200,
                              epsabs=1e-14, epsrel=1e-12)[0]
    g = lambda y: (xx - y) ** (-gamma) * f(y)
    return integrate.quad(g, lo, hi, limit=200, epsabs=1e-14, epsrel=1e-12)[0]
