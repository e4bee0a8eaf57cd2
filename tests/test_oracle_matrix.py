"""Pins of the oracle's Galerkin matrix (Section 2.1) and solve: symmetry, positivity, the
integer-order limit, the template superset of the pattern (Section 2.3) and its density
(Table 1), the manufactured solution's convergence order (Section 3) and the adjoint."""
import math

import numpy as np
import pytest

from oracle import cholesky, chol_solve, solve, riesz_scale
from paper_1811_03339_gb300 import inputs

AFF = ((1.0, 0.3, 0.0), (0.0, 1.0, 0.2), (0.0, 0.0, 0.7))


@pytest.mark.parametrize("n,jit,aff,alpha", [
    (4, 0.0, None, (1.5, 1.5, 1.5)),
    (4, 0.2, None, (1.3, 1.6, 1.8)),
    (3, 0.15, AFF, (1.2, 1.5, 1.9)),
])
def test_symmetric_positive_definite(oracle_for, n, jit, aff, alpha):
    mesh, o = oracle_for(n, jit, 1, aff)
    A = o.assemble(alpha, (1.0, 2.0, 0.5))
    assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0.0


def _p1_laplacian(mesh, o, K):
    """Textbook P1 stiffness sum_T |T| sum_i K_i d_i lambda_a d_i lambda_b, gradients from
    the inverse of the edge matrix (numpy), restricted to interior vertices."""
    A = np.zeros((o.n_dof, o.n_dof))
    for t in range(mesh.n_tets):
        V = mesh.verts[mesh.tets[t]]
        E = (V[1:] - V[0]).T                        # columns v_k - v_0
        G = np.linalg.inv(E)                        # rows: grad lambda_1..3
        grads = np.vstack([-G.sum(axis=0), G])
        vol = abs(np.linalg.det(E)) / 6
        for a in range(4):
            ja = o.dof[mesh.tets[t, a]]
            if ja < 0:
                continue
            for b in range(4):
                jb = o.dof[mesh.tets[t, b]]
                if jb < 0:
                    continue
                A[ja, jb] += vol * sum(K[i] * grads[a, i] * grads[b, i] for i in range(3))
    return A


@pytest.mark.parametrize("n,jit", [(3, 0.0), (4, 0.2)])
def test_integer_order_limit_is_p1_laplacian(oracle_for, n, jit):
    """alpha = 2: s = -1/2, D_L^1 = d/dx, D_R^1 = -d/dx, so A is the anisotropic P1
    Laplacian (the integer-order problem of Table 4)."""
    mesh, o = oracle_for(n, jit, 2)
    K = (1.0, 2.0, 0.5)
    A = o.assemble((2.0, 2.0, 2.0), K)
    ref = _p1_laplacian(mesh, o, K)
    assert np.abs(A - ref).max() <= 1e-12 * np.abs(ref).max()


def _template(mesh, o):
    """T_jk = 1 iff for some axis i the transverse bounding boxes (coordinates != i) of
    the element patches of j and k overlap (closed intervals)."""
    lo = np.full((mesh.n_nodes, 3), np.inf)
    hi = np.full((mesh.n_nodes, 3), -np.inf)
    V = mesh.verts[mesh.tets]
    tlo, thi = V.min(axis=1), V.max(axis=1)
    for k in range(4):
        np.minimum.at(lo, mesh.tets[:, k], tlo)
        np.maximum.at(hi, mesh.tets[:, k], thi)
    dofs = np.nonzero(o.dof >= 0)[0]
    lo, hi = lo[dofs], hi[dofs]
    T = np.zeros((len(dofs), len(dofs)), dtype=bool)
    for i in range(3):
        ok = np.ones_like(T)
        for c in range(3):
            if c == i:
                continue
            ok &= (lo[:, None, c] <= hi[None, :, c]) & (lo[None, :, c] <= hi[:, None, c])
        T |= ok
    return T


@pytest.mark.parametrize("n,jit", [(8, 0.0), (7, 0.2)])
def test_pattern_within_template(oracle_for, n, jit):
    mesh, o = oracle_for(n, jit, 6)
    A = o.assemble((1.4, 1.6, 1.8), (1.0, 1.0, 1.0))
    T = _template(mesh, o)
    assert not np.any((A != 0) & ~T)
    # the template is not trivially full at this size
    assert T.mean() < 0.8


def test_density_scales_like_inverse_square(oracle_for):
    """Table 1: in 3-D the fractional matrix has density O(1/N^2)."""
    dens = []
    ns = (6, 9, 12)
    for n in ns:
        mesh, o = oracle_for(n, 0.0, 0)
        A = o.assemble((1.5, 1.5, 1.5), (1.0, 1.0, 1.0))
        dens.append(np.count_nonzero(np.abs(A) > 1e-14 * np.abs(A).max()) / A.size)
    slope = np.polyfit(np.log(ns), np.log(dens), 1)[0]
    assert -2.6 < slope < -1.5, (dens, slope)


def _l2_error(mesh, o, u):
    full = np.zeros(mesh.n_nodes)
    full[o.dof >= 0] = u[o.dof[o.dof >= 0]]
    a, b = (5 + 3 * 5 ** 0.5) / 20, (5 - 5 ** 0.5) / 20
    lam = np.full((4, 4), b)
    np.fill_diagonal(lam, a)
    uh = (full[mesh.tets][:, None, :] * lam[None]).sum(-1).ravel()
    return math.sqrt(float((o.gw * (uh - inputs.manufactured_u(o.gp)) ** 2).sum()))


def test_manufactured_solution_converges(oracle_for):
    """u = prod x_i^2 (1-x_i)^2 on the unit cube: L2 error of order close to 2
    (Section 3 cites order 2 and observes 1.6-1.95)."""
    alpha, K = (1.5, 1.5, 1.5), (1.0, 1.0, 1.0)
    errs = []
    ns = (4, 8)
    for n in ns:
        mesh, o = oracle_for(n, 0.0, 0)
        A = o.assemble(alpha, K)
        u = solve(A, o.load(inputs.nodal_source(mesh, alpha, K)))
        errs.append(_l2_error(mesh, o, u))
    order = math.log(errs[0] / errs[1]) / math.log(ns[1] / ns[0])
    assert order > 1.4, (errs, order)


def test_cholesky_solve_matches_numpy(oracle_for):
    mesh, o = oracle_for(5, 0.2, 8)
    A = o.assemble((1.3, 1.6, 1.8), (1.0, 2.0, 0.5))
    Lc = cholesky(A)
    assert np.abs(Lc @ Lc.T - A).max() <= 1e-13 * np.abs(A).max()
    assert np.all(np.triu(Lc, 1) == 0)
    b = np.random.default_rng(0).standard_normal((o.n_dof, 3))
    x = chol_solve(Lc, b)
    assert np.abs(A @ x - b).max() <= 1e-10 * np.abs(b).max()


def test_cholesky_reports_non_spd_column():
    from oracle import OracleError
    A = np.eye(4)
    A[2, 2] = -1.0
    with pytest.raises(OracleError) as ei:
        cholesky(A)
    assert ei.value.column == 2


def test_load_vector_is_p1_mass(oracle_for):
    """b = M f with the exact P1 mass matrix |T|/20 (1 + delta_ab)."""
    mesh, o = oracle_for(3, 0.2, 4)
    f = np.random.default_rng(2).standard_normal(mesh.n_nodes)
    ref = np.zeros(o.n_dof)
    for t in range(mesh.n_tets):
        for a in range(4):
            j = o.dof[mesh.tets[t, a]]
            if j < 0:
                continue
            for c in range(4):
                ref[j] += o.vol[t] / 20 * (2.0 if a == c else 1.0) * f[mesh.tets[t, c]]
    assert np.abs(o.load(f) - ref).max() < 1e-15 * mesh.n_tets


def test_adjoint_matches_central_differences(oracle_for):
    """dJ/dK_i and dJ/df of J = 0.5 ||u(K, f) - u_obs||^2 against central differences."""
    mesh, o = oracle_for(3, 0.2, 5)
    alpha = (1.3, 1.6, 1.8)
    K = np.array([1.0, 2.0, 0.5])
    f = inputs.nodal_source(mesh, alpha, K) + 0.1
    u_true = solve(o.assemble(alpha, K), o.load(f))
    u_obs = inputs.noisy_observation(u_true, 0.01, 3) + 0.05 * np.abs(u_true).max()
    J, dK, df, _ = o.adjoint(alpha, K, f, u_obs)

    def Jof(Kv, fv):
        u = solve(o.assemble(alpha, Kv), o.load(fv))
        return 0.5 * float(np.dot(u - u_obs, u - u_obs))

    h = 1e-6
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        fd = (Jof(K + e, f) - Jof(K - e, f)) / (2 * h)
        assert abs(fd - dK[i]) <= 1e-6 * abs(dK[i]) + 1e-14, (i, fd, dK[i])
    for node in (0, 13, 31):
        e = np.zeros_like(f)
        e[node] = h
        fd = (Jof(K, f + e) - Jof(K, f - e)) / (2 * h)
        assert abs(fd - df[node]) <= 1e-6 * abs(df[node]) + 1e-14, (node, fd, df[node])


def test_riesz_scale():
    assert riesz_scale(2.0) == pytest.approx(-0.5, abs=1e-15)
    assert riesz_scale(1.5) < 0


def test_gauss_point_subsets_sum_to_the_assembly(oracle_for):
    """The element sum over a partition of the Gauss points (three interleaved subsets and a
    permuted order) adds up to the whole assembly: the bounded-sample timing of the oracle
    runs the same arithmetic as the full assembly."""
    mesh, o = oracle_for(4, 0.2, 3, None)
    alpha, K = (1.3, 1.6, 1.8), (1.0, 2.0, 0.5)
    A = o.assemble(alpha, K)
    perm = np.random.default_rng(0).permutation(o.n_gp)
    S = np.zeros_like(A)
    for part in (perm[0::3], perm[1::3], perm[2::3]):
        o.assemble_gps(alpha, K, part, S)
    assert np.abs(S - A).max() <= 1e-13 * np.abs(A).max()
    # one Gauss point alone is a rank-2 symmetric update of the matrix
    one = o.assemble_gps(alpha, K, [5])
    assert np.abs(one - one.T).max() <= 1e-15 * np.abs(one).max()
    assert np.linalg.matrix_rank(one, tol=1e-10 * np.abs(one).max()) <= 6


def test_gauss_point_slices_on_threads_sum_to_the_assembly(oracle_for):
    """Slices of the Gauss points assembled at once on four threads, one oracle call per
    thread into its own matrix (as the bench's all-core CPU leg runs it), add up to the
    whole assembly: the oracle's calls share no mutable state."""
    from concurrent.futures import ThreadPoolExecutor
    mesh, o = oracle_for(4, 0.2, 3, None)
    alpha, K = (1.3, 1.6, 1.8), (1.0, 2.0, 0.5)
    A = o.assemble(alpha, K)
    parts = np.array_split(np.arange(o.n_gp, dtype=np.int64), 4)
    with ThreadPoolExecutor(4) as ex:
        mats = list(ex.map(lambda p: o.assemble_gps(alpha, K, p), parts))
    S = sum(mats)
    assert np.abs(S - A).max() <= 1e-13 * np.abs(A).max()
    # each slice alone is what the same call makes on this thread
    for p, Mp in zip(parts, mats):
        assert np.array_equal(Mp, o.assemble_gps(alpha, K, p))
