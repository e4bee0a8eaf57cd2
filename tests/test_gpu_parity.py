"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars: path tet ids bit-exact; path ends and FP64 tables within 1e-10 relative; FP64
matrix and solution within 1e-10; mixed (FP32 contraction and factor + FP64 refinement)
matrix within 1e-4 and solution within 1e-8 of the oracle's FP64 solution.
"""
import numpy as np
import pytest

import oracle
from paper_1811_03339_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1811_03339_gb300 import fem3  # noqa: E402

AFF = ((1.0, 0.3, 0.0), (0.0, 1.0, 0.2), (0.0, 0.0, 0.7))
_CACHE = {}


def _case(name):
    """(mesh, oracle, alpha, K) for a named small case."""
    if name in _CACHE:
        return _CACHE[name]
    specs = {
        "cube4": (4, 0.0, 0, None, (1.5, 1.5, 1.5), (1.0, 1.0, 1.0)),
        "cube3_jitter": (3, 0.2, 5, None, (1.3, 1.6, 1.8), (1.0, 2.0, 0.5)),
        "cube7_jitter": (7, 0.2, 1, None, (1.3, 1.6, 1.8), (1.0, 2.0, 0.5)),
        "ppd5": (5, 0.15, 2, AFF, (1.2, 1.5, 1.9), (1.0, 1.0, 1.0)),
        "cube16_jitter": (16, 0.2, 1, None, (1.3, 1.6, 1.8), (1.0, 2.0, 0.5)),
        # no jitter: Gauss-point lines cross edges and vertices exactly (ties and in-face
        # exits that the walk's FP32 exit filter must leave to the FP64 step)
        "cube6": (6, 0.0, 0, None, (1.4, 1.7, 1.2), (1.0, 1.0, 1.0)),
        # small cells far from the origin: large |x| against the cell size in the filter's
        # error bounds
        "shifted_cube4": (4, 0.2, 7, None, (1.3, 1.6, 1.8), (1.0, 2.0, 0.5)),
    }
    n, jit, seed, aff, alpha, K = specs[name]
    mesh = inputs.cube_mesh(n, jit, seed, aff)
    if name == "shifted_cube4":
        mesh.verts = np.ascontiguousarray(mesh.verts * 0.1 + np.array([10.0, -5.0, 3.0]))
    _CACHE[name] = (mesh, oracle.Oracle.from_mesh(mesh), alpha, K)
    return _CACHE[name]


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("name", ["cube4", "cube3_jitter", "ppd5"])
def test_mesh_records(name):
    mesh, o, _, _ = _case(name)
    m = fem3.Mesh(mesh.verts, mesh.tets)
    assert m.n_dof == o.n_dof and m.n_gp == o.n_gp
    assert np.array_equal(m.dof_of_node, o.dof)
    m.free()


@pytest.mark.parametrize("name", ["cube4", "cube3_jitter", "ppd5", "cube7_jitter", "cube6",
                                  "shifted_cube4"])
def test_paths_bit_exact(name):
    mesh, o, _, _ = _case(name)
    m = fem3.Mesh(mesh.verts, mesh.tets)
    rng = np.random.default_rng(0)
    gps = np.arange(o.n_gp) if o.n_gp <= 1536 else np.sort(rng.choice(o.n_gp, 1500, replace=False))
    # path ends come from lambda_k(x_g) = c_k + grad lambda_k . x_g, whose FP64 rounding scales
    # with |x|, not with the mesh span (the shifted mesh lies 10 spans from the origin)
    tol_r = 1e-12 * max(o.span, float(np.abs(mesh.verts).max()))
    for axis in range(3):
        for d in (-1, 1):
            tet, r0, r1, ns = m.paths(axis, d, gps)
            tet, r0, r1, ns = tet.cpu().numpy(), r0.cpu().numpy(), r1.cpu().numpy(), ns.cpu().numpy()
            for l, g in enumerate(gps):
                st, a, b, _, _ = o.walk(int(g), axis, d)
                assert ns[l] == len(st), (g, axis, d)
                assert np.array_equal(tet[l, :ns[l]], st), (g, axis, d)
                assert np.abs(r0[l, :ns[l]] - a).max(initial=0) <= tol_r
                assert np.abs(r1[l, :ns[l]] - b).max(initial=0) <= tol_r
    m.free()


@pytest.mark.parametrize("name", ["cube4", "cube3_jitter", "ppd5", "cube7_jitter", "cube6",
                                  "shifted_cube4"])
def test_tables_fp64(name):
    mesh, o, alpha, K = _case(name)
    m = fem3.Mesh(mesh.verts, mesh.tets)
    m.assemble(alpha, K, "fp64")
    m.sync()
    rng = np.random.default_rng(1)
    gps = np.sort(rng.choice(o.n_gp, min(o.n_gp, 300), replace=False))
    for axis in range(3):
        gamma = alpha[axis] / 2
        L, R = o.tables(axis, gamma, gps)
        gl = m.table_rows(axis, -1, gps).cpu().numpy()
        gr = m.table_rows(axis, +1, gps).cpu().numpy()
        assert _rel(gl, L) <= 1e-10
        assert _rel(gr, R) <= 1e-10
        # structural: the same nonzero support (exact zeros outside the path's dofs)
        assert np.array_equal(gl != 0, L != 0)
    m.free()


@pytest.mark.parametrize("name", ["cube4", "cube3_jitter", "ppd5", "cube7_jitter"])
def test_assemble_and_solve_fp64(name):
    mesh, o, alpha, K = _case(name)
    m = fem3.Mesh(mesh.verts, mesh.tets)
    A = m.assemble(alpha, K, "fp64", return_matrix=True).cpu().numpy()
    A_ref = o.assemble(alpha, K)
    assert _rel(A, A_ref) <= 1e-10
    f = inputs.nodal_source(mesh, alpha, K) if mesh.affine is None else np.ones(mesh.n_nodes)
    u = m.solve(f).cpu().numpy()
    u_ref = oracle.solve(A_ref, o.load(f))
    assert np.linalg.norm(u - u_ref) <= 1e-10 * np.linalg.norm(u_ref)
    assert m.resid <= 1e-12
    m.free()


@pytest.mark.parametrize("precision", ["fp32", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("name", ["cube4", "cube7_jitter", "ppd5"])
def test_mixed_with_refinement(name, precision):
    mesh, o, alpha, K = _case(name)
    m = fem3.Mesh(mesh.verts, mesh.tets)
    A = m.assemble(alpha, K, precision, return_matrix=True).cpu().numpy()
    A_ref = o.assemble(alpha, K)
    assert _rel(A, A_ref) <= 1e-4
    rng = np.random.default_rng(3)
    f = rng.standard_normal((mesh.n_nodes, 3))
    u = m.solve(f, tol=1e-13).cpu().numpy()
    u_ref = oracle.solve(A_ref, o.load(f))
    assert np.linalg.norm(u - u_ref) <= 1e-8 * np.linalg.norm(u_ref)
    assert m.iters >= 1 and m.resid <= 1e-13
    m.free()


@pytest.mark.parametrize("name", ["cube7_jitter", "ppd5"])
def test_tensor_core_split_products_reach_fp32_accuracy(name):
    """TF32 x 3 (hi*hi + hi*lo + lo*hi) keeps about 22 significant bits: the matrix is
    within 2e-6 of the FP64 oracle (a single TF32 product would be ~1e-3 off)."""
    mesh, o, alpha, K = _case(name)
    m = fem3.Mesh(mesh.verts, mesh.tets)
    A = m.assemble(alpha, K, "tf32x3", return_matrix=True).cpu().numpy()
    m.sync()
    A_ref = o.assemble(alpha, K)
    assert _rel(A, A_ref) <= 2e-6
    # symmetric up to FP32 summation order
    assert np.abs(A - A.T).max() <= 1e-6 * np.abs(A).max()
    m.free()


@pytest.mark.parametrize("name", ["cube7_jitter", "ppd5"])
def test_bf16_split_products_accuracy(name):
    """BF16 x 3 keeps about 16 significant bits (3 * 2^-16 per product): the matrix is
    within 1e-4 of the FP64 oracle, measurably less accurate than TF32 x 3 but far better
    than one BF16 product (2^-8); the two tensor-core forms agree to the BF16 bound."""
    mesh, o, alpha, K = _case(name)
    m = fem3.Mesh(mesh.verts, mesh.tets)
    Ab = m.assemble(alpha, K, "bf16x3", return_matrix=True).cpu().numpy()
    At = m.assemble(alpha, K, "tf32x3", return_matrix=True).cpu().numpy()
    m.sync()
    A_ref = o.assemble(alpha, K)
    eb, et = _rel(Ab, A_ref), _rel(At, A_ref)
    assert eb <= 1e-4
    assert et < eb
    assert _rel(Ab, At) <= 1e-4
    assert np.abs(Ab - Ab.T).max() <= 1e-6 * np.abs(Ab).max()
    m.free()


def test_tensor_core_tile_widths_and_tuner():
    """Both tile widths of the tensor-core contraction give the same matrix (to FP32
    summation order) within the TF32x3 bound of the oracle; with no width forced, the first
    contraction of a size class runs the tuner and later meshes of the class reuse its
    choice."""
    mesh, o, alpha, K = _case("cube7_jitter")
    A_ref = o.assemble(alpha, K)
    As = {}
    for tile in (128, 256):
        m = fem3.Mesh(mesh.verts, mesh.tets, tc_tile=tile)
        As[tile] = m.assemble(alpha, K, "tf32x3", return_matrix=True).cpu().numpy()
        m.sync()
        assert m.tc_tile() == (tile, False)
        assert _rel(As[tile], A_ref) <= 2e-6
        m.free()
    assert _rel(As[128], As[256]) <= 1e-6
    chosen = []
    for rep in range(2):
        m = fem3.Mesh(mesh.verts, mesh.tets)
        A = m.assemble(alpha, K, "bf16x3", return_matrix=True).cpu().numpy()
        m.sync()
        tile, tuned = m.tc_tile()
        assert tile in (128, 256)
        if rep == 1:
            assert not tuned
        chosen.append(tile)
        assert _rel(A, A_ref) <= 1e-4
        m.free()
    assert chosen[0] == chosen[1]
    with pytest.raises(fem3.Fem3Error):
        fem3.Mesh(mesh.verts, mesh.tets, tc_tile=100)


@pytest.mark.parametrize("precision", ["fp64", "tf32x3", "bf16x3"])
def test_adjoint_matches_oracle(precision):
    """dJ/dK and dJ/df of J = 0.5 ||u(K, f) - u_obs||^2 against the oracle's adjoint (which is
    itself pinned to central differences)."""
    mesh, o, alpha, K = _case("cube7_jitter")
    f = inputs.nodal_source(mesh, alpha, K) + 0.1
    u_true = oracle.solve(o.assemble(alpha, K), o.load(f))
    u_obs = inputs.noisy_observation(u_true, 0.01, 3)
    J, dK_ref, df_ref, _ = o.adjoint(alpha, K, f, u_obs)
    m = fem3.Mesh(mesh.verts, mesh.tets)
    m.assemble(alpha, K, precision)
    u = m.solve(f, tol=1e-13)
    dK, dJdf = m.adjoint(u, torch.from_numpy(u_obs).cuda(), tol=1e-13)
    assert np.abs(dK - dK_ref).max() <= 1e-8 * np.abs(dK_ref).max()
    assert _rel(dJdf.cpu().numpy(), df_ref) <= 1e-8
    m.free()


@pytest.mark.parametrize("precision", ["fp64", "tf32x3"])
def test_reassemble_same_mesh(precision):
    """Three assembles with different K on one handle: the second and third factorisations
    run from the captured factorisation graph and must match the oracle like the first."""
    mesh, o, alpha, _ = _case("cube7_jitter")
    f = inputs.nodal_source(mesh, alpha, (1.0, 1.0, 1.0))
    m = fem3.Mesh(mesh.verts, mesh.tets)
    for K in ((1.0, 2.0, 0.5), (0.7, 1.0, 1.3), (2.0, 0.5, 1.0)):
        m.assemble(alpha, K, precision)
        u = m.solve(f, tol=1e-13).cpu().numpy()
        u_ref = oracle.solve(o.assemble(alpha, K), o.load(f))
        assert np.linalg.norm(u - u_ref) <= 1e-8 * np.linalg.norm(u_ref), K
    m.free()


@pytest.mark.parametrize("precision", ["fp64", "tf32x3"])
@pytest.mark.parametrize("nrhs", [16, 17, 21, 30])
def test_many_right_hand_sides(precision, nrhs):
    """Columns go through the wavefront solve up to 24 at a time and through the table
    operator in groups of up to 17 (while 13 or more are left), 8, 4 or 1 (16: one group of
    17 slots; 21: 17 + 4; 30: 17 + 13 and 24 + 6 in the solve); every column must match the
    oracle.  The default bins here fit the list apply, which these groups then run."""
    mesh, o, alpha, K = _case("cube7_jitter")
    f = np.random.default_rng(nrhs).standard_normal((mesh.n_nodes, nrhs))
    m = fem3.Mesh(mesh.verts, mesh.tets)
    assert m.apply_lists()
    m.assemble(alpha, K, precision)
    u = m.solve(f, tol=1e-13).cpu().numpy()
    u_ref = oracle.solve(o.assemble(alpha, K), o.load(f))
    err = np.linalg.norm(u - u_ref, axis=0) / np.linalg.norm(u_ref, axis=0)
    assert err.max() <= (1e-10 if precision == "fp64" else 1e-8), err
    m.free()


@pytest.mark.parametrize("precision", ["tf32x3", "bf16x3"])
def test_dense_apply_for_wide_bins(precision):
    """Bins too wide for the list apply (17 x 8 B x (D + G) above its 112 KB of shared memory,
    or more than 256 template rows in a bin) take the dense-block apply: the refined solution still
    matches the oracle, 17 columns."""
    mesh, o, alpha, K = _case("cube7_jitter")
    m = fem3.Mesh(mesh.verts, mesh.tets, bin_scale=3.0)
    st = [m.bin_stats(a) for a in range(3)]
    md, mg = max(x["max_dof"] for x in st), max(x["max_gp"] for x in st)
    assert not m.apply_lists(), (md, mg)
    assert 17 * 8 * (md + mg) > 112 * 1024 or md > 256, (md, mg)
    m.assemble(alpha, K, precision)
    f = np.random.default_rng(17).standard_normal((mesh.n_nodes, 17))
    u = m.solve(f, tol=1e-13).cpu().numpy()
    u_ref = oracle.solve(o.assemble(alpha, K), o.load(f))
    err = np.linalg.norm(u - u_ref, axis=0) / np.linalg.norm(u_ref, axis=0)
    assert err.max() <= 1e-8, err
    assert m.resid <= 1e-13
    m.free()


def test_load_vector():
    mesh, o, alpha, K = _case("cube3_jitter")
    m = fem3.Mesh(mesh.verts, mesh.tets)
    f = np.random.default_rng(4).standard_normal((mesh.n_nodes, 2))
    b = m.load(f).cpu().numpy()
    assert _rel(b, o.load(f)) <= 1e-13
    m.free()


def test_full_size_cube16_fp64_matrix():
    """16^3 jittered cube (24,576 tets, 3,375 dofs): whole FP64 matrix and solution, then
    the whole tensor-core matrices element by element with each tile width forced: at this
    size many bins hold more than 128 (and 256) dofs, so the multi-tile register epilogue
    (m and n tiles > 0) is compared with the oracle, not only the one-tile shared-memory
    epilogue of the small meshes."""
    mesh, o, alpha, K = _case("cube16_jitter")
    m = fem3.Mesh(mesh.verts, mesh.tets)
    A = m.assemble(alpha, K, "fp64", return_matrix=True).cpu().numpy()
    A_ref = o.assemble(alpha, K)
    assert _rel(A, A_ref) <= 1e-10
    f = inputs.nodal_source(mesh, alpha, K)
    u = m.solve(f).cpu().numpy()
    u_ref = oracle.solve(A_ref, o.load(f))
    assert np.linalg.norm(u - u_ref) <= 1e-10 * np.linalg.norm(u_ref)
    assert max(m.bin_stats(a)["max_dof"] for a in range(3)) > 128
    # mixed form reaches the FP64 solution to 1e-8
    m.assemble(alpha, K, "tf32x3")
    u2 = m.solve(f, tol=1e-13).cpu().numpy()
    assert np.linalg.norm(u2 - u_ref) <= 1e-8 * np.linalg.norm(u_ref)
    m.free()
    for tile in (128, 256):
        mt = fem3.Mesh(mesh.verts, mesh.tets, tc_tile=tile)
        for precision, bar in (("tf32x3", 2e-6), ("bf16x3", 1e-4)):
            At = mt.assemble(alpha, K, precision, return_matrix=True).cpu().numpy()
            mt.sync()
            assert mt.tc_tile() == (tile, False)
            assert _rel(At, A_ref) <= bar, (tile, precision, _rel(At, A_ref))
        mt.free()


@pytest.mark.parametrize("tile", [128, 256])
@pytest.mark.parametrize("precision", ["tf32x3", "bf16x3"])
def test_tensor_core_bins_over_one_tile(tile, precision):
    """A small mesh with wide transverse bins (bin_scale 2.5 on the 10^3 jittered cube):
    bins of more than 128 dofs take the register epilogue over several (m, n) tiles, with
    n tiles > 0 at the 128 width; the whole matrix must match the oracle to the split's bar
    and be symmetric to FP32 summation order."""
    mesh = inputs.cube_mesh(10, 0.2, 4)
    o = oracle.Oracle.from_mesh(mesh)
    alpha, K = (1.3, 1.6, 1.8), (1.0, 2.0, 0.5)
    m = fem3.Mesh(mesh.verts, mesh.tets, bin_scale=2.5, tc_tile=tile)
    assert max(m.bin_stats(a)["max_dof"] for a in range(3)) > 128
    A = m.assemble(alpha, K, precision, return_matrix=True).cpu().numpy()
    m.sync()
    A_ref = o.assemble(alpha, K)
    bar = 2e-6 if precision == "tf32x3" else 1e-4
    assert _rel(A, A_ref) <= bar, _rel(A, A_ref)
    assert np.abs(A - A.T).max() <= 1e-6 * np.abs(A).max()
    f = np.random.default_rng(5).standard_normal((mesh.n_nodes, 2))
    u = m.solve(f, tol=1e-13).cpu().numpy()
    u_ref = oracle.solve(A_ref, o.load(f))
    assert np.linalg.norm(u - u_ref) <= 1e-8 * np.linalg.norm(u_ref)
    m.free()


@pytest.mark.parametrize("alpha", [(2.0, 2.0, 2.0), (2.0, 1.5, 2.0)])
def test_integer_order_axes(alpha):
    """alpha_i = 2 (Table 4's integer-order case): order-1 one-sided derivatives, the slope
    on the Gauss point's tet (the oracle is pinned there to the textbook P1 stiffness
    matrix); all-integer and mixed integer/fractional orders against the oracle."""
    mesh, o, _, K = _case("cube7_jitter")
    A_ref = o.assemble(alpha, K)
    f = inputs.nodal_source(mesh, (1.5, 1.5, 1.5), K) + 0.3
    u_ref = oracle.solve(A_ref, o.load(f))
    m = fem3.Mesh(mesh.verts, mesh.tets)
    A = m.assemble(alpha, K, "fp64", return_matrix=True).cpu().numpy()
    assert _rel(A, A_ref) <= 1e-10
    u = m.solve(f).cpu().numpy()
    assert np.linalg.norm(u - u_ref) <= 1e-10 * np.linalg.norm(u_ref)
    At = m.assemble(alpha, K, "tf32x3", return_matrix=True).cpu().numpy()
    assert _rel(At, A_ref) <= 2e-6
    u = m.solve(f, tol=1e-13).cpu().numpy()
    assert np.linalg.norm(u - u_ref) <= 1e-8 * np.linalg.norm(u_ref)
    m.free()


_PPD24 = {}


def _ppd24():
    """The 24^3 parallelepiped (82,944 tets, 12,167 dofs) with its oracle matrix (about a
    minute of single-threaded host work, computed once per session)."""
    if not _PPD24:
        w = inputs.PARALLELEPIPED24
        mesh = inputs.workload_mesh("parallelepiped24")
        o = oracle.Oracle.from_mesh(mesh)
        _PPD24.update(mesh=mesh, o=o, w=w, A_ref=o.assemble(w["alpha"], w["K"]))
    return _PPD24


def test_full_size_parallelepiped24_paths_and_tables():
    """Paths in both directions and table rows at full size against the oracle."""
    P = _ppd24()
    mesh, o, w = P["mesh"], P["o"], P["w"]
    alpha, K = w["alpha"], w["K"]
    m = fem3.Mesh(mesh.verts, mesh.tets)
    m.assemble(alpha, K, "bf16x3")
    m.sync()
    rng = np.random.default_rng(7)
    gps = np.sort(rng.choice(o.n_gp, 240, replace=False))
    tol_r = 1e-12 * max(o.span, float(np.abs(mesh.verts).max()))
    for axis in range(3):
        for d in (-1, 1):
            tet, r0, r1, ns = m.paths(axis, d, gps)
            tet, r0, r1, ns = (tet.cpu().numpy(), r0.cpu().numpy(), r1.cpu().numpy(),
                               ns.cpu().numpy())
            for l, g in enumerate(gps):
                st, a, b, _, _ = o.walk(int(g), axis, d)
                assert ns[l] == len(st), (g, axis, d)
                assert np.array_equal(tet[l, :ns[l]], st), (g, axis, d)
                assert np.abs(r0[l, :ns[l]] - a).max(initial=0) <= tol_r
                assert np.abs(r1[l, :ns[l]] - b).max(initial=0) <= tol_r
        L, R = o.tables(axis, alpha[axis] / 2, gps[:80])
        assert _rel(m.table_rows(axis, -1, gps[:80]).cpu().numpy(), L) <= 1e-10
        assert _rel(m.table_rows(axis, +1, gps[:80]).cpu().numpy(), R) <= 1e-10
    m.free()


def test_full_size_parallelepiped24_matrix_and_solution():
    """The configuration's own form (BF16 split products, FP32 accumulation, FP32 factor,
    FP64 refinement) at full size: the whole matrix element by element against the oracle
    (1e-4) and the FP64 form's matrix (1e-10); the solution of f = 1 and of 16 seeded normal
    right-hand sides against a solve of the oracle's matrix (1e-8 after refinement, 1e-10
    for the FP64 form).  The reference solve factors the oracle's matrix with LAPACK
    (a library Cholesky as one step; the oracle's own textbook factorisation would take
    several minutes at n = 12,167)."""
    P = _ppd24()
    mesh, o, w, A_ref = P["mesh"], P["o"], P["w"], P["A_ref"]
    alpha, K = w["alpha"], w["K"]
    m = fem3.Mesh(mesh.verts, mesh.tets)
    A = m.assemble(alpha, K, "bf16x3", return_matrix=True).cpu().numpy()
    assert _rel(A, A_ref) <= 1e-4, _rel(A, A_ref)
    assert max(m.bin_stats(a)["max_dof"] for a in range(3)) > 128
    F = np.concatenate([np.ones((mesh.n_nodes, 1)),
                        inputs.random_rhs(mesh.n_nodes, 16, seed=11)], axis=1)
    u = m.solve(F, tol=1e-12).cpu().numpy()
    assert m.iters >= 1 and m.resid <= 1e-12
    scipy_linalg = pytest.importorskip("scipy.linalg")
    cf = scipy_linalg.cho_factor(A_ref, lower=True)
    u_ref = scipy_linalg.cho_solve(cf, o.load(F))
    err = np.linalg.norm(u - u_ref, axis=0) / np.linalg.norm(u_ref, axis=0)
    assert err.max() <= 1e-8, err
    # at the bench's tolerance the late sweeps update the residual from the correction in
    # FP32: the true residual against the oracle's matrix stays within 10% of tol, and the
    # reported one agrees with it
    b_ref = o.load(F)
    u10 = m.solve(F, tol=1e-10).cpu().numpy()
    true_res = (np.linalg.norm(b_ref - A_ref @ u10, axis=0) / np.linalg.norm(b_ref, axis=0)).max()
    assert true_res <= 1.1e-10, true_res
    assert abs(true_res - m.resid) <= 0.05e-10 + 0.1 * true_res, (true_res, m.resid)
    del A
    A64 = m.assemble(alpha, K, "fp64", return_matrix=True).cpu().numpy()
    assert _rel(A64, A_ref) <= 1e-10
    del A64
    u64 = m.solve(F[:, :2]).cpu().numpy()
    err64 = np.linalg.norm(u64 - u_ref[:, :2], axis=0) / np.linalg.norm(u_ref[:, :2], axis=0)
    assert err64.max() <= 1e-10, err64
    m.free()


def test_status_codes():
    mesh, o, alpha, K = _case("cube4")
    m = fem3.Mesh(mesh.verts, mesh.tets)
    with pytest.raises(fem3.Fem3Error) as e:
        m.solve(np.ones(mesh.n_nodes))
    assert e.value.code == fem3.FEM3_E_STATE
    with pytest.raises(fem3.Fem3Error) as e:
        m.assemble((0.9, 1.5, 1.5), K)
    assert e.value.code == fem3.FEM3_E_ARG
    with pytest.raises(fem3.Fem3Error) as e:
        m.assemble(alpha, (1.0, -1.0, 1.0))
    assert e.value.code == fem3.FEM3_E_ARG
    m.free()
    # a walk cap of 2 tets cannot reach the boundary: error status, no hang
    m = fem3.Mesh(mesh.verts, mesh.tets, max_steps=2)
    m.assemble(alpha, K)
    with pytest.raises(fem3.Fem3Error) as e:
        m.sync()
    assert e.value.code == fem3.FEM3_E_WALK
    m.free()
    # zero-volume tet
    bad = mesh.tets.copy()
    bad[0, 3] = bad[0, 2]
    with pytest.raises(fem3.Fem3Error) as e:
        fem3.Mesh(mesh.verts, bad)
    assert e.value.code == fem3.FEM3_E_MESH
    # a face shared by three tets
    dup = np.vstack([mesh.tets, mesh.tets[:1]])
    with pytest.raises(fem3.Fem3Error) as e:
        fem3.Mesh(mesh.verts, dup)
    assert e.value.code == fem3.FEM3_E_MESH


def test_no_interior_dofs():
    """One cell: every vertex is on the boundary, n_dof = 0."""
    mesh = inputs.cube_mesh(1)
    m = fem3.Mesh(mesh.verts, mesh.tets)
    assert m.n_dof == 0
    m.assemble((1.5, 1.5, 1.5), (1.0, 1.0, 1.0), "fp64")
    m.sync()
    m.free()


def test_device_inputs_match_host_inputs():
    mesh, o, alpha, K = _case("cube3_jitter")
    mh = fem3.Mesh(mesh.verts, mesh.tets)
    md = fem3.Mesh(torch.from_numpy(mesh.verts).cuda(), torch.from_numpy(mesh.tets).cuda())
    Ah = mh.assemble(alpha, K, "fp64", return_matrix=True)
    Ad = md.assemble(alpha, K, "fp64", return_matrix=True)
    assert _rel(Ad.cpu().numpy(), Ah.cpu().numpy()) <= 1e-14
    mh.free()
    md.free()


def test_contraction_work_counts_the_oracle_nonzeros():
    """fem3_contract_work = sum over axes and Gauss points of 4 nnz(L[g]) nnz(R[g]), the
    nonzeros of the oracle's table rows (the supports agree exactly)."""
    mesh, o, alpha, K = _case("cube7_jitter")
    m = fem3.Mesh(mesh.verts, mesh.tets)
    m.assemble(alpha, K, "tf32x3")
    got = m.contract_work()
    exp = 0
    for axis in range(3):
        L, R = o.tables(axis, alpha[axis] / 2)
        exp += 4 * int(np.sum((L != 0).sum(1).astype(np.int64) * (R != 0).sum(1)))
    assert got == exp
    nnz = sum(int((L != 0).sum() + (R != 0).sum())
              for L, R in (o.tables(a, alpha[a] / 2) for a in range(3)))
    assert m.table_nnz() == nnz
    m.free()


def test_kernel_class_timing():
    """A profiling handle times every launch of each kernel class on the launch stream; the
    walk class is the walk stage's one launch."""
    mesh, o, alpha, K = _case("cube7_jitter")
    m = fem3.Mesh(mesh.verts, mesh.tets, profile=True)
    m.assemble(alpha, K, "tf32x3")
    m.solve(np.ones((mesh.n_nodes, 3)), tol=1e-12)
    k = m.kernel_ms()
    for name in ("walk_tables", "split", "contract", "factor", "chain", "apply"):
        assert k[name][1] >= 1 and k[name][0] > 0.0, name
    assert k["walk_tables"][1] == 1
    assert k["walk_tables"][0] <= m.stage_ms()[2] * 1.01 + 1e-3
    # a new assemble starts the sums again
    m.assemble(alpha, K, "fp64")
    m.sync()
    k2 = m.kernel_ms()
    assert k2["walk_tables"][1] == 1 and k2["apply"][1] == 0
    m.free()


@pytest.mark.parametrize("name,n_cells", [("cube7_jitter", 7), ("cube10", 10), ("cube16_jitter", 16)])
@pytest.mark.parametrize("precision", ["tf32x3", "bf16x3"])
def test_blocked_tensor_core_factorisation(name, n_cells, precision):
    """The blocked FP32 factorisation with tcgen05 TF32 x 3 trailing updates, forced on
    meshes whose dof counts (216, 729, 3,375) end in ragged panels of 88, 89 and 47 columns:
    the refined solution matches the oracle to 1e-8 in as many refinement sweeps (plus one
    at most) as the tile-task factorisation."""
    if name == "cube10":
        mesh = inputs.cube_mesh(10, 0.2, 4)
        o = oracle.Oracle.from_mesh(mesh)
        alpha, K = (1.3, 1.6, 1.8), (1.0, 2.0, 0.5)
    else:
        mesh, o, alpha, K = _case(name)
    f = np.random.default_rng(8).standard_normal((mesh.n_nodes, 3))
    u_ref = oracle.solve(o.assemble(alpha, K), o.load(f))
    sweeps = {}
    for mode in (1, -1):
        m = fem3.Mesh(mesh.verts, mesh.tets, chol_tc=mode)
        m.assemble(alpha, K, precision)
        u = m.solve(f, tol=1e-13).cpu().numpy()
        err = np.linalg.norm(u - u_ref, axis=0) / np.linalg.norm(u_ref, axis=0)
        assert err.max() <= 1e-8, (mode, err)
        sweeps[mode] = m.iters
        m.free()
    assert sweeps[1] <= sweeps[-1] + 1, sweeps


def test_autograd_gradient_at_full_size():
    """The adjoint configuration: the 16^3 jittered cube, J = 0.5 ||u(K, f) - u_obs||^2 with
    u_obs = u(K_true) + 1% seeded noise, K_true = (1, 2, 0.5), f the manufactured source.
    The gradient from torch.autograd through fem3.frac_solve (backward = fem3_vjp) against
    central differences (h = 1e-6 in each K_i; a direction in f, where J is quadratic), each
    J from the GPU's own FP64 solve, and against the oracle's adjoint gradient (itself pinned
    to central differences); the TF32x3 form with refinement against the oracle too."""
    mesh, o, alpha, K = _case("cube16_jitter")
    f_np = inputs.nodal_source(mesh, alpha, K)
    m = fem3.Mesh(mesh.verts, mesh.tets)
    m.assemble(alpha, K, "fp64")
    u_true = m.solve(f_np).cpu().numpy()
    u_obs = inputs.noisy_observation(u_true, 0.01, 3)
    u_obs_t = torch.from_numpy(u_obs).cuda()

    def grads(precision):
        Kt = torch.tensor(K, dtype=torch.float64, requires_grad=True)
        ft = torch.from_numpy(f_np).cuda().requires_grad_(True)
        u = fem3.frac_solve(m, alpha, Kt, ft, precision, tol=1e-13)
        J = 0.5 * ((u - u_obs_t) ** 2).sum()
        J.backward()
        return float(J.detach()), Kt.grad.numpy().copy(), ft.grad.cpu().numpy()

    def J_of(Kv, fv):
        m.assemble(alpha, Kv, "fp64")
        uu = m.solve(fv)
        return 0.5 * float(((uu - u_obs_t) ** 2).sum())

    J0, gK, gf = grads("fp64")
    assert J0 > 0 and np.all(np.isfinite(gK)) and np.all(np.isfinite(gf))
    h = 1e-6
    for i in range(3):
        Kp, Km = list(K), list(K)
        Kp[i] += h
        Km[i] -= h
        fd = (J_of(Kp, f_np) - J_of(Km, f_np)) / (2 * h)
        assert abs(fd - gK[i]) <= 1e-6 * np.abs(gK).max(), (i, fd, gK[i])
    v = np.random.default_rng(9).standard_normal(mesh.n_nodes)
    hf = 1e-3 * np.abs(f_np).max()
    fdv = (J_of(K, f_np + hf * v) - J_of(K, f_np - hf * v)) / (2 * hf)
    assert abs(fdv - float(gf @ v)) <= 1e-7 * abs(float(gf @ v)) + 1e-12 * np.abs(gf).sum()
    Jo, dK_ref, df_ref, _ = o.adjoint(alpha, K, f_np, u_obs)
    assert abs(J0 - Jo) <= 1e-10 * Jo
    assert np.abs(gK - dK_ref).max() <= 1e-8 * np.abs(dK_ref).max()
    assert _rel(gf, df_ref) <= 1e-8
    _, gK32, gf32 = grads("tf32x3")
    assert np.abs(gK32 - dK_ref).max() <= 1e-8 * np.abs(dK_ref).max()
    assert _rel(gf32, df_ref) <= 1e-8
    m.free()


def test_integer_order_fast_path():
    """fem3_assemble_integer (alpha_i = 2, the element-by-element P1 stiffness, no walk)
    equals the oracle's alpha = 2 matrix (pinned to the textbook P1 Laplacian) and the walk
    path's alpha = 2 matrix; its solve and its gradient (element formula for dA/dK_i) match
    the oracle's; it has no tables to export."""
    mesh, o, _, K = _case("cube7_jitter")
    a2 = (2.0, 2.0, 2.0)
    A_ref = o.assemble(a2, K)
    m = fem3.Mesh(mesh.verts, mesh.tets)
    Aw = m.assemble(a2, K, "fp64", return_matrix=True).cpu().numpy()
    A = m.assemble_integer(K, return_matrix=True).cpu().numpy()
    assert _rel(A, A_ref) <= 1e-12
    assert _rel(A, Aw) <= 1e-12
    f = inputs.nodal_source(mesh, (1.5, 1.5, 1.5), K) + 0.3
    u = m.solve(f)
    u_ref = oracle.solve(A_ref, o.load(f))
    assert np.linalg.norm(u.cpu().numpy() - u_ref) <= 1e-10 * np.linalg.norm(u_ref)
    assert m.resid <= 1e-12
    u_obs = inputs.noisy_observation(u_ref, 0.01, 5)
    dK, dJdf = m.adjoint(u, torch.from_numpy(u_obs).cuda())
    _, dK_ref, df_ref, _ = o.adjoint(a2, K, f, u_obs)
    assert np.abs(dK - dK_ref).max() <= 1e-8 * np.abs(dK_ref).max()
    assert _rel(dJdf.cpu().numpy(), df_ref) <= 1e-8
    with pytest.raises(fem3.Fem3Error) as e:
        m.table_rows(0, -1, [0])
    assert e.value.code == fem3.FEM3_E_STATE
    m.free()


def _coef(o):
    """A positive, non-constant coefficient at the oracle's Gauss points."""
    x = o.gp
    return 1.0 + 0.5 * x[:, 0] - 0.3 * x[:, 1] + 0.8 * x[:, 2] ** 2


@pytest.mark.parametrize("name", ["cube7_jitter", "ppd5"])
@pytest.mark.parametrize("axis,alpha,beta,trial_left", [
    (0, 0.3, 0.8, True), (1, 0.75, 0.6, False), (2, 1.0, 0.0, True), (1, 0.0, 0.0, True),
    (2, 0.65, 0.65, False), (0, 1.0, 1.0, True)])
def test_general_form_matches_oracle(name, axis, alpha, beta, trial_left):
    """fem3_assemble_form (one axis term of (c D^alpha u, D^^beta v), unequal orders in
    [0, 1], a variable coefficient at the Gauss points) against Oracle.assemble_form:
    1e-10 in FP64, 2e-6 with TF32 x 3 and 1e-4 with BF16 x 3 split products, FP32 on CUDA
    cores 1e-5; c = None is c = 1."""
    mesh, o, _, _ = _case(name)
    c = _coef(o)
    K_ref = o.assemble_form(axis, alpha, beta, trial_left, c)
    m = fem3.Mesh(mesh.verts, mesh.tets)
    for precision, bar in (("fp64", 1e-10), ("tf32x3", 2e-6), ("bf16x3", 1e-4), ("fp32", 1e-5)):
        K = m.assemble_form(axis, alpha, beta, trial_left, c, precision).cpu().numpy()
        m.sync()
        assert _rel(K, K_ref) <= bar, (precision, _rel(K, K_ref))
    K1 = m.assemble_form(axis, alpha, beta, trial_left, None, "fp64").cpu().numpy()
    assert _rel(K1, o.assemble_form(axis, alpha, beta, trial_left, None)) <= 1e-10
    # the handle holds no operator for a solve afterwards
    with pytest.raises(fem3.Fem3Error) as e:
        m.solve(np.ones(mesh.n_nodes))
    assert e.value.code == fem3.FEM3_E_STATE
    m.free()


def test_general_form_over_many_tiles():
    """Bins of more than 128 dofs (10^3 cube, bin_scale 2.5) on the tensor cores: the
    non-symmetric epilogue over several (m, n) tiles against the oracle; then the Riesz
    assembly on the same handle is unaffected."""
    mesh = inputs.cube_mesh(10, 0.2, 4)
    o = oracle.Oracle.from_mesh(mesh)
    c = _coef(o)
    m = fem3.Mesh(mesh.verts, mesh.tets, bin_scale=2.5)
    K_ref = o.assemble_form(1, 0.35, 0.9, False, c)
    for precision, bar in (("tf32x3", 2e-6), ("bf16x3", 1e-4)):
        K = m.assemble_form(1, 0.35, 0.9, False, c, precision).cpu().numpy()
        assert _rel(K, K_ref) <= bar, (precision, _rel(K, K_ref))
    alpha, K3 = (1.3, 1.6, 1.8), (1.0, 2.0, 0.5)
    A = m.assemble(alpha, K3, "tf32x3", return_matrix=True).cpu().numpy()
    assert _rel(A, o.assemble(alpha, K3)) <= 2e-6
    m.free()


@pytest.mark.parametrize("name", ["cube7_jitter", "ppd5"])
def test_divergence_form_and_gmres(name):
    """Section 3's divergence form with the paper's coefficients (p_i = cos x_i,
    q_i = 1 - cos x_i) and beta = (0.6, 0.7, 0.8): the matrix against
    Oracle.assemble_divergence (1e-10 FP64, 2e-6 TF32 x 3), and the GMRES solve
    (preconditioned by the SPD part's factor) against a LAPACK solve of the oracle's
    matrix and load vector (1e-10 FP64; the TF32 x 3 operator within its own perturbation)."""
    mesh, o, _, _ = _case(name)
    beta = (0.6, 0.7, 0.8)
    x = o.gp
    p = np.stack([np.cos(x[:, i]) for i in range(3)])
    q = 1.0 - p
    A_ref = o.assemble_divergence(beta, p, q)
    f = np.random.default_rng(12).standard_normal((mesh.n_nodes, 2))
    u_ref = np.linalg.solve(A_ref, o.load(f))
    m = fem3.Mesh(mesh.verts, mesh.tets)
    A = m.assemble_divergence(beta, p, q, "fp64", return_matrix=True).cpu().numpy()
    assert _rel(A, A_ref) <= 1e-10
    assert np.abs(A - A.T).max() > 1e-3 * np.abs(A).max()   # really not symmetric
    u = m.solve(f, tol=1e-13).cpu().numpy()
    err = np.linalg.norm(u - u_ref, axis=0) / np.linalg.norm(u_ref, axis=0)
    assert err.max() <= 1e-10, err
    assert 1 <= m.iters <= 60 and m.resid <= 1e-13
    At = m.assemble_divergence(beta, p, q, "tf32x3", return_matrix=True).cpu().numpy()
    assert _rel(At, A_ref) <= 2e-6
    ut = m.solve(f, tol=1e-12).cpu().numpy()
    errt = np.linalg.norm(ut - u_ref, axis=0) / np.linalg.norm(u_ref, axis=0)
    assert errt.max() <= 1e-4, errt
    with pytest.raises(fem3.Fem3Error):
        m.adjoint(torch.from_numpy(u[:, 0].copy()).cuda(), torch.zeros(m.n_dof, dtype=torch.float64, device="cuda"))
    m.free()
