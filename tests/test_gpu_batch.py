"""Batched assembly and solve (fem3_batch_*): every mesh of a batch gives the result of
the single-mesh path, which is itself pinned to the oracle."""
import numpy as np
import pytest

import oracle
from paper_1811_03339_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1811_03339_gb300 import fem3  # noqa: E402


def _batch_case(seed=0):
    rng = np.random.default_rng(seed)
    ns = [3, 5, 2, 4, 6]
    meshes = [inputs.cube_mesh(n, 0.2, seed + i) for i, n in enumerate(ns)]
    alpha = rng.uniform(1.1, 1.9, size=(len(ns), 3))
    K = rng.uniform(0.5, 2.0, size=(len(ns), 3))
    fs = [rng.standard_normal((m.n_nodes, 4)) for m in meshes]
    return meshes, alpha, K, fs


@pytest.mark.parametrize("precision", ["fp64", "tf32x3", "fp32", "bf16x3"])
def test_batch_matches_single_mesh_and_oracle(precision):
    meshes, alpha, K, fs = _batch_case()
    b = fem3.Batch([(m.verts, m.tets) for m in meshes])
    for rep in range(2):                       # second run: factorisation from its graph
        us = b.run(alpha, K, fs, precision, tol=1e-13)
        for i, m in enumerate(meshes):
            single = fem3.Mesh(m.verts, m.tets)
            single.assemble(alpha[i], K[i], precision)
            u_single = single.solve(fs[i], tol=1e-13).cpu().numpy()
            single.free()
            u = us[i].cpu().numpy()
            assert u.shape == u_single.shape
            tol = 1e-10 if precision == "fp64" else 1e-9
            assert np.linalg.norm(u - u_single) <= tol * np.linalg.norm(u_single), (i, rep)
    for i in (0, 3):
        o = oracle.Oracle.from_mesh(meshes[i])
        u_ref = oracle.solve(o.assemble(alpha[i], K[i]), o.load(fs[i]))
        u = us[i].cpu().numpy()
        assert np.linalg.norm(u - u_ref) <= 1e-8 * np.linalg.norm(u_ref), i
    assert all(r <= 1e-13 for r in b.resid) or precision == "fp64"
    b.free()


def test_batch_rejects_bad_arguments():
    meshes, alpha, K, fs = _batch_case(1)
    b = fem3.Batch([(m.verts, m.tets) for m in meshes[:2]])
    with pytest.raises(fem3.Fem3Error) as e:
        b.run(np.full((2, 3), 2.5), K[:2], fs[:2])
    assert e.value.code == fem3.FEM3_E_ARG
    b.free()


@pytest.mark.parametrize("precision", ["tf32x3", "fp64"])
def test_batch_assembly_replays_as_one_graph(precision):
    """The second run with the same orders, coefficients, precision and right-hand-side
    arrays captures the batch's assembly and factorisation as one CUDA graph, later runs
    replay it; every run matches the single-mesh results, a change of alpha captures again.
    One mesh has 4,096 dofs, so its factorisation (blocked, tensor-core trailing updates on
    a side stream) is inside the graph too."""
    rng = np.random.default_rng(5)
    meshes = [inputs.cube_mesh(n, 0.2, 30 + n) for n in (4, 17, 6)]
    alpha = rng.uniform(1.1, 1.9, size=(3, 3))
    K = rng.uniform(0.5, 2.0, size=(3, 3))
    fs = [rng.standard_normal((m.n_nodes, 3)) for m in meshes]
    fs_dev = [torch.from_numpy(np.asfortranarray(f)).cuda() for f in fs]   # stable pointers

    def singles(al):
        out = []
        for i, m in enumerate(meshes):
            s = fem3.Mesh(m.verts, m.tets)
            s.assemble(al[i], K[i], precision)
            out.append(s.solve(fs[i], tol=1e-13).cpu().numpy())
            s.free()
        return out

    b = fem3.Batch([(m.verts, m.tets) for m in meshes])
    assert b.n_dof[1] == 4096
    tol = 1e-10 if precision == "fp64" else 1e-9
    ref = singles(alpha)
    for rep in range(4):
        us = b.run(alpha, K, fs_dev, precision, tol=1e-13)
        for i in range(3):
            u = us[i].cpu().numpy()
            assert np.linalg.norm(u - ref[i]) <= tol * np.linalg.norm(ref[i]), (rep, i)
    assert b.graph_launches() == 3          # run 2 captured and launched, runs 3-4 replayed
    alpha2 = alpha.copy()
    alpha2[1] = (1.7, 1.4, 1.25)
    ref2 = singles(alpha2)
    for rep in range(2):
        us = b.run(alpha2, K, fs_dev, precision, tol=1e-13)
        for i in range(3):
            u = us[i].cpu().numpy()
            assert np.linalg.norm(u - ref2[i]) <= tol * np.linalg.norm(ref2[i]), (rep, i)
    assert b.graph_launches() == 5
    b.free()
