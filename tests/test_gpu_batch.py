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
