"""One mesh assembled in parts (fem3_assemble_part) and summed over ranks.

CPU (gloo, world size 2, torch.distributed.run on 127.0.0.1): the sum all-reduce of
distributed.sum_parts.  GPU: the parts of every axis's transverse bins add up to the whole
matrix (one process, 1 to 3 parts), and two gloo ranks - both on the one device, their
kernels independent of each other - each assemble their part and all-reduce it on the
host: every rank then holds the one-rank matrix (1e-12) and the oracle's (1e-10)."""
import json
import os
import socket
import subprocess
import sys
import textwrap

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run_ranks(tmp_path, body, nproc=2, timeout=600):
    script = tmp_path / "ranks.py"
    script.write_text(textwrap.dedent(f"""
        import json, sys
        sys.path.insert(0, {ROOT!r})
        import numpy as np
        import torch
        import torch.distributed as dist
        dist.init_process_group("gloo")
        rank, world = dist.get_rank(), dist.get_world_size()
        out = {str(tmp_path)!r}
    """) + textwrap.dedent(body) + "\ndist.destroy_process_group()\n")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node",
           str(nproc), "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           str(script)]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout, env=env)
    assert r.returncode == 0, r.stderr[-3000:]


def test_sum_parts_over_gloo_ranks(tmp_path):
    pytest.importorskip("torch.distributed")
    _run_ranks(tmp_path, """
        from paper_1811_03339_gb300 import distributed
        part = torch.arange(12, dtype=torch.float64).reshape(3, 4) * (rank + 1)
        total = distributed.sum_parts(part.clone())
        np.save(out + f"/sum{rank}.npy", total.numpy())
    """)
    expect = np.arange(12, dtype=np.float64).reshape(3, 4) * 3
    for r in range(2):
        assert np.array_equal(np.load(tmp_path / f"sum{r}.npy"), expect)


@pytest.mark.gpu
def test_parts_add_up_to_the_whole_matrix():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import oracle
    from paper_1811_03339_gb300 import fem3, inputs
    mesh = inputs.cube_mesh(7, 0.2, 1)
    alpha, K = (1.3, 1.6, 1.8), (1.0, 2.0, 0.5)
    A_ref = oracle.Oracle.from_mesh(mesh).assemble(alpha, K)
    m = fem3.Mesh(mesh.verts, mesh.tets)
    for precision, bar in (("fp64", 1e-12), ("tf32x3", 1e-6)):
        whole = m.assemble(alpha, K, precision, return_matrix=True).cpu().numpy()
        for nparts in (1, 2, 3):
            S = sum(m.assemble_part(alpha, K, precision, p, nparts).cpu().numpy()
                    for p in range(nparts))
            assert np.abs(S - whole).max() <= bar * np.abs(whole).max(), (precision, nparts)
        part0 = m.assemble_part(alpha, K, precision, 0, 2).cpu().numpy()
        assert 0 < np.abs(part0).max() and np.abs(part0 - whole).max() > 1e-3 * np.abs(whole).max()
    assert np.abs(whole - A_ref).max() <= 2e-6 * np.abs(A_ref).max()
    with pytest.raises(fem3.Fem3Error) as e:
        m.solve(np.ones(mesh.n_nodes))
    assert e.value.code == fem3.FEM3_E_STATE
    m.free()


@pytest.mark.gpu
def test_two_ranks_assemble_one_mesh(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    _run_ranks(tmp_path, """
        torch.cuda.set_device(0)
        from paper_1811_03339_gb300 import distributed, fem3, inputs
        mesh = inputs.cube_mesh(7, 0.2, 1)
        m = fem3.Mesh(mesh.verts, mesh.tets)
        A = distributed.assemble_distributed(m, (1.3, 1.6, 1.8), (1.0, 2.0, 0.5), "fp64",
                                             reduce_on_host=True)
        np.save(out + f"/A{rank}.npy", A.numpy())
        m.free()
    """)
    import oracle
    from paper_1811_03339_gb300 import fem3, inputs
    mesh = inputs.cube_mesh(7, 0.2, 1)
    alpha, K = (1.3, 1.6, 1.8), (1.0, 2.0, 0.5)
    m = fem3.Mesh(mesh.verts, mesh.tets)
    one = m.assemble(alpha, K, "fp64", return_matrix=True).cpu().numpy()
    m.free()
    A_ref = oracle.Oracle.from_mesh(mesh).assemble(alpha, K)
    for r in range(2):
        A = np.load(tmp_path / f"A{r}.npy")
        assert np.abs(A - one).max() <= 1e-12 * np.abs(one).max()
        assert np.abs(A - A_ref).max() <= 1e-10 * np.abs(A_ref).max()
