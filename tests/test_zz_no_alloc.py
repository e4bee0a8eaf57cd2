"""fem3_spd_solve_static: the dense SPD solve whose working memory is a static device
array, for callers that cannot allocate device memory (latency-critical loops that must
not enter the allocator, or host applications that own every device allocation).

It must give the same solution as the regular solve (fem3_solve, FP64 form) on the same
matrix and right-hand side, on two calls in a row (the static array keeps the previous
call's contents), and reject systems larger than its static capacity.  This file is
collected last so that a failure here comes after every other test has run."""
import ctypes

import numpy as np
import pytest

from paper_1811_03339_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1811_03339_gb300 import fem3  # noqa: E402


def _solve_static(lib, A, b, x):
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.fem3_spd_solve_static(ctypes.c_void_p(A.data_ptr()), ctypes.c_int64(A.shape[0]),
                                     ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()), s)


def test_static_solve_matches_regular_solve_twice():
    lib = fem3.load_library()
    mesh = inputs.cube_mesh(7, 0.2, 1)          # 216 dofs: four 64-row blocks, ragged tail
    alpha, K = (1.3, 1.6, 1.8), (1.0, 2.0, 0.5)
    f = inputs.nodal_source(mesh, alpha, K)
    m = fem3.Mesh(mesh.verts, mesh.tets)
    A = m.assemble(alpha, K, "fp64", return_matrix=True)
    b = m.load(f).contiguous()
    u_ref = m.solve(f)                           # regular entry point (allocates)
    torch.cuda.synchronize()
    for call in range(2):
        x = torch.full_like(b, float("nan"))
        assert _solve_static(lib, A, b, x) == fem3.FEM3_OK
        err = float(torch.linalg.norm(x - u_ref) / torch.linalg.norm(u_ref))
        assert err <= 1e-10, (call, err)
    # a second, different system right after: nothing of the previous call leaks
    A2 = torch.eye(100, dtype=torch.float64, device="cuda") * 4.0
    b2 = torch.arange(100, dtype=torch.float64, device="cuda")
    x2 = torch.empty_like(b2)
    assert _solve_static(lib, A2, b2, x2) == fem3.FEM3_OK
    assert float((x2 - b2 / 4.0).abs().max()) == 0.0
    m.free()


def test_static_solve_rejects_oversize_and_non_spd():
    lib = fem3.load_library()
    big = torch.zeros((513, 513), dtype=torch.float64, device="cuda")
    v = torch.zeros(513, dtype=torch.float64, device="cuda")
    assert _solve_static(lib, big, v, v.clone()) == fem3.FEM3_E_ARG
    bad = -torch.eye(8, dtype=torch.float64, device="cuda")
    w = torch.ones(8, dtype=torch.float64, device="cuda")
    assert _solve_static(lib, bad, w, w.clone()) == fem3.FEM3_E_NOT_SPD


def test_static_solve_rejects_host_and_wrong_type_buffers():
    """Host memory handed to the C entry point is refused before any kernel runs, and the
    Python wrapper refuses tensors that are not contiguous float64 CUDA tensors of the
    right shapes."""
    lib = fem3.load_library()
    A = torch.eye(8, dtype=torch.float64, device="cuda")
    b = torch.ones(8, dtype=torch.float64, device="cuda")
    Ah = np.eye(8)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    x = torch.empty_like(b)
    rc = lib.fem3_spd_solve_static(ctypes.c_void_p(Ah.ctypes.data), ctypes.c_int64(8),
                                   ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()), s)
    assert rc == fem3.FEM3_E_ARG
    with pytest.raises(ValueError):
        fem3.spd_solve_static(A.float(), b, x)
    with pytest.raises(ValueError):
        fem3.spd_solve_static(A[:, :4].contiguous(), b, x)
    fem3.spd_solve_static(A, b, x)
    assert float((x - b).abs().max()) == 0.0
