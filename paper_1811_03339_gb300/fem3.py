"""Thin Python binding of libfem3 (argument marshalling only).

Every step of the method runs in the CUDA library; this module converts torch tensors
or numpy arrays into pointers, passes the current torch stream, and turns status codes
into exceptions.  There is no CPU fallback: if the library is missing the calls raise.

The functions mirror the C ABI of ``include/fem3.h`` (``fem3_mesh_upload`` ->
``mesh_upload`` ...); ``Mesh`` wraps a handle for convenience.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build_lib

FEM3_OK = 0
FEM3_E_ARG, FEM3_E_MESH, FEM3_E_WALK, FEM3_E_NOT_SPD = -1, -2, -3, -4
FEM3_E_NO_CONVERGE, FEM3_E_CUDA, FEM3_E_OOM, FEM3_E_STATE, FEM3_E_TEMPLATE = -5, -6, -7, -8, -9

PRECISIONS = {"fp64": 0, "tf32x3": 1, "fp32": 2, "bf16x3": 3}

# every entry point declared in include/fem3.h
SYMBOLS = ("fem3_mesh_upload", "fem3_mesh_info", "fem3_assemble", "fem3_assemble_integer",
           "fem3_assemble_form", "fem3_assemble_divergence", "fem3_assemble_part",
           "fem3_load", "fem3_solve",
           "fem3_adjoint", "fem3_vjp", "fem3_paths", "fem3_table_rows", "fem3_sync", "fem3_stage_ms",
           "fem3_counters", "fem3_bin_stats", "fem3_kernel_ms", "fem3_contract_work",
           "fem3_table_nnz",
           "fem3_tc_tile", "fem3_apply_lists",
           "fem3_last_error",
           "fem3_mesh_free",
           "fem3_spd_solve_static",
           "fem3_batch_create", "fem3_batch_mesh", "fem3_batch_run", "fem3_batch_graph_launches",
           "fem3_batch_free")

_lib = None


class Fem3Error(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"fem3 status {code}: {msg}")
        self.code = code


class Options(C.Structure):
    _fields_ = [("bin_scale", C.c_double), ("max_steps", C.c_int32), ("profile", C.c_int32),
                ("tc_tile", C.c_int32), ("chol_tc", C.c_int32)]


def lib_path() -> str:
    return _build_lib.LIB


def load_library(build_if_missing: bool = True):
    """Load libfem3.so (compiling it first if it is missing or stale and nvcc exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build_lib.up_to_date():
        _build_lib.build()
    if not os.path.exists(_build_lib.LIB):
        raise RuntimeError("libfem3.so is not built; call __graft_entry__.build()")
    lib = C.CDLL(_build_lib.LIB)
    p, i64, i32, dbl, ci = C.c_void_p, C.c_int64, C.c_int32, C.c_double, C.c_int
    sig = {
        "fem3_mesh_upload": [p, i64, p, i64, C.POINTER(Options), p, C.POINTER(p)],
        "fem3_mesh_info": [p, C.POINTER(i64), C.POINTER(i64), p],
        "fem3_assemble": [p, p, p, ci, p, p],
        "fem3_assemble_integer": [p, p, p, p],
        "fem3_assemble_form": [p, ci, dbl, dbl, ci, p, ci, p, p],
        "fem3_assemble_part": [p, p, p, ci, ci, ci, p, p],
        "fem3_assemble_divergence": [p, p, p, p, ci, p, p],
        "fem3_load": [p, p, ci, p, p],
        "fem3_solve": [p, p, ci, dbl, ci, p, C.POINTER(ci), C.POINTER(dbl), p],
        "fem3_adjoint": [p, p, p, dbl, ci, p, p, p],
        "fem3_vjp": [p, p, p, dbl, ci, p, p, p],
        "fem3_paths": [p, ci, ci, p, i64, ci, p, p, p, p, p],
        "fem3_table_rows": [p, ci, ci, p, i64, p, p],
        "fem3_sync": [p, p],
        "fem3_stage_ms": [p, ci, C.POINTER(C.c_float)],
        "fem3_counters": [p, C.POINTER(i64), C.POINTER(dbl), C.POINTER(i64), C.POINTER(i64)],
        "fem3_tc_tile": [p, C.POINTER(C.c_int32), C.POINTER(C.c_int32)],
        "fem3_apply_lists": [p, C.POINTER(C.c_int32)],
        "fem3_bin_stats": [p, ci, C.POINTER(i64), C.POINTER(i64), C.POINTER(i32), C.POINTER(i32)],
        "fem3_kernel_ms": [p, ci, C.POINTER(C.c_float), C.POINTER(i32)],
        "fem3_contract_work": [p, C.POINTER(dbl), p],
        "fem3_table_nnz": [p, C.POINTER(i64), p],
        "fem3_last_error": [C.c_char_p, C.c_size_t],
        "fem3_mesh_free": [p],
        "fem3_spd_solve_static": [p, i64, p, p, p],
        "fem3_batch_create": [ci, p, p, p, p, C.POINTER(Options), p, C.POINTER(p)],
        "fem3_batch_mesh": [p, ci, C.POINTER(p)],
        "fem3_batch_run": [p, p, p, ci, p, ci, dbl, ci, p, p, p, p],
        "fem3_batch_graph_launches": [p, C.POINTER(i64)],
        "fem3_batch_free": [p],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = None if name in ("fem3_mesh_free", "fem3_batch_free") else ci
    _lib = lib
    return lib


def _check(code: int):
    if code != FEM3_OK:
        buf = C.create_string_buffer(512)
        _lib.fem3_last_error(buf, 512)
        raise Fem3Error(code, buf.value.decode(errors="replace"))


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _ptr(x):
    """Pointer of a torch tensor (any device) or a numpy array (host)."""
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"] or x.flags["F_CONTIGUOUS"]
        return C.c_void_p(x.ctypes.data)
    assert x.is_contiguous(), "tensor must be contiguous"
    return C.c_void_p(x.data_ptr())


# ---------------------------------------------------------------------------------
# functions with the C ABI's names
# ---------------------------------------------------------------------------------
def mesh_upload(verts, tets, bin_scale: float = 0.5, max_steps: int = 0, profile: bool = False,
                stream=None, tc_tile: int = 0, chol_tc: int = 0):
    lib = load_library()
    opt = Options(bin_scale, max_steps, 1 if profile else 0, tc_tile, chol_tc)
    h = C.c_void_p()
    _check(lib.fem3_mesh_upload(_ptr(verts), int(verts.shape[0]), _ptr(tets), int(tets.shape[0]),
                                C.byref(opt), _stream(stream), C.byref(h)))
    return h


def mesh_info(h, n_nodes: int | None = None):
    n_dof, n_gp = C.c_int64(), C.c_int64()
    dof = np.empty(n_nodes, dtype=np.int32) if n_nodes else None
    _check(_lib.fem3_mesh_info(h, C.byref(n_dof), C.byref(n_gp),
                               _ptr(dof) if dof is not None else None))
    return n_dof.value, n_gp.value, dof


def assemble(h, alpha, K, precision="fp64", A_out=None, stream=None):
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    k = np.ascontiguousarray(K, dtype=np.float64)
    _check(_lib.fem3_assemble(h, _ptr(a), _ptr(k), PRECISIONS[precision],
                              _ptr(A_out) if A_out is not None else None, _stream(stream)))


def assemble_part(h, alpha, K, precision, part, nparts, A_out, stream=None):
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    k = np.ascontiguousarray(K, dtype=np.float64)
    _check(_lib.fem3_assemble_part(h, _ptr(a), _ptr(k), PRECISIONS[precision], int(part),
                                   int(nparts), _ptr(A_out), _stream(stream)))


def assemble_integer(h, K, A_out=None, stream=None):
    k = np.ascontiguousarray(K, dtype=np.float64)
    _check(_lib.fem3_assemble_integer(h, _ptr(k), _ptr(A_out) if A_out is not None else None,
                                      _stream(stream)))


def assemble_form(h, axis, alpha, beta, trial_left, c, precision, K_out, stream=None):
    _check(_lib.fem3_assemble_form(h, int(axis), float(alpha), float(beta), int(bool(trial_left)),
                                   _ptr(c) if c is not None else None, PRECISIONS[precision],
                                   _ptr(K_out), _stream(stream)))


def assemble_divergence(h, beta, p, q, precision, A_out=None, stream=None):
    b = np.ascontiguousarray(beta, dtype=np.float64)
    _check(_lib.fem3_assemble_divergence(h, _ptr(b), _ptr(p), _ptr(q), PRECISIONS[precision],
                                         _ptr(A_out) if A_out is not None else None,
                                         _stream(stream)))


def load(h, f, nrhs, b, stream=None):
    _check(_lib.fem3_load(h, _ptr(f), int(nrhs), _ptr(b), _stream(stream)))


def solve(h, f, nrhs, u, tol=1e-12, max_iter=50, stream=None):
    it, res = C.c_int(0), C.c_double(0)
    _check(_lib.fem3_solve(h, _ptr(f), int(nrhs), float(tol), int(max_iter), _ptr(u),
                           C.byref(it), C.byref(res), _stream(stream)))
    return it.value, res.value


def adjoint(h, u, u_obs, dJ_df=None, tol=1e-12, max_iter=50, stream=None):
    dK = np.zeros(3)
    _check(_lib.fem3_adjoint(h, _ptr(u), _ptr(u_obs), float(tol), int(max_iter), _ptr(dK),
                             _ptr(dJ_df) if dJ_df is not None else None, _stream(stream)))
    return dK


def vjp(h, u, g, df=None, tol=1e-12, max_iter=50, stream=None):
    dK = np.zeros(3)
    _check(_lib.fem3_vjp(h, _ptr(u), _ptr(g), float(tol), int(max_iter), _ptr(dK),
                         _ptr(df) if df is not None else None, _stream(stream)))
    return dK


def paths(h, axis, direction, gps, cap, tet_out, r_in, r_out, nseg, stream=None):
    _check(_lib.fem3_paths(h, int(axis), int(direction), _ptr(gps), int(gps.shape[0]), int(cap),
                           _ptr(tet_out), _ptr(r_in), _ptr(r_out), _ptr(nseg), _stream(stream)))


def table_rows(h, axis, direction, gps, rows, stream=None):
    _check(_lib.fem3_table_rows(h, int(axis), int(direction), _ptr(gps), int(gps.shape[0]),
                                _ptr(rows), _stream(stream)))


def sync(h, stream=None):
    _check(_lib.fem3_sync(h, _stream(stream)))


def stage_ms(h):
    out = []
    for k in range(7):
        v = C.c_float(0)
        _check(_lib.fem3_stage_ms(h, k, C.byref(v)))
        out.append(v.value)
    return out


def counters(h):
    s, f, b, n = C.c_int64(), C.c_double(), C.c_int64(), C.c_int64()
    _check(_lib.fem3_counters(h, C.byref(s), C.byref(f), C.byref(b), C.byref(n)))
    return dict(segments=s.value, contract_flops=f.value, table_bytes=b.value, launches=n.value)


def contract_work(h, stream=None):
    f = C.c_double(0)
    _check(_lib.fem3_contract_work(h, C.byref(f), _stream(stream)))
    return f.value


def table_nnz(h, stream=None):
    v = C.c_int64(0)
    _check(_lib.fem3_table_nnz(h, C.byref(v), _stream(stream)))
    return v.value


KERNEL_CLASSES = ("walk_tables", "split", "contract", "factor", "chain", "apply")


def kernel_ms(h):
    """{class: (summed ms, launches)} of the profiled launches since the last assemble"""
    out = {}
    for k, name in enumerate(KERNEL_CLASSES):
        v, n = C.c_float(0), C.c_int32(0)
        _check(_lib.fem3_kernel_ms(h, k, C.byref(v), C.byref(n)))
        out[name] = (v.value, n.value)
    return out


def bin_stats(h, axis):
    nb, nt, md, mg = C.c_int64(), C.c_int64(), C.c_int32(), C.c_int32()
    _check(_lib.fem3_bin_stats(h, int(axis), C.byref(nb), C.byref(nt), C.byref(md), C.byref(mg)))
    return dict(n_bins=nb.value, n_tmpl=nt.value, max_dof=md.value, max_gp=mg.value)


def tc_tile(h):
    t, u = C.c_int32(), C.c_int32()
    _check(_lib.fem3_tc_tile(h, C.byref(t), C.byref(u)))
    return t.value, bool(u.value)


def apply_lists(h):
    v = C.c_int32()
    _check(_lib.fem3_apply_lists(h, C.byref(v)))
    return bool(v.value)


def spd_solve_static(A, b, x, stream=None):
    """Dense SPD solve with no device allocation (n <= 512): A (n, n), b and x (n,), all
    contiguous float64 CUDA tensors on the current device (see include/fem3.h)."""
    import torch
    lib = load_library()
    dev = torch.cuda.current_device()
    for name, t in (("A", A), ("b", b), ("x", x)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
                and t.is_contiguous() and t.device.index == dev):
            raise ValueError(f"{name} must be a contiguous float64 CUDA tensor on device {dev}")
    n = A.shape[0] if A.dim() == 2 else -1
    if A.dim() != 2 or A.shape[1] != n or b.shape != (n,) or x.shape != (n,):
        raise ValueError("A must be (n, n), b and x (n,)")
    _check(lib.fem3_spd_solve_static(_ptr(A), int(A.shape[0]), _ptr(b), _ptr(x), _stream(stream)))


def mesh_free(h):
    if h and _lib is not None:
        _lib.fem3_mesh_free(h)


# ---------------------------------------------------------------------------------
class Mesh:
    """A mesh uploaded to the current CUDA device (torch's current stream by default)."""

    def __init__(self, verts, tets, bin_scale: float = 0.5, max_steps: int = 0,
                 profile: bool = False, stream=None, tc_tile: int = 0, chol_tc: int = 0):
        import torch
        self._torch = torch
        self.stream = stream
        if isinstance(verts, np.ndarray):
            verts = np.ascontiguousarray(verts, dtype=np.float64)
            tets = np.ascontiguousarray(tets, dtype=np.int32)
        self.n_nodes = int(verts.shape[0])
        self.n_tets = int(tets.shape[0])
        self.h = mesh_upload(verts, tets, bin_scale, max_steps, profile, stream, tc_tile, chol_tc)
        self.n_dof, self.n_gp, self.dof_of_node = mesh_info(self.h, self.n_nodes)
        self.precision = None

    def _dev(self, shape, dtype=None):
        t = self._torch
        return t.empty(shape, dtype=dtype or t.float64, device="cuda")

    def assemble(self, alpha, K, precision="fp64", return_matrix=False):
        A = self._dev((self.n_dof, self.n_dof)) if return_matrix else None
        assemble(self.h, alpha, K, precision, A, self.stream)
        self.precision = precision
        return A

    def assemble_part(self, alpha, K, precision, part, nparts):
        """Part `part` of `nparts` of the matrix (the bins [nb part/nparts, nb (part+1)/nparts)
        of every axis); the parts sum to the whole matrix."""
        A = self._dev((self.n_dof, self.n_dof))
        assemble_part(self.h, alpha, K, precision, part, nparts, A, self.stream)
        self.precision = None
        return A

    def assemble_integer(self, K, return_matrix=False):
        """alpha_i = 2 on every axis: the P1 stiffness matrix, assembled tet by tet"""
        A = self._dev((self.n_dof, self.n_dof)) if return_matrix else None
        assemble_integer(self.h, K, A, self.stream)
        self.precision = "fp64"
        return A

    def assemble_form(self, axis, alpha, beta, trial_left=True, c=None, precision="fp64"):
        """One axis term K[k, l] = sum_g w_g c_g (D^alpha psi_l)(x_g) (D^^beta psi_k)(x_g)
        (left trial operator when trial_left); c: values at the Gauss points or None."""
        if c is not None and isinstance(c, np.ndarray):
            c = np.ascontiguousarray(c, dtype=np.float64)
        K = self._dev((self.n_dof, self.n_dof))
        assemble_form(self.h, axis, alpha, beta, trial_left, c, precision, K, self.stream)
        self.precision = None
        return K

    def assemble_divergence(self, beta, p, q, precision="fp64", return_matrix=False):
        """Section 3's divergence form; p, q [3, n_gp] at the Gauss points.  fem3_solve then
        runs preconditioned GMRES on it."""
        if isinstance(p, np.ndarray):
            p = np.ascontiguousarray(p, dtype=np.float64)
            q = np.ascontiguousarray(q, dtype=np.float64)
        A = self._dev((self.n_dof, self.n_dof)) if return_matrix else None
        assemble_divergence(self.h, beta, p, q, precision, A, self.stream)
        self.precision = precision
        return A

    def load(self, f):
        f = self._as_nodal(f)
        nrhs = 1 if f.dim() == 1 else f.shape[0]
        b = self._dev((nrhs, self.n_dof))
        load(self.h, f, nrhs, b, self.stream)
        return b[0] if nrhs == 1 else b.T

    def _as_nodal(self, f):
        t = self._torch
        if isinstance(f, np.ndarray):
            f = t.from_numpy(np.ascontiguousarray(f, dtype=np.float64))
        if f.dim() == 2:
            f = f.T.contiguous()   # column-major [n_nodes][nrhs] = row-major [nrhs][n_nodes]
        return f.contiguous()

    def solve(self, f, tol=1e-12, max_iter=50):
        """u = A^{-1} M f; f nodal [n_nodes] or [n_nodes, nrhs] (host or device)."""
        f = self._as_nodal(f)
        nrhs = 1 if f.dim() == 1 else f.shape[0]
        u = self._dev((nrhs, self.n_dof))
        self.iters, self.resid = solve(self.h, f, nrhs, u, tol, max_iter, self.stream)
        return u[0] if nrhs == 1 else u.T

    def adjoint(self, u, u_obs, tol=1e-12, max_iter=50):
        dJdf = self._dev((self.n_nodes,))
        dK = adjoint(self.h, u.contiguous(), u_obs.contiguous(), dJdf, tol, max_iter, self.stream)
        return dK, dJdf

    def vjp(self, u, g, tol=1e-12, max_iter=50):
        """(dL/dK [3] host, dL/df [n_nodes] device) for an upstream gradient g = dL/du of the
        last solve's solution u (one right-hand side)."""
        df = self._dev((self.n_nodes,))
        dK = vjp(self.h, u.contiguous(), g.contiguous(), df, tol, max_iter, self.stream)
        return dK, df

    def paths(self, axis, direction, gps, cap=None):
        t = self._torch
        gps = t.as_tensor(gps, dtype=t.int64, device="cuda").contiguous()
        cap = cap or int(8 * round(self.n_tets ** (1 / 3))) + 64
        n = gps.shape[0]
        tet = t.full((n, cap), -1, dtype=t.int32, device="cuda")
        r0 = t.zeros((n, cap), dtype=t.float64, device="cuda")
        r1 = t.zeros((n, cap), dtype=t.float64, device="cuda")
        ns = t.zeros((n,), dtype=t.int32, device="cuda")
        paths(self.h, axis, direction, gps, cap, tet, r0, r1, ns, self.stream)
        return tet, r0, r1, ns

    def table_rows(self, axis, direction, gps):
        t = self._torch
        gps = t.as_tensor(gps, dtype=t.int64, device="cuda").contiguous()
        rows = self._dev((gps.shape[0], self.n_dof))
        table_rows(self.h, axis, direction, gps, rows, self.stream)
        return rows

    def sync(self):
        sync(self.h, self.stream)

    def stage_ms(self):
        return stage_ms(self.h)

    def counters(self):
        return counters(self.h)

    def contract_work(self):
        """algorithmic flops of the last contraction: sum_g 4 nnz(L[g]) nnz(R[g]) per axis"""
        return contract_work(self.h, self.stream)

    def table_nnz(self):
        """nonzeros of the last assemble's tables: sum over axes and g of nnz(L[g]) + nnz(R[g])"""
        return table_nnz(self.h, self.stream)

    def kernel_ms(self):
        """{kernel class: (ms, launches)} timed on the launch stream (profiling handles)"""
        return kernel_ms(self.h)

    def bin_stats(self, axis):
        """bins of one axis: count, template rows, largest dof set and Gauss-point count"""
        return bin_stats(self.h, axis)

    def tc_tile(self):
        """(tile width of the last tensor-core contraction, whether it ran the tuner)"""
        return tc_tile(self.h)

    def apply_lists(self):
        """whether the refinement's operator apply runs from the tables' nonzero lists (else
        from the dense table blocks of the bins)"""
        return apply_lists(self.h)

    def free(self):
        if getattr(self, "h", None):
            mesh_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Batch:
    """Many meshes assembled and solved together (fem3_batch_*).

    meshes: list of (verts, tets) host arrays.  run() takes per-mesh alpha and K
    ([n][3]) and per-mesh nodal right-hand sides ([n_nodes_i, nrhs] host or device) and
    returns per-mesh solutions ([n_dof_i, nrhs] device tensors)."""

    def __init__(self, meshes, bin_scale: float = 0.5, max_steps: int = 0, stream=None):
        import torch
        self._torch = torch
        lib = load_library()
        self.stream = stream
        self._keep = [(np.ascontiguousarray(v, dtype=np.float64), np.ascontiguousarray(t, dtype=np.int32))
                      for v, t in meshes]
        n = len(self._keep)
        vp = (C.c_void_p * n)(*[v.ctypes.data for v, _ in self._keep])
        tp = (C.c_void_p * n)(*[t.ctypes.data for _, t in self._keep])
        nn = (C.c_int64 * n)(*[v.shape[0] for v, _ in self._keep])
        nt = (C.c_int64 * n)(*[t.shape[0] for _, t in self._keep])
        opt = Options(bin_scale, max_steps, 0, 0, 0)
        h = C.c_void_p()
        _check(lib.fem3_batch_create(n, vp, nn, tp, nt, C.byref(opt), _stream(stream), C.byref(h)))
        self.h = h
        self.n = n
        self.n_dof, self.n_nodes = [], []
        for i in range(n):
            mh = C.c_void_p()
            _check(lib.fem3_batch_mesh(self.h, i, C.byref(mh)))
            nd, _, _ = mesh_info(mh)
            self.n_dof.append(nd)
            self.n_nodes.append(self._keep[i][0].shape[0])

    def run(self, alpha, K, fs, precision="tf32x3", tol=1e-12, max_iter=50):
        t = self._torch
        a = np.ascontiguousarray(alpha, dtype=np.float64).reshape(self.n, 3)
        k = np.ascontiguousarray(K, dtype=np.float64).reshape(self.n, 3)
        f_dev = []
        nrhs = None
        for i, f in enumerate(fs):
            ft = t.as_tensor(f, dtype=t.float64)
            if ft.dim() == 1:
                ft = ft[:, None]
            nrhs = ft.shape[1]
            f_dev.append(ft.T.contiguous().cuda())       # column-major [n_nodes][nrhs]
        u_dev = [t.empty((nrhs, self.n_dof[i]), dtype=t.float64, device="cuda") for i in range(self.n)]
        fp = (C.c_void_p * self.n)(*[x.data_ptr() for x in f_dev])
        up = (C.c_void_p * self.n)(*[x.data_ptr() for x in u_dev])
        it = (C.c_int * self.n)()
        rs = (C.c_double * self.n)()
        _check(_lib.fem3_batch_run(self.h, _ptr(a), _ptr(k), PRECISIONS[precision], fp, int(nrhs),
                                   float(tol), int(max_iter), up, it, rs, _stream(self.stream)))
        self.iters, self.resid = list(it), list(rs)
        return [x.T for x in u_dev]

    def graph_launches(self):
        """launches of the captured assembly + factorisation graph so far (the capturing run's
        own launch included)"""
        v = C.c_int64(0)
        _check(_lib.fem3_batch_graph_launches(self.h, C.byref(v)))
        return v.value

    def free(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.fem3_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ---------------------------------------------------------------------------------
# autograd
# ---------------------------------------------------------------------------------
def _frac_solve_function():
    import torch

    class FracSolve(torch.autograd.Function):
        """u = A(K)^{-1} M f on one mesh, differentiable in K (3 axis coefficients) and in
        the nodal source f (one right-hand side).  Forward: fem3_assemble + fem3_solve;
        backward: fem3_vjp (one adjoint solve with the same factorisation, the axis forms
        of the tables and M^T lambda)."""

        @staticmethod
        def forward(ctx, K, f, mesh, alpha, precision, tol):
            mesh.assemble(alpha, [float(x) for x in K.detach().cpu()], precision)
            u = mesh.solve(f.detach(), tol=tol)
            ctx.mesh, ctx.tol = mesh, tol
            ctx.k_device, ctx.k_dtype = K.device, K.dtype
            ctx.save_for_backward(u)
            return u

        @staticmethod
        def backward(ctx, grad_u):
            (u,) = ctx.saved_tensors
            dK, df = ctx.mesh.vjp(u, grad_u.to(u.dtype).contiguous(), tol=ctx.tol)
            gK = torch.as_tensor(dK, dtype=ctx.k_dtype, device=ctx.k_device)
            return gK, df, None, None, None, None

    return FracSolve


_FRAC_SOLVE = None


def frac_solve(mesh, alpha, K, f, precision="fp64", tol=1e-12):
    """Differentiable solve: K a float64 tensor [3] (any device), f a float64 CUDA tensor
    [n_nodes]; returns u [n_dof] on the device.  Gradients flow to K and f through the
    library's adjoint (fem3_vjp)."""
    global _FRAC_SOLVE
    if _FRAC_SOLVE is None:
        _FRAC_SOLVE = _frac_solve_function()
    return _FRAC_SOLVE.apply(K, f, mesh, tuple(float(a) for a in alpha), precision, tol)
