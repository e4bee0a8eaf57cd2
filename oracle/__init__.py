"""Plain FP64 CPU oracle for the fractional FEM assembly (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  The product path (``paper_1811_03339_gb300``) never does.

The arithmetic lives in ``fem3_oracle.c`` (plain C, no blocking, no fusion); this file
compiles it with gcc on first use and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fem3_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libfem3_oracle.so")
_lock = threading.Lock()
_lib = None

OR_E_WALK = -3
OR_E_NOT_SPD = -4


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, FP64, no FMA contraction so x86 and Arm agree)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        p = C.c_void_p
        i64, i32, dbl = C.c_int64, C.c_int32, C.c_double
        lib.or_mesh_build.restype = p
        lib.or_mesh_build.argtypes = [p, i64, p, i64, C.POINTER(C.c_int)]
        lib.or_mesh_free.argtypes = [p]
        lib.or_mesh_info.argtypes = [p, C.POINTER(i64), C.POINTER(i64), C.POINTER(dbl)]
        lib.or_mesh_get.argtypes = [p, p, p, p, p, p, p]
        lib.or_walk.restype = C.c_int
        lib.or_walk.argtypes = [p, i64, C.c_int, C.c_int, C.c_int, p, p, p,
                                C.POINTER(dbl), C.POINTER(i32)]
        lib.or_walk_point.restype = C.c_int
        lib.or_walk_point.argtypes = [p, p, i32, C.c_int, C.c_int, C.c_int, p, p, p,
                                      C.POINTER(dbl), C.POINTER(i32)]
        lib.or_table_row.restype = C.c_int
        lib.or_table_row.argtypes = [p, i64, C.c_int, C.c_int, dbl, C.c_int, p]
        lib.or_assemble.restype = C.c_int
        lib.or_assemble.argtypes = [p, p, p, p]
        lib.or_assemble_gps.restype = C.c_int
        lib.or_assemble_gps.argtypes = [p, p, p, p, i64, p]
        lib.or_assemble_form.restype = C.c_int
        lib.or_assemble_form.argtypes = [p, C.c_int, dbl, dbl, C.c_int, p, C.c_int, p]
        lib.or_assemble_divergence.restype = C.c_int
        lib.or_assemble_divergence.argtypes = [p, p, p, p, C.c_int, p]
        lib.or_load.restype = C.c_int
        lib.or_load.argtypes = [p, p, C.c_int, p]
        lib.or_load_T.restype = C.c_int
        lib.or_load_T.argtypes = [p, p, C.c_int, p]
        lib.or_cholesky.restype = C.c_int
        lib.or_cholesky.argtypes = [i64, p, p, C.POINTER(i64)]
        lib.or_chol_solve.argtypes = [i64, p, C.c_int, p]
        lib.or_axis_forms.restype = C.c_int
        lib.or_axis_forms.argtypes = [p, p, p, p, p]
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return C.c_void_p(a.ctypes.data)


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with status {code}")
        self.code = code


class Oracle:
    """Oracle bound to one mesh (verts float64 [n,3], tets int32 [T,4])."""

    def __init__(self, verts: np.ndarray, tets: np.ndarray):
        self._lib = _load()
        self.verts = np.ascontiguousarray(verts, dtype=np.float64)
        self.tets = np.ascontiguousarray(tets, dtype=np.int32)
        st = C.c_int(0)
        h = self._lib.or_mesh_build(_ptr(self.verts), self.verts.shape[0], _ptr(self.tets),
                                    self.tets.shape[0], C.byref(st))
        if not h:
            raise OracleError(st.value, "mesh_build")
        self._h = C.c_void_p(h)
        nd, ng, sp = C.c_int64(), C.c_int64(), C.c_double()
        self._lib.or_mesh_info(self._h, C.byref(nd), C.byref(ng), C.byref(sp))
        self.n_dof, self.n_gp, self.span = nd.value, ng.value, sp.value
        self.n_nodes = self.verts.shape[0]
        self.n_tets = self.tets.shape[0]
        T = self.n_tets
        self.M = np.empty((T, 4, 4))
        self.vol = np.empty(T)
        self.nbr = np.empty((T, 4), dtype=np.int32)
        self.dof = np.empty(self.n_nodes, dtype=np.int32)
        self.gp = np.empty((4 * T, 3))
        self.gw = np.empty(4 * T)
        self._lib.or_mesh_get(self._h, _ptr(self.M), _ptr(self.vol), _ptr(self.nbr),
                              _ptr(self.dof), _ptr(self.gp), _ptr(self.gw))
        self.max_steps = int(8.0 * np.cbrt(float(T))) + 64

    @classmethod
    def from_mesh(cls, mesh) -> "Oracle":
        return cls(mesh.verts, mesh.tets)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and self._lib is not None:
            self._lib.or_mesh_free(h)
            self._h = None

    # -- Section 2.2: path search ---------------------------------------------------
    def walk(self, g: int, axis: int, direction: int):
        """Ordered segments of the path from Gauss point g along -e_axis (direction=-1)
        or +e_axis (direction=+1): (tet ids, r_in, r_out, r_end, end tet)."""
        cap = self.max_steps
        st = np.empty(cap, dtype=np.int32)
        r0 = np.empty(cap)
        r1 = np.empty(cap)
        re, te = C.c_double(), C.c_int32()
        n = self._lib.or_walk(self._h, int(g), int(axis), int(direction), cap, _ptr(st),
                              _ptr(r0), _ptr(r1), C.byref(re), C.byref(te))
        if n < 0:
            raise OracleError(n, "walk")
        return st[:n].copy(), r0[:n].copy(), r1[:n].copy(), re.value, te.value

    def walk_point(self, x, tet: int, axis: int, direction: int):
        """Same walk from an arbitrary point x inside tet (used for degenerate rays)."""
        cap = self.max_steps
        xx = np.ascontiguousarray(x, dtype=np.float64)
        st = np.empty(cap, dtype=np.int32)
        r0 = np.empty(cap)
        r1 = np.empty(cap)
        re, te = C.c_double(), C.c_int32()
        n = self._lib.or_walk_point(self._h, _ptr(xx), int(tet), int(axis), int(direction),
                                    cap, _ptr(st), _ptr(r0), _ptr(r1), C.byref(re),
                                    C.byref(te))
        if n < 0:
            raise OracleError(n, "walk_point")
        return st[:n].copy(), r0[:n].copy(), r1[:n].copy(), re.value, te.value

    # -- Section 2.1: derivative tables ---------------------------------------------
    def table_row(self, g: int, axis: int, direction: int, gamma: float,
                  all_nodes: bool = False) -> np.ndarray:
        row = np.empty(self.n_nodes if all_nodes else self.n_dof)
        e = self._lib.or_table_row(self._h, int(g), int(axis), int(direction), float(gamma),
                                   int(bool(all_nodes)), _ptr(row))
        if e:
            raise OracleError(e, "table_row")
        return row

    def tables(self, axis: int, gamma: float, gps=None, all_nodes: bool = False):
        """Dense rows of L (left, direction -1) and R (right, +1) for the given Gauss points."""
        gps = np.arange(self.n_gp) if gps is None else np.asarray(gps)
        width = self.n_nodes if all_nodes else self.n_dof
        Lt = np.empty((len(gps), width))
        Rt = np.empty((len(gps), width))
        for r, g in enumerate(gps):
            Lt[r] = self.table_row(int(g), axis, -1, gamma, all_nodes)
            Rt[r] = self.table_row(int(g), axis, +1, gamma, all_nodes)
        return Lt, Rt

    # -- Section 2.1: Galerkin matrix -----------------------------------------------
    def assemble(self, alpha, K) -> np.ndarray:
        a = np.ascontiguousarray(alpha, dtype=np.float64)
        k = np.ascontiguousarray(K, dtype=np.float64)
        A = np.empty((self.n_dof, self.n_dof))
        e = self._lib.or_assemble(self._h, _ptr(a), _ptr(k), _ptr(A))
        if e:
            raise OracleError(e, "assemble")
        return A

    def assemble_gps(self, alpha, K, gps, A: np.ndarray | None = None) -> np.ndarray:
        """Add the element-sum terms of the listed Gauss points (all axes) to A (a new zero
        matrix when None); a partition of the Gauss points sums to ``assemble``."""
        a = np.ascontiguousarray(alpha, dtype=np.float64)
        k = np.ascontiguousarray(K, dtype=np.float64)
        g = np.ascontiguousarray(gps, dtype=np.int64)
        if A is None:
            A = np.zeros((self.n_dof, self.n_dof))
        assert A.flags["C_CONTIGUOUS"] and A.shape == (self.n_dof, self.n_dof)
        e = self._lib.or_assemble_gps(self._h, _ptr(a), _ptr(k), _ptr(g), len(g), _ptr(A))
        if e:
            raise OracleError(e, "assemble_gps")
        return A

    def assemble_form(self, axis: int, alpha: float, beta: float, trial_left: bool = True,
                      c=None, all_nodes: bool = False) -> np.ndarray:
        """One axis term of (c D^alpha u, D^^beta v) (Section 2.1, eq. "equ:varsss"):
        K[k, l] = sum_g w_g c_g (D^alpha psi_l)(x_g) (D^^beta psi_k)(x_g), D^alpha the left
        operator when trial_left (D^^beta the right one), orders in [0, 1]; c: values at the
        Gauss points (``self.gp`` order) or None for 1."""
        n = self.n_nodes if all_nodes else self.n_dof
        K = np.empty((n, n))
        cg = None
        if c is not None:
            cg = np.ascontiguousarray(c, dtype=np.float64)
            if cg.shape != (self.n_gp,):
                raise ValueError("c must hold one value per Gauss point")
        e = self._lib.or_assemble_form(self._h, int(axis), float(alpha), float(beta),
                                       int(bool(trial_left)),
                                       None if cg is None else _ptr(cg), int(bool(all_nodes)),
                                       _ptr(K))
        if e:
            raise OracleError(e, "assemble_form")
        return K

    def assemble_divergence(self, beta, p, q, all_nodes: bool = False) -> np.ndarray:
        """Section 3 (eq. "equ:sfde2"): A[k, l] = a(psi_l, psi_k) with
        a(u, v) = -sum_i ((p_i D_L^{beta_i} u, D_i v) - (q_i D_R^{beta_i} u, D_i v));
        p, q: [3, n_gp] coefficient values at the Gauss points (``self.gp`` order)."""
        n = self.n_nodes if all_nodes else self.n_dof
        b = np.ascontiguousarray(beta, dtype=np.float64)
        pg = np.ascontiguousarray(p, dtype=np.float64)
        qg = np.ascontiguousarray(q, dtype=np.float64)
        if b.shape != (3,) or pg.shape != (3, self.n_gp) or qg.shape != (3, self.n_gp):
            raise ValueError("beta [3], p and q [3, n_gp]")
        A = np.empty((n, n))
        e = self._lib.or_assemble_divergence(self._h, _ptr(b), _ptr(pg), _ptr(qg),
                                             int(bool(all_nodes)), _ptr(A))
        if e:
            raise OracleError(e, "assemble_divergence")
        return A

    def load(self, f: np.ndarray) -> np.ndarray:
        """b = M f; f nodal [n_nodes] or [n_nodes, nrhs]; returns [n_dof] or [n_dof, nrhs]."""
        f = np.asarray(f, dtype=np.float64)
        vec = f.ndim == 1
        F = np.asfortranarray(f.reshape(self.n_nodes, -1))
        nrhs = F.shape[1]
        b = np.empty((self.n_dof, nrhs), order="F")
        self._lib.or_load(self._h, _ptr(F), nrhs, _ptr(b))
        return b[:, 0].copy() if vec else b

    def load_T(self, lam: np.ndarray) -> np.ndarray:
        lam = np.asarray(lam, dtype=np.float64)
        vec = lam.ndim == 1
        Lm = np.asfortranarray(lam.reshape(self.n_dof, -1))
        nrhs = Lm.shape[1]
        out = np.empty((self.n_nodes, nrhs), order="F")
        self._lib.or_load_T(self._h, _ptr(Lm), nrhs, _ptr(out))
        return out[:, 0].copy() if vec else out

    def axis_forms(self, alpha, u: np.ndarray, lam: np.ndarray) -> np.ndarray:
        a = np.ascontiguousarray(alpha, dtype=np.float64)
        u = np.ascontiguousarray(u, dtype=np.float64)
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        out = np.empty(3)
        e = self._lib.or_axis_forms(self._h, _ptr(a), _ptr(u), _ptr(lam), _ptr(out))
        if e:
            raise OracleError(e, "axis_forms")
        return out

    # -- adjoint: J = 0.5 ||u - u_obs||^2, u = A^{-1} M f ---------------------------
    def adjoint(self, alpha, K, f: np.ndarray, u_obs: np.ndarray, A: np.ndarray | None = None):
        A = self.assemble(alpha, K) if A is None else A
        Lc = cholesky(A)
        u = chol_solve(Lc, self.load(f))
        lam = chol_solve(Lc, u - u_obs)
        dK = -self.axis_forms(alpha, u, lam)
        df = self.load_T(lam)
        J = 0.5 * float(np.dot(u - u_obs, u - u_obs))
        return J, dK, df, u


def cholesky(A: np.ndarray) -> np.ndarray:
    lib = _load()
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    Lc = np.empty_like(A)
    bad = C.c_int64(-1)
    e = lib.or_cholesky(n, _ptr(A), _ptr(Lc), C.byref(bad))
    if e:
        err = OracleError(e, f"cholesky (column {bad.value})")
        err.column = bad.value
        raise err
    return Lc


def chol_solve(Lc: np.ndarray, b: np.ndarray) -> np.ndarray:
    lib = _load()
    b = np.asarray(b, dtype=np.float64)
    vec = b.ndim == 1
    X = np.asfortranarray(b.reshape(Lc.shape[0], -1)).copy(order="F")
    lib.or_chol_solve(Lc.shape[0], _ptr(np.ascontiguousarray(Lc)), X.shape[1], _ptr(X))
    return X[:, 0].copy() if vec else X


def solve(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    return chol_solve(cholesky(A), b)


def riesz_scale(alpha: float) -> float:
    """s = 1 / (2 cos(pi alpha / 2)), the Riesz constant folded into the Galerkin matrix."""
    return 1.0 / (2.0 * math.cos(math.pi * alpha / 2.0))
