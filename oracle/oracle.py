"""Oracle for the FC-RKPM hot path: traditional neighbour-loop RKPM in FP64 (plain C).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this module.  It shares no
code with the CUDA library and never imports it.  The C source
(``rkpm_oracle.c``) works on the domain nodes only -- explicit neighbour search,
explicit moment matrices (Eq. 3), shape functions (Eq. 2), implicit gradients
(Eq. 15-16), the stiffness matrix assembled with direct nodal integration
(Eq. 26, 50, 54), the force vector (Eq. 27, 59), field evaluation (Eq. 62) and a
strongly enforced Dirichlet solve (Eq. 25, 29).

Every function here takes grid-indexed numpy arrays (x fastest, shape (nz, ny, nx)
or flat) and returns grid-indexed arrays; values off the domain are zero.

Parity pins (tests/test_oracle_pins.py) fix it against the paper: reproducing
conditions, the closed-form interior stencil at a = 2h (cubic B-spline weights
1/6, 2/3, 1/6), interior neighbour counts of Tab. 4-5, symmetry of K and K.1 = 0,
the energy of linear fields, f^r moments, and convergence to a manufactured
solution.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rkpm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, f"liboracle_{platform.machine()}.so")
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_intp = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (plain C, no arch flags; OpenMP
    when available, which threads the loops over nodes, rows and samples)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        try:  # all host threads where the compiler has OpenMP; serial otherwise
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    lib.orc_threads.restype = ctypes.c_int
    lib.orc_threads.argtypes = []
    lib.orc_phi1.restype = ctypes.c_double
    lib.orc_phi1.argtypes = [ctypes.c_double]
    lib.orc_create.restype = ctypes.c_void_p
    lib.orc_create.argtypes = [_intp, _f64p, ctypes.c_double, ctypes.c_int, _u8p]
    lib.orc_destroy.argtypes = [ctypes.c_void_p]
    for name in ("orc_nnode", "orc_nsingular", "orc_first_singular"):
        getattr(lib, name).restype = ctypes.c_int64
        getattr(lib, name).argtypes = [ctypes.c_void_p]
    lib.orc_nslot.restype = ctypes.c_int
    lib.orc_nslot.argtypes = [ctypes.c_void_p]
    lib.orc_reach.restype = ctypes.c_int
    lib.orc_reach.argtypes = [ctypes.c_void_p, ctypes.c_int]
    for name in ("orc_s", "orc_dim"):
        getattr(lib, name).restype = ctypes.c_int
        getattr(lib, name).argtypes = [ctypes.c_void_p]
    lib.orc_eval_points_1d.restype = ctypes.c_int64
    lib.orc_eval_points_1d.argtypes = [ctypes.c_void_p, ctypes.c_int64, _f64p, _f64p, _f64p]
    lib.orc_grid_dim.restype = ctypes.c_int
    lib.orc_grid_dim.argtypes = [_intp]
    lib.orc_basis_size_dim.restype = ctypes.c_int
    lib.orc_basis_size_dim.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.orc_node_box.argtypes = [ctypes.c_void_p, _i64p]
    lib.orc_shape_tables.argtypes = [ctypes.c_void_p, _i64p, _f64p, _f64p]
    lib.orc_neighbour_count.restype = ctypes.c_int
    lib.orc_neighbour_count.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    lib.orc_neighbour_count_bruteforce.restype = ctypes.c_int
    lib.orc_neighbour_count_bruteforce.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    lib.orc_b_fields.argtypes = [ctypes.c_void_p, _f64p]
    lib.orc_apply_K.argtypes = [ctypes.c_void_p, _f64p, _f64p, _f64p]
    lib.orc_rhs.argtypes = [ctypes.c_void_p, _f64p, _f64p, _f64p]
    lib.orc_eval_u.argtypes = [ctypes.c_void_p, _f64p, _f64p]
    lib.orc_eval_u_transpose.argtypes = [ctypes.c_void_p, _f64p, _f64p]
    lib.orc_grad_transpose.argtypes = [ctypes.c_void_p, _f64p, _f64p, _f64p]
    lib.orc_assemble_K.restype = ctypes.c_int64
    lib.orc_assemble_K.argtypes = [ctypes.c_void_p, _f64p]
    lib.orc_get_K.argtypes = [ctypes.c_void_p, _i64p, _i64p, _f64p]
    lib.orc_solve_dirichlet.restype = ctypes.c_int
    lib.orc_solve_dirichlet.argtypes = [ctypes.c_void_p, _u8p, _f64p, _f64p, ctypes.c_double,
                                        ctypes.c_int, ctypes.c_int, _f64p, _f64p]
    lib.orc_spmv.argtypes = [ctypes.c_void_p, _f64p, _f64p]
    lib.orc_apply_K_sampled.restype = ctypes.c_int64
    lib.orc_apply_K_sampled.argtypes = [_intp, _f64p, ctypes.c_double, ctypes.c_int, _u8p, _f64p,
                                        _f64p, ctypes.c_int64, _i64p, _f64p]
    lib.orc_b_sampled.restype = ctypes.c_int64
    lib.orc_b_sampled.argtypes = [_intp, _f64p, ctypes.c_double, ctypes.c_int, _u8p,
                                  ctypes.c_int64, _i64p, _f64p]
    _lib = lib
    return lib


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_f64p)


def _u8(a):
    a = np.ascontiguousarray(a, dtype=np.uint8)
    return a, a.ctypes.data_as(_u8p)


def _i64(a):
    a = np.ascontiguousarray(a, dtype=np.int64)
    return a, a.ctypes.data_as(_i64p)


def threads() -> int:
    """Host threads the oracle's loops run on (1 without OpenMP)."""
    return int(_load().orc_threads())


def phi1(z: float) -> float:
    """Eq. 7 on one axis, z = |x|/a."""
    return _load().orc_phi1(float(z))


class Oracle:
    """Traditional RKPM discretisation of one domain (chi nodes of a grid).

    n: (nx, ny, nz) grid points; h: (hx, hy, hz) spacing; a_tilde: support in
    units of h (Eq. 64); degree: 1 or 2; chi: grid-indexed 0/1.  A grid with
    nz = 1 is two-dimensional and one with ny = nz = 1 one-dimensional: the
    absent axes carry no kernel factor, monomial or gradient (s = 4 / 10 in 3D,
    3 / 6 in 2D, 2 / 3 in 1D; b^k = 0 on an absent axis).
    """

    def __init__(self, n, h, a_tilde, degree, chi):
        lib = _load()
        self.n = tuple(int(v) for v in n)
        self.h = tuple(float(v) for v in h)
        self.a_tilde = float(a_tilde)
        self.degree = int(degree)
        self.nbox = self.n[0] * self.n[1] * self.n[2]
        self._chi, pchi = _u8(np.asarray(chi).reshape(-1))
        nn = (ctypes.c_int * 3)(*self.n)
        hh = (ctypes.c_double * 3)(*self.h)
        if lib.orc_grid_dim(nn) < 0 or self.degree not in (1, 2):
            raise ValueError("oracle: grid must be (n, 1, 1), (n, m, 1) or (n, m, l) with n > 1; degree 1 or 2")
        self._h = lib.orc_create(nn, hh, self.a_tilde, self.degree, pchi)
        if not self._h:
            raise MemoryError("oracle: allocation failed")
        self.s = lib.orc_s(self._h)
        self.dim = lib.orc_dim(self._h)
        self.nnode = lib.orc_nnode(self._h)
        self.nslot = lib.orc_nslot(self._h)
        self.reach = tuple(lib.orc_reach(self._h, k) for k in range(3))
        self.nsingular = lib.orc_nsingular(self._h)
        self.first_singular = lib.orc_first_singular(self._h)
        self._assembled = False
        self._nnz = 0

    def __del__(self):
        if getattr(self, "_h", None):
            _load().orc_destroy(self._h)
            self._h = None

    # -- tables ---------------------------------------------------------------
    def node_box(self) -> np.ndarray:
        out = np.zeros(self.nnode, dtype=np.int64)
        _load().orc_node_box(self._h, out.ctypes.data_as(_i64p))
        return out

    def shape_tables(self):
        """(nbr, psi, dpsi): per evaluation node S and slot, neighbour node number
        (-1 if none), Psi_I(x_S) (Eq. 2) and Psi^{grad k}_I(x_S) (Eq. 15)."""
        nbr = np.zeros((self.nnode, self.nslot), dtype=np.int64)
        psi = np.zeros((self.nnode, self.nslot))
        dpsi = np.zeros((self.nnode, self.nslot, 3))
        _load().orc_shape_tables(self._h, nbr.ctypes.data_as(_i64p), psi.ctypes.data_as(_f64p),
                                 dpsi.ctypes.data_as(_f64p))
        return nbr, psi, dpsi

    def neighbour_count(self, node: int, brute_force: bool = False) -> int:
        f = _load().orc_neighbour_count_bruteforce if brute_force else _load().orc_neighbour_count
        return f(self._h, int(node))

    def b_fields(self) -> np.ndarray:
        """(4, s, nbox): b^0, b^x, b^y, b^z on the grid (Eq. 45-47, scaled basis)."""
        out = np.zeros((4, self.s, self.nbox))
        _load().orc_b_fields(self._h, out.ctypes.data_as(_f64p))
        return out

    # -- operators ------------------------------------------------------------
    def apply_K(self, V, d) -> np.ndarray:
        """f = K d (Eq. 50/54), matrix-free neighbour loops."""
        V, pV = _f64(np.asarray(V).reshape(-1))
        d, pd = _f64(np.asarray(d).reshape(-1))
        f = np.zeros(self.nbox)
        _load().orc_apply_K(self._h, pV, pd, f.ctypes.data_as(_f64p))
        return f

    def rhs(self, V, r) -> np.ndarray:
        """f^r (Eq. 27/59)."""
        V, pV = _f64(np.asarray(V).reshape(-1))
        r, pr = _f64(np.asarray(r).reshape(-1))
        f = np.zeros(self.nbox)
        _load().orc_rhs(self._h, pV, pr, f.ctypes.data_as(_f64p))
        return f

    def eval_u(self, d) -> np.ndarray:
        """u^h at the nodes (Eq. 62)."""
        d, pd = _f64(np.asarray(d).reshape(-1))
        u = np.zeros(self.nbox)
        _load().orc_eval_u(self._h, pd, u.ctypes.data_as(_f64p))
        return u

    def eval_points_1d(self, x, d) -> np.ndarray:
        """u^h(x) = sum_I Psi_I(x) d_I at arbitrary points of a 1D grid (Eq. 1-2); x is
        measured from grid node 0."""
        x, px = _f64(np.asarray(x).reshape(-1))
        d, pd = _f64(np.asarray(d).reshape(-1))
        u = np.zeros(x.size)
        bad = _load().orc_eval_points_1d(self._h, x.size, px, pd, u.ctypes.data_as(_f64p))
        if bad < 0:
            raise ValueError("oracle: eval_points_1d needs a 1D grid")
        if bad > 0:
            raise ArithmeticError(f"oracle: {bad} points with a singular moment matrix")
        return u

    def eval_u_transpose(self, e) -> np.ndarray:
        """Transpose of Eq. 62: w_J = sum_I Psi_J(x_I) e_I."""
        e, pe = _f64(np.asarray(e).reshape(-1))
        w = np.zeros(self.nbox)
        _load().orc_eval_u_transpose(self._h, pe, w.ctypes.data_as(_f64p))
        return w

    def grad_transpose(self, V, N) -> np.ndarray:
        """Gradient-type nonlinear force (Eq. B.6-B.8, DNI): f_J = sum_S V_S
        sum_k Psi^{grad k}_J(x_S) N^k_S, i.e. B^T N; N has shape (3, nbox)
        (rows beyond the grid's dimension are ignored by the zero gradients)."""
        V, pV = _f64(np.asarray(V).reshape(-1))
        N, pN = _f64(np.asarray(N, dtype=np.float64).reshape(3, -1))
        f = np.zeros(self.nbox)
        _load().orc_grad_transpose(self._h, pV, pN, f.ctypes.data_as(_f64p))
        return f

    def assemble_K(self, V):
        """Assemble K (Eq. 26 with direct nodal integration) as CSR over node numbers."""
        V, pV = _f64(np.asarray(V).reshape(-1))
        nnz = _load().orc_assemble_K(self._h, pV)
        if nnz < 0:
            raise MemoryError("oracle: K assembly failed")
        self._assembled = True
        self._nnz = int(nnz)
        return self._nnz

    def K_csr(self):
        """(indptr, indices, data) of the assembled K over node numbers."""
        if not self._assembled:
            raise RuntimeError("assemble_K first")
        ptr = np.zeros(self.nnode + 1, dtype=np.int64)
        col = np.zeros(self._nnz, dtype=np.int64)
        val = np.zeros(self._nnz)
        _load().orc_get_K(self._h, ptr.ctypes.data_as(_i64p), col.ctypes.data_as(_i64p),
                          val.ctypes.data_as(_f64p))
        return ptr, col, val

    def spmv(self, x) -> np.ndarray:
        """y = K x with the assembled K (grid-indexed)."""
        if not self._assembled:
            raise RuntimeError("assemble_K first")
        x, px = _f64(np.asarray(x).reshape(-1))
        y = np.zeros(self.nbox)
        _load().orc_spmv(self._h, px, y.ctypes.data_as(_f64p))
        return y

    def solve(self, V, chi_gamma, r, g, tol=1e-14, max_iter=200000, dense_max=3000):
        """Alg. 5 done the traditional way: assemble K, f^r; d = g on Gamma_g
        (Eq. 29); solve K_OO d_O = f^r_O - K_OG g_G (dense Cholesky for small
        systems, CG on the CSR otherwise).  Returns (d, info)."""
        self.assemble_K(V)
        fr = self.rhs(V, r)
        cg, pcg = _u8(np.asarray(chi_gamma).reshape(-1))
        fr, pfr = _f64(fr)
        g, pg = _f64(np.asarray(g).reshape(-1))
        d = np.zeros(self.nbox)
        res = ctypes.c_double(0.0)
        ret = _load().orc_solve_dirichlet(self._h, pcg, pfr, pg, float(tol), int(max_iter), int(dense_max),
                                         d.ctypes.data_as(_f64p), ctypes.byref(res))
        if ret in (-1, -2):
            raise RuntimeError(f"oracle solve failed ({ret})")
        return d, {"iterations": ret, "rel_residual": res.value, "converged": ret != -3}

    def solve_rhs(self, chi_gamma, rhs, g, tol=1e-14, max_iter=200000, dense_max=3000):
        """Dirichlet solve with a given right-hand side vector (K must be assembled)."""
        if not self._assembled:
            raise RuntimeError("assemble_K first")
        cg, pcg = _u8(np.asarray(chi_gamma).reshape(-1))
        rhs, prhs = _f64(np.asarray(rhs).reshape(-1))
        g, pg = _f64(np.asarray(g).reshape(-1))
        d = np.zeros(self.nbox)
        res = ctypes.c_double(0.0)
        ret = _load().orc_solve_dirichlet(self._h, pcg, prhs, pg, float(tol), int(max_iter), int(dense_max),
                                         d.ctypes.data_as(_f64p), ctypes.byref(res))
        if ret in (-1, -2):
            raise RuntimeError(f"oracle solve failed ({ret})")
        return d, {"iterations": ret, "rel_residual": res.value, "converged": ret != -3}

    def adjoint(self, V, chi, chi_gamma, r, g, u_target, tol=1e-14, dense_max=3000):
        """J = 1/2 sum_chi (u^h - u_target)^2 and its gradients with respect to r and
        g, from the assembled K (derivation: d = P_G g + P_O x, K_OO x = P_O(f^r - K P_G g),
        f^r = R r with dR/dr_S = V_S Psi_I(x_S)).  Returns (J, dJ_dr, dJ_dg, u, d)."""
        chi = np.asarray(chi).reshape(-1).astype(bool)
        gam = np.asarray(chi_gamma).reshape(-1).astype(bool)
        free = chi & ~gam
        d, _ = self.solve(V, chi_gamma, r, g, tol=tol, dense_max=dense_max)
        u = self.eval_u(d)
        e = np.where(chi, u - np.asarray(u_target).reshape(-1), 0.0)
        J = 0.5 * float(np.dot(e, e))
        w = self.eval_u_transpose(e)                # U^T e
        zeros = np.zeros(self.nbox)
        lam, _ = self.solve_rhs(chi_gamma, np.where(free, w, 0.0), zeros, tol=tol, dense_max=dense_max)
        lam = np.where(free, lam, 0.0)
        Vf = np.asarray(V, dtype=np.float64).reshape(-1)
        dJ_dr = np.where(chi, Vf * self.eval_u(lam), 0.0)
        Klam = self.spmv(lam)
        dJ_dg = np.where(gam, w - Klam, 0.0)
        return J, dJ_dr, dJ_dg, u, d


def apply_K_sampled(n, h, a_tilde, degree, chi, V, d, sample) -> np.ndarray:
    """(K d)_I at the given grid points, each built from scratch (large grids)."""
    lib = _load()
    chi, pchi = _u8(np.asarray(chi).reshape(-1))
    V, pV = _f64(np.asarray(V).reshape(-1))
    d, pd = _f64(np.asarray(d).reshape(-1))
    sample, ps = _i64(np.asarray(sample).reshape(-1))
    out = np.zeros(sample.size)
    nn = (ctypes.c_int * 3)(*[int(v) for v in n])
    hh = (ctypes.c_double * 3)(*[float(v) for v in h])
    bad = lib.orc_apply_K_sampled(nn, hh, float(a_tilde), int(degree), pchi, pV, pd, sample.size, ps,
                                  out.ctypes.data_as(_f64p))
    if bad < 0:
        raise MemoryError("oracle: allocation failed")
    return out


def b_sampled(n, h, a_tilde, degree, chi, sample) -> np.ndarray:
    """(nsample, 4, s) correction coefficients at the given grid points."""
    lib = _load()
    nn = (ctypes.c_int * 3)(*[int(v) for v in n])
    s = lib.orc_basis_size_dim(int(degree), lib.orc_grid_dim(nn))
    if s < 0:
        raise ValueError("oracle: bad grid or degree")
    chi, pchi = _u8(np.asarray(chi).reshape(-1))
    sample, ps = _i64(np.asarray(sample).reshape(-1))
    out = np.zeros((sample.size, 4, s))
    nn = (ctypes.c_int * 3)(*[int(v) for v in n])
    hh = (ctypes.c_double * 3)(*[float(v) for v in h])
    bad = lib.orc_b_sampled(nn, hh, float(a_tilde), int(degree), pchi, sample.size, ps,
                            out.ctypes.data_as(_f64p))
    if bad < 0:
        raise MemoryError("oracle: allocation failed")
    return out
