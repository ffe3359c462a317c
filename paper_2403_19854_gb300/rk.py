"""Python binding of the FC-RKPM C ABI (include/fcrkpm.h).

Argument marshalling only: every step of set-up, K.u, f^r, u^h and the solves runs
in the CUDA library.  Arrays may be torch tensors (CUDA or CPU) or numpy arrays;
CUDA tensors are passed as device pointers, everything else as host pointers
(the library stages host arrays itself).  If the shared library has not been
built, loading raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfcrkpm.so")
_lib = None

RK_OK = 0
STATUS = ["RK_OK", "RK_ERR_INVALID_ARG", "RK_ERR_CUDA", "RK_ERR_OOM", "RK_ERR_SINGULAR_MOMENT",
          "RK_ERR_NOT_CONVERGED", "RK_ERR_BREAKDOWN", "RK_ERR_TIMEOUT", "RK_ERR_UNSUPPORTED"]
RK_F64, RK_F32 = 0, 1
RK_PREC_FP64, RK_PREC_MIXED = 0, 1

EXPORTED = ["rk_default_solve_opts", "rk_supported_length", "rk_setup", "rk_singular_nodes", "rk_apply_K",
            "rk_rhs", "rk_eval_u", "rk_eval_u_transpose", "rk_get_b", "rk_get_shape", "rk_solve",
            "rk_solve_adjoint", "rk_destroy", "rk_status_string", "rk_last_error_message",
            "rk_kernel_launches", "rk_profile_enable", "rk_profile_read", "rk_profile_class_name",
            "rk_solve_vjp", "rk_clone", "rk_solve_batched", "rk_apply_precond", "rk_boundary_rhs",
            "rk_solve_neumann", "rk_apply_M", "rk_lumped_mass", "rk_transient_explicit", "rk_transient_implicit",
            "rk_nonlinear_force", "rk_nonlinear_grad_force", "rk_solve_penalty", "rk_solve_nonlinear", "rk_debug_short_waits", "rk_apply_K_noalloc"]
NONLINEARITIES = {"cubic": 0, "sinh": 1, "exp": 2}
PROF_CLASSES = 12


class RKError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        super().__init__(f"{STATUS[status] if 0 <= status < len(STATUS) else status}: {msg}")


class Grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32 * 3), ("h", ctypes.c_double * 3)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("inner_tol", ctypes.c_double), ("max_outer", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("x0_given", ctypes.c_int32), ("fp64_finish", ctypes.c_int32),
                ("precond", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class BatchItem(ctypes.Structure):
    _fields_ = [("h", ctypes.c_void_p), ("r", ctypes.c_void_p), ("g", ctypes.c_void_p), ("d", ctypes.c_void_p),
                ("u", ctypes.c_void_p)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("outer", ctypes.c_int32), ("matvec_f32", ctypes.c_int32),
                ("matvec_f64", ctypes.c_int32), ("rel_residual", ctypes.c_double), ("f_norm", ctypes.c_double),
                ("setup_ms", ctypes.c_double), ("solve_ms", ctypes.c_double), ("status", ctypes.c_int32),
                ("fp64_iterations", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


def lib():
    """Load libfcrkpm.so (built by paper_2403_19854_gb300.build / __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"FC-RKPM CUDA library not built ({LIB_PATH}); run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
    L.rk_default_solve_opts.argtypes = [ctypes.POINTER(SolveOpts)]
    L.rk_default_solve_opts.restype = None
    L.rk_supported_length.argtypes = [ctypes.c_int]
    L.rk_supported_length.restype = ctypes.c_int
    L.rk_setup.argtypes = [ctypes.POINTER(Grid), vp, vp, vp, i32, f64, vp, ctypes.POINTER(vp)]
    L.rk_singular_nodes.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    L.rk_apply_K.argtypes = [vp, vp, vp, i32, vp]
    L.rk_apply_precond.argtypes = [vp, vp, vp, i32, vp]
    L.rk_boundary_rhs.argtypes = [vp, vp, vp, vp, vp]
    L.rk_apply_M.argtypes = [vp, vp, vp, i32, vp]
    L.rk_nonlinear_force.argtypes = [vp, vp, i32, ctypes.c_double, vp, vp]
    L.rk_solve_penalty.argtypes = [vp, vp, vp, vp, ctypes.c_double, vp, vp, ctypes.POINTER(SolveOpts),
                                   ctypes.POINTER(SolveInfo), vp]
    L.rk_nonlinear_grad_force.argtypes = [vp, vp, i32, ctypes.c_double, ctypes.POINTER(ctypes.c_double), vp, vp]
    L.rk_solve_nonlinear.argtypes = [vp, vp, vp, i32, ctypes.c_double, vp, vp, ctypes.POINTER(SolveOpts),
                                     ctypes.POINTER(SolveInfo), vp]
    L.rk_lumped_mass.argtypes = [vp, vp, vp]
    L.rk_transient_explicit.argtypes = [vp, vp, vp, ctypes.c_double, i32, vp, vp]
    L.rk_transient_implicit.argtypes = [vp, vp, vp, ctypes.c_double, i32, vp, ctypes.POINTER(SolveOpts),
                                        ctypes.POINTER(SolveInfo), vp]
    L.rk_solve_neumann.argtypes = [vp, vp, vp, vp, vp, vp, vp, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo),
                                   vp]
    for name in ("rk_rhs", "rk_eval_u", "rk_eval_u_transpose"):
        getattr(L, name).argtypes = [vp, vp, vp, vp]
    L.rk_get_b.argtypes = [vp, vp, vp]
    L.rk_get_shape.argtypes = [vp, ctypes.POINTER(ctypes.c_int32 * 3), ctypes.POINTER(i32),
                               ctypes.POINTER(ctypes.c_int64)]
    L.rk_solve.argtypes = [vp, vp, vp, vp, vp, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo), vp]
    L.rk_solve_adjoint.argtypes = [vp, vp, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo), vp]
    L.rk_solve_vjp.argtypes = [vp, vp, vp, vp, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo), vp]
    L.rk_clone.argtypes = [vp, ctypes.POINTER(vp)]
    L.rk_solve_batched.argtypes = [ctypes.POINTER(BatchItem), i32, ctypes.POINTER(SolveOpts),
                                   ctypes.POINTER(SolveInfo), vp]
    L.rk_destroy.argtypes = [vp]
    L.rk_status_string.argtypes = [ctypes.c_int]
    L.rk_status_string.restype = ctypes.c_char_p
    L.rk_last_error_message.argtypes = []
    L.rk_last_error_message.restype = ctypes.c_char_p
    L.rk_kernel_launches.argtypes = []
    L.rk_kernel_launches.restype = ctypes.c_int64
    L.rk_profile_enable.argtypes = [vp, i32]
    L.rk_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64), i32]
    L.rk_profile_class_name.argtypes = [i32]
    L.rk_profile_class_name.restype = ctypes.c_char_p
    L.rk_debug_short_waits.argtypes = [vp, i32]
    L.rk_apply_K_noalloc.argtypes = [ctypes.POINTER(Grid), i32, f64, vp, vp, vp, vp, vp, vp]
    for name in EXPORTED:
        if getattr(L, name).restype is ctypes.c_int:  # default
            pass
    _lib = L
    return L


def _check(status):
    if status != RK_OK:
        raise RKError(status, lib().rk_last_error_message().decode())


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """(pointer, keep-alive) of a torch tensor or numpy array; None -> NULL."""
    if x is None:
        return None, None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr()), x
    a = np.ascontiguousarray(x)
    return ctypes.c_void_p(a.ctypes.data), a


def _stream(x=None):
    """Current torch CUDA stream handle when x is a CUDA tensor (else the default stream)."""
    try:
        import torch
        if torch.cuda.is_available() and (x is None or (_is_torch(x) and x.is_cuda)):
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return ctypes.c_void_p(0)


def _like(x, dtype, n):
    if _is_torch(x):
        import torch
        return torch.empty(n, dtype=torch.float64 if dtype == RK_F64 else torch.float32, device=x.device)
    return np.empty(n, dtype=np.float64 if dtype == RK_F64 else np.float32)


def default_opts(**kw) -> SolveOpts:
    o = SolveOpts()
    lib().rk_default_solve_opts(ctypes.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": RK_PREC_FP64, "mixed": RK_PREC_MIXED}[v]
        if k == "precond" and isinstance(v, str):
            v = {"none": 0, "spectral": 1}[v]
        setattr(o, k, v)
    return o


def supported_length(n: int) -> bool:
    return bool(lib().rk_supported_length(int(n)))


def kernel_launches() -> int:
    """Kernels launched by the library in this process so far."""
    return int(lib().rk_kernel_launches())


class Handle:
    """An rk_handle: set-up (Alg. 1) done on construction, freed by close()/del."""

    def __init__(self, n, h, chi, chi_gamma, V, degree, a_tilde, stream=None):
        g = Grid()
        for k in range(3):
            g.n[k] = int(n[k])
            g.h[k] = float(h[k])
        self.n = tuple(int(v) for v in n)
        self.nbox = self.n[0] * self.n[1] * self.n[2]
        self.degree = int(degree)
        dim = 3 if self.n[2] > 1 else (2 if self.n[1] > 1 else 1)
        self.s = {3: (4, 10), 2: (3, 6), 1: (2, 3)}[dim][self.degree - 1]  # basis size of the box's dimension
        pc, kc = _ptr(chi)
        pg, kg = _ptr(chi_gamma)
        pV, kV = _ptr(V)
        out = ctypes.c_void_p()
        st = lib().rk_setup(ctypes.byref(g), pc, pg, pV, self.degree, float(a_tilde),
                            stream if stream is not None else _stream(chi), ctypes.byref(out))
        self._h = out
        self.singular = (0, -1)
        if st != RK_OK and not out:
            _check(st)
        cnt, first = ctypes.c_int64(), ctypes.c_int64()
        lib().rk_singular_nodes(self._h, ctypes.byref(cnt), ctypes.byref(first))
        self.singular = (cnt.value, first.value)
        if st != RK_OK and st != 4:
            _check(st)
        self.setup_status = st

    @classmethod
    def from_problem(cls, p, device=None):
        """Set up from a workloads.Problem (inputs copied to `device` as torch tensors
        when given, else passed as host arrays)."""
        if device is not None:
            import torch
            chi = torch.as_tensor(p.chi, device=device)
            cg = torch.as_tensor(p.chi_gamma, device=device)
            V = torch.as_tensor(p.V, device=device)
            return cls(p.n, p.h, chi, cg, V, p.degree, p.a_tilde)
        return cls(p.n, p.h, p.chi, p.chi_gamma, p.V, p.degree, p.a_tilde)

    def clone(self):
        """A handle sharing this set-up with its own workspaces (another right-hand side)."""
        out = ctypes.c_void_p()
        _check(lib().rk_clone(self._h, ctypes.byref(out)))
        c = Handle.__new__(Handle)
        c.n, c.nbox, c.degree, c.s = self.n, self.nbox, self.degree, self.s
        c.singular, c.setup_status = self.singular, self.setup_status
        c._h = out
        c._parent = self  # the parent must outlive the clone
        return c

    def close(self):
        if getattr(self, "_h", None):
            lib().rk_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -------------------------------------------------------------- operators
    def apply_K(self, d, f=None, stream=None):
        """f = K d (Alg. 2); float32 input -> FP32 path, float64 -> FP64 path."""
        is32 = (str(d.dtype).endswith("float32"))
        dt = RK_F32 if is32 else RK_F64
        if f is None:
            f = _like(d, dt, self.nbox)
        pd, kd = _ptr(d)
        pf, kf = _ptr(f)
        _check(lib().rk_apply_K(self._h, pd, pf, dt, stream if stream is not None else _stream(d)))
        return f

    def apply_precond(self, r, z=None, stream=None):
        """z = M^{-1} r, the spectral preconditioner (float32 -> FP32 path, float64 -> FP64)."""
        is32 = (str(r.dtype).endswith("float32"))
        dt = RK_F32 if is32 else RK_F64
        if z is None:
            z = _like(r, dt, self.nbox)
        pr, kr = _ptr(r)
        pz, kz = _ptr(z)
        _check(lib().rk_apply_precond(self._h, pr, pz, dt, stream if stream is not None else _stream(r)))
        return z

    def _unary(self, fn, x, out, stream):
        if out is None:
            out = _like(x, RK_F64, self.nbox)
        px, kx = _ptr(x)
        po, ko = _ptr(out)
        _check(fn(self._h, px, po, stream if stream is not None else _stream(x)))
        return out

    def rhs(self, r, out=None, stream=None):
        """f^r (Alg. 4)."""
        return self._unary(lib().rk_rhs, r, out, stream)

    def eval_u(self, d, out=None, stream=None):
        """u^h at the nodes (Alg. 3)."""
        return self._unary(lib().rk_eval_u, d, out, stream)

    def eval_u_transpose(self, e, out=None, stream=None):
        """Transpose of Alg. 3."""
        return self._unary(lib().rk_eval_u_transpose, e, out, stream)

    def get_b(self, out=None):
        """(4, s, nbox) FP64 correction coefficients b^0, b^x, b^y, b^z."""
        if out is None:
            out = np.empty(4 * self.s * self.nbox)
        po, ko = _ptr(out)
        _check(lib().rk_get_b(self._h, po, _stream(out)))
        return out.reshape(4, self.s, self.nbox) if not _is_torch(out) else out.view(4, self.s, self.nbox)

    def shape(self):
        n = (ctypes.c_int32 * 3)()
        s = ctypes.c_int32()
        nom = ctypes.c_int64()
        _check(lib().rk_get_shape(self._h, ctypes.byref(n), ctypes.byref(s), ctypes.byref(nom)))
        return tuple(n), s.value, nom.value

    # ---------------------------------------------------------- instrumentation
    def debug_short_waits(self, enable=True):
        """Diagnostic: make the first bounded wait for each input tile of the TMA-fed
        passes give up at once (the next synchronising call reports RK_ERR_TIMEOUT)."""
        _check(lib().rk_debug_short_waits(self._h, 1 if enable else 0))

    def profile(self, enable=True):
        """Start/stop per-kernel-class CUDA-event timing (counters cleared)."""
        _check(lib().rk_profile_enable(self._h, 1 if enable else 0))

    def profile_read(self):
        """{(class name, 'f32'|'f64'): (ms, launches)} since profile(True)."""
        n = 2 * PROF_CLASSES
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int64 * n)()
        _check(lib().rk_profile_read(self._h, ms, cnt, n))
        out = {}
        for i in range(n):
            if cnt[i]:
                name = lib().rk_profile_class_name(i % PROF_CLASSES).decode()
                out[(name, "f64" if i >= PROF_CLASSES else "f32")] = (ms[i], cnt[i])
        return out

    # ------------------------------------------------------------------ solves
    # ------------------------------------------------------- time-dependent
    def apply_M(self, v, out=None, stream=None):
        """f^m = M v (Alg. C.1); float32 -> FP32 path, float64 -> FP64."""
        is32 = (str(v.dtype).endswith("float32"))
        dt = RK_F32 if is32 else RK_F64
        if out is None:
            out = _like(v, dt, self.nbox)
        pv, kv = _ptr(v)
        po, ko = _ptr(out)
        _check(lib().rk_apply_M(self._h, pv, po, dt, stream if stream is not None else _stream(v)))
        return out

    def lumped_mass(self, out=None, like=None, stream=None):
        """M^l (Alg. C.2), FP64."""
        if out is None:
            out = _like(like if like is not None else np.empty(1), RK_F64, self.nbox)
        po, ko = _ptr(out)
        _check(lib().rk_lumped_mass(self._h, po, stream if stream is not None else _stream(out)))
        return out

    def transient_explicit(self, f, g, dt, n_steps, d, stream=None):
        """Alg. C.3 (forward Euler, lumped mass): advances d in place by n_steps."""
        pf, kf = _ptr(f)
        pg, kg = _ptr(g)
        pd, kd = _ptr(d)
        _check(lib().rk_transient_explicit(self._h, pf, pg, float(dt), int(n_steps), pd,
                                           stream if stream is not None else _stream(d)))
        return d

    def transient_implicit(self, f, g, dt, n_steps, d, opts=None, stream=None, **kw):
        """Alg. C.4 (backward Euler, FP64 CG per step): advances d in place; returns info."""
        if opts is None:
            opts = default_opts(**kw)
        info = SolveInfo()
        pf, kf = _ptr(f)
        pg, kg = _ptr(g)
        pd, kd = _ptr(d)
        _check(lib().rk_transient_implicit(self._h, pf, pg, float(dt), int(n_steps), pd, ctypes.byref(opts),
                                           ctypes.byref(info), stream if stream is not None else _stream(d)))
        return info.as_dict()

    # ------------------------------------------------------------ nonlinear
    def nonlinear_force(self, d, kind, c, out=None, stream=None):
        """f^N(d) of Appendix B for N in NONLINEARITIES ("cubic", "sinh", "exp") times c."""
        if out is None:
            out = _like(d, RK_F64, self.nbox)
        pd, kd = _ptr(d)
        po, ko = _ptr(out)
        _check(lib().rk_nonlinear_force(self._h, pd, NONLINEARITIES[kind], float(c), po,
                                        stream if stream is not None else _stream(d)))
        return out

    def nonlinear_grad_force(self, d, kind, c, a, out=None, stream=None):
        """Gradient-type force of Eq. B.5-B.8 / B.10: B^T N with N^k = a_k N(u^h),
        N in NONLINEARITIES times c, a a 3-vector (a[2] unused in 2D)."""
        if out is None:
            out = _like(d, RK_F64, self.nbox)
        av = (ctypes.c_double * 3)(*[float(v) for v in a])
        pd, kd = _ptr(d)
        po, ko = _ptr(out)
        _check(lib().rk_nonlinear_grad_force(self._h, pd, NONLINEARITIES[kind], float(c), av, po,
                                             stream if stream is not None else _stream(d)))
        return out

    def solve_nonlinear(self, r, g, kind, c, d=None, u=None, opts=None, stream=None, raise_on_error=True, **kw):
        """Alg. B.3 (nonlinear CG): returns (d, u, info dict)."""
        if opts is None:
            opts = default_opts(**kw)
        if d is None:
            d = _like(r, RK_F64, self.nbox)
        if u is None:
            u = _like(r, RK_F64, self.nbox)
        info = SolveInfo()
        pr, kr = _ptr(r)
        pg, kg = _ptr(g)
        pd, kd = _ptr(d)
        pu, ku = _ptr(u)
        st = lib().rk_solve_nonlinear(self._h, pr, pg, NONLINEARITIES[kind], float(c), pd, pu, ctypes.byref(opts),
                                      ctypes.byref(info), stream if stream is not None else _stream(r))
        if raise_on_error:
            _check(st)
        return d, u, info.as_dict()

    def solve_penalty(self, r, g, A, beta, d=None, u=None, opts=None, stream=None, raise_on_error=True, **kw):
        """Essential conditions by the penalty method (Sec. 2.4): (K + beta U^T diag(A) U) d =
        f^r + beta U^T (A g) over every chi node, FP64 CG.  Returns (d, u, info dict)."""
        if opts is None:
            opts = default_opts(**kw)
        if d is None:
            d = _like(r, RK_F64, self.nbox)
        if u is None:
            u = _like(r, RK_F64, self.nbox)
        info = SolveInfo()
        pr, kr = _ptr(r)
        pg, kg = _ptr(g)
        pa, ka = _ptr(A)
        pd, kd = _ptr(d)
        pu, ku = _ptr(u)
        st = lib().rk_solve_penalty(self._h, pr, pg, pa, float(beta), pd, pu, ctypes.byref(opts), ctypes.byref(info),
                                    stream if stream is not None else _stream(r))
        if raise_on_error:
            _check(st)
        return d, u, info.as_dict()

    def boundary_rhs(self, q, A, out=None, stream=None):
        """f^q of Alg. A.1 for Neumann data q and boundary weights A (FP64)."""
        if out is None:
            out = _like(q, RK_F64, self.nbox)
        pq, kq = _ptr(q)
        pa, ka = _ptr(A)
        po, ko = _ptr(out)
        _check(lib().rk_boundary_rhs(self._h, pq, pa, po, stream if stream is not None else _stream(q)))
        return out

    def solve(self, r, g=None, d=None, u=None, opts=None, want_u=True, stream=None, raise_on_error=True, q=None,
              A=None, **kw):
        """Alg. 5: returns (d, u, info dict); with q and A the Neumann term f^q of
        Alg. A.1 joins the right-hand side."""
        if opts is None:
            opts = default_opts(**kw)
        if d is None:
            d = _like(r, RK_F64, self.nbox)
        if u is None and want_u:
            u = _like(r, RK_F64, self.nbox)
        info = SolveInfo()
        pr, kr = _ptr(r)
        pg, kg = _ptr(g)
        pd, kd = _ptr(d)
        pu, ku = _ptr(u)
        if q is not None:
            pq, kq = _ptr(q)
            pa, ka = _ptr(A)
            st = lib().rk_solve_neumann(self._h, pr, pg, pq, pa, pd, pu, ctypes.byref(opts), ctypes.byref(info),
                                        stream if stream is not None else _stream(r))
        else:
            st = lib().rk_solve(self._h, pr, pg, pd, pu, ctypes.byref(opts), ctypes.byref(info),
                                stream if stream is not None else _stream(r))
        if raise_on_error:
            _check(st)
        return d, u, info.as_dict()

    def solve_vjp(self, u_bar, opts=None, stream=None, **kw):
        """(r_bar, g_bar, info): vector-Jacobian product of u^h(r, g) for the cotangent u_bar."""
        if opts is None:
            opts = default_opts(**kw)
        rb = _like(u_bar, RK_F64, self.nbox)
        gb = _like(u_bar, RK_F64, self.nbox)
        info = SolveInfo()
        pu, ku = _ptr(u_bar)
        pr, k1 = _ptr(rb)
        pg, k2 = _ptr(gb)
        _check(lib().rk_solve_vjp(self._h, pu, pr, pg, ctypes.byref(opts), ctypes.byref(info),
                                  stream if stream is not None else _stream(u_bar)))
        return rb, gb, info.as_dict()

    def solve_adjoint(self, r, g, u_target, opts=None, stream=None, **kw):
        """Gradient of J = 1/2 |u^h - u_target|^2 over chi: returns (J, dJ/dr, dJ/dg, info)."""
        if opts is None:
            opts = default_opts(**kw)
        dr = _like(r, RK_F64, self.nbox)
        dg = _like(r, RK_F64, self.nbox)
        J = ctypes.c_double()
        info = SolveInfo()
        pr, kr = _ptr(r)
        pg, kg = _ptr(g)
        pt, kt = _ptr(u_target)
        pdr, k1 = _ptr(dr)
        pdg, k2 = _ptr(dg)
        _check(lib().rk_solve_adjoint(self._h, pr, pg, pt, pdr, pdg, ctypes.byref(J), ctypes.byref(opts),
                                      ctypes.byref(info), stream if stream is not None else _stream(r)))
        return J.value, dr, dg, info.as_dict()


def solve_batched(items, opts=None, stream=None, raise_on_error=True, **kw):
    """Alg. 5 for many problems at once (mixed precision).  items: sequence of
    (handle, r, g, d, u) with distinct handles (Handle.clone() for several
    right-hand sides of one domain); d and u are outputs (u may be None).
    Returns the list of per-item info dicts."""
    if opts is None:
        opts = default_opts(**kw)
    n = len(items)
    arr = (BatchItem * n)()
    keep = []
    for i, (h, r, g, d, u) in enumerate(items):
        pr, kr = _ptr(r)
        pg, kg = _ptr(g)
        pd, kd = _ptr(d)
        pu, ku = _ptr(u)
        keep += [kr, kg, kd, ku]
        arr[i].h = h._h.value if isinstance(h._h, ctypes.c_void_p) else h._h
        arr[i].r, arr[i].g, arr[i].d, arr[i].u = (pr.value if pr else None, pg.value if pg else None,
                                                 pd.value if pd else None, pu.value if pu else None)
    infos = (SolveInfo * n)()
    st = lib().rk_solve_batched(arr, n, ctypes.byref(opts), infos, stream if stream is not None else _stream(items[0][1]))
    if raise_on_error:
        _check(st)
    return [infos[i].as_dict() for i in range(n)]


def poisson_solve(handle, r, g, opts=None, **kw):
    """u^h(r, g) of Alg. 5 as a differentiable torch operation (CUDA float64 tensors).

    Backward is one adjoint solve through rk_solve_vjp (the map is linear, so the
    forward solve is recomputed from nothing and no forward state is stored)."""
    import torch

    if opts is None:
        opts = default_opts(**kw)

    class _Solve(torch.autograd.Function):
        @staticmethod
        def forward(ctx, r_, g_):
            _, u, _ = handle.solve(r_.detach().contiguous(), g_.detach().contiguous(), opts=opts)
            return u

        @staticmethod
        def backward(ctx, u_bar):
            rb, gb, _ = handle.solve_vjp(u_bar.detach().contiguous(), opts=opts)
            return rb, gb

    return _Solve.apply(r, g)
