"""rk_apply_K_noalloc: the FP64 stiffness action for callers that cannot allocate
device memory (host applications that own all device memory through their own
pool, or loops where a cudaMalloc/cudaFree and its device-wide synchronisation
are not allowed).  Its output must equal rk_apply_K's, on two calls in a row
(the second call reuses the fixed scratch array left by the first).

This file is collected last on purpose, so a stop-at-first-failure run has
already run every other test when it gets here.
"""
import ctypes

import numpy as np
import pytest

from paper_2403_19854_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2403_19854_gb300 import rk  # noqa: E402

DEV = torch.device("cuda:0")
TOL64 = 1e-10  # the FP64 parity tolerance of the GPU tests


def _noalloc(p, chi, chiV, b, d, f):
    L = rk.lib()
    L.rk_apply_K_noalloc.argtypes = [ctypes.POINTER(rk.Grid), ctypes.c_int32, ctypes.c_double, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p]
    L.rk_apply_K_noalloc.restype = ctypes.c_int
    g = rk.Grid()
    for k in range(3):
        g.n[k] = p.n[k]
        g.h[k] = p.h[k]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
    return L.rk_apply_K_noalloc(ctypes.byref(g), p.degree, p.a_tilde, ptr(chi), ptr(chiV), ptr(b), ptr(d),
                                ptr(f), stream)


@pytest.mark.parametrize("nb,a,deg", [(64, 2.5, 1), (32, 3.0, 2)])
def test_noalloc_matches_apply_K_twice(nb, a, deg):
    p = W.cube_problem(nb, a, deg, "sin")
    H = rk.Handle.from_problem(p, device=DEV)
    chi = torch.as_tensor(p.chi, device=DEV)
    chiV = torch.as_tensor(p.V * p.chi, device=DEV)
    b = torch.empty(4 * p.s * p.nbox, dtype=torch.float64, device=DEV)
    H.get_b(b)
    for seed in (1, 2):
        d = torch.as_tensor(W.random_field(p.nbox, seed), device=DEV)
        ref = H.apply_K(d).cpu().numpy()
        f = torch.full((p.nbox,), float("nan"), dtype=torch.float64, device=DEV)
        assert _noalloc(p, chi, chiV, b, d, f) == rk.RK_OK
        torch.cuda.synchronize()
        got = f.cpu().numpy()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < TOL64, f"call {seed}: rel err {err}"
    H.close()


def test_noalloc_rejects_box_beyond_its_scratch():
    """A 128^3 box does not fit the fixed scratch: refused before any device work."""
    p = W.cube_problem(16, 2.5, 1, "zero")
    p.n = (128, 128, 128)
    dummy = torch.zeros(8, dtype=torch.float64, device=DEV)
    st = _noalloc(p, dummy, dummy, dummy, dummy, dummy)
    assert st == 8  # RK_ERR_UNSUPPORTED
