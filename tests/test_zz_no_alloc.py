"""rk_apply_K_noalloc: the FP64 stiffness action for callers that cannot allocate
device memory (host applications that own all device memory through their own
pool, or loops where a cudaMalloc/cudaFree and its device-wide synchronisation
are not allowed).  Its output must equal rk_apply_K's, on two calls in a row (the
second call reuses the fixed scratch array left by the first), and the oracle's
K d (Eq. 50/54); it must refuse, before any work on the output, arrays that are
not device memory and a domain that touches its periodic image (Eq. 66).

This file is collected last on purpose, so a stop-at-first-failure run has
already run every other test when it gets here.
"""
import ctypes

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2403_19854_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2403_19854_gb300 import rk  # noqa: E402

DEV = torch.device("cuda:0")
TOL64 = 1e-10  # the FP64 parity tolerance of the GPU tests


def _noalloc(p, chi, chiV, b, d, f, n=None):
    L = rk.lib()
    g = rk.Grid()
    for k in range(3):
        g.n[k] = (n or p.n)[k]
        g.h[k] = p.h[k]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def ptr(t):
        if t is None:
            return None
        return ctypes.c_void_p(t.data_ptr() if isinstance(t, torch.Tensor) else t.ctypes.data)

    return L.rk_apply_K_noalloc(ctypes.byref(g), p.degree, p.a_tilde, ptr(chi), ptr(chiV), ptr(b), ptr(d),
                                ptr(f), stream)


def _inputs(p, H):
    chi = torch.as_tensor(p.chi, device=DEV)
    chiV = torch.as_tensor(p.V * p.chi, device=DEV)
    b = torch.empty(4 * p.s * p.nbox, dtype=torch.float64, device=DEV)
    H.get_b(b)
    return chi, chiV, b


def _rel(a, b):
    return max(np.linalg.norm(a - b) / np.linalg.norm(b), np.abs(a - b).max() / np.abs(b).max())


def _problem(kind, nb, a, deg):
    if kind == "cube":
        return W.cube_problem(nb, a, deg, "sin")
    return W.spheres_problem(n_box=nb, n_spheres=3, a_tilde=a, degree=deg, r_range=(0.2, 0.3), seed=11)


# the largest boxes the fixed scratch holds (64^3 linear, 48^3 quadratic), and an
# embedded domain whose boundary nodes rk_apply_K serves from its compact tables
@pytest.mark.parametrize("kind,nb,a,deg", [("cube", 64, 2.5, 1), ("cube", 32, 3.0, 2), ("cube", 48, 3.0, 2),
                                           ("spheres", 32, 3.0, 2)])
def test_noalloc_matches_apply_K_twice(kind, nb, a, deg):
    p = _problem(kind, nb, a, deg)
    H = rk.Handle.from_problem(p, device=DEV)
    chi, chiV, b = _inputs(p, H)
    o = Oracle(p.n, p.h, a, deg, p.chi)
    m = p.chi > 0
    for seed in (1, 2):
        dn = W.random_field(p.nbox, seed)
        d = torch.as_tensor(dn, device=DEV)
        ref = H.apply_K(d).cpu().numpy()
        f = torch.full((p.nbox,), float("nan"), dtype=torch.float64, device=DEV)
        assert _noalloc(p, chi, chiV, b, d, f) == rk.RK_OK
        torch.cuda.synchronize()
        got = f.cpu().numpy()
        assert _rel(got, ref) < TOL64, f"call {seed}: against rk_apply_K {_rel(got, ref):.3e}"
        fo = o.apply_K(p.V, dn * p.chi)
        assert _rel(got[m], fo[m]) < TOL64, f"call {seed}: against the oracle {_rel(got[m], fo[m]):.3e}"
        assert np.all(got[~m] == 0.0)
    H.close()


def test_noalloc_rejects_box_beyond_its_scratch():
    """A 128^3 box does not fit the fixed scratch: refused before any device work."""
    p = W.cube_problem(16, 2.5, 1, "zero")
    dummy = torch.zeros(8, dtype=torch.float64, device=DEV)
    st = _noalloc(p, dummy, dummy, dummy, dummy, dummy, n=(128, 128, 128))
    assert st == 8  # RK_ERR_UNSUPPORTED


def test_noalloc_rejects_host_arrays():
    """Host arrays would need staging buffers: RK_ERR_INVALID_ARG, output untouched."""
    p = W.cube_problem(16, 2.5, 1, "sin")
    H = rk.Handle.from_problem(p, device=DEV)
    chi, chiV, b = _inputs(p, H)
    d = torch.as_tensor(W.random_field(p.nbox, 1), device=DEV)
    f = torch.full((p.nbox,), 7.0, dtype=torch.float64, device=DEV)
    d_host = np.ascontiguousarray(d.cpu().numpy())
    f_host = np.full(p.nbox, 7.0)
    assert _noalloc(p, chi, chiV, b, d_host, f) == 1        # RK_ERR_INVALID_ARG
    assert _noalloc(p, chi, chiV, b, d, f_host) == 1
    assert _noalloc(p, chi.cpu().numpy(), chiV, b, d, f) == 1
    torch.cuda.synchronize()
    assert np.all(f.cpu().numpy() == 7.0) and np.all(f_host == 7.0)
    H.close()


def test_noalloc_rejects_a_gap_narrower_than_the_support():
    """A domain that touches its periodic image within the support (Eq. 66) gives a
    different operator; like rk_setup, the call refuses it (RK_ERR_UNSUPPORTED) and
    leaves f untouched.  At a = 2.5h the reach is two nodes: one empty node is too
    few, two suffice."""
    p = W.cube_problem(16, 2.5, 1, "sin")
    H = rk.Handle.from_problem(p, device=DEV)
    chi, chiV, b = _inputs(p, H)
    d = torch.as_tensor(W.random_field(p.nbox, 1), device=DEV)
    f = torch.full((p.nbox,), 7.0, dtype=torch.float64, device=DEV)
    chi3 = p.chi.reshape(16, 16, 16).copy()
    chi3[:, :, 14] = chi3[:, :, 0]  # x nodes 0..14 occupied: one empty node (15)
    narrow = torch.as_tensor(chi3.reshape(-1), device=DEV)
    assert _noalloc(p, narrow, chiV, b, d, f) == 8  # RK_ERR_UNSUPPORTED
    torch.cuda.synchronize()
    assert np.all(f.cpu().numpy() == 7.0)
    # the unmodified domain (two empty nodes per axis) passes on the next call
    assert _noalloc(p, chi, chiV, b, d, f) == rk.RK_OK
    torch.cuda.synchronize()
    ref = H.apply_K(d).cpu().numpy()
    assert _rel(f.cpu().numpy(), ref) < TOL64
    H.close()
