"""One-dimensional boxes (grid (n, 1, 1), Sec. 6.1.1): set-up, operators and solves
of the CUDA path against the oracle on the same 1D grid, and the convergence of
the paper's 1D problem (Eq. 97-98) on the GPU, measured with the Gauss-quadrature
L2 error of Eq. 100 through the oracle's u^h between the nodes.

On a 1D box the x pass is the whole chain: its outputs are the D_p, and its single
row is paired with a row of zeros.  Same tolerances as the 3D parity tests: FP64
1e-10, FP32 2e-6, solves 1e-9.
"""
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


def close(a, b, tol, m=None, what=""):
    """relative L2 and max-norm error against b, over the mask m"""
    a, b = np.asarray(a), np.asarray(b)
    if m is not None:
        a, b = a[m], b[m]
    l2 = float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    mx = float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
    assert l2 < tol and mx < tol, f"{what}: rel L2 {l2:.3e}, max {mx:.3e}"


def tdev(x):
    return torch.as_tensor(np.ascontiguousarray(x), device=DEV)


def np_(t):
    return t.detach().cpu().numpy()


CASES = [(16, 1.5, 1), (32, 2.5, 1), (32, 2.5, 2), (36, 3.0, 2), (64, 2.0, 1), (256, 4.5, 2)]


@pytest.mark.parametrize("nb,a,deg", CASES)
def test_setup_and_operators_1d(nb, a, deg):
    p = W.line_problem(nb, a, deg)
    H = rk.Handle.from_problem(p, device=DEV)
    o = Oracle(p.n, p.h, a, deg, p.chi)
    assert H.s == o.s == p.s == deg + 1 and H.singular == (0, -1)
    m = p.chi > 0
    bg = np_(H.get_b(torch.empty(4 * p.s * p.nbox, dtype=torch.float64, device=DEV)))
    bo = o.b_fields()
    for i in range(2):
        close(bg[i][:, m], bo[i][:, m], 1e-10, what=f"b family {i}")
    assert np.all(bg[2] == 0.0) and np.all(bg[3] == 0.0)
    d = W.random_field(p.nbox, 3)
    close(np_(H.apply_K(tdev(d))), o.apply_K(p.V, d * p.chi), 1e-10, m, "K.u FP64")
    d32 = d.astype(np.float32)
    f32 = np_(H.apply_K(tdev(d32))).astype(np.float64)
    close(f32, o.apply_K(p.V, d32.astype(np.float64) * p.chi), 2e-6, m, "K.u FP32")
    close(np_(H.eval_u(tdev(d))), o.eval_u(d * p.chi), 1e-10, m, "u^h")
    close(np_(H.eval_u_transpose(tdev(d))), o.eval_u_transpose(d * p.chi), 1e-10, m, "U^T")
    r = W.random_field(p.nbox, 5)
    fr = np_(H.rhs(tdev(r)))
    close(fr, o.rhs(p.V, r * p.chi), 1e-10, m, "f^r")
    assert np.all(fr[~m] == 0.0)
    H.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("nb,a,deg", [(16, 1.5, 1), (64, 2.5, 1), (32, 3.0, 2)])
def test_solve_1d_matches_oracle(nb, a, deg, prec):
    p = W.line_problem(nb, a, deg)
    p.g = np.where(p.chi_gamma > 0, 0.3, 0.0)
    H = rk.Handle.from_problem(p, device=DEV)
    o = Oracle(p.n, p.h, a, deg, p.chi)
    do, _ = o.solve(p.V, p.chi_gamma, p.r, p.g, tol=1e-14)
    d, u, info = H.solve(tdev(p.r), tdev(p.g), precision=prec, tol=1e-12)
    assert info["status"] == 0
    close(np_(d), do, 1e-9, what="d")
    H.close()


def test_paper_1d_problem_converges_quadratically():
    """Sec. 6.1.1 (Eq. 97-98, a = 1.5h, linear basis): the L2 error of Eq. 100 (5
    Gauss points per cell, u^h between the nodes from the GPU's d through the
    oracle's shape functions) at 16 ... 256 nodes falls at the quadratic rate of
    Fig. 9.  (The solve stops at 1e-11: its condition number times the double
    precision bounds the reachable residual near 1e-11 at 256 nodes.)"""
    gx, gw = np.polynomial.legendre.leggauss(5)
    errs, hs = [], []
    for nb in (16, 32, 64, 128, 256):
        p = W.line_problem(nb, 1.5, 1)
        H = rk.Handle.from_problem(p, device=DEV)
        d, u, info = H.solve(tdev(p.r), tdev(p.g), precision="fp64", tol=1e-11)
        assert info["status"] == 0
        o = Oracle(p.n, p.h, 1.5, 1, p.chi)
        h = p.h[0]
        n_om = p.meta["n_omega_side"]
        left = np.arange(n_om - 1) * h
        xq = (left[:, None] + 0.5 * h * (gx[None, :] + 1.0)).reshape(-1)
        wq = np.tile(0.5 * h * gw, n_om - 1)
        uh = o.eval_points_1d(xq, np_(d))
        ue = 1.0 - (xq - 1.0) ** 2  # node 0 sits at x = -1
        errs.append(np.sqrt((wq * (uh - ue) ** 2).sum()))
        hs.append(h)
        H.close()
    rates = np.diff(np.log(errs)) / np.diff(np.log(hs))
    assert np.all(rates > 1.9) and np.all(rates < 2.1), rates


def test_1d_rejects_the_spectral_preconditioner():
    p = W.line_problem(32, 1.5, 1)
    H = rk.Handle.from_problem(p, device=DEV)
    with pytest.raises(rk.RKError):
        H.apply_precond(tdev(W.random_field(p.nbox, 1)))
    H.close()


def test_1d_gap_narrower_than_support_is_rejected():
    """Eq. 66 on a line: with a = 2h the reach is one node, so a domain that fills
    every node of the line touches its periodic image and the set-up refuses it."""
    p = W.line_problem(16, 2.0, 1)
    chi = p.chi.copy()
    chi[14] = 1
    chi[15] = 1
    with pytest.raises(rk.RKError) as e:
        rk.Handle(p.n, p.h, tdev(chi), tdev(p.chi_gamma), tdev(p.V), 1, 2.0)
    assert e.value.status == 8
    H = rk.Handle(p.n, p.h, tdev(p.chi), tdev(p.chi_gamma), tdev(p.V), 1, 2.0)
    H.close()
