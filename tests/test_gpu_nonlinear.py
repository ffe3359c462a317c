"""Nonlinear reaction terms (Appendix B) against the oracle: f^N(d) = U^T(V N(U d))
from the oracle's explicit shape functions (Eq. B.4), and Alg. B.3's nonlinear CG
against a dense Newton solve of K d + f^N(d) = f^r assembled from the oracle."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.oracle import Oracle
from paper_2403_19854_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2403_19854_gb300 import rk  # noqa: E402

DEV = torch.device("cuda:0")
N = {"cubic": (lambda u: u ** 3, lambda u: 3 * u ** 2), "sinh": (np.sinh, np.cosh), "exp": (np.exp, np.exp)}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def tdev(x):
    return torch.as_tensor(np.ascontiguousarray(x), device=DEV)


def np_(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("kind", ["cubic", "sinh", "exp"])
@pytest.mark.parametrize("deg,a", [(1, 2.5), (2, 3.0)])
def test_nonlinear_force(kind, deg, a):
    p = W.cube_problem(16, a, deg, "sin")
    H = rk.Handle.from_problem(p, device=DEV)
    o = Oracle(p.n, p.h, a, deg, p.chi)
    d = 0.5 * W.random_field(p.nbox, 3) * p.chi
    u = o.eval_u(d)
    fo = o.eval_u_transpose(p.V * 2.0 * N[kind][0](u) * p.chi)
    f = np_(H.nonlinear_force(tdev(d), kind, 2.0))
    assert rel(f, fo) < 1e-10
    H.close()


GRAD_CASES = [("cube", 16, 2.5, 1), ("cube", 16, 3.0, 2), ("spheres", 32, 2.5, 1), ("plane", 32, 2.5, 2),
              ("line", 64, 3.0, 2)]


@pytest.mark.parametrize("kind", ["cubic", "sinh", "exp"])
@pytest.mark.parametrize("geom,nb,a,deg", GRAD_CASES)
def test_gradient_type_force_eq_b10(kind, geom, nb, a, deg):
    """f^N = B^T N with N^k = a_k N(u^h) (Eq. B.5-B.8 in the form of Eq. B.10),
    against the oracle's explicit shape-function gradients (Eq. B.6 with direct
    nodal integration); the oracle's B^T is pinned by gradient reproduction."""
    if geom == "cube":
        p = W.cube_problem(nb, a, deg, "sin")
    elif geom == "spheres":
        p = W.spheres_problem(n_box=nb, n_spheres=3, a_tilde=a, degree=deg, r_range=(0.2, 0.3), seed=8)
    elif geom == "plane":
        p = W.plane_problem(nb, a, deg)
    else:
        p = W.line_problem(nb, a, deg)
    H = rk.Handle.from_problem(p, device=DEV)
    o = Oracle(p.n, p.h, a, deg, p.chi)
    av = [0.7, -1.3 if p.n[1] > 1 else 0.0, 0.4 if p.n[2] > 1 else 0.0]
    d = 0.5 * W.random_field(p.nbox, 3) * p.chi
    u = o.eval_u(d)
    Nu = 2.0 * N[kind][0](u) * p.chi
    fo = o.grad_transpose(p.V, np.stack([av[k] * Nu for k in range(3)]))
    f = np_(H.nonlinear_grad_force(tdev(d), kind, 2.0, av))
    assert rel(f, fo) < 1e-10, rel(f, fo)
    assert np.abs(f - fo).max() <= 1e-10 * np.abs(fo).max()
    assert np.all(f[p.chi == 0] == 0.0)
    H.close()


def _newton_reference(p, o, kind, c):
    o.assemble_K(p.V)
    ptr, col, val = o.K_csr()
    nodes = np.flatnonzero(p.chi)
    nn = len(nodes)
    K = sp.csr_matrix((val, col, ptr), shape=(nn, nn)).toarray()
    nbr, psi, _ = o.shape_tables()
    rows, cols = np.nonzero(nbr >= 0)
    U = sp.csr_matrix((psi[rows, cols], (rows, nbr[rows, cols])), shape=(nn, nn)).toarray()
    V = p.V[nodes]
    free = p.chi_gamma[nodes] == 0
    fr = o.rhs(p.V, p.r)[nodes]
    d = np.where(free, 0.0, p.g[nodes])
    f, fp = N[kind]
    for _ in range(50):
        u = U @ d
        R = (K @ d + U.T @ (V * c * f(u)) - fr)[free]
        if np.linalg.norm(R) <= 1e-14 * np.linalg.norm(fr[free]):
            break
        J = K + U.T @ ((V * c * fp(u))[:, None] * U)
        d[free] -= np.linalg.solve(J[np.ix_(free, free)], R)
    out = np.zeros(p.nbox)
    out[nodes] = d
    return out


@pytest.mark.parametrize("kind,c", [("cubic", 50.0), ("sinh", 5.0), ("exp", 1.0)])
def test_nonlinear_cg_alg_b3(kind, c):
    p = W.cube_problem(16, 2.5, 1, "sin")
    p.g = np.where(p.chi_gamma > 0, 0.2 * W.random_field(p.nbox, 4), 0.0)
    H = rk.Handle.from_problem(p, device=DEV)
    o = Oracle(p.n, p.h, 2.5, 1, p.chi)
    ref = _newton_reference(p, o, kind, c)
    d, u, info = H.solve_nonlinear(tdev(p.r), tdev(p.g), kind, c, tol=1e-12, max_iter=20000)
    assert info["status"] == 0
    assert rel(np_(d), ref) < 1e-8
    gam = p.chi_gamma > 0
    assert np.array_equal(np_(d)[gam], p.g[gam])
    H.close()


def test_zero_nonlinearity_is_the_linear_solve():
    p = W.cube_problem(16, 2.5, 1, "sin")
    H = rk.Handle.from_problem(p, device=DEV)
    d, _, info = H.solve_nonlinear(tdev(p.r), tdev(p.g), "cubic", 0.0, tol=1e-12, max_iter=20000)
    d0, _, _ = H.solve(tdev(p.r), tdev(p.g), precision="fp64", tol=1e-13)
    assert rel(np_(d), np_(d0)) < 1e-9
    H.close()
