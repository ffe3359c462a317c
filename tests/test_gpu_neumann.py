"""Neumann data (Appendix A): f^q of Alg. A.1 and solves with mixed boundary
conditions, against the oracle.

The oracle's f^q is sum_S Psi_I(x_S) q_S A_S (Eq. A.2) from its explicit shape
functions; its solve assembles K and the right-hand side f^r + f^q, fixes d = g on
Gamma_g and factors the rest.
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


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def tdev(x):
    return torch.as_tensor(np.ascontiguousarray(x), device=DEV)


def np_(t):
    return t.detach().cpu().numpy()


def mixed_bc_cube(nb, a, deg):
    """Cube with Dirichlet data on the two x faces and Neumann data on the other
    four (weights h^2 halved on edges, random flux), random source and g."""
    p = W.cube_problem(nb, a, deg, "zero")
    n_om = p.meta["n_omega_side"]
    k, j, i = np.meshgrid(np.arange(nb), np.arange(nb), np.arange(nb), indexing="ij")
    i, j, k = i.reshape(-1), j.reshape(-1), k.reshape(-1)
    inside = p.chi > 0
    xface = inside & ((i == 0) | (i == n_om - 1))
    yzface = inside & ~xface & ((j == 0) | (j == n_om - 1) | (k == 0) | (k == n_om - 1))
    edge = yzface & ((j == 0) | (j == n_om - 1)) & ((k == 0) | (k == n_om - 1))
    rng = np.random.default_rng(nb)
    A = np.where(yzface, p.h[0] ** 2 * np.where(edge, 0.5, 1.0), 0.0)
    q = np.where(yzface, rng.standard_normal(p.nbox), 0.0)
    p.chi_gamma = xface.astype(np.uint8)
    p.r = np.where(inside, rng.standard_normal(p.nbox), 0.0)
    p.g = np.where(xface, 0.1 * rng.standard_normal(p.nbox), 0.0)
    return p, q, A


@pytest.mark.parametrize("nb,a,deg", [(16, 2.5, 1), (16, 3.0, 2), (32, 2.0, 1)])
def test_boundary_rhs_alg_a1(nb, a, deg):
    p, q, A = mixed_bc_cube(nb, a, deg)
    H = rk.Handle.from_problem(p, device=DEV)
    o = Oracle(p.n, p.h, a, deg, p.chi)
    fo = o.eval_u_transpose(q * A)
    f = np_(H.boundary_rhs(tdev(q), tdev(A)))
    assert rel(f, fo) < 1e-10
    assert np.all(f[p.chi == 0] == 0.0)
    H.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_mixed_boundary_solve(prec):
    p, q, A = mixed_bc_cube(16, 2.5, 1)
    H = rk.Handle.from_problem(p, device=DEV)
    o = Oracle(p.n, p.h, 2.5, 1, p.chi)
    o.assemble_K(p.V)
    rhs = o.rhs(p.V, p.r) + o.eval_u_transpose(q * A)
    do, _ = o.solve_rhs(p.chi_gamma, rhs, p.g, tol=1e-14)
    d, u, info = H.solve(tdev(p.r), tdev(p.g), q=tdev(q), A=tdev(A), precision=prec, tol=1e-13)
    assert info["status"] == 0
    assert rel(np_(d), do) < 1e-9
    gam = p.chi_gamma > 0
    assert np.array_equal(np_(d)[gam], p.g[gam])
    # without the Neumann term the solution differs
    d0, _, _ = H.solve(tdev(p.r), tdev(p.g), precision=prec, tol=1e-13)
    assert rel(np_(d0), do) > 1e-3
    H.close()


def _dense_tables(p, o):
    import scipy.sparse as sp
    o.assemble_K(p.V)
    ptr, col, val = o.K_csr()
    nodes = np.flatnonzero(p.chi)
    nn = len(nodes)
    K = sp.csr_matrix((val, col, ptr), shape=(nn, nn)).toarray()
    nbr, psi, _ = o.shape_tables()
    rows, cols = np.nonzero(nbr >= 0)
    U = sp.csr_matrix((psi[rows, cols], (rows, nbr[rows, cols])), shape=(nn, nn)).toarray()
    return nodes, K, U


def _penalty_system(p, a, deg, seed=29):
    o = Oracle(p.n, p.h, a, deg, p.chi)
    nodes, K, U = _dense_tables(p, o)
    A = W.cube_surface_weights(p)
    rng = np.random.default_rng(seed)
    r = W.random_field(p.nbox, 11) * p.chi
    g = np.where(A > 0, rng.standard_normal(p.nbox), 0.0)
    beta = 100.0 * np.abs(K).max() / A.max()
    An = A[nodes]
    M = K + beta * (U.T * An) @ U
    rhs = o.rhs(p.V, r)[nodes] + beta * U.T @ (An * g[nodes])
    return nodes, U, M, rhs, r, g, A, beta


def test_penalty_solve_matches_oracle():
    """Essential conditions by the penalty method (Sec. 2.4): the GPU solve of
    M d = (K + beta U^T diag(A) U) d = f^r + beta U^T (A g) against the dense solve of
    the same system built from the oracle's assembled K and shape functions U
    (linear basis, cube face weights A, beta = 100 max|K| / max A): d and u^h to 1e-9."""
    p = W.cube_problem(16, 2.5, 1, "zero")
    nodes, U, M, rhs, r, g, A, beta = _penalty_system(p, 2.5, 1)
    H = rk.Handle.from_problem(p, device=DEV)
    d, u, info = H.solve_penalty(tdev(r), tdev(g), tdev(A), beta, tol=1e-13, max_iter=100000)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-13
    dn = np_(d)
    assert np.all(dn[p.chi == 0] == 0.0)
    do = np.zeros(p.nbox)
    do[nodes] = np.linalg.solve(M, rhs)
    uo = np.zeros(p.nbox)
    uo[nodes] = U @ do[nodes]
    assert rel(dn, do) < 1e-9, rel(dn, do)
    assert rel(np_(u), uo) < 1e-9
    H.close()


@pytest.mark.parametrize("a,deg", [(2.5, 1), (3.0, 2), (3.5, 2)])
def test_penalty_cg_iterates_match_dense_cg(a, deg):
    """The penalty operator and right-hand side, checked through the CG iterates:
    k iterations from d = 0 give a fixed polynomial in M applied to the right-hand
    side, so the GPU's d after 8 iterations must equal 8 iterations of the same CG
    on the dense M and f^r + beta U^T (A g) from the oracle.  (With the quadratic
    basis the system keeps the near-zero-energy modes of direct nodal integration,
    too ill-conditioned for plain CG to converge, so this is how its operator is
    checked.)"""
    p = W.cube_problem(16, a, deg, "zero")
    nodes, U, M, rhs, r, g, A, beta = _penalty_system(p, a, deg)
    x = np.zeros(len(nodes))
    res = rhs.copy()
    pv = res.copy()
    rr = res @ res
    for _ in range(8):
        Ap = M @ pv
        al = rr / (pv @ Ap)
        x += al * pv
        res -= al * Ap
        rr_new = res @ res
        pv = res + (rr_new / rr) * pv
        rr = rr_new
    H = rk.Handle.from_problem(p, device=DEV)
    d, u, info = H.solve_penalty(tdev(r), tdev(g), tdev(A), beta, tol=1e-30, max_iter=8, raise_on_error=False)
    assert info["status"] == 5 and info["iterations"] == 8  # RK_ERR_NOT_CONVERGED at the cap
    dn = np_(d)
    assert rel(dn[nodes], x) < 1e-10, rel(dn[nodes], x)
    assert np.all(dn[p.chi == 0] == 0.0)
    H.close()
