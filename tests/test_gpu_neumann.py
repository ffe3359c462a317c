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


@pytest.mark.parametrize("a,deg", [(2.5, 1), (3.0, 2)])
def test_penalty_solve_matches_oracle(a, deg):
    """Essential conditions by the penalty method (Sec. 2.4): the GPU solve of
    (K + beta U^T diag(A) U) d = f^r + beta U^T (A g) against the dense solve of the
    same system built from the oracle's assembled K and shape functions U, with the
    cube's face weights A and beta = 100 max|K| / max A; d and u^h to 1e-9."""
    p = W.cube_problem(16, a, deg, "zero")
    o = Oracle(p.n, p.h, a, deg, p.chi)
    nodes, K, U = _dense_tables(p, o)
    A = W.cube_surface_weights(p)
    rng = np.random.default_rng(29)
    r = W.random_field(p.nbox, 11) * p.chi
    g = np.where(A > 0, rng.standard_normal(p.nbox), 0.0)
    beta = 100.0 * np.abs(K).max() / A.max()
    An = A[nodes]
    M = K + beta * (U.T * An) @ U
    rhs = o.rhs(p.V, r)[nodes] + beta * U.T @ (An * g[nodes])
    do = np.zeros(p.nbox)
    do[nodes] = np.linalg.solve(M, rhs)
    uo = np.zeros(p.nbox)
    uo[nodes] = U @ do[nodes]
    H = rk.Handle.from_problem(p, device=DEV)
    d, u, info = H.solve_penalty(tdev(r), tdev(g), tdev(A), beta, tol=1e-13, max_iter=20000)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-13
    assert rel(np_(d), do) < 1e-9, rel(np_(d), do)
    assert rel(np_(u), uo) < 1e-9
    assert np.all(np_(d)[p.chi == 0] == 0.0)
    H.close()
