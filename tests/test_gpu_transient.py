"""Time-dependent terms of Appendix C against the oracle: the consistent mass
action (Alg. C.1), the lumped mass (Alg. C.2), forward Euler with the lumped mass
(Alg. C.3) and backward Euler (Alg. C.4).

The oracle's M v is U^T (V o U v) from its explicit shape functions (Eq. C.5 with
DNI); its lumped mass is U^T V; the reference steppers repeat the same updates
with the oracle's operators (forward Euler) or a dense solve of the assembled
(M + dt K) restricted to the free nodes (backward Euler).
"""
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


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def tdev(x):
    return torch.as_tensor(np.ascontiguousarray(x), device=DEV)


def np_(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("kind,nb,a,deg", [("cube", 16, 2.5, 1), ("cube", 16, 3.0, 2), ("spheres", 32, 2.5, 1)])
def test_mass_action_and_lumped_mass(kind, nb, a, deg):
    if kind == "cube":
        p = W.cube_problem(nb, a, deg, "zero")
    else:
        p = W.spheres_problem(n_box=nb, n_spheres=3, a_tilde=a, degree=deg, r_range=(0.2, 0.3), seed=11)
    H = rk.Handle.from_problem(p, device=DEV)
    o = Oracle(p.n, p.h, a, deg, p.chi)
    v = W.random_field(p.nbox, 3) * p.chi
    mo = o.eval_u_transpose(p.V * o.eval_u(v))
    assert rel(np_(H.apply_M(tdev(v))), mo) < 1e-10
    m32 = np_(H.apply_M(tdev(v.astype(np.float32)))).astype(np.float64)
    assert rel(m32, o.eval_u_transpose(p.V * o.eval_u(v.astype(np.float32).astype(np.float64)))) < 2e-6
    assert rel(np_(H.lumped_mass(like=tdev(v))), o.eval_u_transpose(p.V)) < 1e-10
    H.close()


def _problem():
    p = W.cube_problem(16, 2.5, 1, "sin")
    p.g = np.where(p.chi_gamma > 0, 0.1 * W.random_field(p.nbox, 5), 0.0)
    return p


def test_forward_euler_lumped_mass_alg_c3():
    p = _problem()
    H = rk.Handle.from_problem(p, device=DEV)
    o = Oracle(p.n, p.h, 2.5, 1, p.chi)
    free = (p.chi > 0) & (p.chi_gamma == 0)
    gam = p.chi_gamma > 0
    f = o.rhs(p.V, p.r)
    ml = o.eval_u_transpose(p.V)
    d0 = np.where(free, W.random_field(p.nbox, 7), 0.0) + np.where(gam, p.g, 0.0)
    dt = 0.02 * p.h[0] ** 2
    d = d0.copy()
    for _ in range(10):
        Kd = o.apply_K(p.V, d)
        d = np.where(free, d + dt * (f - Kd) / np.where(free, ml, 1.0), d)
    dg = tdev(d0)
    H.transient_explicit(tdev(f), tdev(p.g), dt, 10, dg)
    assert rel(np_(dg), d) < 1e-10
    assert np.array_equal(np_(dg)[gam], p.g[gam])
    H.close()


def test_backward_euler_alg_c4():
    p = _problem()
    H = rk.Handle.from_problem(p, device=DEV)
    o = Oracle(p.n, p.h, 2.5, 1, p.chi)
    o.assemble_K(p.V)
    ptr, col, val = o.K_csr()
    nodes = np.flatnonzero(p.chi)
    nn = len(nodes)
    K = sp.csr_matrix((val, col, ptr), shape=(nn, nn)).toarray()
    nbr, psi, _ = o.shape_tables()
    rows, cols = np.nonzero(nbr >= 0)
    U = sp.csr_matrix((psi[rows, cols], (rows, nbr[rows, cols])), shape=(nn, nn)).toarray()
    M = U.T @ (p.V[nodes][:, None] * U)
    free = p.chi_gamma[nodes] == 0
    f = o.rhs(p.V, p.r)[nodes]
    gG = np.where(free, 0.0, p.g[nodes])
    dt = 0.01
    x = np.where(free, W.random_field(p.nbox, 8)[nodes], 0.0)
    d0 = np.zeros(p.nbox)
    d0[nodes] = x + gG
    A = (M + dt * K)[np.ix_(free, free)]
    for _ in range(2):
        b = (M @ x + dt * f - dt * (K @ gG))[free]
        x = np.zeros(nn)
        x[free] = np.linalg.solve(A, b)
    ref = np.zeros(p.nbox)
    ref[nodes] = x + gG
    dg = tdev(d0)
    info = H.transient_implicit(tdev(p.r * 0 + o.rhs(p.V, p.r)), tdev(p.g), dt, 2, dg, tol=1e-13)
    assert info["outer"] == 2
    assert rel(np_(dg), ref) < 1e-9
    H.close()
