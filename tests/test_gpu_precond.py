"""The spectral preconditioner of RK_PRECOND_SPECTRAL and preconditioned solves.

M^{-1} r = chi_Omega o F^{-1}[F(r) / (lam + shift)], lam the eigenvalues of K on a
periodic box of regular nodes.  The reference here takes lam from the oracle:
the row of the oracle's assembled K at a deep-interior node of a cube is the
stencil of that periodic operator, so its 3D DFT (numpy) is lam; shift is
1e-3 lam(2 pi / n_x, 0, 0).  PCG solves are compared with the oracle's solution.
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


def interior_stencil(a_tilde, degree, h):
    """{(dx, dy, dz): K_IJ} at a deep-interior node, from the oracle's assembled K
    on a 20^3-box cube with spacing h (trapezoidal V does not reach the centre)."""
    nb = 20
    p = W.cube_problem(nb, a_tilde, degree, "zero")
    o = Oracle(p.n, (h, h, h), a_tilde, degree, p.chi)
    V = np.where(p.chi > 0, h ** 3, 0.0)
    o.assemble_K(V)
    ptr, col, val = o.K_csr()
    nodes = np.flatnonzero(p.chi)
    K = sp.csr_matrix((val, col, ptr), shape=(o.nnode, o.nnode))
    c = 9 + nb * (9 + nb * 9)
    row = K[np.searchsorted(nodes, c)]
    st = {}
    for j, v in zip(row.indices, row.data):
        g = nodes[j]
        st[(g % nb - 9, (g // nb) % nb - 9, g // (nb * nb) - 9)] = v
    return st


def reference_precond(n, stencil, r, mask):
    nx, ny, nz = n
    a = np.zeros((nz, ny, nx))
    for (dx, dy, dz), v in stencil.items():
        a[dz % nz, dy % ny, dx % nx] += v
    lam = np.real(np.fft.fftn(a))
    shift = 1e-3 * lam[0, 0, 1]
    z = np.real(np.fft.ifftn(np.fft.fftn(r.reshape(nz, ny, nx)) / (lam + shift))).reshape(-1)
    return z * mask


@pytest.mark.parametrize("box,a,deg", [((32, 32, 32), 2.5, 1), ((36, 48, 32), 2.5, 1), ((32, 32, 32), 2.0, 1),
                                       ((16, 16, 16), 3.0, 2), ((64, 36, 72), 2.5, 1)])
def test_precond_equals_fft_of_the_oracle_stencil(box, a, deg):
    p = W.embed(W.cube_problem(16, a, deg, "zero"), box)
    H = rk.Handle.from_problem(p, device=DEV)
    st = interior_stencil(a, deg, p.h[0])
    m = p.chi_gamma == 0
    m &= p.chi > 0
    r = W.random_field(p.nbox, 3) * m
    z_ref = reference_precond(p.n, st, r, m)
    z64 = np_(H.apply_precond(tdev(r)))
    assert rel(z64, z_ref) < 1e-9
    z32 = np_(H.apply_precond(tdev(r.astype(np.float32)))).astype(np.float64)
    assert rel(z32, z_ref) < 2e-5
    assert np.all(z64[~m] == 0.0)
    H.close()


def test_precond_is_symmetric_positive():
    p = W.cube_problem(32, 2.5, 1, "zero")
    H = rk.Handle.from_problem(p, device=DEV)
    m = (p.chi > 0) & (p.chi_gamma == 0)
    x = W.random_field(p.nbox, 4) * m
    y = W.random_field(p.nbox, 5) * m
    Mx = np_(H.apply_precond(tdev(x)))
    My = np_(H.apply_precond(tdev(y)))
    assert abs(np.dot(y, Mx) - np.dot(x, My)) <= 1e-12 * abs(np.dot(x, Mx))
    assert np.dot(x, Mx) > 0 and np.dot(y, My) > 0
    H.close()


# sizes whose free nodes the oracle factors directly (dense Cholesky, <= 3000)
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("kind,nb,a", [("cube", 16, 2.5), ("cube", 16, 2.0), ("spheres", 24, 2.5), ("box", 36, 2.5)])
def test_pcg_solve_matches_oracle(kind, nb, a, prec):
    if kind == "cube":
        p = W.cube_problem(nb, a, 1, "sin")
        p.g = np.where(p.chi_gamma > 0, 0.1 * W.random_field(p.nbox, 5), 0.0)
    elif kind == "box":
        p = W.embed(W.spheres_problem(n_box=24, n_spheres=2, a_tilde=a, degree=1, r_range=(0.2, 0.25), seed=12),
                    (nb, 32, 48))
    else:
        p = W.embed(W.spheres_problem(n_box=nb, n_spheres=3, a_tilde=a, degree=1, r_range=(0.2, 0.3), seed=11),
                    (32, 32, 32))
    assert int(((p.chi > 0) & (p.chi_gamma == 0)).sum()) <= 3000
    H = rk.Handle.from_problem(p, device=DEV)
    o = Oracle(p.n, p.h, a, 1, p.chi)
    do, _ = o.solve(p.V, p.chi_gamma, p.r, p.g, tol=1e-14)
    d0, _, i0 = H.solve(tdev(p.r), tdev(p.g), precision=prec, tol=1e-12)
    d1, _, i1 = H.solve(tdev(p.r), tdev(p.g), precision=prec, tol=1e-12, precond="spectral")
    assert i1["status"] == 0 and i1["rel_residual"] <= 1e-12
    assert rel(np_(d1), do) < 1e-9
    assert i1["iterations"] < i0["iterations"]
    H.close()


def test_pcg_batched_equals_single():
    p = W.spheres_problem(n_box=32, n_spheres=2, a_tilde=2.5, degree=1, r_range=(0.2, 0.25), seed=4)
    H = rk.Handle.from_problem(p, device=DEV)
    C = H.clone()
    r2 = W.random_field(p.nbox, 9) * p.chi
    opts = dict(precision="mixed", tol=1e-10, check_every=8, precond="spectral")
    items = [(H, tdev(p.r), tdev(p.g), torch.empty(p.nbox, dtype=torch.float64, device=DEV), None),
             (C, tdev(r2), tdev(p.g), torch.empty(p.nbox, dtype=torch.float64, device=DEV), None)]
    infos = rk.solve_batched(items, **opts)
    for (h, r, g, d, _), ib in zip(items, infos):
        d1, _, i1 = h.solve(r, g, **opts)
        assert ib["iterations"] == i1["iterations"]
        assert rel(np_(d), np_(d1)) <= 1e-13
    C.close()
    H.close()
