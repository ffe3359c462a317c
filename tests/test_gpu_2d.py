"""Two-dimensional boxes (grid n_z = 1, Sec. 6.1.2): set-up, operators and solves
of the CUDA path against the oracle on the same 2D grid, and the convergence of
the paper's 2D problem (Eq. 101-102) on the GPU.

Same tolerances as the 3D parity tests: FP64 1e-10, FP32 2e-6, solves 1e-9.
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


def rel(a, b, m=None):
    a, b = np.asarray(a), np.asarray(b)
    if m is not None:
        a, b = a[m], b[m]
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def tdev(x):
    return torch.as_tensor(np.ascontiguousarray(x), device=DEV)


def np_(t):
    return t.detach().cpu().numpy()


CASES = [(16, 1.5, 1), (32, 2.5, 1), (32, 2.5, 2), (36, 3.0, 2), (64, 2.0, 1)]


@pytest.mark.parametrize("nb,a,deg", CASES)
def test_setup_and_operators_2d(nb, a, deg):
    p = W.plane_problem(nb, a, deg)
    H = rk.Handle.from_problem(p, device=DEV)
    o = Oracle(p.n, p.h, a, deg, p.chi)
    assert H.s == o.s == p.s and H.singular == (0, -1)
    m = p.chi > 0
    bg = np_(H.get_b(torch.empty(4 * p.s * p.nbox, dtype=torch.float64, device=DEV)))
    bo = o.b_fields()
    for i in range(3):
        assert rel(bg[i][:, m], bo[i][:, m]) < 1e-10, f"b family {i}"
    assert np.all(bg[3] == 0.0)
    d = W.random_field(p.nbox, 3)
    assert rel(np_(H.apply_K(tdev(d))), o.apply_K(p.V, d * p.chi), m) < 1e-10
    d32 = d.astype(np.float32)
    f32 = np_(H.apply_K(tdev(d32))).astype(np.float64)
    assert rel(f32, o.apply_K(p.V, d32.astype(np.float64) * p.chi), m) < 2e-6
    assert rel(np_(H.eval_u(tdev(d))), o.eval_u(d * p.chi), m) < 1e-10
    assert rel(np_(H.eval_u_transpose(tdev(d))), o.eval_u_transpose(d * p.chi), m) < 1e-10
    r = W.random_field(p.nbox, 5)
    fr = np_(H.rhs(tdev(r)))
    assert rel(fr, o.rhs(p.V, r * p.chi), m) < 1e-10
    assert np.all(fr[~m] == 0.0)
    H.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("nb,a,deg", [(16, 1.5, 1), (32, 2.5, 1), (16, 2.5, 2)])
def test_solve_2d_matches_oracle(nb, a, deg, prec):
    p = W.plane_problem(nb, a, deg)
    H = rk.Handle.from_problem(p, device=DEV)
    o = Oracle(p.n, p.h, a, deg, p.chi)
    do, _ = o.solve(p.V, p.chi_gamma, p.r, p.g, tol=1e-14)
    d, u, info = H.solve(tdev(p.r), tdev(p.g), precision=prec, tol=1e-12)
    assert info["status"] == 0
    assert rel(np_(d), do) < 1e-9
    H.close()


def test_paper_2d_problem_converges_quadratically():
    """Sec. 6.1.2 (Eq. 101-103, a = 1.5h, linear basis): nodal normalised L2 error of
    Eq. 104 at boxes 32^2 ... 256^2 on the GPU falls at the quadratic rate of Fig. 11."""
    errs, hs = [], []
    for nb in (32, 64, 128, 256):
        p = W.plane_problem(nb, 1.5, 1)
        H = rk.Handle.from_problem(p, device=DEV)
        d, u, info = H.solve(tdev(p.r), tdev(p.g), precision="fp64", tol=1e-12)
        assert info["status"] == 0
        m = p.chi > 0
        uu = np_(u)
        errs.append(np.sqrt(((uu - p.u_exact)[m] ** 2).sum() / (p.u_exact[m] ** 2).sum()))
        hs.append(p.h[0])
        H.close()
    rates = np.diff(np.log(errs)) / np.diff(np.log(hs))
    assert np.all(rates > 1.9) and np.all(rates < 2.1), rates


def test_2d_rejects_the_spectral_preconditioner():
    p = W.plane_problem(16, 1.5, 1)
    H = rk.Handle.from_problem(p, device=DEV)
    with pytest.raises(rk.RKError):
        H.apply_precond(tdev(W.random_field(p.nbox, 1)))
    H.close()


@pytest.mark.parametrize("axis", [0, 1])
def test_2d_gap_narrower_than_support_is_rejected(axis):
    """Eq. 66 on a plane: with a = 2h the reach is one node, so a domain that fills
    every index of x (or of y) touches its periodic image and the set-up refuses it;
    the single z index, which every node occupies, is not an axis of the problem."""
    p = W.plane_problem(16, 2.0, 1)
    chi = p.chi.reshape(16, 16).copy()          # [y, x]
    if axis == 0:
        chi[:, 14] = chi[:, 0]
        chi[:, 15] = chi[:, 0]
    else:
        chi[14, :] = chi[0, :]
        chi[15, :] = chi[0, :]
    with pytest.raises(rk.RKError) as e:
        rk.Handle(p.n, p.h, tdev(chi.reshape(-1)), tdev(p.chi_gamma), tdev(p.V), 1, 2.0)
    assert e.value.status == 8
    H = rk.Handle(p.n, p.h, tdev(p.chi), tdev(p.chi_gamma), tdev(p.V), 1, 2.0)   # the gap kept: accepted
    H.close()
