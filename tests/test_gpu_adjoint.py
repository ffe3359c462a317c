"""Adjoint gradients of J = 1/2 sum_chi (u^h - u_target)^2 on the 96^3-box cube
(a = 2.5h, linear basis, Gaussian random source sigma = 0.1, cosine Dirichlet data).

* rk_solve_adjoint against autograd through poisson_solve (rk_solve_vjp backward);
* both against central finite differences on seeded directions: J is an exact
  quadratic in (r, g), so (J(t + e d) - J(t - e d)) / 2e equals grad . d up to the
  solve tolerance, for any e.  The step e is half the size of r itself: a large
  step leaves the difference exact and makes the solve error small against it.
  Solves run to a relative residual of 1e-13 and the gradients must agree to
  1e-8 relative.  3 directions with plain CG solves, and the 32 seeded directions
  of the workload with preconditioned solves (the solver only evaluates J; any
  solve to the tolerance gives the same quadratic).
"""
import numpy as np
import pytest

from paper_2403_19854_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2403_19854_gb300 import rk  # noqa: E402

DEV = torch.device("cuda:0")
SOLVE_TOL = 1e-13  # relative FP64 residual of every solve
FD_TOL = 1e-8      # relative agreement of central differences with grad . d


@pytest.fixture(scope="module")
def problem():
    p = W.adjoint_problem(n_box=96, a_tilde=2.5, degree=1)
    H = rk.Handle.from_problem(p, device=DEV)
    t = {k: torch.as_tensor(getattr(p, k), device=DEV) for k in ("r", "g", "chi", "chi_gamma")}
    t["ut"] = torch.as_tensor(p.meta["u_target"], device=DEV)
    yield p, H, t
    H.close()


def _J(H, t, r, g, prec):
    _, u, _ = H.solve(r, g, precision=prec, tol=SOLVE_TOL)
    e = (u - t["ut"]) * t["chi"]
    return 0.5 * float((e * e).sum())


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_adjoint_equals_autograd(problem, prec):
    p, H, t = problem
    J, gr, gg, info = H.solve_adjoint(t["r"], t["g"], t["ut"], precision=prec, tol=SOLVE_TOL)
    r = t["r"].clone().requires_grad_(True)
    g = t["g"].clone().requires_grad_(True)
    u = rk.poisson_solve(H, r, g, precision=prec, tol=SOLVE_TOL)
    e = (u - t["ut"]) * t["chi"]
    Ja = 0.5 * (e * e).sum()
    Ja.backward()
    assert abs(float(Ja) - J) <= 1e-10 * J
    assert float((r.grad - gr).norm() / gr.norm()) < 1e-8
    assert float((g.grad - gg).norm() / gg.norm()) < 1e-8
    # gradients vanish where the inputs are not read
    assert float(gr[t["chi"] == 0].abs().max()) == 0.0
    assert float(gg[t["chi_gamma"] == 0].abs().max()) == 0.0


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_adjoint_central_differences(problem, prec):
    p, H, t = problem
    J, gr, gg, info = H.solve_adjoint(t["r"], t["g"], t["ut"], precision=prec, tol=SOLVE_TOL)
    rng = np.random.default_rng(20240328 + 4001)
    for _ in range(3):
        dr = torch.as_tensor(rng.standard_normal(p.nbox), device=DEV) * t["chi"]
        dg = torch.as_tensor(rng.standard_normal(p.nbox), device=DEV) * t["chi_gamma"]
        eps = 0.5 * float(t["r"].norm()) / float(dr.norm())
        fd = (_J(H, t, t["r"] + eps * dr, t["g"] + eps * dg, prec)
              - _J(H, t, t["r"] - eps * dr, t["g"] - eps * dg, prec)) / (2 * eps)
        an = float((gr * dr).sum() + (gg * dg).sum())
        assert abs(an - fd) <= FD_TOL * abs(fd), f"rel {abs(an - fd) / abs(fd):.3e}"


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_adjoint_32_directions(problem, prec):
    p, H, t = problem
    J, gr, gg, info = H.solve_adjoint(t["r"], t["g"], t["ut"], precision=prec, tol=SOLVE_TOL, precond="spectral")
    Jp, grp, ggp, _ = H.solve_adjoint(t["r"], t["g"], t["ut"], precision=prec, tol=SOLVE_TOL)
    # the gradient does not depend on the solver used for it
    assert float((gr - grp).norm() / grp.norm()) < 1e-8 and float((gg - ggp).norm() / ggp.norm()) < 1e-8

    def Jp_(r, g):
        _, u, _ = H.solve(r, g, precision=prec, tol=SOLVE_TOL, precond="spectral")
        e = (u - t["ut"]) * t["chi"]
        return 0.5 * float((e * e).sum())

    rng = np.random.default_rng(20240328 + 4032)
    worst = 0.0
    for _ in range(32):
        dr = torch.as_tensor(rng.standard_normal(p.nbox), device=DEV) * t["chi"]
        dg = torch.as_tensor(rng.standard_normal(p.nbox), device=DEV) * t["chi_gamma"]
        eps = 0.5 * float(t["r"].norm()) / float(dr.norm())
        fd = (Jp_(t["r"] + eps * dr, t["g"] + eps * dg) - Jp_(t["r"] - eps * dr, t["g"] - eps * dg)) / (2 * eps)
        an = float((gr * dr).sum() + (gg * dg).sum())
        worst = max(worst, abs(an - fd) / abs(fd))
    assert worst < FD_TOL, f"worst rel {worst:.3e}"
