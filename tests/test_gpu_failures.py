"""Failure detection of the solve, made on the host (no GPU fault, trap or hang):
a non-finite right-hand side is rejected before any iteration and leaves the
handle usable, and an iteration cap ends the solve with RK_ERR_NOT_CONVERGED and
a finite residual."""
import numpy as np
import pytest

from paper_2403_19854_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2403_19854_gb300 import rk  # noqa: E402

DEV = torch.device("cuda:0")


def tdev(x):
    return torch.as_tensor(np.ascontiguousarray(x), device=DEV)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_nan_source_is_rejected_and_handle_stays_usable(prec):
    p = W.cube_problem(16, 2.5, 1, "sin")
    H = rk.Handle.from_problem(p, device=DEV)
    r = p.r.copy()
    r[6 + 16 * (7 + 16 * 6)] = np.nan
    with pytest.raises(rk.RKError) as e:
        H.solve(tdev(r), tdev(p.g), precision=prec, tol=1e-10)
    assert rk.STATUS[e.value.status] == "RK_ERR_INVALID_ARG"
    d, u, info = H.solve(tdev(p.r), tdev(p.g), precision=prec, tol=1e-10)
    assert info["status"] == 0 and np.isfinite(d.cpu().numpy()).all()
    H.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_iteration_cap_reports_not_converged(prec):
    p = W.cube_problem(32, 2.5, 1, "sin")
    H = rk.Handle.from_problem(p, device=DEV)
    d, u, info = H.solve(tdev(p.r), tdev(p.g), precision=prec, tol=1e-12, max_iter=50, raise_on_error=False)
    assert rk.STATUS[info["status"]] == "RK_ERR_NOT_CONVERGED"
    assert 0 < info["iterations"] <= 50
    assert np.isfinite(info["rel_residual"]) and info["rel_residual"] > 1e-12
    assert np.isfinite(d.cpu().numpy()).all()
    H.close()
