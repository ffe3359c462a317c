"""Failure detection without a GPU fault, trap or hang: a non-finite right-hand
side is rejected before any iteration and leaves the handle usable; an iteration
cap ends the solve with RK_ERR_NOT_CONVERGED and a finite residual; and a bounded
device wait that gives up is reported as RK_ERR_TIMEOUT (the waits are made to
give up at once while every copy still completes), after which the handle
computes correct results again."""
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


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_bounded_wait_that_gives_up_reports_timeout(dtype):
    """rk_debug_short_waits: the first wait of every block of the TMA-fed y and z
    passes for its input tile gives up at once; the block waits for the copy in
    flight with the normal limit, records the time-out and returns.  A call on host
    arrays synchronises and must report RK_ERR_TIMEOUT; with normal waits the same
    handle matches the oracle again (Alg. 2 against Eq. 50/54)."""
    from oracle.oracle import Oracle
    p = W.cube_problem(32, 2.5, 1, "sin")
    H = rk.Handle.from_problem(p, device=DEV)
    d = W.random_field(p.nbox, 3).astype(dtype)
    H.debug_short_waits(True)
    with pytest.raises(rk.RKError) as e:
        H.apply_K(d)  # host arrays: the call synchronises and checks the error word
    assert rk.STATUS[e.value.status] == "RK_ERR_TIMEOUT"
    H.debug_short_waits(False)
    f = H.apply_K(d).astype(np.float64)
    fo = Oracle(p.n, p.h, 2.5, 1, p.chi).apply_K(p.V, d.astype(np.float64) * p.chi)
    tol = 1e-10 if dtype == np.float64 else 2e-6
    assert np.linalg.norm(f - fo) / np.linalg.norm(fo) < tol
    H.close()


def test_solve_reports_timeout_and_recovers():
    """The same in a mixed solve (TMA-fed strided passes inside the captured CG
    chunks, and the bulk-copy x split of the fused CG step): RK_ERR_TIMEOUT, then a
    normal solve on the same handle converges."""
    p = W.cube_problem(32, 2.5, 1, "sin")
    H = rk.Handle.from_problem(p, device=DEV)
    H.debug_short_waits(True)
    _, _, info = H.solve(tdev(p.r), tdev(p.g), precision="mixed", tol=1e-10, raise_on_error=False)
    assert rk.STATUS[info["status"]] == "RK_ERR_TIMEOUT"
    H.debug_short_waits(False)
    d, u, info = H.solve(tdev(p.r), tdev(p.g), precision="mixed", tol=1e-10)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-10
    H.close()
