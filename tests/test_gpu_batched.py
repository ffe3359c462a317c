"""Uneven domains: the 7-smooth box sides, non-cubic boxes, embedding, and the
batched persistent solve.

* K.u (FP64, FP32) on every built side that is not a power of two, in non-cubic
  boxes holding an embedded sphere domain, against the oracle;
* a domain embedded in a larger box gives the same K.u and u^h on its nodes
  (the extra nodes are outside chi, Eq. 40);
* rk_solve_batched over several domains and right-hand sides (clones) gives the
  same iterates as rk_solve of each item alone: same kernels, same
  deterministic reductions, hence the same bits;
* one batched item against the oracle's solve.
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
TOL64 = 1e-10
TOL32 = 2e-6


def rel(a, b, m=None):
    a = np.asarray(a)
    b = np.asarray(b)
    if m is not None:
        a, b = a[m], b[m]
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def tdev(x):
    return torch.as_tensor(np.ascontiguousarray(x), device=DEV)


def np_(t):
    return t.detach().cpu().numpy()


SMOOTH = (36, 48, 72, 96, 100, 144, 162)
# every 7-smooth side on every axis (the x pass and the strided y / z passes map
# lines to threads differently), both bases
BOXES = ([((n, 32, 36), 2.5, 1) for n in SMOOTH] + [((32, n, 36), 3.0, 2) for n in SMOOTH]
         + [((36, 32, n), 2.5, 1) for n in SMOOTH] + [((32, 36, n), 3.0, 2) for n in (72, 144, 162)])


@pytest.mark.parametrize("box,a,deg", BOXES, ids=lambda v: str(v))
def test_seven_smooth_sides_noncubic(box, a, deg):
    p0 = W.spheres_problem(n_box=32, n_spheres=3, a_tilde=a, degree=deg, r_range=(0.2, 0.3), seed=31)
    p = W.embed(p0, box)
    H = rk.Handle.from_problem(p, device=DEV)
    o = Oracle(p.n, p.h, a, deg, p.chi)
    m = p.chi > 0
    d = W.random_field(p.nbox, 3)
    fo = o.apply_K(p.V, d * p.chi)
    f = np_(H.apply_K(tdev(d)))
    assert rel(f, fo, m) < TOL64
    assert np.all(f[~m] == 0.0)
    f32 = np_(H.apply_K(tdev(d.astype(np.float32)))).astype(np.float64)
    fo32 = o.apply_K(p.V, d.astype(np.float32).astype(np.float64) * p.chi)
    assert rel(f32, fo32, m) < TOL32
    H.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("nx", SMOOTH)
def test_solve_on_seven_smooth_x_sides(nx, prec):
    """Alg. 5 on boxes whose x side gives P = 4, 6, 9, 10 or 12 threads per line: the
    CG steps fused into the x passes (direction update, p.Ap and alpha) run with
    those block shapes.  Against the oracle's direct solve."""
    p0 = W.spheres_problem(n_box=32, n_spheres=2, a_tilde=2.5, degree=1, r_range=(0.18, 0.22), seed=77)
    p = W.embed(p0, (nx, 32, 36))
    p.g = np.where(p.chi_gamma > 0, 0.1 * W.random_field(p.nbox, 5), 0.0)
    H = rk.Handle.from_problem(p, device=DEV)
    o = Oracle(p.n, p.h, 2.5, 1, p.chi)
    do, _ = o.solve(p.V, p.chi_gamma, p.r, p.g, tol=1e-14)
    d, u, info = H.solve(tdev(p.r), tdev(p.g), precision=prec, tol=1e-12)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-12
    assert rel(np_(d), do) < 1e-9
    H.close()


def test_embedding_leaves_the_operator_unchanged():
    p0 = W.spheres_problem(n_box=32, n_spheres=4, a_tilde=2.5, degree=1, r_range=(0.15, 0.25), seed=5)
    p1 = W.embed(p0, (48, 36, 64))
    H0 = rk.Handle.from_problem(p0, device=DEV)
    H1 = rk.Handle.from_problem(p1, device=DEV)
    d0 = W.random_field(p0.nbox, 8) * p0.chi
    d1 = W.embed(W.Problem(n=p0.n, h=p0.h, a_tilde=2.5, degree=1, chi=p0.chi, chi_gamma=p0.chi_gamma,
                           V=p0.V, r=d0, g=p0.g), p1.n).r
    m0 = p0.chi > 0
    m1 = p1.chi > 0
    f0 = np_(H0.apply_K(tdev(d0)))[m0]
    f1 = np_(H1.apply_K(tdev(d1)))[m1]
    assert rel(f1, f0) < 1e-12
    _, u0, _ = H0.solve(tdev(p0.r), tdev(p0.g), precision="fp64", tol=1e-12)
    _, u1, _ = H1.solve(tdev(p1.r), tdev(p1.g), precision="fp64", tol=1e-12)
    assert rel(np_(u1)[m1], np_(u0)[m0]) < 1e-9
    H0.close()
    H1.close()


def test_full_size_sphere_box144_sampled():
    """A 130-node sphere domain in a 144^3 box (a side that is not a power of two on
    all three axes): K.u and b on sampled nodes against the oracle."""
    from oracle.oracle import apply_K_sampled, b_sampled
    p0, _ = W.batched_domains(n_domains=10, n_rhs=1)[9]
    p = W.embed(p0, (144, 144, 144))
    H = rk.Handle.from_problem(p, device=DEV)
    rng = np.random.default_rng(144)
    idx = np.flatnonzero(p.chi)
    sample = np.sort(rng.choice(idx, 64, replace=False))
    bnd = np.flatnonzero(p.chi_gamma)
    sample = np.unique(np.concatenate([sample, rng.choice(bnd, 16, replace=False)]))
    d = W.random_field(p.nbox, 9) * p.chi
    f64 = np_(H.apply_K(tdev(d)))
    fo = apply_K_sampled(p.n, p.h, p.a_tilde, p.degree, p.chi, p.V, d, sample)
    assert rel(f64[sample], fo) < TOL64
    bg = np_(H.get_b(torch.empty(4 * p.s * p.nbox, dtype=torch.float64, device=DEV)))
    bo = b_sampled(p.n, p.h, p.a_tilde, p.degree, p.chi, sample)
    for i in range(4):
        assert rel(bg[i][:, sample].T, bo[:, i, :]) < TOL64
    H.close()


def _smallest_side(S):
    return next(n for n in range(S, 513) if rk.supported_length(n))


@pytest.fixture(scope="module")
def batch():
    doms = W.batched_domains(n_domains=4, side_range=(30, 40), n_rhs=2, seed=20240328 + 5102)
    items, keep = [], []
    for p0, rhs in doms:
        p = W.embed(p0, (_smallest_side(p0.n[0]),) * 3)
        H = rk.Handle.from_problem(p, device=DEV)
        hs = [H] + [H.clone() for _ in rhs[1:]]
        pad = [W.embed(W.Problem(n=p0.n, h=p0.h, a_tilde=p0.a_tilde, degree=p0.degree, chi=p0.chi,
                                 chi_gamma=p0.chi_gamma, V=p0.V, r=r, g=p0.g), p.n).r for r in rhs]
        for h, r in zip(hs, pad):
            items.append((p, h, r))
        keep.append((H, hs))
    yield items
    for H, hs in keep:
        for h in hs[1:]:
            h.close()
        H.close()


def test_batched_equals_individual_solves(batch):
    """Same iterations and bits as one rk_solve per item.  The n = 2 items (a = 3h)
    carry the near-zero-energy modes of direct nodal integration (kappa ~ 1e8 already
    at 20^3), which FP32 cannot resolve: they stop at the iteration cap or when the
    FP32 iterations stall, and the comparison covers them all the same."""
    opts = dict(precision="mixed", tol=1e-10, check_every=8, max_iter=3000, fp64_finish=0)
    args = []
    for p, h, r in batch:
        args.append((h, tdev(r), tdev(p.g), torch.empty(p.nbox, dtype=torch.float64, device=DEV),
                     torch.empty(p.nbox, dtype=torch.float64, device=DEV)))
    infos = rk.solve_batched(args, raise_on_error=False, **opts)
    for (p, h, r), (_, rt, gt, d, u), ib in zip(batch, args, infos):
        d1, u1, i1 = h.solve(rt, gt, raise_on_error=False, **opts)
        if p.degree == 1:
            assert ib["status"] == 0 and ib["rel_residual"] <= 1e-10 and ib["fp64_iterations"] == 0
        assert ib["status"] == i1["status"]
        assert ib["iterations"] == i1["iterations"] and ib["outer"] == i1["outer"]
        assert rel(np_(d), np_(d1)) <= 1e-13
        assert rel(np_(u), np_(u1)) <= 1e-13
        assert np.array_equal(np_(d)[p.chi_gamma > 0], p.g[p.chi_gamma > 0])


def test_batched_item_matches_oracle(batch):
    p, h, r = min((it for it in batch if it[0].degree == 1), key=lambda it: it[0].n_omega)
    d = torch.empty(p.nbox, dtype=torch.float64, device=DEV)
    rk.solve_batched([(h, tdev(r), tdev(p.g), d, None)], precision="mixed", tol=1e-13)
    o = Oracle(p.n, p.h, p.a_tilde, p.degree, p.chi)
    do, _ = o.solve(p.V, p.chi_gamma, r, p.g, tol=1e-14)
    assert rel(np_(d), do) < 1e-9


def test_stalled_mixed_solve_finishes_in_fp64():
    """The hand-over of a mixed solve to FP64 CG (Alg. 5 with iterative refinement:
    when the FP32 iterations stop reducing the FP64 residual, or the refinement-step
    cap is reached, the solve continues with FP64 CG from the current iterate).
    The cap of two refinement steps forces the hand-over on any device: after two
    residual replacements (each at a tenth of the previous FP64 residual) the
    residual is near 1e-2, far above tol.  The finished solve must reach tol with
    FP64 iterations, and its d must match the oracle's direct solve of the assembled
    Dirichlet system (Eq. 29) to 1e-9; with fp64_finish = 0 the same cap ends the
    solve unconverged at the residual of the mixed iterations."""
    p = W.cube_problem(32, 2.5, 1, "sin")
    p.g = np.where(p.chi_gamma > 0, 0.1 * W.random_field(p.nbox, 5), 0.0)
    H = rk.Handle.from_problem(p, device=DEV)
    r, g = tdev(p.r), tdev(p.g)
    _, _, i0 = H.solve(r, g, precision="mixed", tol=1e-13, fp64_finish=0, max_outer=2, raise_on_error=False)
    d1, u1, i1 = H.solve(r, g, precision="mixed", tol=1e-13, fp64_finish=1, max_outer=2, raise_on_error=False)
    assert i0["status"] == 5 and i0["fp64_iterations"] == 0 and i0["outer"] == 2
    assert i0["rel_residual"] > 1e-6
    assert i1["status"] == 0 and i1["fp64_iterations"] > 0
    assert i1["rel_residual"] <= 1e-13 < i0["rel_residual"]
    o = Oracle(p.n, p.h, p.a_tilde, p.degree, p.chi)
    do, _ = o.solve(p.V, p.chi_gamma, p.r, p.g, tol=1e-13)  # CG on the assembled CSR
    assert rel(np_(d1), do) < 1e-9
    assert rel(np_(u1), o.eval_u(do)) < 1e-9
    H.close()


def test_batched_rejects_shared_handles(batch):
    p, h, r = batch[0]
    d = torch.empty(p.nbox, dtype=torch.float64, device=DEV)
    e = torch.empty(p.nbox, dtype=torch.float64, device=DEV)
    with pytest.raises(rk.RKError):
        rk.solve_batched([(h, tdev(r), None, d, None), (h, tdev(r), None, e, None)])


def test_autotune_picks_a_built_side():
    from paper_2403_19854_gb300 import autotune
    S = 37
    n = autotune.best_side(S, 1, max_candidates=2)
    assert n >= S and rk.supported_length(n)


def test_autotune_mixed_opts_picks_a_converging_candidate():
    """autotune.best_mixed_opts times one mixed solve per replacement setting and
    returns the fastest one that reached tol; the solve with it matches the oracle."""
    from paper_2403_19854_gb300 import autotune
    p = W.cube_problem(16, 2.0, 1, "sin")
    H = rk.Handle.from_problem(p, device=DEV)
    r, g = tdev(p.r), tdev(p.g)
    itol, ce, t = autotune.best_mixed_opts(H, r, g, tol=1e-12)
    assert (itol, ce) in autotune.MIXED_CANDIDATES
    assert len(t) == len(autotune.MIXED_CANDIDATES)
    assert t[f"{itol}/{ce}"][2] == 0
    d, _, info = H.solve(r, g, precision="mixed", tol=1e-12, inner_tol=itol, check_every=ce)
    o = Oracle(p.n, p.h, p.a_tilde, p.degree, p.chi)
    do, _ = o.solve(p.V, p.chi_gamma, p.r, p.g, tol=1e-14)
    assert rel(np_(d), do) < 1e-9
    H.close()
