"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (relative L2 over the domain nodes, 0 required off the domain):
  FP64 path   1e-10   (the FC-RKPM result is the traditional RKPM result up to
                       rounding: Sec. 6.1, "identical up to the machine precision")
  FP32 path   2e-6    (single-precision FFT convolutions: a few ulps of FP32,
                       ~6e-8, times the O(log N) growth of the transforms and the
                       two chained convolutions of Alg. 2; measured 2-5e-7 at
                       16^3-32^3 and 4.6e-7 / 9.4e-7 (L2 / max) at 256^3, where
                       log2 N is twice that of 16^3)
  mixed solve 1e-9 against the FP64 solution after FP64 refinement.
Each comparison checks the relative L2 error and the max-norm error relative to
the largest reference value, both against the same tolerance.
"""
import functools

import numpy as np
import pytest

from oracle.oracle import Oracle, apply_K_sampled, b_sampled
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


def relmax(a, b, m=None):
    """Max-norm error relative to the largest reference value: one wrong node among
    many cannot hide under a small relative L2 error."""
    a = np.asarray(a)
    b = np.asarray(b)
    if m is not None:
        a, b = a[m], b[m]
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def close(a, b, tol, m=None, what=""):
    """Relative L2 and relative max-norm error both within tol."""
    e2, ei = rel(a, b, m), relmax(a, b, m)
    assert e2 < tol and ei < tol, f"{what}: rel L2 {e2:.3e}, rel max {ei:.3e} (tol {tol:.0e})"


def tdev(x, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(x), device=DEV)
    return t.to(dtype) if dtype is not None else t


def np_(t):
    return t.detach().cpu().numpy()


def _problem(kind, nb, a, deg, seed=11):
    if kind == "cube":
        return W.cube_problem(nb, a, deg, "sin")
    if kind == "paper":
        return W.cube_problem(nb, a, deg, "paper", -1.0, 1.0)
    return W.spheres_problem(n_box=nb, n_spheres=3, a_tilde=a, degree=deg, r_range=(0.2, 0.3), seed=seed)


CASES = [("cube", 16, 2.0, 1), ("cube", 16, 2.5, 1), ("cube", 16, 3.0, 2), ("spheres", 16, 2.5, 1),
         ("spheres", 32, 3.0, 2), ("paper", 8, 1.5, 1), ("cube", 32, 3.5, 1)]


@pytest.fixture(scope="module", params=CASES, ids=lambda c: f"{c[0]}{c[1]}-a{c[2]}-n{c[3]}")
def case(request):
    kind, nb, a, deg = request.param
    p = _problem(kind, nb, a, deg)
    H = rk.Handle.from_problem(p, device=DEV)
    o = Oracle(p.n, p.h, a, deg, p.chi)
    yield p, H, o
    H.close()


def test_setup_coefficients_alg1(case):
    """b^0, b^x, b^y, b^z of Alg. 1 (FFT moments + per-node Cholesky) == oracle rows of
    M^{-1} built from explicit neighbour sums, per coefficient family."""
    p, H, o = case
    m = p.chi > 0
    bg = np_(H.get_b(torch.empty(4 * p.s * p.nbox, dtype=torch.float64, device=DEV)))
    bo = o.b_fields()
    for i in range(4):
        close(bg[i][:, m], bo[i][:, m], TOL64, what=f"b family {i}")
    assert H.singular == (0, -1)


def test_stiffness_action_fp64_alg2(case):
    p, H, o = case
    m = p.chi > 0
    d = W.random_field(p.nbox, 3)
    f = np_(H.apply_K(tdev(d)))
    fo = o.apply_K(p.V, d * p.chi)
    close(f, fo, TOL64, m)
    assert np.all(f[~m] == 0.0)


def test_stiffness_action_fp32_alg2(case):
    p, H, o = case
    m = p.chi > 0
    d = W.random_field(p.nbox, 4).astype(np.float32)
    f = np_(H.apply_K(tdev(d))).astype(np.float64)
    fo = o.apply_K(p.V, d.astype(np.float64) * p.chi)
    close(f, fo, TOL32, m)
    assert np.all(f[~m] == 0.0)


def test_rhs_alg4(case):
    p, H, o = case
    m = p.chi > 0
    r = W.random_field(p.nbox, 5)
    fr = np_(H.rhs(tdev(r)))
    close(fr, o.rhs(p.V, r * p.chi), TOL64, m)
    assert np.all(fr[~m] == 0.0)


def test_eval_u_alg3_and_transpose(case):
    p, H, o = case
    m = p.chi > 0
    d = W.random_field(p.nbox, 6)
    u = np_(H.eval_u(tdev(d)))
    close(u, o.eval_u(d * p.chi), TOL64, m)
    w = np_(H.eval_u_transpose(tdev(d)))
    close(w, o.eval_u_transpose(d * p.chi), TOL64, m)
    assert np.all(u[~m] == 0.0) and np.all(w[~m] == 0.0)


def test_host_pointers_same_result(case):
    """The ABI accepts host arrays (staged by the library) with the same result."""
    p, H, o = case
    d = W.random_field(p.nbox, 7)
    f_host = H.apply_K(d)
    f_dev = np_(H.apply_K(tdev(d)))
    assert np.array_equal(f_host, f_dev)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("nb,a", [(16, 2.0), (16, 2.5), (32, 2.0)])
def test_solve_alg5_matches_oracle(nb, a, prec):
    """Alg. 5 with strong Dirichlet data (random g on Gamma_g): d and u^h against the
    oracle's direct / CG solve of the assembled system."""
    p = W.cube_problem(nb, a, 1, "sin")
    p.g = np.where(p.chi_gamma > 0, 0.1 * W.random_field(p.nbox, 5), 0.0)
    H = rk.Handle.from_problem(p, device=DEV)
    o = Oracle(p.n, p.h, a, 1, p.chi)
    do, info_o = o.solve(p.V, p.chi_gamma, p.r, p.g, tol=1e-14)
    uo = o.eval_u(do)
    d, u, info = H.solve(tdev(p.r), tdev(p.g), precision=prec, tol=1e-13)
    assert info["rel_residual"] <= 1e-13
    close(np_(d), do, 1e-9)
    close(np_(u), uo, 1e-9)
    gam = p.chi_gamma > 0
    assert np.array_equal(np_(d)[gam], p.g[gam])


@functools.lru_cache(maxsize=None)
def _oracle_adjoint(nb):
    """The oracle's gradient: direct solves at 16^3; at 32^3 CG on the assembled
    CSR to 1e-13 (the adjoint system does not reach 1e-14 in FP64 CG there)."""
    p = W.adjoint_problem(n_box=nb, a_tilde=2.5, degree=1, sigma=0.2)
    o = Oracle(p.n, p.h, 2.5, 1, p.chi)
    Jo, gro, ggo, _, _ = o.adjoint(p.V, p.chi, p.chi_gamma, p.r, p.g, p.meta["u_target"],
                                   tol=1e-14 if nb <= 16 else 1e-13)
    return p, Jo, gro, ggo


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("nb", [16, 32])
def test_adjoint_matches_oracle_gradient(prec, nb):
    """dJ/dr and dJ/dg from the adjoint solve against the oracle's assembled-K
    gradient."""
    p, Jo, gro, ggo = _oracle_adjoint(nb)
    H = rk.Handle.from_problem(p, device=DEV)
    ut = p.meta["u_target"]
    J, gr, gg, info = H.solve_adjoint(tdev(p.r), tdev(p.g), tdev(ut), precision=prec, tol=1e-13)
    assert abs(J - Jo) <= 1e-10 * Jo
    close(np_(gr), gro, 1e-8)
    close(np_(gg), ggo, 1e-8)


@pytest.mark.parametrize("nb,a,deg", [(128, 2.5, 1), (96, 2.5, 1), (64, 3.0, 2)])
def test_full_size_sampled_parity(nb, a, deg):
    """At full sizes: K.u (FP64 and FP32) and b on sampled nodes, each recomputed by the
    oracle from scratch; the sample includes faces, edges and corners of the cube."""
    p = W.cube_problem(nb, a, deg, "sin")
    H = rk.Handle.from_problem(p, device=DEV)
    rng = np.random.default_rng(nb)
    n_om = p.meta["n_omega_side"]
    pts = [(0, 0, 0), (n_om - 1, 0, 0), (1, n_om - 1, 2), (n_om - 1, n_om - 1, n_om - 1), (n_om // 2,) * 3]
    pts += [tuple(rng.integers(0, n_om, 3)) for _ in range(40)]
    sample = np.array([i + nb * (j + nb * k) for i, j, k in pts], dtype=np.int64)
    d = W.random_field(p.nbox, 9)
    f64 = np_(H.apply_K(tdev(d)))
    f32 = np_(H.apply_K(tdev(d.astype(np.float32)))).astype(np.float64)
    fo = apply_K_sampled(p.n, p.h, a, deg, p.chi, p.V, d, sample)
    close(f64[sample], fo, TOL64)
    fo32 = apply_K_sampled(p.n, p.h, a, deg, p.chi, p.V, d.astype(np.float32).astype(np.float64), sample)
    close(f32[sample], fo32, TOL32)
    bg = np_(H.get_b(torch.empty(4 * p.s * p.nbox, dtype=torch.float64, device=DEV)))
    bo = b_sampled(p.n, p.h, a, deg, p.chi, sample)
    for i in range(4):
        close(bg[i][:, sample].T, bo[:, i, :], TOL64)


def cube_sample(nb, a, n_random=24, seed=0):
    """Grid indices of a structured sample of the cube's domain nodes: the 8 corners,
    nodes on the 12 edges, on the 6 faces, on every layer from the face inwards to
    the first regular layer (the first whose support lies in the domain) on each
    axis, and random interior nodes."""
    n_om = nb - int(np.floor(a))
    reach = int(np.ceil(a)) - 1
    L = n_om - 1
    rng = np.random.default_rng(seed)
    pts = [(i, j, k) for i in (0, L) for j in (0, L) for k in (0, L)]
    for t in (1, L // 3, L - 1):
        pts += [(t, 0, 0), (0, t, L), (L, L, t), (0, L, t), (t, L, 0), (L, t, L)]
    for f in range(6):
        ax, side = f // 2, (0 if f % 2 == 0 else L)
        for _ in range(2):
            c = list(rng.integers(1, L, 2))
            c.insert(ax, side)
            pts.append(tuple(c))
    for layer in range(1, reach + 2):
        for ax in range(3):
            for side in (layer, L - layer):
                c = list(rng.integers(reach + 1, L - reach, 2))
                c.insert(ax, side)
                pts.append(tuple(c))
    pts += [tuple(rng.integers(0, n_om, 3)) for _ in range(n_random)]
    return np.unique(np.array([i + nb * (j + nb * k) for i, j, k in pts], dtype=np.int64))


def test_full_size_sampled_parity_cube256_linear():
    """The benchmarked operator itself: the 256^3-box cube, a = 2.5h, linear basis,
    whose z split writes g of the regular nodes through the scaled multiplier rows
    and leaves the boundary groups to the pointwise kernel.  K.u in FP64 and FP32
    and b at >= 64 structured sample nodes (corners, edges, faces, each layer up to
    the first regular one, interior), each recomputed by the oracle from scratch
    (Alg. 2 against the neighbour sums of Eq. 50/54)."""
    nb, a = 256, 2.5
    p = W.cube_problem(nb, a, 1, "sin")
    H = rk.Handle.from_problem(p, device=DEV)
    sample = cube_sample(nb, a, seed=256)
    assert sample.size >= 64 and np.all(p.chi[sample] == 1)
    d = W.random_field(p.nbox, 9)
    f64 = np_(H.apply_K(tdev(d)))
    fo = apply_K_sampled(p.n, p.h, a, 1, p.chi, p.V, d, sample)
    close(f64[sample], fo, TOL64, what="FP64 K.u")
    d32 = d.astype(np.float32)
    f32 = np_(H.apply_K(tdev(d32))).astype(np.float64)
    fo32 = apply_K_sampled(p.n, p.h, a, 1, p.chi, p.V, d32.astype(np.float64), sample)
    close(f32[sample], fo32, TOL32, what="FP32 K.u")
    assert np.all(f64[p.chi == 0] == 0.0) and np.all(f32[p.chi == 0] == 0.0)
    bg = np_(H.get_b(torch.empty(4 * p.s * p.nbox, dtype=torch.float64, device=DEV)))
    bo = b_sampled(p.n, p.h, a, 1, p.chi, sample)
    for i in range(4):
        close(bg[i][:, sample].T, bo[:, i, :], TOL64, what=f"b family {i}")
    H.close()


def test_full_size_sampled_parity_spheres256_quadratic():
    """The embedded-domain workload at full size: 12 spheres in a 256^3 box, quadratic
    basis, a = 3h.  K.u (FP64, FP32) and b at sampled nodes (interior, boundary and
    near-boundary), each recomputed by the oracle from scratch."""
    p = W.spheres_problem(n_box=256, n_spheres=12, a_tilde=3.0, degree=2)
    H = rk.Handle.from_problem(p, device=DEV)
    rng = np.random.default_rng(256)
    inside = np.flatnonzero(p.chi)
    bnd = np.flatnonzero(p.chi_gamma)
    sample = np.unique(np.concatenate([rng.choice(inside, 40, replace=False), rng.choice(bnd, 24, replace=False)]))
    d = W.random_field(p.nbox, 9) * p.chi
    f64 = np_(H.apply_K(tdev(d)))
    fo = apply_K_sampled(p.n, p.h, 3.0, 2, p.chi, p.V, d, sample)
    close(f64[sample], fo, TOL64)
    f32 = np_(H.apply_K(tdev(d.astype(np.float32)))).astype(np.float64)
    fo32 = apply_K_sampled(p.n, p.h, 3.0, 2, p.chi, p.V, d.astype(np.float32).astype(np.float64), sample)
    close(f32[sample], fo32, TOL32)
    bg = np_(H.get_b(torch.empty(4 * p.s * p.nbox, dtype=torch.float64, device=DEV)))
    bo = b_sampled(p.n, p.h, 3.0, 2, p.chi, sample)
    for i in range(4):
        close(bg[i][:, sample].T, bo[:, i, :], TOL64)
    H.close()


def test_gap_narrower_than_support_is_rejected():
    """A domain that touches its periodic image within the support is refused (Eq. 66).
    At a = 2h the reach is one node (phi(2h) = 0), so one empty node suffices; with
    no empty node along x the set-up must fail."""
    p = W.cube_problem(16, 2.0, 1, "sin")
    chi = p.chi.reshape(16, 16, 16).copy()
    chi[:, :, 14] = chi[:, :, 0]   # close the gap on x: nodes 13 and 0 become neighbours
    chi[:, :, 15] = chi[:, :, 0]   # through the periodic boundary
    with pytest.raises(rk.RKError) as e:
        rk.Handle(p.n, p.h, tdev(chi.reshape(-1)), tdev(p.chi_gamma), tdev(p.V), 1, 2.0)
    assert e.value.status == 8


def test_singular_moment_reported():
    """An isolated node has too few neighbours for a linear basis (Eq. 5): reported,
    not fatal."""
    chi = np.zeros(16 ** 3, dtype=np.uint8)
    chi[5 + 16 * (5 + 16 * 5)] = 1
    V = chi * 1e-3
    H = rk.Handle((16, 16, 16), (0.1, 0.1, 0.1), tdev(chi), tdev(np.zeros_like(chi)), tdev(V), 1, 2.0)
    assert H.setup_status == 4
    assert H.singular == (1, 5 + 16 * (5 + 16 * 5))


# Support sweep with the shapes of Tab. 4-5: a 20^3-node cube domain (box side
# 20 + floor(a~), Eq. 64-67) for a~ = 1.5 ... 4.5, i.e. M = 27 ... 729 neighbours,
# embedded in a 32^3 box; both bases where the moment matrices are regular.
@pytest.mark.parametrize("a,deg", [(1.5, 1), (2.0, 1), (2.5, 1), (3.0, 1), (3.5, 1), (4.0, 1), (4.5, 1),
                                   (2.5, 2), (3.5, 2), (4.5, 2)])
def test_support_sweep_tab4_tab5(a, deg):
    nb = 20 + int(np.floor(a))
    p = W.embed(W.cube_problem(nb, a, deg, "zero"), (32, 32, 32))
    assert int(p.chi.sum()) == 20 ** 3
    H = rk.Handle.from_problem(p, device=DEV)
    o = Oracle(p.n, p.h, a, deg, p.chi)
    m = p.chi > 0
    bg = np_(H.get_b(torch.empty(4 * p.s * p.nbox, dtype=torch.float64, device=DEV)))
    bo = o.b_fields()
    for i in range(4):
        close(bg[i][:, m], bo[i][:, m], TOL64, what=f"b family {i}")
    d = W.random_field(p.nbox, 13)
    fo = o.apply_K(p.V, d * p.chi)
    f = np_(H.apply_K(tdev(d)))
    close(f, fo, TOL64, m)
    assert np.all(f[~m] == 0.0)
    f32 = np_(H.apply_K(tdev(d.astype(np.float32)))).astype(np.float64)
    close(f32, o.apply_K(p.V, d.astype(np.float32).astype(np.float64) * p.chi), TOL32, m)
    H.close()


def test_paper_3d_problem_converges_quadratically_on_the_gpu():
    """Sec. 6.1.3 (Eq. 106-108: a = 1.5h, linear basis, u = prod(1 - x_k^2) on
    [-1, 1]^3), solved on the GPU (mixed precision with FP64 refinement) at boxes
    16^3 ... 256^3: the nodal normalised L2 error of Eq. 104 falls at the quadratic
    rate the paper states for n = 1 (the oracle gives 1.95-1.99 over 16^3-48^3)."""
    errs, hs = [], []
    for nb in (16, 32, 64, 128, 256):
        p = W.cube_problem(nb, 1.5, 1, "paper", -1.0, 1.0)
        H = rk.Handle.from_problem(p, device=DEV)
        d, u, info = H.solve(tdev(p.r), tdev(p.g), precision="mixed", tol=1e-11)
        assert info["status"] == 0
        m = p.chi > 0
        uu = np_(u)
        errs.append(np.sqrt(((uu - p.u_exact)[m] ** 2).sum() / (p.u_exact[m] ** 2).sum()))
        hs.append(p.h[0])
        H.close()
    rates = np.diff(np.log(errs)) / np.diff(np.log(hs))
    assert np.all(rates > 1.85) and np.all(rates < 2.15), rates
