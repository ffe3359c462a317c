"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each checks a value printed in the
paper, a closed form derived by hand from Eq. 7, an identity that the reproducing
construction (Eq. 2-3, 15-16) guarantees, or the paper's stated convergence rate.
A dropped term, a wrong sign or index, or a transposed operand in the oracle fails
at least one of them (noted per test).
"""
from fractions import Fraction

import numpy as np
import pytest

from conftest import read_golden
from oracle.oracle import Oracle, apply_K_sampled, b_sampled, phi1
from paper_2403_19854_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore")


def _cube(nb, a, deg=1, kind="sin"):
    lohi = (-1.0, 1.0) if kind == "paper" else (0.0, 1.0)
    return W.cube_problem(nb, a, deg, kind, *lohi)


def _coords(p):
    X, Y, Z = p.coords()
    return np.stack([X, Y, Z], 1)


# --------------------------------------------------------------------------- Eq. 7
def test_kernel_values_eq7():
    """phi at hand-evaluated points of Eq. 7 (golden), both branches, the support end."""
    for z, num, den in read_golden("phi_eq7.txt"):
        assert phi1(float(z)) == pytest.approx(int(num) / int(den), abs=1e-15)
        assert phi1(-float(z)) == phi1(float(z))


def test_kernel_c2_continuity_eq7():
    """Eq. 7 is a cubic B-spline: value, slope and curvature continuous at z = 1/2, and
    it reaches 0 with zero slope at z = 1 (a wrong coefficient breaks one of these)."""
    e = 1e-5
    for z0 in (0.5, 1.0):
        left = [phi1(z0 - k * e) for k in (0, 1, 2)]
        right = [phi1(z0 + k * e) for k in (0, 1, 2)] if z0 < 1 else [0.0, 0.0, 0.0]
        dl = (left[0] - left[1]) / e
        dr = (right[1] - right[0]) / e if z0 < 1 else 0.0
        assert abs(dl - dr) < 1e-4
    # curvature at 1/2: 4 from both sides (second differences)
    c_left = (phi1(0.5) - 2 * phi1(0.5 - 1e-3) + phi1(0.5 - 2e-3)) / 1e-6
    c_right = (phi1(0.5) - 2 * phi1(0.5 + 1e-3) + phi1(0.5 + 2e-3)) / 1e-6
    assert abs(c_left - c_right) < 0.05


def test_bspline_partition_of_unity_at_a2():
    """With a = 2h the profile is the uniform cubic B-spline, whose integer shifts sum
    to one at every point: sum_i phi(|u - i| / 2) = 1."""
    for u in np.linspace(0.0, 1.0, 11):
        s = sum(phi1(abs(u - i) / 2.0) for i in range(-3, 5))
        assert s == pytest.approx(1.0, abs=1e-15)


# ------------------------------------------------------------------ Sec. 5.1, Tab.
def test_box_rule_tab1_tab10():
    """Domain nodes per box side match Tab. 1 (a = 1.5h) and Tab. 10 (a = 3.5h)."""
    for side, a, total in read_golden("tab1_tab10_box_nodes.txt"):
        assert W.domain_side(int(side), float(a)) ** 3 == int(total)


def test_neighbour_counts_tab4_tab5():
    """Interior neighbour count M of Tab. 4-5 from the oracle's grid search."""
    for a, M in read_golden("tab4_tab5_neighbours.txt"):
        a = float(a)
        p = _cube(14, a)
        o = Oracle(p.n, p.h, a, 1, p.chi)
        nb = o.node_box()
        c = 4 + 14 * (4 + 14 * 4)
        assert o.neighbour_count(int(np.searchsorted(nb, c))) == int(M)


def test_neighbour_search_equals_brute_force():
    """Grid search over +-reach == O(N^2) scan over all nodes, on an irregular domain."""
    p = W.spheres_problem(n_box=12, n_spheres=3, a_tilde=2.5, degree=1, r_range=(0.15, 0.3), seed=7)
    o = Oracle(p.n, p.h, 2.5, 1, p.chi)
    for S in range(0, o.nnode, max(1, o.nnode // 97)):
        assert o.neighbour_count(S) == o.neighbour_count(S, brute_force=True)


# ----------------------------------------------------------- reproducing conditions
def _monomials(deg):
    out = [(0, 0, 0)]
    out += [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
    if deg == 2:
        out += [(2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2)]
    return out


@pytest.mark.parametrize("case", ["cube1", "cube2", "spheres1", "spheres2"])
def test_reproducing_conditions(case):
    """sum_I Psi_I(x_S) (x_I - x_S)^alpha = delta_{alpha,0} and
    sum_I Psi^{grad k}_I(x_S) (x_I - x_S)^alpha = delta_{alpha,e_k} for |alpha| <= n at every
    node (Eq. 2-3 and 15-16).  A wrong row of M^{-1}, a wrong basis entry or a sign
    error in Eq. 46-47 fails this."""
    deg = 1 if case.endswith("1") else 2
    a = 2.5 if deg == 1 else 3.0
    if case.startswith("cube"):
        p = _cube(12, a, deg)
    else:
        p = W.spheres_problem(n_box=16, n_spheres=3, a_tilde=a, degree=deg, r_range=(0.2, 0.3), seed=11)
    o = Oracle(p.n, p.h, a, deg, p.chi)
    assert o.nsingular == 0
    nbr, psi, dpsi = o.shape_tables()
    nb = o.node_box()
    X = _coords(p)
    xs = X[nb]
    valid = nbr >= 0
    xI = X[nb[np.where(valid, nbr, 0)]]
    rel = (xI - xs[:, None, :]) / (a * np.asarray(p.h))  # scaled offsets, O(1)
    hh = np.asarray(p.h)
    for al in _monomials(deg):
        mono = np.where(valid, rel[..., 0] ** al[0] * rel[..., 1] ** al[1] * rel[..., 2] ** al[2], 0.0)
        target = 1.0 if al == (0, 0, 0) else 0.0
        assert np.abs((psi * mono).sum(1) - target).max() < 1e-12
        for k in range(3):
            ek = tuple(1 if j == k else 0 for j in range(3))
            # Psi^grad has units 1/length; with scaled offsets the identity reads
            # sum Psi^grad_k * rel^alpha * a = delta_{alpha, e_k}
            t = 1.0 if al == ek else 0.0
            got = (dpsi[..., k] * mono).sum(1) * a * hh[k]
            assert np.abs(got - t).max() < 1e-11


# ------------------------------------------------------ closed-form interior stencil
def _w_a2():
    return {-1: Fraction(1, 6), 0: Fraction(2, 3), 1: Fraction(1, 6)}


def test_interior_shape_functions_closed_form_a2():
    """At a = 2h the interior moment matrix is diag(1, 1/12, 1/12, 1/12) (scaled basis):
    Psi_I(x_S) = w w w and Psi^{grad x}_I(x_S) = o_x/(2h) w(o_y) w(o_z) with the B-spline
    weights w = (1/6, 2/3, 1/6), i.e. a central difference smoothed by the B-spline."""
    p = _cube(14, 2.0)
    o = Oracle(p.n, p.h, 2.0, 1, p.chi)
    nbr, psi, dpsi = o.shape_tables()
    nb = o.node_box()
    h = p.h[0]
    w = _w_a2()
    S = int(np.searchsorted(nb, 5 + 14 * (6 + 14 * 5)))
    for sl in range(27):
        ox, oy, oz = sl % 3 - 1, (sl // 3) % 3 - 1, sl // 9 - 1
        assert psi[S, sl] == pytest.approx(float(w[ox] * w[oy] * w[oz]), abs=1e-15)
        assert dpsi[S, sl, 0] * 2 * h == pytest.approx(float(ox * w[oy] * w[oz]), abs=1e-14)
        assert dpsi[S, sl, 1] * 2 * h == pytest.approx(float(oy * w[ox] * w[oz]), abs=1e-14)
        assert dpsi[S, sl, 2] * 2 * h == pytest.approx(float(oz * w[ox] * w[oy]), abs=1e-14)
    bf = o.b_fields()
    c = 5 + 14 * (6 + 14 * 5)
    assert bf[0, :, c] == pytest.approx([1, 0, 0, 0], abs=1e-14)
    assert bf[1, :, c] * h == pytest.approx([0, -6, 0, 0], abs=1e-12)   # -(1/a) * 12, a = 2h


def test_interior_stiffness_row_closed_form_a2():
    """Deep-interior rows of K at a = 2h equal h^3 sum_k D_k^T D_k with the exact
    rational stencil above (K_{I,I+D} = (h/4) * integer/1296), computed with fractions.
    Pins V, the DNI sum of Eq. 54 and the pairing of I and J."""
    p = _cube(14, 2.0)
    o = Oracle(p.n, p.h, 2.0, 1, p.chi)
    o.assemble_K(p.V)
    ptr, col, val = o.K_csr()
    nb = o.node_box()
    h = p.h[0]
    w = _w_a2()
    offs = [(x, y, z) for z in (-1, 0, 1) for y in (-1, 0, 1) for x in (-1, 0, 1)]

    def c(k, o3):
        others = [w[o3[j]] for j in range(3) if j != k]
        return o3[k] * others[0] * others[1]

    exact = {}
    for D in [(x, y, z) for z in range(-2, 3) for y in range(-2, 3) for x in range(-2, 3)]:
        s = Fraction(0)
        for o3 in offs:
            o2 = (o3[0] + D[0], o3[1] + D[1], o3[2] + D[2])
            if max(abs(v) for v in o2) > 1:
                continue
            for k in range(3):
                s += c(k, o3) * c(k, o2)
        exact[D] = s
    n = 14
    for (i, j, k) in [(5, 6, 5), (2, 2, 2), (6, 4, 7)]:
        I = int(np.searchsorted(nb, i + n * (j + n * k)))
        row = {}
        for e in range(ptr[I], ptr[I + 1]):
            J = nb[col[e]]
            D = (J % n - i, (J // n) % n - j, J // (n * n) - k)
            row[D] = val[e]
        for D, v in exact.items():
            assert row.get(D, 0.0) == pytest.approx(float(v) * h / 4.0, rel=1e-12, abs=1e-15 * h)


def test_interior_gradient_stencil_a25_properties():
    """At a = 2.5h (reach 2) the interior implicit gradient is antisymmetric in the
    derivative axis, exact on linear functions (sum_o c(o) o_x h = 1), and proportional
    to o_x phi(|o_x|/2.5) along that axis (the diagonal moment matrix of the interior)."""
    p = _cube(14, 2.5)
    o = Oracle(p.n, p.h, 2.5, 1, p.chi)
    nbr, psi, dpsi = o.shape_tables()
    nb = o.node_box()
    h = p.h[0]
    S = int(np.searchsorted(nb, 5 + 14 * (5 + 14 * 5)))
    g = dpsi[S, :, 0].reshape(5, 5, 5)  # [oz, oy, ox]
    assert np.abs(g + g[:, :, ::-1]).max() < 1e-13 / h
    ox = np.arange(-2, 3)
    assert (g.sum(axis=(0, 1)) * ox * h).sum() == pytest.approx(1.0, abs=1e-13)
    prof = g.sum(axis=(0, 1))
    ratio = prof[3] / prof[4]
    assert ratio == pytest.approx((1 * phi1(1 / 2.5)) / (2 * phi1(2 / 2.5)), rel=1e-12)


# ------------------------------------------------------------------ stiffness matrix
@pytest.mark.parametrize("deg,a,geom", [(1, 2.0, "cube"), (1, 2.5, "spheres"), (2, 3.0, "cube")])
def test_stiffness_symmetric_psd_constants_in_null_space(deg, a, geom):
    """K of Eq. 26 is symmetric, positive semidefinite, and K.1 = 0 before boundary
    conditions (the implicit gradient reproduces constants with zero gradient)."""
    if geom == "cube":
        p = _cube(10 if deg == 1 else 12, a, deg)
    else:
        p = W.spheres_problem(n_box=14, n_spheres=2, a_tilde=a, degree=deg, r_range=(0.25, 0.3), seed=5)
    o = Oracle(p.n, p.h, a, deg, p.chi)
    o.assemble_K(p.V)
    ptr, col, val = o.K_csr()
    K = np.zeros((o.nnode, o.nnode))
    for I in range(o.nnode):
        K[I, col[ptr[I]:ptr[I + 1]]] = val[ptr[I]:ptr[I + 1]]
    nrm = np.abs(K).max()
    assert np.abs(K - K.T).max() <= 1e-14 * nrm
    assert np.abs(K.sum(1)).max() <= 1e-13 * nrm
    assert np.linalg.eigvalsh(K).min() >= -1e-12 * nrm


def test_energy_of_linear_field_equals_volume():
    """For d = a.x + c the implicit gradient is exactly a at every node, so
    d^T K d = |a|^2 sum_S V_S = |a|^2 (unit cube, trapezoidal V sums to 1).
    A wrong V, a dropped gradient component or a missing DNI weight fails this."""
    for a_t, deg in ((2.0, 1), (2.5, 1), (3.0, 2)):
        p = _cube(12, a_t, deg)
        o = Oracle(p.n, p.h, a_t, deg, p.chi)
        X = _coords(p)
        av = np.array([0.3, -1.2, 0.7])
        d = np.where(p.chi > 0, X @ av + 0.4, 0.0)
        f = o.apply_K(p.V, d)
        assert p.V.sum() == pytest.approx(1.0, abs=1e-14)
        assert float(d @ f) == pytest.approx(float(av @ av), rel=1e-12)


def test_matrix_free_equals_assembled():
    """Matrix-free neighbour loops (g = B d, f = B^T V g) == assembled CSR SpMV."""
    p = W.spheres_problem(n_box=14, n_spheres=3, a_tilde=2.5, degree=1, r_range=(0.2, 0.3), seed=3)
    o = Oracle(p.n, p.h, 2.5, 1, p.chi)
    d = W.random_field(p.nbox, 1) * p.chi
    f1 = o.apply_K(p.V, d)
    o.assemble_K(p.V)
    f2 = o.spmv(d)
    assert np.abs(f1 - f2).max() <= 1e-13 * np.abs(f1).max()


def test_sampled_mode_equals_tables():
    """Per-node recomputation (used at full sizes) == the tabulated discretisation."""
    p = W.spheres_problem(n_box=14, n_spheres=3, a_tilde=3.0, degree=2, r_range=(0.15, 0.25), seed=9)
    o = Oracle(p.n, p.h, 3.0, 2, p.chi)
    d = W.random_field(p.nbox, 2) * p.chi
    f = o.apply_K(p.V, d)
    sample = np.flatnonzero(p.chi)[::7]
    fs = apply_K_sampled(p.n, p.h, 3.0, 2, p.chi, p.V, d, sample)
    assert np.abs(fs - f[sample]).max() <= 1e-13 * np.abs(f).max()
    bs = b_sampled(p.n, p.h, 3.0, 2, p.chi, sample)
    bf = o.b_fields()
    assert np.abs(bs - np.transpose(bf[:, :, sample], (2, 0, 1))).max() <= 1e-12 * np.abs(bf).max()


# ---------------------------------------------------------------- f^r and u^h
def test_rhs_moments():
    """sum_I f^r_I x_I^alpha = sum_S V_S r_S x_S^alpha for |alpha| <= n (Eq. 59 with the
    reproducing condition).  Transposing Psi_I(x_S) into Psi_S(x_I) breaks it."""
    p = W.spheres_problem(n_box=16, n_spheres=3, a_tilde=2.5, degree=1, r_range=(0.2, 0.3), seed=4)
    o = Oracle(p.n, p.h, 2.5, 1, p.chi)
    r = W.random_field(p.nbox, 5) * p.chi
    fr = o.rhs(p.V, r)
    X = _coords(p)
    for al in _monomials(1):
        mono = X[:, 0] ** al[0] * X[:, 1] ** al[1] * X[:, 2] ** al[2]
        lhs = float(fr @ mono)
        rhs = float((p.V * r * p.chi) @ mono)
        assert lhs == pytest.approx(rhs, rel=1e-12, abs=1e-15)


def _dense_tables(p, o):
    """(nodes, K, U) over the chi nodes in node order: the oracle's assembled K
    (Eq. 26, DNI) and U[S, J] = Psi_J(x_S) (Eq. 2) from its shape tables."""
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


def test_penalty_solution_tends_to_the_constrained_one():
    """Essential conditions by the penalty method (Sec. 2.4): the solution of
    (K + beta U^T diag(A) U) d = f^r + beta U^T (A g) tends, as beta grows, to the
    Lagrange-multiplier solution of min 1/2 d.K d - d.f^r subject to u^h = g on the
    boundary nodes, with an error O(1/beta).  Built densely from the oracle's K and
    U on a 10^3-node cube (surface weights A of its faces)."""
    p = W.cube_problem(12, 2.5, 1, "zero")
    o = Oracle(p.n, p.h, 2.5, 1, p.chi)
    nodes, K, U = _dense_tables(p, o)
    A = W.cube_surface_weights(p)[nodes]
    gam = A > 0
    assert gam.sum() == 10 ** 3 - 8 ** 3
    rng = np.random.default_rng(23)
    r = W.random_field(p.nbox, 7) * p.chi
    f = o.rhs(p.V, r)[nodes]
    g = np.where(gam, rng.standard_normal(len(nodes)), 0.0)
    C = U[gam]
    nc = C.shape[0]
    kkt = np.block([[K, C.T], [C, np.zeros((nc, nc))]])
    d_kkt = np.linalg.solve(kkt, np.concatenate([f, g[gam]]))[: len(nodes)]
    assert np.abs(C @ d_kkt - g[gam]).max() < 1e-9
    scale = np.abs(K).max() / A.max()
    errs = []
    for bt in (1e2, 1e3, 1e4, 1e5):
        beta = bt * scale
        M = K + beta * (U.T * A) @ U
        d = np.linalg.solve(M, f + beta * U.T @ (A * g))
        errs.append(np.linalg.norm(d - d_kkt) / np.linalg.norm(d_kkt))
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(5.0 < q < 20.0 for q in ratios), (errs, ratios)
    assert errs[-1] < 1e-3


@pytest.mark.parametrize("deg,a", [(1, 2.5), (2, 3.0)])
def test_grad_force_moments(deg, a):
    """The gradient-type nonlinear force of Eq. B.6-B.8, f_J = sum_S V_S sum_k
    Psi^{grad k}_J(x_S) N^k_S, against the reproduction of gradients
    (sum_J Psi^{grad k}_J(x) m(x_J) = d_k m(x) for monomials |m| <= n):
    sum_J f_J m(x_J) = sum_S V_S sum_k N^k_S d_k m(x_S).  A transposed Psi
    (Psi_S at x_J), a dropped component or a sign flips it."""
    p = W.spheres_problem(n_box=16, n_spheres=3, a_tilde=a, degree=deg, r_range=(0.2, 0.3), seed=6)
    o = Oracle(p.n, p.h, a, deg, p.chi)
    rng = np.random.default_rng(17)
    N = rng.standard_normal((3, p.nbox)) * p.chi
    f = o.grad_transpose(p.V, N)
    assert np.all(f[p.chi == 0] == 0.0)
    X = _coords(p)
    for al in _monomials(deg):
        mono = X[:, 0] ** al[0] * X[:, 1] ** al[1] * X[:, 2] ** al[2]
        rhs = 0.0
        for k in range(3):
            if al[k] == 0:
                continue
            e = list(al)
            e[k] -= 1
            dmono = al[k] * X[:, 0] ** e[0] * X[:, 1] ** e[1] * X[:, 2] ** e[2]
            rhs += float((p.V * p.chi * N[k]) @ dmono)
        lhs = float(f @ mono)
        scale = float(np.abs(p.V * N).sum()) + 1e-300
        assert abs(lhs - rhs) <= 1e-12 * scale, (al, lhs, rhs)


@pytest.mark.parametrize("deg,a", [(1, 2.5), (2, 3.0)])
def test_eval_u_reproduces_polynomials(deg, a):
    """u^h of Eq. 62 with d = a polynomial of degree <= n returns that polynomial at every
    node (near boundaries too)."""
    p = W.spheres_problem(n_box=16, n_spheres=3, a_tilde=a, degree=deg, r_range=(0.2, 0.3), seed=6)
    o = Oracle(p.n, p.h, a, deg, p.chi)
    X = _coords(p)
    q = 0.2 + 0.5 * X[:, 0] - 0.3 * X[:, 1] + 0.9 * X[:, 2]
    if deg == 2:
        q = q + 0.7 * X[:, 0] * X[:, 1] - 0.4 * X[:, 2] ** 2
    d = np.where(p.chi > 0, q, 0.0)
    u = o.eval_u(d)
    m = p.chi > 0
    assert np.abs(u[m] - q[m]).max() < 1e-12


# ---------------------------------------------------------------- solve
def test_solve_satisfies_dirichlet_system():
    """d = g on Gamma_g (Eq. 29) and K_OO d_O = f^r_O - K_OG g_G on the free nodes."""
    p = _cube(10, 2.0)
    p.g = np.where(p.chi_gamma > 0, W.random_field(p.nbox, 8), 0.0)
    o = Oracle(p.n, p.h, 2.0, 1, p.chi)
    d, info = o.solve(p.V, p.chi_gamma, p.r, p.g)
    gam = p.chi_gamma > 0
    free = (p.chi > 0) & ~gam
    assert np.array_equal(d[gam], p.g[gam])
    res = o.spmv(d) - o.rhs(p.V, p.r)
    assert np.abs(res[free]).max() <= 1e-12 * np.abs(o.rhs(p.V, p.r)).max()


@pytest.mark.slow
def test_manufactured_solution_quadratic_rate_paper_3d():
    """The 3D problem of Sec. 6.1.3 (Eq. 106-108: a = 1.5h, linear basis, u = prod(1-x_k^2)
    on [-1,1]^3) converges at the quadratic rate the paper states for RKPM with n = 1
    (Sec. 6.1.1-6.1.2; the 3D plot is Fig. 13).  Nodal normalised L2 error of Eq. 104."""
    errs, hs = [], []
    for nb in (12, 16, 24, 32):
        p = _cube(nb, 1.5, 1, "paper")
        o = Oracle(p.n, p.h, 1.5, 1, p.chi)
        d, info = o.solve(p.V, p.chi_gamma, p.r, p.g, tol=1e-13)
        assert info["converged"]
        u = o.eval_u(d)
        m = p.chi > 0
        errs.append(np.sqrt(((u - p.u_exact)[m] ** 2).sum() / (p.u_exact[m] ** 2).sum()))
        hs.append(p.h[0])
    rates = np.diff(np.log(errs)) / np.diff(np.log(hs))
    assert rates[-1] > 1.8 and rates[-1] < 2.3
    assert np.polyfit(np.log(hs), np.log(errs), 1)[0] > 1.8


def test_adjoint_gradient_matches_central_differences():
    """J(r, g) = 1/2 |u^h - u_t|^2 is quadratic in (r, g), so central differences are exact
    up to rounding; the oracle's adjoint gradient (assembled K) must match on seeded
    directions."""
    p = W.adjoint_problem(n_box=9, a_tilde=2.0, degree=1, seed=123, sigma=0.3)
    o = Oracle(p.n, p.h, 2.0, 1, p.chi)
    ut = p.meta["u_target"]
    J, gr, gg, _, _ = o.adjoint(p.V, p.chi, p.chi_gamma, p.r, p.g, ut)
    rng = np.random.default_rng(77)

    def Jof(r, g):
        d, _ = o.solve(p.V, p.chi_gamma, r, g)
        e = np.where(p.chi > 0, o.eval_u(d) - ut, 0.0)
        return 0.5 * float(e @ e)

    for _ in range(4):
        dr = rng.standard_normal(p.nbox) * p.chi
        dg = rng.standard_normal(p.nbox) * p.chi_gamma
        eps = 1e-2
        fd = (Jof(p.r + eps * dr, p.g + eps * dg) - Jof(p.r - eps * dr, p.g - eps * dg)) / (2 * eps)
        an = float(gr @ dr + gg @ dg)
        assert an == pytest.approx(fd, rel=1e-9, abs=1e-12)


def test_singular_moment_is_detected():
    """A node with too few neighbours (an isolated node) has a singular M (Eq. 5 count)."""
    chi = np.zeros(8 ** 3, dtype=np.uint8)
    chi[3 + 8 * (3 + 8 * 3)] = 1
    o = Oracle((8, 8, 8), (0.1, 0.1, 0.1), 2.0, 1, chi)
    assert o.nsingular == 1 and o.first_singular == 3 + 8 * (3 + 8 * 3)


def test_boundary_integral_moments_alg_a1():
    """f^q of Alg. A.1 (Eq. A.2): f^q_I = sum_S Psi_I(x_S) q_S A_S.  Partition of
    unity and linear reproduction of Psi fix its zeroth and first moments:
    sum_I f^q_I = sum_S q_S A_S and sum_I f^q_I x_I = sum_S q_S A_S x_S."""
    p = W.cube_problem(12, 2.5, 1, "zero")
    o = Oracle(p.n, p.h, 2.5, 1, p.chi)
    rng = np.random.default_rng(7)
    gam = p.chi_gamma > 0
    A = np.where(gam, p.h[0] ** 2 * rng.uniform(0.5, 1.0, p.nbox), 0.0)
    q = np.where(gam, rng.standard_normal(p.nbox), 0.0)
    fq = o.eval_u_transpose(q * A)
    X, Y, Z = p.coords()
    tot = np.sum(q * A)
    assert abs(fq.sum() - tot) <= 1e-12 * np.sum(np.abs(q * A))
    for c in (X, Y, Z):
        assert abs(np.sum(fq * c) - np.sum(q * A * c)) <= 1e-12 * np.sum(np.abs(q * A))
    assert np.all(fq[p.chi == 0] == 0)


def test_mass_terms_appendix_c():
    """M = sum_S V_S Psi(x_S) Psi(x_S)^T (Eq. C.5, DNI) applied as U^T (V o U v):
    symmetric; the lumped mass (row sums, Eq. C.9) equals U^T V by partition of
    unity and sums to the volume; a linear field v_I = x_I gives sum_I (Mv)_I =
    sum_S V_S x_S (linear reproduction)."""
    p = W.cube_problem(12, 2.5, 1, "zero")
    o = Oracle(p.n, p.h, 2.5, 1, p.chi)
    m = p.chi > 0

    def M(v):
        return o.eval_u_transpose(p.V * o.eval_u(v))

    rng = np.random.default_rng(9)
    x = rng.standard_normal(p.nbox) * m
    y = rng.standard_normal(p.nbox) * m
    assert abs(np.dot(y, M(x)) - np.dot(x, M(y))) <= 1e-13 * abs(np.dot(x, M(x)))
    assert np.dot(x, M(x)) > 0
    ml = o.eval_u_transpose(p.V)
    assert np.allclose(M(m.astype(float)), ml, rtol=0, atol=1e-14 * ml.max())
    assert abs(ml.sum() - p.V.sum()) <= 1e-13 * p.V.sum()
    X, _, _ = p.coords()
    assert abs(M(X * m).sum() - np.sum(p.V * X)) <= 1e-13 * np.sum(np.abs(p.V * X))


# ----------------------------------------------------------- 1D and 2D (Sec. 6.1)
def _monomials_dim(deg, dim):
    """Exponent triples of the degree <= deg monomials in the first dim coordinates."""
    return [al for al in _monomials(deg) if all(al[k] == 0 for k in range(dim, 3))]


@pytest.mark.parametrize("dim,deg,a", [(1, 1, 1.5), (1, 2, 2.5), (2, 1, 1.5), (2, 2, 2.5)])
def test_reproducing_conditions_1d_2d(dim, deg, a):
    """The reproducing conditions of Eq. 2-3 and 15-16 on the 1D and 2D grids of
    Sec. 6.1.1-6.1.2 (the paper states the method in 2D; 1D drops a coordinate):
    monomials of the present coordinates are reproduced, and the gradient along an
    absent axis is 0.  A basis that kept an absent coordinate would make M singular."""
    p = W.line_problem(24, a, deg) if dim == 1 else W.plane_problem(14, a, deg)
    o = Oracle(p.n, p.h, a, deg, p.chi)
    assert o.dim == dim and o.s == p.s and o.nsingular == 0
    nbr, psi, dpsi = o.shape_tables()
    nb = o.node_box()
    X = _coords(p)
    valid = nbr >= 0
    rel = (X[nb[np.where(valid, nbr, 0)]] - X[nb][:, None, :]) / (a * np.asarray(p.h))
    hh = np.asarray(p.h)
    for al in _monomials_dim(deg, dim):
        mono = np.where(valid, rel[..., 0] ** al[0] * rel[..., 1] ** al[1] * rel[..., 2] ** al[2], 0.0)
        assert np.abs((psi * mono).sum(1) - (1.0 if al == (0, 0, 0) else 0.0)).max() < 1e-12
        for k in range(3):
            t = 1.0 if (k < dim and al == tuple(1 if j == k else 0 for j in range(3))) else 0.0
            assert np.abs((dpsi[..., k] * mono).sum(1) * a * hh[k] - t).max() < 1e-11
    assert np.all(dpsi[..., dim:] == 0.0)


def test_interior_stiffness_row_1d_a2():
    """1D at a = 2h: the interior moment matrix is diag(1, 1/12) in the scaled basis, so
    Psi^grad_{S+o}(x_S) = 3 o w_o / h with w = (1/6, 2/3, 1/6): the central difference
    (d_{S+1} - d_{S-1}) / (2h).  With V = h (Eq. 54) a deep-interior row of K is
    [-1/(4h), 0, 1/(2h), 0, -1/(4h)] at offsets -2 .. 2 (the checkerboard null mode
    of DNI that the paper notes)."""
    p = W.line_problem(32, 2.0, 1)
    o = Oracle(p.n, p.h, 2.0, 1, p.chi)
    h = p.h[0]
    nbr, psi, dpsi = o.shape_tables()
    nb = o.node_box()
    S = int(np.searchsorted(nb, 12))
    for sl, off in enumerate((-1, 0, 1)):
        assert psi[S, sl] == pytest.approx(float(_w_a2()[off]), abs=1e-15)
        assert dpsi[S, sl, 0] * 2 * h == pytest.approx(float(off), abs=1e-13)
    o.assemble_K(p.V)
    ptr, col, val = o.K_csr()
    I = int(np.searchsorted(nb, 12))
    row = {int(nb[col[e]]) - 12: val[e] for e in range(ptr[I], ptr[I + 1])}
    exact = {-2: -0.25 / h, -1: 0.0, 0: 0.5 / h, 1: 0.0, 2: -0.25 / h}
    for D, v in exact.items():
        assert row.get(D, 0.0) == pytest.approx(v, rel=1e-12, abs=1e-12 / h)
    assert set(row) <= set(exact)


@pytest.mark.parametrize("dim", [1, 2])
def test_stiffness_symmetric_constants_in_null_space_1d_2d(dim):
    """K of Eq. 50 is symmetric and annihilates constants (gradient reproduction)."""
    p = W.line_problem(24, 2.5, 1) if dim == 1 else W.plane_problem(16, 2.5, 1)
    o = Oracle(p.n, p.h, 2.5, 1, p.chi)
    o.assemble_K(p.V)
    ptr, col, val = o.K_csr()
    import scipy.sparse as sp
    K = sp.csr_matrix((val, col, ptr), shape=(o.nnode, o.nnode))
    nK = abs(K).max()
    assert abs(K - K.T).max() <= 1e-14 * nK
    assert np.abs(K @ np.ones(o.nnode)).max() <= 1e-13 * nK


@pytest.mark.parametrize("dim", [1, 2])
def test_manufactured_solution_quadratic_rate_1d_2d(dim):
    """Sec. 6.1.1 (Eq. 97-99) and Sec. 6.1.2 (Eq. 101-103): a = 1.5h, linear basis; the
    paper reports quadratic convergence (Fig. 9, Fig. 11).  Nodal normalised L2 error
    of Eq. 104."""
    sizes = (16, 32, 64, 128) if dim == 1 else (12, 16, 24, 32)
    errs, hs = [], []
    for nb in sizes:
        p = W.line_problem(nb, 1.5, 1) if dim == 1 else W.plane_problem(nb, 1.5, 1)
        o = Oracle(p.n, p.h, 1.5, 1, p.chi)
        d, info = o.solve(p.V, p.chi_gamma, p.r, p.g, tol=1e-13)
        assert info["converged"]
        m = p.chi > 0
        u = o.eval_u(d)
        errs.append(np.sqrt(((u - p.u_exact)[m] ** 2).sum() / (p.u_exact[m] ** 2).sum()))
        hs.append(p.h[0])
    rates = np.diff(np.log(errs)) / np.diff(np.log(hs))
    assert np.all(rates > 1.9) and np.all(rates < 2.1)


def test_interior_shape_functions_closed_form_2d_a2():
    """2D at a = 2h: the interior moment matrix is diag(1, 1/12, 1/12) (scaled basis),
    so Psi_I(x_S) = w(o_x) w(o_y) and Psi^{grad x}_I(x_S) = o_x/(2h) w(o_y) with the
    B-spline weights w = (1/6, 2/3, 1/6); the z gradient is 0 (no z axis)."""
    p = W.plane_problem(16, 2.0, 1)
    o = Oracle(p.n, p.h, 2.0, 1, p.chi)
    nbr, psi, dpsi = o.shape_tables()
    nb = o.node_box()
    h = p.h[0]
    w = _w_a2()
    c = 6 + 16 * 7
    S = int(np.searchsorted(nb, c))
    assert o.nslot == 9
    for sl in range(9):
        ox, oy = sl % 3 - 1, sl // 3 - 1
        assert psi[S, sl] == pytest.approx(float(w[ox] * w[oy]), abs=1e-15)
        assert dpsi[S, sl, 0] * 2 * h == pytest.approx(float(ox * w[oy]), abs=1e-14)
        assert dpsi[S, sl, 1] * 2 * h == pytest.approx(float(oy * w[ox]), abs=1e-14)
        assert dpsi[S, sl, 2] == 0.0
    bf = o.b_fields()
    assert bf[0, :, c] == pytest.approx([1, 0, 0], abs=1e-14)
    assert bf[1, :, c] * h == pytest.approx([0, -6, 0], abs=1e-12)   # -(1/a) * 12, a = 2h
    assert np.all(bf[3] == 0.0)


@pytest.mark.parametrize("dim", [1, 2])
def test_line_plane_inputs_trapezoidal_measure(dim):
    """The nodal volumes of the line and plane problems are the trapezoidal rule on
    [-1, 1]^dim: they sum to 2^dim and integrate the exact solution (a polynomial of
    degree 2 per axis) with error O(h^2); the Dirichlet nodes are the boundary."""
    p = W.line_problem(33, 1.5) if dim == 1 else W.plane_problem(33, 1.5)
    assert p.V.sum() == pytest.approx(2.0 ** dim, rel=1e-14)
    exact = 4.0 / 3.0 if dim == 1 else (4.0 / 3.0) ** 2
    assert abs((p.V * p.u_exact).sum() - exact) < 2 * p.h[0] ** 2
    X, Y, _ = p.coords()
    X, Y = X - 1.0, Y - 1.0
    on = p.chi > 0
    bnd = (np.isclose(np.abs(X), 1.0) | ((dim == 2) & np.isclose(np.abs(Y), 1.0))) & on
    assert np.array_equal(p.chi_gamma > 0, bnd)


def test_arbitrary_point_evaluation_1d_reproduces_and_matches_nodes():
    """Eq. 1-2 at arbitrary points: the linear basis reproduces any linear field
    exactly everywhere (d_I = alpha + beta x_I gives u^h(x) = alpha + beta x), and at
    the nodes the value equals Eq. 62 (the nodal evaluation)."""
    p = W.line_problem(40, 2.5, 1)
    o = Oracle(p.n, p.h, 2.5, 1, p.chi)
    h = p.h[0]
    n_om = p.meta["n_omega_side"]
    rng = np.random.default_rng(7)
    x = rng.uniform(0.0, (n_om - 1) * h, 200)
    X = np.arange(p.nbox) * h
    d = np.where(p.chi > 0, 0.3 - 1.7 * X, 0.0)
    assert np.abs(o.eval_points_1d(x, d) - (0.3 - 1.7 * x)).max() < 1e-12
    d2 = W.random_field(p.nbox, 3)
    nodes = np.arange(n_om) * h
    assert np.abs(o.eval_points_1d(nodes, d2) - o.eval_u(d2 * p.chi)[:n_om]).max() < 1e-13


def test_paper_1d_gauss_quadrature_error_rate():
    """Sec. 6.1.1 measures the L2 error of Eq. 100 with 5 Gauss points per cell; the
    paper reports the quadratic rate (Fig. 9).  a = 1.5h, linear basis, N = 2^4 ... 2^8."""
    gx, gw = np.polynomial.legendre.leggauss(5)
    errs, hs = [], []
    for nb in (16, 32, 64, 128, 256):
        p = W.line_problem(nb, 1.5, 1)
        o = Oracle(p.n, p.h, 1.5, 1, p.chi)
        d, info = o.solve(p.V, p.chi_gamma, p.r, p.g, tol=1e-13)
        assert info["converged"]
        h = p.h[0]
        n_om = p.meta["n_omega_side"]
        left = np.arange(n_om - 1) * h
        xq = (left[:, None] + 0.5 * h * (gx[None, :] + 1.0)).reshape(-1)
        wq = np.tile(0.5 * h * gw, n_om - 1)
        uh = o.eval_points_1d(xq, d)
        ue = 1.0 - (xq - 1.0) ** 2           # node 0 sits at x = -1
        errs.append(np.sqrt((wq * (uh - ue) ** 2).sum()))
        hs.append(h)
    rates = np.diff(np.log(errs)) / np.diff(np.log(hs))
    assert np.all(rates > 1.9) and np.all(rates < 2.1), rates
