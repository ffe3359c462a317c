"""Seeded synthetic inputs for the 3D Poisson problem of Eq. 8 (geometry, nodal
volumes, sources, boundary data).

This module holds no part of the method's arithmetic: it only builds the input
arrays that Alg. 5 reads (chi, chi_Gamma_g, V, r, g -- Eq. 40, 87, 93, 95) on a
uniform grid, plus analytic reference fields.  Both the CUDA path and the oracle
consume what it produces; neither is imported here.

Grid convention: a periodic box of nx x ny x nz nodes (x fastest, flat index
i + nx*(j + ny*k)), node (i, j, k) at (i*h_x, j*h_y, k*h_z) relative to the box
origin.  The domain Omega occupies the first n_omega nodes of each axis and the
remaining floor(a_tilde) nodes per axis form the gap of Eq. 66
(l_e = (floor(a_tilde) + 1) h), so a box side N holds N - floor(a_tilde) domain
nodes (Tab. 1: 343 domain nodes in an 8^3 box at a_tilde = 1.5; Tab. 10:
2,048,383 = 127^3 at a_tilde = 3.5 in a 130^3 box).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 20240328


@dataclass
class Problem:
    """Inputs of Alg. 5 on one box, grid-indexed flat arrays (x fastest)."""

    n: tuple            # (nx, ny, nz) box nodes
    h: tuple            # (hx, hy, hz) spacing
    a_tilde: float      # support in units of h (Eq. 64)
    degree: int         # monomial degree n (1 or 2)
    chi: np.ndarray     # uint8, Eq. 40
    chi_gamma: np.ndarray  # uint8, Eq. 95
    V: np.ndarray       # float64 nodal volumes, Eq. 87
    r: np.ndarray       # float64 source, Eq. 93
    g: np.ndarray       # float64 Dirichlet data (read on chi_gamma only)
    u_exact: np.ndarray | None = None
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nbox(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    @property
    def n_omega(self) -> int:
        return int(self.chi.sum())

    @property
    def dim(self) -> int:
        """3, or 2 when nz = 1, or 1 when ny = nz = 1 (absent axes are trailing)."""
        return 1 if self.n[1] == 1 and self.n[2] == 1 else (2 if self.n[2] == 1 else 3)

    @property
    def s(self) -> int:
        """Monomials of degree <= n in dim coordinates (Eq. 5)."""
        return {1: self.degree + 1, 2: 3 if self.degree == 1 else 6, 3: 4 if self.degree == 1 else 10}[self.dim]

    def coords(self):
        """(X, Y, Z) flat coordinate arrays of the box nodes (Eq. 71)."""
        nx, ny, nz = self.n
        k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        return (i.reshape(-1) * self.h[0], j.reshape(-1) * self.h[1], k.reshape(-1) * self.h[2])


def domain_side(n_box: int, a_tilde: float) -> int:
    """Domain nodes per axis in a box of n_box nodes (gap of floor(a_tilde) nodes)."""
    return int(n_box) - int(math.floor(a_tilde))


def _face_flags(n_box, n_omega):
    """Per-axis masks: inside the domain, and on a face of the domain."""
    idx = np.arange(n_box)
    inside = idx < n_omega
    face = (idx == 0) | (idx == n_omega - 1)
    return inside, face


def cube_surface_weights(p):
    """Boundary quadrature weights A of a cube_problem domain (the boundary
    integrals of Sec. 2.4 and Appendix A with direct nodal quadrature): a node on a
    face normal to axis k gets the 2D trapezoidal share of that face, h^2 halved
    once per in-face axis on which it lies on the face's edge; a node on several
    faces (an edge or a corner of the cube) sums its shares.  Zero off the faces."""
    nb = p.n[0]
    h = p.h[0]
    chi3 = p.chi.reshape(p.n[2], p.n[1], p.n[0])
    n_om = int(chi3[0, 0, :].sum())
    inside, face = _face_flags(nb, n_om)
    ins3 = inside[None, None, :] & inside[None, :, None] & inside[:, None, None]
    fk = [face[None, None, :], face[None, :, None], face[:, None, None]]  # x, y, z
    A = np.zeros((nb, nb, nb))
    for k in range(3):
        o1, o2 = [fk[m] for m in range(3) if m != k]
        w = h * h * 0.5 ** (o1.astype(np.int32) + o2.astype(np.int32))
        A = A + np.where(ins3 & fk[k], w, 0.0)
    return A.reshape(-1)


def cube_problem(n_box, a_tilde, degree=1, kind="sin", lo=0.0, hi=1.0):
    """Cube domain [lo, hi]^3 meshed by n_omega = n_box - floor(a_tilde) nodes per
    axis (h = (hi - lo)/(n_omega - 1)), embedded in an n_box^3 periodic box.

    kind "sin": u = sin(pi x) sin(pi y) sin(pi z) on [0,1]^3, r = 3 pi^2 u, g = 0.
    kind "paper": Eq. 106-107, u = (1-x^2)(1-y^2)(1-z^2) on [-1,1]^3,
        r = 2[3 - 2(x^2+y^2+z^2) + x^2y^2 + x^2z^2 + y^2z^2], g = 0.
    kind "zero": r = 0, g = 0 (geometry only).
    V is the trapezoidal cell share: h^3 halved once per axis on which the node
    lies on a face (faces h^3/2, edges h^3/4, corners h^3/8).
    Gamma_g = all nodes on the faces of the cube.
    """
    nb = int(n_box)
    n_om = domain_side(nb, a_tilde)
    if n_om < 2:
        raise ValueError("box too small for this support")
    h = (hi - lo) / (n_om - 1)
    inside, face = _face_flags(nb, n_om)
    ins3 = inside[None, None, :] & inside[None, :, None] & inside[:, None, None]
    facecount = (face[None, None, :].astype(np.int32) + face[None, :, None] + face[:, None, None])
    onface = ins3 & (facecount > 0)
    chi = ins3.astype(np.uint8).reshape(-1)
    chi_gamma = onface.astype(np.uint8).reshape(-1)
    V = np.where(ins3, h ** 3 * 0.5 ** facecount, 0.0).reshape(-1)
    x1 = lo + np.arange(nb) * h
    X = x1[None, None, :]
    Y = x1[None, :, None]
    Z = x1[:, None, None]
    if kind == "sin":
        u = np.sin(np.pi * X) * np.sin(np.pi * Y) * np.sin(np.pi * Z)
        r = 3.0 * np.pi ** 2 * u
    elif kind == "paper":
        u = (1 - X ** 2) * (1 - Y ** 2) * (1 - Z ** 2)
        r = 2.0 * (3.0 - 2.0 * (X ** 2 + Y ** 2 + Z ** 2) + X ** 2 * Y ** 2 + X ** 2 * Z ** 2 + Y ** 2 * Z ** 2)
    elif kind == "zero":
        u = np.zeros((nb, nb, nb))
        r = np.zeros((nb, nb, nb))
    else:
        raise ValueError(kind)
    u = np.where(ins3, u, 0.0).reshape(-1)
    r = np.where(ins3, r, 0.0).reshape(-1)
    g = np.zeros(nb ** 3)
    return Problem(n=(nb, nb, nb), h=(h, h, h), a_tilde=float(a_tilde), degree=int(degree), chi=chi,
                   chi_gamma=chi_gamma, V=V, r=r, g=g, u_exact=u, name=f"cube{nb}-{kind}",
                   meta={"n_omega_side": n_om, "lo": lo, "hi": hi})


def line_problem(n_box, a_tilde=1.5, degree=1):
    """The 1D problem of Sec. 6.1.1 (Eq. 97-98): -u'' = 2 on [-1, 1], u(-1) = u(1) = 0,
    exact u = 1 - x^2.  A line of n_box nodes (grid (n_box, 1, 1)), of which
    n_box - floor(a_tilde) span [-1, 1] (the box rule of Eq. 64-67); V = h, halved
    at the two end nodes (trapezoidal share); Gamma_g = the two end nodes."""
    nb = int(n_box)
    n_om = domain_side(nb, a_tilde)
    if n_om < 2:
        raise ValueError("box too small for this support")
    h = 2.0 / (n_om - 1)
    x = -1.0 + np.arange(nb) * h
    inside, face = _face_flags(nb, n_om)
    chi = inside.astype(np.uint8)
    chi_gamma = (inside & face).astype(np.uint8)
    V = np.where(inside, h * np.where(face, 0.5, 1.0), 0.0)
    u = np.where(inside, 1.0 - x ** 2, 0.0)
    r = np.where(inside, 2.0, 0.0)
    return Problem(n=(nb, 1, 1), h=(h, h, h), a_tilde=float(a_tilde), degree=int(degree), chi=chi,
                   chi_gamma=chi_gamma, V=V, r=r, g=np.zeros(nb), u_exact=u, name=f"line{nb}",
                   meta={"n_omega_side": n_om, "lo": -1.0, "hi": 1.0})


def plane_problem(n_box, a_tilde=1.5, degree=1):
    """The 2D problem of Sec. 6.1.2 (Eq. 101-102): -Lap u = 4 - 2x^2 - 2y^2 on
    [-1, 1]^2, u = 0 on the boundary, exact u = (1 - x^2)(1 - y^2).  A square of
    n_box^2 nodes (grid (n_box, n_box, 1)) with n_box - floor(a_tilde) domain nodes
    per axis; V = h^2 halved once per axis on which a node lies on the boundary;
    Gamma_g = the boundary nodes."""
    nb = int(n_box)
    n_om = domain_side(nb, a_tilde)
    if n_om < 2:
        raise ValueError("box too small for this support")
    h = 2.0 / (n_om - 1)
    inside, face = _face_flags(nb, n_om)
    ins2 = inside[None, :] & inside[:, None]
    fc = face[None, :].astype(np.int32) + face[:, None]
    x1 = -1.0 + np.arange(nb) * h
    X, Y = x1[None, :], x1[:, None]
    u = np.where(ins2, (1 - X ** 2) * (1 - Y ** 2), 0.0).reshape(-1)
    r = np.where(ins2, 4.0 - 2.0 * X ** 2 - 2.0 * Y ** 2, 0.0).reshape(-1)
    V = np.where(ins2, h ** 2 * 0.5 ** fc, 0.0).reshape(-1)
    return Problem(n=(nb, nb, 1), h=(h, h, h), a_tilde=float(a_tilde), degree=int(degree),
                   chi=ins2.astype(np.uint8).reshape(-1), chi_gamma=(ins2 & (fc > 0)).astype(np.uint8).reshape(-1),
                   V=V, r=r, g=np.zeros(nb * nb), u_exact=u, name=f"plane{nb}",
                   meta={"n_omega_side": n_om, "lo": -1.0, "hi": 1.0})


def boundary_of(chi3: np.ndarray) -> np.ndarray:
    """Nodes of chi with at least one of their 6 face-neighbours outside chi
    (periodic indexing of the box)."""
    c = chi3.astype(bool)
    out = np.zeros_like(c)
    for ax in range(3):
        for sh in (1, -1):
            out |= c & ~np.roll(c, sh, axis=ax)
    return out


def spheres_problem(n_box=256, n_spheres=12, a_tilde=3.0, degree=2, seed=BASE_SEED + 3000,
                    r_range=(0.1, 0.3), n_gauss=8):
    """Embedded domain: union of seeded spheres in the box [0,1)^3, h = 1/n_box.

    Radius ~ U[r_range]; centre ~ U[rad + h, 1 - rad - (floor(a_tilde) + 2) h]^3, so
    every sphere keeps a gap >= l_e = (floor(a_tilde)+1) h to the periodic image.
    r(x) = sum_k A_k exp(-|x - c_k|^2 / (2 s_k^2)), A ~ U[-1,1], c ~ U[0,1]^3,
    s ~ U[0.05, 0.15].  g = 0 on Gamma_g (chi nodes with a face-neighbour outside
    chi).  V = h^3 on every chi node.
    """
    rng = np.random.default_rng(seed)
    nb = int(n_box)
    h = 1.0 / nb
    x1 = np.arange(nb) * h
    X = x1[None, None, :]
    Y = x1[None, :, None]
    Z = x1[:, None, None]
    chi3 = np.zeros((nb, nb, nb), dtype=bool)
    m = math.floor(a_tilde)
    spheres = []
    for _ in range(n_spheres):
        rad = rng.uniform(*r_range)
        lo_c = rad + h
        hi_c = 1.0 - rad - (m + 2) * h
        c = rng.uniform(lo_c, hi_c, size=3)
        spheres.append((float(rad), c.tolist()))
        chi3 |= (X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2 <= rad * rad
    gam3 = boundary_of(chi3)
    r3 = np.zeros((nb, nb, nb))
    for _ in range(n_gauss):
        A = rng.uniform(-1.0, 1.0)
        c = rng.uniform(0.0, 1.0, size=3)
        sg = rng.uniform(0.05, 0.15)
        r3 += A * np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) / (2 * sg * sg))
    chi = chi3.astype(np.uint8).reshape(-1)
    return Problem(n=(nb, nb, nb), h=(h, h, h), a_tilde=float(a_tilde), degree=int(degree), chi=chi,
                   chi_gamma=gam3.astype(np.uint8).reshape(-1), V=np.where(chi3, h ** 3, 0.0).reshape(-1),
                   r=np.where(chi3, r3, 0.0).reshape(-1), g=np.zeros(nb ** 3), u_exact=None,
                   name=f"spheres{nb}", meta={"spheres": spheres, "seed": seed})


def gaussian_random_field(n, sigma, h, seed):
    """Smooth random field on a periodic grid: seeded white noise filtered by a
    Gaussian of standard deviation sigma (physical units), unit RMS.  (Input
    generation; the FFT here is a library filter, not part of the method.)"""
    rng = np.random.default_rng(seed)
    nx, ny, nz = n
    w = rng.standard_normal((nz, ny, nx))
    kx = np.fft.fftfreq(nx, d=h[0]) * 2 * np.pi
    ky = np.fft.fftfreq(ny, d=h[1]) * 2 * np.pi
    kz = np.fft.fftfreq(nz, d=h[2]) * 2 * np.pi
    K2 = kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2
    f = np.real(np.fft.ifftn(np.fft.fftn(w) * np.exp(-0.5 * sigma * sigma * K2)))
    f /= np.sqrt(np.mean(f * f))
    return f.reshape(-1)


def adjoint_problem(n_box=96, a_tilde=2.5, degree=1, seed=BASE_SEED + 4000, sigma=0.1):
    """Unit-cube problem for J = 1/2 |u - u_target|^2: r is a Gaussian random field
    (sigma = 0.1), u_target = sin(pi x) sin(pi y) sin(pi z), g = a low-frequency sum
    of three cosines restricted to Gamma_g."""
    p = cube_problem(n_box, a_tilde, degree, kind="sin")
    rng = np.random.default_rng(seed)
    r = gaussian_random_field(p.n, sigma, p.h, seed)
    X, Y, Z = p.coords()
    g = np.zeros(p.nbox)
    for _ in range(3):
        kv = rng.integers(1, 3, size=3)
        ph = rng.uniform(0, 2 * np.pi)
        A = rng.uniform(0.2, 1.0)
        g += A * np.cos(np.pi * (kv[0] * X + kv[1] * Y + kv[2] * Z) + ph)
    p.r = np.where(p.chi > 0, r, 0.0)
    p.g = np.where(p.chi_gamma > 0, g, 0.0)
    p.meta["u_target"] = p.u_exact.copy()
    p.name = f"adjoint{n_box}"
    return p


def random_field(nbox, seed, dtype=np.float64):
    """Seeded uniform(-1, 1) values, one per box node."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=int(nbox)).astype(dtype)


def fourier_mode(n, kvec):
    """cos(2 pi (kx i/nx + ky j/ny + kz k/nz)) on the box grid (flat)."""
    nx, ny, nz = n
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ph = 2 * np.pi * (kvec[0] * i / nx + kvec[1] * j / ny + kvec[2] * k / nz)
    return np.cos(ph).reshape(-1)


def embed(p: Problem, n_box) -> Problem:
    """The same problem in a larger periodic box (extra nodes outside the domain:
    chi = 0, V = 0, r = 0, g = 0; spacing unchanged)."""
    nb = tuple(int(v) for v in n_box)
    if any(a < b for a, b in zip(nb, p.n)):
        raise ValueError("box must not shrink")

    def pad(a):
        out = np.zeros((nb[2], nb[1], nb[0]), dtype=a.dtype)
        out[:p.n[2], :p.n[1], :p.n[0]] = a.reshape(p.n[2], p.n[1], p.n[0])
        return out.reshape(-1)

    q = Problem(n=nb, h=p.h, a_tilde=p.a_tilde, degree=p.degree, chi=pad(p.chi), chi_gamma=pad(p.chi_gamma),
                V=pad(p.V), r=pad(p.r), g=pad(p.g), u_exact=None if p.u_exact is None else pad(p.u_exact),
                name=p.name + f"@{nb[0]}", meta=dict(p.meta))
    q.meta["embedded_from"] = p.n
    return q


def gaussian_sources(n_box, h, n_gauss, rng):
    """sum_k A_k exp(-|x - c_k|^2 / (2 s_k^2)) on the box grid, A ~ U[-1,1],
    c ~ U[0,1]^3, s ~ U[0.05, 0.15]."""
    nb = int(n_box)
    x1 = np.arange(nb) * h
    X = x1[None, None, :]
    Y = x1[None, :, None]
    Z = x1[:, None, None]
    r3 = np.zeros((nb, nb, nb))
    for _ in range(n_gauss):
        A = rng.uniform(-1.0, 1.0)
        c = rng.uniform(0.0, 1.0, size=3)
        sg = rng.uniform(0.05, 0.15)
        r3 += A * np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) / (2 * sg * sg))
    return r3.reshape(-1)


def batched_domains(n_domains=64, side_range=(32, 160), n_rhs=4, seed=BASE_SEED + 5000):
    """Seeded domains of uneven size: box side S ~ U{side_range}, a union of 1..12
    spheres (radius U[0.1, 0.3] of the unit box, h = 1/S), basis linear (a = 2.5h)
    or quadratic (a = 3.0h) with probability 1/2, and n_rhs sources of 8 Gaussians
    each.  Returns a list of (Problem, [r_1, ..., r_nrhs])."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_domains):
        S = int(rng.integers(side_range[0], side_range[1] + 1))
        deg = 1 if rng.random() < 0.5 else 2
        a = 2.5 if deg == 1 else 3.0
        ns = int(rng.integers(1, 13))
        p = spheres_problem(n_box=S, n_spheres=ns, a_tilde=a, degree=deg, seed=seed + 1 + i, n_gauss=8)
        p.name = f"batch{i}-S{S}-n{deg}"
        rhs = [np.where(p.chi > 0, gaussian_sources(S, p.h[0], 8, rng), 0.0) for _ in range(n_rhs)]
        out.append((p, rhs))
    return out
