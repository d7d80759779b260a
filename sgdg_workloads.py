"""Seeded synthetic workloads shared by the oracle, the tests and the benchmark.

This module holds only *inputs*: coarse simplicial meshes, the coefficient
functions of the transport problem (beta, sigma, u0) and seeded random
coefficient vectors.  It contains none of the method's arithmetic (no
refinement, no assembly, no operator, no solver); the oracle and the CUDA
library each implement those on their own.

Problem statement (Sect. 1, Eqs. 1-2): d_t u + beta . grad u + sigma u = f on
(0,T) x Omega_x x Omega_v with inflow data g and initial data u0.  Coefficients
are given in the tensor-product form of Sect. 4.2: every one of the 2d
components of beta is a single product coef * fx(x) * fv(v); sigma likewise.
A ``None`` factor means the constant 1.

All callables take an array of points of shape (npts, d) and return (npts,).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Optional, Tuple

import numpy as np

Fn = Optional[Callable[[np.ndarray], np.ndarray]]


@dataclass
class CoarseMesh:
    """A coarse simplicial mesh on a box domain.

    coords: (nv, d) float64; cells: (nc, d+1) int32, vertex indices.
    lo/hi: box bounds per axis.  periodic: per-axis periodicity flag.
    """
    coords: np.ndarray
    cells: np.ndarray
    lo: Tuple[float, ...]
    hi: Tuple[float, ...]
    periodic: Tuple[bool, ...]

    @property
    def dim(self) -> int:
        return self.coords.shape[1]


@dataclass
class Product:
    """coef * ft(t) * fx(x) * fv(v); ``None`` factors are the constant 1.
    ft (time-dependent beta and sigma, Sect. 4.2) maps an array of times to
    values; u0 products leave it None."""
    coef: float
    fx: Fn = None
    fv: Fn = None
    ft: Optional[Callable[[np.ndarray], np.ndarray]] = None


@dataclass
class Source:
    """coef * ft(t) * fx(x) * fv(v), one term of the source f; ``None``
    factors are the constant 1 (ft maps an array of times to values)."""
    coef: float
    fx: Fn = None
    fv: Fn = None
    ft: Optional[Callable[[np.ndarray], np.ndarray]] = None


@dataclass
class Problem:
    """One transport problem on a product phase space (Sect. 1-2)."""
    name: str
    d: int
    mesh_x: CoarseMesh
    mesh_v: CoarseMesh
    L: int                      # sparse level, 0-based: grids (l, L-l), l = 0..L
    r: int                      # time-DG degree (1)
    dt: float
    delta: float                # streamline-diffusion parameter
    n_strips: int
    beta: List[Product]         # 2d components: x-components then v-components
    sigma: Product
    u0: List[Product]           # sum of separable products
    exact: Optional[Callable[[float, np.ndarray, np.ndarray], np.ndarray]] = None
    f: List[Source] = field(default_factory=list)   # source, sum of separable terms
    g: List[Source] = field(default_factory=list)   # inflow data on Gamma^-, sum of separable terms
    order: int = 1              # polynomial order of the continuous spatial elements (P1, P2)
    element: str = "P"          # "P": simplices (P_order); "Q": tensor-product Q_order on the squares


# ----------------------------------------------------------------------------
# coarse meshes (input data: the vertex/cell lists a user would hand over)
# ----------------------------------------------------------------------------

def interval_mesh(a: float, b: float, n_cells: int = 4, periodic: bool = False) -> CoarseMesh:
    x = np.linspace(a, b, n_cells + 1)
    cells = np.array([[i, i + 1] for i in range(n_cells)], dtype=np.int32)
    return CoarseMesh(x[:, None].copy(), cells, (a,), (b,), (periodic,))


def square_mesh(a: float, b: float, n_sq: int = 2, periodic: bool = False) -> CoarseMesh:
    """n_sq x n_sq squares, each cut along the same diagonal (lower-left to
    upper-right); 2 n_sq^2 triangles.  n_sq = 2 gives the 8-triangle mesh."""
    t = np.linspace(a, b, n_sq + 1)
    X, Y = np.meshgrid(t, t, indexing="xy")
    coords = np.stack([X.ravel(), Y.ravel()], axis=1)
    vid = lambda i, j: j * (n_sq + 1) + i
    cells = []
    for j in range(n_sq):
        for i in range(n_sq):
            p00, p10, p01, p11 = vid(i, j), vid(i + 1, j), vid(i, j + 1), vid(i + 1, j + 1)
            cells.append([p00, p10, p11])
            cells.append([p00, p11, p01])
    return CoarseMesh(coords, np.array(cells, dtype=np.int32), (a, a), (b, b), (periodic, periodic))


def cube_mesh(a: float, b: float, n_cb: int = 1, periodic: bool = False) -> CoarseMesh:
    """n_cb^3 cubes, each cut into the 6 Kuhn (Freudenthal) tetrahedra that
    share its main diagonal; every tetrahedron lists its vertices along a
    monotone lattice path (corner, + e_i, + e_i + e_j, opposite corner).
    n_cb = 1 gives the 6-tetrahedron coarse mesh."""
    t = np.linspace(a, b, n_cb + 1)
    Z, Y, X = np.meshgrid(t, t, t, indexing="ij")
    coords = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    vid = lambda i, j, k: (k * (n_cb + 1) + j) * (n_cb + 1) + i
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    cells = []
    for k in range(n_cb):
        for j in range(n_cb):
            for i in range(n_cb):
                for pm in perms:
                    p = [i, j, k]
                    path = [vid(*p)]
                    for ax in pm:
                        p[ax] += 1
                        path.append(vid(*p))
                    cells.append(path)
    return CoarseMesh(coords, np.array(cells, dtype=np.int32), (a, a, a), (b, b, b), (periodic,) * 3)


# ----------------------------------------------------------------------------
# problems
# ----------------------------------------------------------------------------

def _gauss(c: float, var2: float):
    # exp(-(s - c)^2 / var2) along axis 0
    return lambda p: np.exp(-((p[:, 0] - c) ** 2) / var2)


def free_streaming_1d(L: int = 6, n_strips: int = 16, dt: float = 1.0 / 32.0) -> Problem:
    """d=1 free streaming: x in [0,1], v in [-1,1], beta = (v, 0), sigma = 0,
    f = 0, g = 0, u0 = exp(-(x-0.5)^2/0.01) exp(-v^2/0.1).  delta = finest
    edge length of the two meshes (the smaller one).  Exact solution
    u0(x - v t, v) where x - v t stays in [0,1] (inflow g = 0), else 0."""
    mx = interval_mesh(0.0, 1.0, 4)
    mv = interval_mesh(-1.0, 1.0, 4)
    hx = 1.0 / (4 * 2 ** L)
    hv = 2.0 / (4 * 2 ** L)
    ux = _gauss(0.5, 0.01)
    uv = lambda p: np.exp(-(p[:, 0] ** 2) / 0.1)

    def exact(t, x, v):
        xs = x - v * t
        inside = (xs >= 0.0) & (xs <= 1.0)
        return np.where(inside, np.exp(-((xs - 0.5) ** 2) / 0.01) * np.exp(-(v ** 2) / 0.1), 0.0)

    return Problem(
        name=f"free_streaming_1d_L{L}", d=1, mesh_x=mx, mesh_v=mv, L=L, r=1, dt=dt,
        delta=min(hx, hv), n_strips=n_strips,
        beta=[Product(1.0, None, lambda p: p[:, 0]), Product(0.0)],
        sigma=Product(0.0), u0=[Product(1.0, ux, uv)], exact=exact)


def transport_2d(L: int = 9, sigma: float = 0.1, dt: float = 1.0 / 64.0, n_strips: int = 16) -> Problem:
    """d=2: Omega_x = [0,1]^2, Omega_v = [-1,1]^2, 8-triangle coarse meshes,
    beta = (v1, v2, E1(x), E2(x)) with E = 0.5 (sin 2 pi x2, cos 2 pi x1),
    constant sigma, Gaussian u0, f = 0, g = 0.  delta = finest edge leg."""
    mx = square_mesh(0.0, 1.0, 2)
    mv = square_mesh(-1.0, 1.0, 2)
    hx = 1.0 / 2 ** (L + 1)
    hv = 2.0 / 2 ** (L + 1)
    beta = [
        Product(1.0, None, lambda p: p[:, 0]),
        Product(1.0, None, lambda p: p[:, 1]),
        Product(0.5, lambda p: np.sin(2 * np.pi * p[:, 1]), None),
        Product(0.5, lambda p: np.cos(2 * np.pi * p[:, 0]), None),
    ]
    ux = lambda p: np.exp(-((p[:, 0] - 0.5) ** 2 + (p[:, 1] - 0.5) ** 2) / 0.01)
    uv = lambda p: np.exp(-(p[:, 0] ** 2 + p[:, 1] ** 2) / 0.1)
    return Problem(
        name=f"transport_2d_L{L}", d=2, mesh_x=mx, mesh_v=mv, L=L, r=1, dt=dt,
        delta=min(hx, hv), n_strips=n_strips, beta=beta,
        sigma=Product(sigma) if sigma != 0.0 else Product(0.0),
        u0=[Product(1.0, ux, uv)])


def periodic_advection_1d(L: int, r: int = 1) -> Problem:
    """Sect. 5.1 (Eq. 25) with d = 1: beta = (1, 1) on the periodic unit
    square, u0 = sin(2 pi (x + v)); coarse meshes of 4 cells; 2^(L_paper+1)
    strips over one period T = 1/2; delta = finest edge length.  Here L is
    0-based (L_paper = L + 1).  r is the order of both the spatial elements
    (P_r) and the time-DG polynomials, as in Table 1."""
    mx = interval_mesh(0.0, 1.0, 4, periodic=True)
    mv = interval_mesh(0.0, 1.0, 4, periodic=True)
    Lp = L + 1
    n_strips = 2 ** (Lp + 1)
    T = 0.5
    h = 1.0 / (4 * 2 ** L)
    # sin(2 pi (x + v)) = sin(2 pi x) cos(2 pi v) + cos(2 pi x) sin(2 pi v)
    u0 = [Product(1.0, lambda p: np.sin(2 * np.pi * p[:, 0]), lambda p: np.cos(2 * np.pi * p[:, 0])),
          Product(1.0, lambda p: np.cos(2 * np.pi * p[:, 0]), lambda p: np.sin(2 * np.pi * p[:, 0]))]

    def exact(t, x, v):
        return np.sin(2 * np.pi * (x + v - 2 * t))

    return Problem(name=f"periodic_advection_1d_L{L}" + ("" if r == 1 else f"_r{r}"), d=1, mesh_x=mx, mesh_v=mv,
                   L=L, r=r, dt=T / n_strips, delta=h, n_strips=n_strips,
                   beta=[Product(1.0), Product(1.0)], sigma=Product(0.0), u0=u0, exact=exact, order=r)


def periodic_advection_2d(L: int, r: int = 1, element: str = "P") -> Problem:
    """Sect. 5.1 (Eq. 25) with d = 2: beta = (1, 1, 1, 1) on the periodic unit
    cubes, u0 = sin(2 pi (x1 + x2 + v1 + v2)); coarse meshes of 4 x 4 squares
    (two triangles each); 2^(L_paper+1) strips over one period T = 1/4;
    delta = finest edge length along the axes.  L is 0-based; r is the order
    of the spatial elements and of the time-DG polynomials, as in Table 1;
    element "P" uses the triangles, "Q" tensor-product elements on the
    squares."""
    mx = square_mesh(0.0, 1.0, 4, periodic=True)
    mv = square_mesh(0.0, 1.0, 4, periodic=True)
    Lp = L + 1
    n_strips = 2 ** (Lp + 1)
    T = 0.25
    h = 1.0 / (4 * 2 ** L)
    s2 = lambda p: np.sin(2 * np.pi * (p[:, 0] + p[:, 1]))
    c2 = lambda p: np.cos(2 * np.pi * (p[:, 0] + p[:, 1]))
    u0 = [Product(1.0, s2, c2), Product(1.0, c2, s2)]

    def exact(t, x, v):
        return np.sin(2 * np.pi * (x[..., 0] + x[..., 1] + v[..., 0] + v[..., 1] - 4 * t))

    return Problem(name=f"periodic_advection_2d_L{L}" + ("" if r == 1 else f"_r{r}"), d=2, mesh_x=mx, mesh_v=mv,
                   L=L, r=r, dt=T / n_strips, delta=h, n_strips=n_strips, beta=[Product(1.0)] * 4,
                   sigma=Product(0.0), u0=u0, exact=exact, order=r, element=element)


def transport_3d(L: int = 7, dt: float = 1.0 / 32.0, n_strips: int = 8) -> Problem:
    """d=3 (6-D phase space): Omega_x = [0,1]^3, Omega_v = [-1,1]^3, 6-tetrahedron
    Kuhn coarse meshes refined uniformly ((2^l + 1)^3 vertices on level l),
    beta = (v, E(x)) with E = 0.5 (sin 2 pi x2, sin 2 pi x3, sin 2 pi x1),
    sigma = 0, u0 = exp(-|x - 1/2|^2 / 0.01) exp(-|v|^2 / 0.1), delta = the
    shortest finest edge (the x mesh's, 2^-L)."""
    mx = cube_mesh(0.0, 1.0, 1)
    mv = cube_mesh(-1.0, 1.0, 1)
    hx = 1.0 / 2 ** L
    beta = [Product(1.0, None, lambda p: p[:, 0]), Product(1.0, None, lambda p: p[:, 1]),
            Product(1.0, None, lambda p: p[:, 2]),
            Product(0.5, lambda p: np.sin(2 * np.pi * p[:, 1]), None),
            Product(0.5, lambda p: np.sin(2 * np.pi * p[:, 2]), None),
            Product(0.5, lambda p: np.sin(2 * np.pi * p[:, 0]), None)]
    ux = lambda p: np.exp(-((p[:, 0] - 0.5) ** 2 + (p[:, 1] - 0.5) ** 2 + (p[:, 2] - 0.5) ** 2) / 0.01)
    uv = lambda p: np.exp(-(p[:, 0] ** 2 + p[:, 1] ** 2 + p[:, 2] ** 2) / 0.1)
    return Problem(name=f"transport_3d_L{L}", d=3, mesh_x=mx, mesh_v=mv, L=L, r=1, dt=dt, delta=hx,
                   n_strips=n_strips, beta=beta, sigma=Product(0.0), u0=[Product(1.0, ux, uv)])


def time_dependent_1d(L: int = 3, dt: float = 1.0 / 8.0, n_strips: int = 4, omega: float = 3.0,
                      sigma0: float = 0.4) -> Problem:
    """d=1 transport with coefficients that vary in time (Sect. 4.2 allows
    beta(t, x, v) and sigma(t, x, v) in tensor form): x in [0,1], v in [-1,1],
    beta = (v (1 + t/2), cos(omega t) (x - 1/2)), sigma = sigma0 (1 + sin(omega t)/2).
    The v-component changes sign in time (at t = pi / (2 omega) = 0.52 for
    omega = 3) and in space on the mesh line x = 1/2, so the inflow part of
    the v-boundary switches sides within the run.  u0 = config-1 Gaussian."""
    mx = interval_mesh(0.0, 1.0, 4)
    mv = interval_mesh(-1.0, 1.0, 4)
    h = 1.0 / (4 * 2 ** L)
    ux = _gauss(0.5, 0.01)
    uv = lambda p: np.exp(-(p[:, 0] ** 2) / 0.1)
    return Problem(
        name=f"time_dependent_1d_L{L}", d=1, mesh_x=mx, mesh_v=mv, L=L, r=1, dt=dt, delta=h, n_strips=n_strips,
        beta=[Product(1.0, None, lambda p: p[:, 0], lambda t: 1.0 + 0.5 * np.asarray(t)),
              Product(1.0, lambda p: p[:, 0] - 0.5, None, lambda t: np.cos(omega * np.asarray(t)))],
        sigma=Product(sigma0, None, None, lambda t: 1.0 + 0.5 * np.sin(omega * np.asarray(t))),
        u0=[Product(1.0, ux, uv)])


def time_dependent_2d(L: int = 3, dt: float = 1.0 / 16.0, n_strips: int = 4, omega: float = 6.0) -> Problem:
    """The transport_2d problem with a field that rotates its sign in time:
    E(t, x) = cos(omega t) 0.5 (sin 2 pi x2, cos 2 pi x1) and
    sigma = 0.1 (1 + t); beta = (v, E(t, x))."""
    p = transport_2d(L=L, sigma=0.1, dt=dt, n_strips=n_strips)
    c = lambda t: np.cos(omega * np.asarray(t))
    p.beta[2] = Product(0.5, lambda q: np.sin(2 * np.pi * q[:, 1]), None, c)
    p.beta[3] = Product(0.5, lambda q: np.cos(2 * np.pi * q[:, 0]), None, c)
    p.sigma = Product(0.1, None, None, lambda t: 1.0 + np.asarray(t))
    p.name = f"time_dependent_2d_L{L}"
    return p


def landau_4d(L: int = 8, alpha: float = 0.01, k: float = 0.5, n_strips: int = 200, dt: float = None,
              phase: float = 0.0) -> Problem:
    """2+2-dimensional Landau damping (Sect. 5.3): periodic x in [0, 4 pi]^2,
    v in [-6, 6]^2 (8-triangle coarse meshes), f0 = (1 + alpha cos(k x1 +
    phase)) exp(-|v|^2/2) / (2 pi), Vlasov beta = (v, -E(x)) with E from the
    Poisson problem of the density; the initial E callback is zero (the first
    field update replaces it).  dt halves per level: 1/32 at L = 8 (100 steps
    on [0, 50] at the paper's level 5, doubled per level)."""
    four_pi = 4.0 * np.pi
    mx = square_mesh(0.0, four_pi, 2, periodic=True)
    mv = square_mesh(-6.0, 6.0, 2)
    if dt is None:
        dt = 0.5 / 2 ** (L - 4)
    hx = four_pi / 2 ** (L + 1)
    hv = 12.0 / 2 ** (L + 1)
    zero = lambda p: np.zeros(p.shape[0])
    fx = lambda p: 1.0 + alpha * np.cos(k * p[:, 0] + phase)
    fv = lambda p: np.exp(-(p[:, 0] ** 2 + p[:, 1] ** 2) / 2.0) / (2.0 * np.pi)
    return Problem(
        name=f"landau_4d_L{L}", d=2, mesh_x=mx, mesh_v=mv, L=L, r=1, dt=dt, delta=min(hx, hv),
        n_strips=n_strips,
        beta=[Product(1.0, None, lambda p: p[:, 0]), Product(1.0, None, lambda p: p[:, 1]),
              Product(-1.0, zero, None), Product(-1.0, zero, None)],
        sigma=Product(0.0), u0=[Product(1.0, fx, fv)])


def _poly(c):
    """t -> c[0] + c[1] t + c[2] t^2 and its derivative."""
    a = lambda t: c[0] + c[1] * np.asarray(t) + c[2] * np.asarray(t) ** 2
    da = lambda t: c[1] + 2.0 * c[2] * np.asarray(t)
    return a, da


def manufactured_1d(L: int = 4, sigma: float = 0.5, dt: float = 1.0 / 16.0, n_strips: int = 4,
                    seed: int = 0) -> Problem:
    """d=1 manufactured solution u*(t, x, v) = a(t) X(x) V(v) on [0,1] x [-1,1]
    with X = sin^2(pi x), V = cos^2(pi v / 2) (1 + b v), a a seeded quadratic;
    beta = (v, 0), constant sigma; f = d_t u* + v d_x u* + sigma u* as three
    separable terms.  u* vanishes on the boundary, so the inflow data g is 0."""
    rng = np.random.default_rng(seed)
    c = (1.0, float(rng.uniform(-0.5, 0.5)), float(rng.uniform(-0.5, 0.5)))
    b = float(rng.uniform(-0.3, 0.3))
    a, da = _poly(c)
    X = lambda p: np.sin(np.pi * p[:, 0]) ** 2
    dX = lambda p: np.pi * np.sin(2 * np.pi * p[:, 0])
    V = lambda p: np.cos(0.5 * np.pi * p[:, 0]) ** 2 * (1.0 + b * p[:, 0])
    vV = lambda p: p[:, 0] * V(p)

    def exact(t, x, v):
        return a(t) * np.sin(np.pi * x) ** 2 * np.cos(0.5 * np.pi * v) ** 2 * (1.0 + b * v)

    f = [Source(1.0, X, V, da), Source(sigma, X, V, a), Source(1.0, dX, vV, a)]
    h = 1.0 / (4 * 2 ** L)
    return Problem(name=f"manufactured_1d_L{L}", d=1, mesh_x=interval_mesh(0.0, 1.0, 4),
                   mesh_v=interval_mesh(-1.0, 1.0, 4), L=L, r=1, dt=dt, delta=h, n_strips=n_strips,
                   beta=[Product(1.0, None, lambda p: p[:, 0]), Product(0.0)],
                   sigma=Product(sigma) if sigma != 0.0 else Product(0.0),
                   u0=[Product(float(a(0.0)), X, V)], exact=exact, f=f)


def discrete_manufactured_1d(L: int = 3, sigma: float = 0.5, dt: float = 1.0 / 8.0, n_strips: int = 2,
                             c0: float = 1.0, c1: float = 0.75) -> Problem:
    """d=1 solution inside the discrete space: u*(t, x, v) = (c0 + c1 t)
    phi(x) psi(v) with phi, psi the level-0 hat functions at x = 1/2 and v = 0
    (supports inside the domain, so the inflow data g = 0), beta = (v, 0),
    constant sigma; f = d_t u* + v d_x u* + sigma u* as three separable terms
    (piecewise polynomial, kinks on coarse mesh lines).  A consistent scheme
    with exact quadrature reproduces u* up to the solver tolerance."""
    phi = lambda p: np.maximum(0.0, 1.0 - np.abs(p[:, 0] - 0.5) / 0.25)
    dphi = lambda p: np.where(np.abs(p[:, 0] - 0.5) < 0.25, -np.sign(p[:, 0] - 0.5) / 0.25, 0.0)
    psi = lambda p: np.maximum(0.0, 1.0 - np.abs(p[:, 0]) / 0.5)
    vpsi = lambda p: p[:, 0] * psi(p)
    a = lambda t: c0 + c1 * np.asarray(t)
    da = lambda t: c1 + 0.0 * np.asarray(t)

    def exact(t, x, v):
        return (c0 + c1 * t) * np.maximum(0.0, 1.0 - np.abs(x - 0.5) / 0.25) * np.maximum(0.0, 1.0 - np.abs(v) / 0.5)

    f = [Source(1.0, phi, psi, da), Source(sigma, phi, psi, a), Source(1.0, dphi, vpsi, a)]
    h = 1.0 / (4 * 2 ** L)
    return Problem(name=f"discrete_manufactured_1d_L{L}", d=1, mesh_x=interval_mesh(0.0, 1.0, 4),
                   mesh_v=interval_mesh(-1.0, 1.0, 4), L=L, r=1, dt=dt, delta=h, n_strips=n_strips,
                   beta=[Product(1.0, None, lambda p: p[:, 0]), Product(0.0)],
                   sigma=Product(sigma) if sigma != 0.0 else Product(0.0),
                   u0=[Product(c0, phi, psi)], exact=exact, f=f)


def inflow_manufactured_1d(L: int = 3, sigma: float = 0.3, dt: float = 1.0 / 8.0, n_strips: int = 2,
                           c0: float = 1.0, c1: float = 0.5) -> Problem:
    """d=1 solution inside the discrete space that does not vanish on the
    boundary: u*(t, x, v) = (c0 + c1 t)(1 + x)(1 + v/2) on x in [0,1],
    v in [-1,1] (P1 in x and v, linear in t), beta = (v, x - 1/2) (inflow on
    all four sides, sign changes on the mesh lines v = 0 and x = 1/2),
    constant sigma; f = d_t u* + beta . grad u* + sigma u* as four separable
    terms and the inflow data g = u* on Gamma^-.  Exact quadrature of the
    polynomial data lets a consistent scheme reproduce u* up to the solver
    tolerance."""
    X = lambda p: 1.0 + p[:, 0]
    V = lambda p: 1.0 + 0.5 * p[:, 0]
    vV = lambda p: p[:, 0] * V(p)
    eX = lambda p: (p[:, 0] - 0.5) * X(p)
    a = lambda t: c0 + c1 * np.asarray(t)
    da = lambda t: c1 + 0.0 * np.asarray(t)

    def exact(t, x, v):
        return (c0 + c1 * t) * (1.0 + x) * (1.0 + 0.5 * v)

    f = [Source(1.0, X, V, da), Source(sigma, X, V, a), Source(1.0, None, vV, a), Source(0.5, eX, None, a)]
    h = 1.0 / (4 * 2 ** L)
    return Problem(name=f"inflow_manufactured_1d_L{L}", d=1, mesh_x=interval_mesh(0.0, 1.0, 4),
                   mesh_v=interval_mesh(-1.0, 1.0, 4), L=L, r=1, dt=dt, delta=h, n_strips=n_strips,
                   beta=[Product(1.0, None, lambda p: p[:, 0]), Product(1.0, lambda p: p[:, 0] - 0.5, None)],
                   sigma=Product(sigma) if sigma != 0.0 else Product(0.0),
                   u0=[Product(c0, X, V)], exact=exact, f=f, g=[Source(1.0, X, V, a)])


def inflow_time_dependent_1d(L: int = 3, sigma: float = 0.3, dt: float = 1.0 / 8.0, n_strips: int = 4,
                             c0: float = 1.0, c1: float = 0.5) -> Problem:
    """The inflow_manufactured_1d solution u* = (c0 + c1 t)(1 + x)(1 + v/2)
    with a field that changes sign in time: beta = (v, (1 - 3t)(x - 1/2))
    (sign change at t = 1/3, inside the third strip of dt = 1/8), so the
    inflow part of the v-boundary moves between the two halves of the x
    range within a strip.  f = d_t u* + beta . grad u* + sigma u* as
    separable terms with polynomial time factors, g = u* on Gamma^-(t)."""
    X = lambda p: 1.0 + p[:, 0]
    V = lambda p: 1.0 + 0.5 * p[:, 0]
    vV = lambda p: p[:, 0] * V(p)
    eX = lambda p: (p[:, 0] - 0.5) * X(p)
    a = lambda t: c0 + c1 * np.asarray(t)
    da = lambda t: c1 + 0.0 * np.asarray(t)
    e = lambda t: 1.0 - 3.0 * np.asarray(t)

    def exact(t, x, v):
        return (c0 + c1 * t) * (1.0 + x) * (1.0 + 0.5 * v)

    f = [Source(1.0, X, V, da), Source(sigma, X, V, a), Source(1.0, None, vV, a),
         Source(0.5, eX, None, lambda t: e(t) * a(t))]
    h = 1.0 / (4 * 2 ** L)
    return Problem(name=f"inflow_time_dependent_1d_L{L}", d=1, mesh_x=interval_mesh(0.0, 1.0, 4),
                   mesh_v=interval_mesh(-1.0, 1.0, 4), L=L, r=1, dt=dt, delta=h, n_strips=n_strips,
                   beta=[Product(1.0, None, lambda p: p[:, 0]), Product(1.0, lambda p: p[:, 0] - 0.5, None, e)],
                   sigma=Product(sigma) if sigma != 0.0 else Product(0.0),
                   u0=[Product(c0, X, V)], exact=exact, f=f, g=[Source(1.0, X, V, a)])


def inflow_manufactured_2d(L: int = 2, sigma: float = 0.2, dt: float = 1.0 / 8.0, n_strips: int = 2,
                           c0: float = 1.0, c1: float = -0.4) -> Problem:
    """d=2 analogue on [0,1]^2 x [-1,1]^2: u* = (c0 + c1 t)(1 + x1 + 2 x2)
    (1 + v1/2 - 0.3 v2), beta = (v1, v2, x2 - 1/2, 1/2 - x1) (inflow on every
    side of both boxes), f as separable polynomial terms, g = u* on Gamma^-."""
    X = lambda p: 1.0 + p[:, 0] + 2.0 * p[:, 1]
    V = lambda p: 1.0 + 0.5 * p[:, 0] - 0.3 * p[:, 1]
    a = lambda t: c0 + c1 * np.asarray(t)
    da = lambda t: c1 + 0.0 * np.asarray(t)

    def exact(t, x, v):
        return (c0 + c1 * t) * (1.0 + x[..., 0] + 2.0 * x[..., 1]) * (1.0 + 0.5 * v[..., 0] - 0.3 * v[..., 1])

    f = [Source(1.0, X, V, da), Source(sigma, X, V, a),
         Source(1.0, None, lambda p: p[:, 0] * V(p), a),            # v1 d_x1 u*, d_x1 X = 1
         Source(2.0, None, lambda p: p[:, 1] * V(p), a),            # v2 d_x2 u*, d_x2 X = 2
         Source(0.5, lambda p: (p[:, 1] - 0.5) * X(p), None, a),     # E1 d_v1 u*, d_v1 V = 1/2
         Source(-0.3, lambda p: (0.5 - p[:, 0]) * X(p), None, a)]    # E2 d_v2 u*, d_v2 V = -0.3
    hx = 1.0 / 2 ** (L + 1)
    return Problem(name=f"inflow_manufactured_2d_L{L}", d=2, mesh_x=square_mesh(0.0, 1.0, 2),
                   mesh_v=square_mesh(-1.0, 1.0, 2), L=L, r=1, dt=dt, delta=hx, n_strips=n_strips,
                   beta=[Product(1.0, None, lambda p: p[:, 0]), Product(1.0, None, lambda p: p[:, 1]),
                         Product(1.0, lambda p: p[:, 1] - 0.5, None), Product(1.0, lambda p: 0.5 - p[:, 0], None)],
                   sigma=Product(sigma) if sigma != 0.0 else Product(0.0),
                   u0=[Product(c0, X, V)], exact=exact, f=f, g=[Source(1.0, X, V, a)])


def inflow_time_dependent_2d(L: int = 1, sigma: float = 0.2, dt: float = 1.0 / 8.0, n_strips: int = 3,
                             c0: float = 1.0, c1: float = -0.4) -> Problem:
    """inflow_manufactured_2d with time factors on the v-components of beta:
    E1 = (1 - 3t)(x2 - 1/2) changes sign at t = 1/3 (inside the third strip
    of dt = 1/8) and E2 = (1 + t)(1/2 - x1); the sources carry the same time
    factors, g = u* on Gamma^-(t)."""
    X = lambda p: 1.0 + p[:, 0] + 2.0 * p[:, 1]
    V = lambda p: 1.0 + 0.5 * p[:, 0] - 0.3 * p[:, 1]
    a = lambda t: c0 + c1 * np.asarray(t)
    da = lambda t: c1 + 0.0 * np.asarray(t)
    e1 = lambda t: 1.0 - 3.0 * np.asarray(t)
    e2 = lambda t: 1.0 + np.asarray(t)

    def exact(t, x, v):
        return (c0 + c1 * t) * (1.0 + x[..., 0] + 2.0 * x[..., 1]) * (1.0 + 0.5 * v[..., 0] - 0.3 * v[..., 1])

    f = [Source(1.0, X, V, da), Source(sigma, X, V, a),
         Source(1.0, None, lambda p: p[:, 0] * V(p), a),
         Source(2.0, None, lambda p: p[:, 1] * V(p), a),
         Source(0.5, lambda p: (p[:, 1] - 0.5) * X(p), None, lambda t: e1(t) * a(t)),
         Source(-0.3, lambda p: (0.5 - p[:, 0]) * X(p), None, lambda t: e2(t) * a(t))]
    hx = 1.0 / 2 ** (L + 1)
    return Problem(name=f"inflow_time_dependent_2d_L{L}", d=2, mesh_x=square_mesh(0.0, 1.0, 2),
                   mesh_v=square_mesh(-1.0, 1.0, 2), L=L, r=1, dt=dt, delta=hx, n_strips=n_strips,
                   beta=[Product(1.0, None, lambda p: p[:, 0]), Product(1.0, None, lambda p: p[:, 1]),
                         Product(1.0, lambda p: p[:, 1] - 0.5, None, e1),
                         Product(1.0, lambda p: 0.5 - p[:, 0], None, e2)],
                   sigma=Product(sigma) if sigma != 0.0 else Product(0.0),
                   u0=[Product(c0, X, V)], exact=exact, f=f, g=[Source(1.0, X, V, a)])


def manufactured_2d(L: int = 9, sigma: float = 0.1, dt: float = 1.0 / 64.0, n_strips: int = 16,
                    seed: int = 0) -> Problem:
    """d=2 manufactured solution on the transport_2d problem (beta = (v1, v2,
    E1(x), E2(x)), E = 0.5 (sin 2 pi x2, cos 2 pi x1), constant sigma):
    u* = a(t) X(x) V(v), X = sin^2(pi x1) sin^2(pi x2),
    V = cos^2(pi v1 / 2) cos^2(pi v2 / 2) (1 + b1 v1 + b2 v2), a a seeded
    quadratic; f = d_t u* + beta . grad u* + sigma u* as six separable terms.
    u* vanishes on the boundary, so the inflow data g is 0."""
    base = transport_2d(L=L, sigma=sigma, dt=dt, n_strips=n_strips)
    rng = np.random.default_rng(seed)
    c = (1.0, float(rng.uniform(-0.5, 0.5)), float(rng.uniform(-0.5, 0.5)))
    b1, b2 = (float(x) for x in rng.uniform(-0.3, 0.3, size=2))
    a, da = _poly(c)
    pi = np.pi
    X = lambda p: np.sin(pi * p[:, 0]) ** 2 * np.sin(pi * p[:, 1]) ** 2
    d1X = lambda p: pi * np.sin(2 * pi * p[:, 0]) * np.sin(pi * p[:, 1]) ** 2
    d2X = lambda p: pi * np.sin(pi * p[:, 0]) ** 2 * np.sin(2 * pi * p[:, 1])
    C = lambda p: np.cos(0.5 * pi * p[:, 0]) ** 2 * np.cos(0.5 * pi * p[:, 1]) ** 2
    lin = lambda p: 1.0 + b1 * p[:, 0] + b2 * p[:, 1]
    V = lambda p: C(p) * lin(p)
    v1V = lambda p: p[:, 0] * V(p)
    v2V = lambda p: p[:, 1] * V(p)
    d1V = lambda p: (-0.5 * pi * np.sin(pi * p[:, 0]) * np.cos(0.5 * pi * p[:, 1]) ** 2 * lin(p) + C(p) * b1)
    d2V = lambda p: (-0.5 * pi * np.cos(0.5 * pi * p[:, 0]) ** 2 * np.sin(pi * p[:, 1]) * lin(p) + C(p) * b2)
    E1X = lambda p: np.sin(2 * pi * p[:, 1]) * X(p)
    E2X = lambda p: np.cos(2 * pi * p[:, 0]) * X(p)

    def exact(t, x, v):
        return a(t) * X(x) * V(v)

    base.name = f"manufactured_2d_L{L}"
    base.u0 = [Product(float(a(0.0)), X, V)]
    base.exact = exact
    base.f = [Source(1.0, X, V, da), Source(sigma, X, V, a), Source(1.0, d1X, v1V, a), Source(1.0, d2X, v2V, a),
              Source(0.5, E1X, d1V, a), Source(0.5, E2X, d2V, a)]
    return base


def batched_4d(n: int = 48, seed: int = 0, levels=(6, 7, 8, 9), dt: float = 1.0 / 32.0,
               n_strips: int = 16) -> List[Problem]:
    """Many independent 4D instances with the d=1 free-streaming physics on the
    d=2 geometry: beta = (v1, v2, 0, 0), sigma = f = g = 0, 8-triangle coarse
    meshes, L drawn uniformly from ``levels``, u0 = exp(-|x-c|^2/(2 s))
    exp(-|v|^2/0.1) with c ~ U[0.3, 0.7]^2 and s ~ U[0.005, 0.02] (seeded)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        L = int(rng.choice(levels))
        c = rng.uniform(0.3, 0.7, size=2)
        s = float(rng.uniform(0.005, 0.02))
        ux = (lambda c0, c1, s2: (lambda p: np.exp(-((p[:, 0] - c0) ** 2 + (p[:, 1] - c1) ** 2) / s2)))(
            float(c[0]), float(c[1]), 2.0 * s)
        uv = lambda p: np.exp(-(p[:, 0] ** 2 + p[:, 1] ** 2) / 0.1)
        hx = 1.0 / 2 ** (L + 1)
        out.append(Problem(
            name=f"batched_4d_{k}_L{L}", d=2, mesh_x=square_mesh(0.0, 1.0, 2), mesh_v=square_mesh(-1.0, 1.0, 2),
            L=L, r=1, dt=dt, delta=hx, n_strips=n_strips,
            beta=[Product(1.0, None, lambda p: p[:, 0]), Product(1.0, None, lambda p: p[:, 1]),
                  Product(0.0), Product(0.0)],
            sigma=Product(0.0), u0=[Product(1.0, ux, uv)]))
    return out


# ----------------------------------------------------------------------------
# seeded random inputs
# ----------------------------------------------------------------------------

def uniform_vector(n: int, seed: int) -> np.ndarray:
    """U[-1, 1] float64 values, seeded (PCG64)."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=n)


def round_to_bf16(x: np.ndarray) -> np.ndarray:
    """The nearest bfloat16 values of x (rounded to float32, then to 8
    significant bits, ties to even), returned as float64: inputs that a
    bfloat16-storage apply and an FP64 reference read identically."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    return (b.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def grid_samples(shapes, per_grid: int, seed: int):
    """(grid, k1, k2) output positions, per_grid >= 2 on every grid: the
    last row and column (the ragged edges of any tiling), then seeded
    interior positions."""
    rng = np.random.default_rng(seed)
    out = []
    for i, (n1, n2) in enumerate(shapes):
        out.append((i, n1 - 1, n2 - 1))
        for _ in range(per_grid - 1):
            out.append((i, int(rng.integers(0, n1)), int(rng.integers(0, n2))))
    return out


def sample_indices(n: int, k: int, seed: int) -> np.ndarray:
    """k distinct sorted indices in [0, n), seeded."""
    rng = np.random.default_rng(seed)
    k = min(k, n)
    return np.sort(rng.choice(n, size=k, replace=False))
