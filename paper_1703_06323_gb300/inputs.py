"""Seeded synthetic problems for the unfitted-FE BDDC solver.

This module holds only *problem definitions*: level-set geometry sampled at
the background-mesh nodes, source terms, Neumann flux fields, Dirichlet data,
per-cell coefficients, and the random draws behind them.  None of the solver's
arithmetic (classification, integration, assembly, BDDC, PCG) lives here, so
both the CUDA path and the FP64 oracle can consume the same arrays.

Elasticity problems (ncomp = 3) carry nodal body forces f of shape (n_nodes, 3),
an optional nodal stress field q of shape (n_nodes, 9) (row-major sigma_ij; the
boundary traction is sigma n), Dirichlet values of shape (n_nodes, 3) and the
material (E, nu) in ``lame``.

Array conventions (shared with the C ABI):
  * nodes of an ``nx x ny x nz`` cell grid are numbered ``i + (nx+1)*(j + (ny+1)*k)``
    (x fastest); cells are numbered ``i + nx*(j + ny*k)``;
  * nodal scalars are float64 arrays of length ``(nx+1)(ny+1)(nz+1)``;
  * nodal flux vectors are float64 arrays of shape ``(n_nodes, 3)``;
  * the domain is ``{phi < 0}`` (Sect. 2.1: the boundary is the zero level set).

Workloads (the sphere, the bumpy sphere with forced small cuts, the batched
spheres and the random-coefficient sphere) follow the paper's experiment setup
(Sect. 5.1: sphere geometry, Neumann data on the unfitted boundary, one pinned
interior node when no box face carries a Dirichlet condition).
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

# Bit of ``dirichlet_face_mask`` per box face: x=lo, x=hi, y=lo, y=hi, z=lo, z=hi.
FACE_XLO, FACE_XHI, FACE_YLO, FACE_YHI, FACE_ZLO, FACE_ZHI = (1 << b for b in range(6))
ALL_FACES = 0x3F

PIN_NONE = -1
PIN_AUTO = -2


@dataclasses.dataclass
class Problem:
    """One Poisson problem on a Cartesian background mesh of a box."""

    name: str
    box_lo: np.ndarray          # (3,) float64
    box_hi: np.ndarray          # (3,) float64
    cells: tuple                # (nx, ny, nz)
    sub_cells: tuple            # cells per subdomain block edge, e.g. (8, 8, 8)
    phi: np.ndarray             # nodal level set, domain = {phi < 0}
    f: np.ndarray               # nodal source values (Q1 interpolated)
    q: Optional[np.ndarray] = None          # nodal flux vector, Neumann data g = q . n
    dirichlet_face_mask: int = 0
    pin_node: int = PIN_AUTO
    dirichlet_values: Optional[np.ndarray] = None   # nodal values read at constrained nodes
    kappa: Optional[np.ndarray] = None      # per-cell diffusion coefficient (None = 1)
    u_exact: Optional[np.ndarray] = None    # nodal exact solution when manufactured
    meta: dict = dataclasses.field(default_factory=dict)
    ncomp: int = 1                          # 1 Poisson; 3 linear elasticity
    lame: Optional[tuple] = None            # elasticity: (E, nu); kappa then scales E per cell
    weak_dirichlet: bool = False            # Poisson: Dirichlet data (dirichlet_values, Q1 interpolated)
                                            # imposed weakly (Nitsche) on the unfitted boundary

    @property
    def n_nodes(self) -> int:
        nx, ny, nz = self.cells
        return (nx + 1) * (ny + 1) * (nz + 1)

    @property
    def h(self) -> float:
        return float((self.box_hi[0] - self.box_lo[0]) / self.cells[0])


def node_coords(box_lo, box_hi, cells):
    """Return (X, Y, Z) node coordinates, flattened x-fastest."""
    nx, ny, nz = cells
    lo = np.asarray(box_lo, dtype=np.float64)
    hi = np.asarray(box_hi, dtype=np.float64)
    xs = lo[0] + (hi[0] - lo[0]) * np.arange(nx + 1) / nx
    ys = lo[1] + (hi[1] - lo[1]) * np.arange(ny + 1) / ny
    zs = lo[2] + (hi[2] - lo[2]) * np.arange(nz + 1) / nz
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    return X.ravel(), Y.ravel(), Z.ravel()


def cell_centres(box_lo, box_hi, cells):
    nx, ny, nz = cells
    lo = np.asarray(box_lo, dtype=np.float64)
    hi = np.asarray(box_hi, dtype=np.float64)
    xs = lo[0] + (hi[0] - lo[0]) * (np.arange(nx) + 0.5) / nx
    ys = lo[1] + (hi[1] - lo[1]) * (np.arange(ny) + 0.5) / ny
    zs = lo[2] + (hi[2] - lo[2]) * (np.arange(nz) + 0.5) / nz
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    return X.ravel(), Y.ravel(), Z.ravel()


def _sines(X, Y, Z):
    """u = sin(pi x) sin(pi y) sin(pi z), its flux grad u and source -lap u."""
    sx, sy, sz = np.sin(np.pi * X), np.sin(np.pi * Y), np.sin(np.pi * Z)
    cx, cy, cz = np.cos(np.pi * X), np.cos(np.pi * Y), np.cos(np.pi * Z)
    u = sx * sy * sz
    q = np.pi * np.stack([cx * sy * sz, sx * cy * sz, sx * sy * cz], axis=1)
    f = 3.0 * np.pi ** 2 * u
    return u, q, f


# ---------------------------------------------------------------------------
# Generic small geometries (used by tests and examples)
# ---------------------------------------------------------------------------

def sphere_problem(cells=(16, 16, 16), sub_cells=(8, 8, 8), centre=(0.5, 0.5, 0.5),
                   radius=0.4, box_lo=(0.0, 0.0, 0.0), box_hi=(1.0, 1.0, 1.0),
                   dirichlet_face_mask=ALL_FACES, pin_node=PIN_AUTO, name="sphere"):
    """Sphere {|x-c| < r} with manufactured u = sin(pi x) sin(pi y) sin(pi z)."""
    X, Y, Z = node_coords(box_lo, box_hi, cells)
    c = np.asarray(centre, dtype=np.float64)
    phi = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) - radius
    u, q, f = _sines(X, Y, Z)
    return Problem(name=name, box_lo=np.asarray(box_lo, float), box_hi=np.asarray(box_hi, float),
                   cells=tuple(cells), sub_cells=tuple(sub_cells), phi=phi, f=f, q=q,
                   dirichlet_face_mask=dirichlet_face_mask, pin_node=pin_node,
                   dirichlet_values=u.copy(), u_exact=u,
                   meta={"centre": c.tolist(), "radius": radius})


def plane_problem(cells=(16, 16, 16), sub_cells=(8, 8, 8), normal=(1.0, 0.0, 0.0), offset=0.5,
                  box_lo=(0.0, 0.0, 0.0), box_hi=(1.0, 1.0, 1.0), dirichlet_face_mask=FACE_XLO,
                  linear=(0.3, 1.0, -0.5, 0.25), pin_node=PIN_AUTO, name="plane"):
    """Half-space {n.x < offset} clipped to the box, with a linear exact solution.

    u = a + b.x solves -lap u = 0 with flux q = b; the plane level set is
    resolved exactly by the tet-linear geometry, so u is reproduced by Q1.
    """
    X, Y, Z = node_coords(box_lo, box_hi, cells)
    n = np.asarray(normal, dtype=np.float64)
    phi = n[0] * X + n[1] * Y + n[2] * Z - offset
    a, bx, by, bz = linear
    u = a + bx * X + by * Y + bz * Z
    q = np.tile(np.array([bx, by, bz], dtype=np.float64), (X.size, 1))
    return Problem(name=name, box_lo=np.asarray(box_lo, float), box_hi=np.asarray(box_hi, float),
                   cells=tuple(cells), sub_cells=tuple(sub_cells), phi=phi, f=np.zeros_like(X), q=q,
                   dirichlet_face_mask=dirichlet_face_mask, pin_node=pin_node,
                   dirichlet_values=u.copy(), u_exact=u,
                   meta={"normal": n.tolist(), "offset": offset})


def box_problem(cells=(16, 16, 16), sub_cells=(8, 8, 8), dirichlet_face_mask=ALL_FACES, seed=0,
                name="box"):
    """Whole box active (no cut cells), random nodal source: the body-fitted case."""
    X, Y, Z = node_coords((0, 0, 0), (1, 1, 1), cells)
    rng = np.random.default_rng(seed)
    phi = -np.ones_like(X)
    f = rng.uniform(-1.0, 1.0, X.size)
    return Problem(name=name, box_lo=np.zeros(3), box_hi=np.ones(3), cells=tuple(cells),
                   sub_cells=tuple(sub_cells), phi=phi, f=f, q=None,
                   dirichlet_face_mask=dirichlet_face_mask, pin_node=PIN_AUTO,
                   dirichlet_values=np.zeros_like(X))


# ---------------------------------------------------------------------------
# Benchmark workloads
# ---------------------------------------------------------------------------

def manufactured_sphere(seed=0, n=16, sub=8, radius=0.4):
    """Sphere radius 0.4 in the unit cube (16^3 cells, 2^3 blocks of 8^3).

    Centre (0.5,0.5,0.5) + U(-0.02,0.02)^3 from ``seed``; u = 0 on the box faces
    (never reached by the sphere, so one interior node is pinned to u_exact);
    Neumann data g = grad(u_exact).n on the unfitted boundary; f = -lap u_exact.
    """
    rng = np.random.default_rng(seed)
    c = 0.5 + rng.uniform(-0.02, 0.02, 3)
    p = sphere_problem(cells=(n, n, n), sub_cells=(sub, sub, sub), centre=c, radius=radius,
                       dirichlet_face_mask=ALL_FACES, pin_node=PIN_AUTO,
                       name=f"sphere{n}_r{radius}_seed{seed}")
    p.meta["seed"] = seed
    return p


def _bumpy_phi(X, Y, Z, c, dirs, r0=0.3, amp=0.05, width=20.0):
    d = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2)
    bump = np.zeros_like(d)
    for k in range(dirs.shape[0]):
        p = c + r0 * dirs[k]
        bump += np.exp(-width * ((X - p[0]) ** 2 + (Y - p[1]) ** 2 + (Z - p[2]) ** 2))
    return d - r0 - amp * bump


def bumpy_sphere(seed=0, n=64, sub=8, eta_target=1e-6, n_bumps=6):
    """Bumpy sphere phi = |x-c| - 0.3 - 0.05 sum_k exp(-20|x-p_k|^2), 64^3 cells.

    * ``c`` = (0.5,0.5,0.5) + a seeded sub-cell offset U(-h/2,h/2)^3;
    * bump points p_k = c + 0.3 d_k with seeded unit directions d_k;
    * then the x coordinate of ``c`` is adjusted so that the grid node x* nearest
      the surface along (1,1,1)/sqrt(3) sits at depth phi(x*) = -delta, where
      delta = h (6 eta_target n_x n_y n_z)^(1/3) is the depth at which a plane
      with unit normal n cuts a corner piece of volume fraction eta_target off
      the cell beyond x*.  The achieved minimum cut fraction is a solver output.
    f ~ U(-1,1) per node, Neumann (zero flux) on the whole boundary, one pinned node.
    """
    rng = np.random.default_rng(seed)
    h = 1.0 / n
    c0 = np.full(3, 0.5) + rng.uniform(-0.5 * h, 0.5 * h, 3)
    dirs = rng.normal(size=(n_bumps, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    f = rng.uniform(-1.0, 1.0, (n + 1) ** 3)

    def phi_at(pts, c):
        return _bumpy_phi(pts[:, 0], pts[:, 1], pts[:, 2], c, dirs)

    dstar = np.ones(3) / np.sqrt(3.0)
    # surface point along the ray c0 + t dstar (bisection on phi)
    lo_t, hi_t = 0.0, 0.49
    for _ in range(200):
        mid = 0.5 * (lo_t + hi_t)
        if phi_at((c0 + mid * dstar)[None, :], c0)[0] < 0:
            lo_t = mid
        else:
            hi_t = mid
    P = c0 + lo_t * dstar
    xstar = np.floor(P / h) * h            # grid node on the -(1,1,1) side of P
    # local unit normal at P by central differences of the level set
    eps = 1e-6
    g = np.array([(phi_at((P + eps * e)[None], c0)[0] - phi_at((P - eps * e)[None], c0)[0]) / (2 * eps)
                  for e in np.eye(3)])
    nrm = g / np.linalg.norm(g)
    prod = max(float(nrm[0] * nrm[1] * nrm[2]), 1e-3)
    delta = h * (6.0 * eta_target * prod) ** (1.0 / 3.0)
    # shift c_x by s so that phi(x*; c0 + s e_x) = -delta (bisection; phi decreases with s here)
    s_lo, s_hi = -2.0 * h, 2.0 * h
    def gfun(s):
        return phi_at(xstar[None], c0 + np.array([s, 0.0, 0.0]))[0] + delta
    for _ in range(200):
        mid = 0.5 * (s_lo + s_hi)
        if gfun(mid) > 0:
            s_lo = mid
        else:
            s_hi = mid
    c = c0 + np.array([0.5 * (s_lo + s_hi), 0.0, 0.0])
    X, Y, Z = node_coords((0, 0, 0), (1, 1, 1), (n, n, n))
    phi = _bumpy_phi(X, Y, Z, c, dirs)
    return Problem(name=f"bumpy_sphere{n}_seed{seed}", box_lo=np.zeros(3), box_hi=np.ones(3),
                   cells=(n, n, n), sub_cells=(sub, sub, sub), phi=phi, f=f, q=None,
                   dirichlet_face_mask=0, pin_node=PIN_AUTO,
                   dirichlet_values=np.zeros_like(phi),
                   meta={"seed": seed, "centre": c.tolist(), "bump_dirs": dirs.tolist(),
                         "xstar": xstar.tolist(), "delta": delta, "eta_target": eta_target})


def random_field_kappa(cells, seed=0, sigma=1.0, ell=0.1, n_features=1024):
    """kappa = exp(g) per cell, g a squared-exponential Gaussian field (std sigma,
    correlation length ell) drawn by random Fourier features (Rahimi & Recht 2007)."""
    rng = np.random.default_rng(seed + 7919)
    w = rng.normal(scale=1.0 / ell, size=(n_features, 3))
    b = rng.uniform(0.0, 2.0 * np.pi, n_features)
    a = rng.normal(size=n_features)
    # cell centres form a tensor grid, so cos(w.x + b) = Re(e^{ib} e^{i w_x x} e^{i w_y y} e^{i w_z z})
    # and the feature sum is a product of three 1-D factors contracted over the features
    nx, ny, nz = cells
    cx, cy, cz = ((np.arange(n) + 0.5) / n for n in (nx, ny, nz))
    Ex, Ey, Ez = (np.exp(1j * np.outer(w[:, d], c)) for d, c in enumerate((cx, cy, cz)))
    T = (a * np.exp(1j * b))[:, None] * Ez                     # features x nz
    g = np.empty((nz, ny, nx))
    for k in range(nz):
        g[k] = ((Ey * T[:, k:k + 1]).T @ Ex).real               # (ny x M) (M x nx)
    g = g.ravel() * (sigma * np.sqrt(2.0 / n_features))
    return np.exp(g)


def coefficient_sphere(seed=0, n=128, sub=8, radius=0.45):
    """Sphere radius 0.45 with a log-normal per-cell coefficient (adjoint workload)."""
    X, Y, Z = node_coords((0, 0, 0), (1, 1, 1), (n, n, n))
    phi = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2) - radius
    u_d = np.sin(np.pi * X) * np.sin(np.pi * Y) * np.sin(np.pi * Z)
    kappa = random_field_kappa((n, n, n), seed=seed)
    return Problem(name=f"kappa_sphere{n}_seed{seed}", box_lo=np.zeros(3), box_hi=np.ones(3),
                   cells=(n, n, n), sub_cells=(sub, sub, sub), phi=phi, f=np.ones_like(phi), q=None,
                   dirichlet_face_mask=0, pin_node=PIN_AUTO, dirichlet_values=np.zeros_like(phi),
                   kappa=kappa, meta={"seed": seed, "u_d": u_d})


def batched_spheres(count=256, seed=0, sizes=(24, 32, 48, 64), sub=8):
    """Independent sphere problems with seeded size, centre and radius U(0.25,0.45)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(sizes[rng.integers(len(sizes))])
        r = float(rng.uniform(0.25, 0.45))
        delta = max(0.5 - r - 2.0 / n, 0.0)    # the sphere stays 2h inside the box where it can
        c = 0.5 + rng.uniform(-delta, delta, 3)
        p = sphere_problem(cells=(n, n, n), sub_cells=(sub, sub, sub), centre=c, radius=r,
                           dirichlet_face_mask=0, pin_node=PIN_AUTO, name=f"batch{i}_n{n}")
        p.f = rng.uniform(-1.0, 1.0, p.n_nodes)
        p.q = None
        p.dirichlet_values = np.zeros(p.n_nodes)
        out.append(p)
    return out


# ---------------------------------------------------------------------------
# Linear elasticity (vector Q1, 3 DOFs per node)
# ---------------------------------------------------------------------------

def _sphere_union_phi(X, Y, Z, centres, radii):
    phi = np.full(X.shape, np.inf)
    for c, r in zip(centres, radii):
        phi = np.minimum(phi, np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) - r)
    return phi


def elastic_patch(cells=(8, 8, 8), sub_cells=(4, 4, 4), normal=(1.0, 0.2, 0.1), offset=0.56,
                  grad=((0.02, 0.01, -0.03), (0.015, -0.01, 0.02), (-0.025, 0.03, 0.01)),
                  shift=(0.1, -0.2, 0.05), E=1.0, nu=0.3, name="elastic_patch"):
    """Plane-cut box with the linear displacement u = shift + grad x.

    The uniform stress sigma = lambda tr(eps) I + 2 mu eps of u is prescribed as
    the traction sigma n on the unfitted plane; the box faces the domain reaches
    (all but x = 1) carry u as a strong Dirichlet condition; no body force."""
    X, Y, Z = node_coords((0, 0, 0), (1, 1, 1), cells)
    n = np.asarray(normal, dtype=np.float64)
    n = n / np.linalg.norm(n)
    phi = n[0] * X + n[1] * Y + n[2] * Z - offset
    B = np.asarray(grad, dtype=np.float64)
    P = np.stack([X, Y, Z], axis=1)
    u = np.asarray(shift, dtype=np.float64)[None, :] + P @ B.T
    eps = 0.5 * (B + B.T)
    lam, mu = E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))
    sigma = lam * np.trace(eps) * np.eye(3) + 2 * mu * eps
    mask = FACE_XLO | FACE_YLO | FACE_YHI | FACE_ZLO | FACE_ZHI
    return Problem(name=name, box_lo=np.zeros(3), box_hi=np.ones(3), cells=tuple(cells),
                   sub_cells=tuple(sub_cells), phi=phi, f=np.zeros((X.size, 3)),
                   q=np.tile(sigma.ravel(), (X.size, 1)), dirichlet_face_mask=mask, pin_node=PIN_NONE,
                   dirichlet_values=u.copy(), u_exact=u, ncomp=3, lame=(E, nu),
                   meta={"normal": n.tolist(), "offset": offset})


def elastic_spheres(seed=0, n=96, sub=8, count=8, r_range=(0.1, 0.2), E=1.0, nu=0.3, snap=0.0):
    """Union of seeded spheres clamped on the box face x = 0 (body force (0,0,-1)).

    The spheres form a chain: the first one crosses x = 0, each next one is
    centred at a seeded direction from the previous centre, at a seeded fraction
    U(0.5, 0.9) of the sum of the two radii, and kept inside [r, 1 - r] in y, z and
    [.., 1 - r] in x; the union is therefore connected and touches x = 0.  Cut
    boundary traction-free; other box faces natural.  Nodal level-set values
    closer to zero than snap * h are moved to +-snap * h (sign kept), which keeps
    every cut volume fraction above ~snap^3 / 6; snap = 0 keeps the raw union."""
    rng = np.random.default_rng(seed)
    radii = rng.uniform(r_range[0], r_range[1], count)
    centres = np.zeros((count, 3))
    centres[0] = [rng.uniform(0.3, 0.7) * radii[0], rng.uniform(0.3, 0.7), rng.uniform(0.3, 0.7)]
    for i in range(1, count):
        for _ in range(1000):
            d = rng.normal(size=3)
            d /= np.linalg.norm(d)
            c = centres[i - 1] + d * rng.uniform(0.5, 0.9) * (radii[i - 1] + radii[i])
            lo = np.array([0.0, radii[i], radii[i]])
            hi = 1.0 - radii[i]
            if np.all(c >= lo) and np.all(c <= hi):
                break
        centres[i] = np.clip(c, [0.0, radii[i], radii[i]], 1.0 - radii[i])
    X, Y, Z = node_coords((0, 0, 0), (1, 1, 1), (n, n, n))
    phi = _sphere_union_phi(X, Y, Z, centres, radii)
    if snap > 0:
        g = snap / n
        near = np.abs(phi) < g
        phi[near] = np.where(phi[near] < 0, -g, g)
    f = np.zeros((X.size, 3))
    f[:, 2] = -1.0
    return Problem(name=f"elastic_spheres{n}_seed{seed}", box_lo=np.zeros(3), box_hi=np.ones(3),
                   cells=(n, n, n), sub_cells=(sub, sub, sub), phi=phi, f=f, q=None,
                   dirichlet_face_mask=FACE_XLO, pin_node=PIN_NONE,
                   dirichlet_values=np.zeros((X.size, 3)), ncomp=3, lame=(E, nu),
                   meta={"seed": seed, "centres": centres.tolist(), "radii": radii.tolist(), "snap": snap})
