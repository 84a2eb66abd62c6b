"""Oracle runs shared by the GPU parity tests (computed once per test session)."""
import functools

import numpy as np

from oracle import elasticity as EL
from oracle.assembly import System
from oracle.bddc import BDDC
from oracle.integration import Integration
from oracle.mesh import Mesh
from oracle.pcg import pcg
from paper_1703_06323_gb300 import inputs


def small_problems():
    """Small cases that span several blocks, ragged tails and the degenerate cases."""
    isl_cells = (16, 16, 16)
    X, Y, Z = inputs.node_coords((0, 0, 0), (1, 1, 1), isl_cells)
    a = np.sqrt((X - 0.125) ** 2 + (Y - 0.125) ** 2 + (Z - 0.125) ** 2) - 0.04
    b = np.sqrt((X - 0.375) ** 2 + (Y - 0.375) ** 2 + (Z - 0.125) ** 2) - 0.04
    c = np.sqrt((X - 0.75) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2) - 0.2
    islands = inputs.Problem(name="two_pieces", box_lo=np.zeros(3), box_hi=np.ones(3), cells=isl_cells,
                             sub_cells=(8, 8, 8), phi=np.minimum(np.minimum(a, b), c), f=np.ones_like(X),
                             dirichlet_face_mask=0, pin_node=inputs.PIN_NONE)
    return {
        "sphere16": inputs.manufactured_sphere(0),
        "sphere_ragged": inputs.sphere_problem(cells=(12, 9, 6), sub_cells=(4, 3, 3), centre=(0.52, 0.41, 0.27),
                                               radius=0.22, box_lo=(0, 0, 0), box_hi=(1.0, 0.75, 0.5),
                                               dirichlet_face_mask=0, pin_node=inputs.PIN_AUTO, name="ragged"),
        "plane": inputs.plane_problem(cells=(8, 8, 8), sub_cells=(4, 4, 4), normal=(0.6, 0.8, 0.1), offset=0.61,
                                      dirichlet_face_mask=inputs.ALL_FACES),
        "box_dirichlet": inputs.box_problem(cells=(8, 8, 8), sub_cells=(4, 4, 4),
                                            dirichlet_face_mask=inputs.ALL_FACES),
        "one_subdomain": inputs.manufactured_sphere(0, n=8, sub=8, radius=0.4),
        "slab_sliver": _slab(1e-5),
        "two_pieces": islands,      # floating islands: integer parity, then SINGULAR_LOCAL
        "u_shape": _u_shape(),      # block 0 holds two separate subdomains
        "tower": _tower(),          # 8 z layers of blocks: multi-level coarse cyclic reduction
    }


def large_block_problems():
    """Blocks of more than 8 cells per edge (Sect. 5.2 studies H/h up to 16): a sphere
    in 16^3-cell blocks, a plane cut that leaves whole blocks nearly full (17^3 local
    nodes, interiors near 15^3), and a ragged 16 x 12 x 16 block shape."""
    return {
        "lb_sphere": inputs.sphere_problem(cells=(32, 32, 32), sub_cells=(16, 16, 16), centre=(0.02, -0.01, 0.03),
                                           radius=0.7, box_lo=(-1, -1, -1), box_hi=(1, 1, 1),
                                           dirichlet_face_mask=0, pin_node=inputs.PIN_AUTO, name="lb_sphere"),
        "lb_plane": inputs.plane_problem(cells=(32, 32, 32), sub_cells=(16, 16, 16), normal=(0.3, 0.2, 0.93),
                                         offset=0.97, dirichlet_face_mask=inputs.ALL_FACES, name="lb_plane"),
        "lb_ragged": inputs.sphere_problem(cells=(32, 24, 16), sub_cells=(16, 12, 16), centre=(0.55, 0.4, 0.26),
                                           radius=0.4, box_lo=(0, 0, 0), box_hi=(1.0, 0.75, 0.5),
                                           dirichlet_face_mask=inputs.FACE_XLO, pin_node=inputs.PIN_AUTO,
                                           name="lb_ragged"),
    }


def _tower():
    """A wavy cylinder along z through 8 layers of 4^3-cell blocks (pure Neumann, pinned)."""
    cells = (8, 8, 32)
    X, Y, Z = inputs.node_coords((0, 0, 0), (1, 1, 4), cells)
    r = 0.33 + 0.06 * np.sin(2 * np.pi * Z / 1.3)
    phi = np.sqrt((X - 0.5) ** 2 + (Y - 0.47) ** 2) - r
    f = np.random.default_rng(7).uniform(-1, 1, X.size)
    return inputs.Problem(name="tower", box_lo=np.zeros(3), box_hi=np.array([1.0, 1.0, 4.0]), cells=cells,
                          sub_cells=(4, 4, 4), phi=phi, f=f, dirichlet_face_mask=0, pin_node=inputs.PIN_AUTO)


def _box_phi(X, Y, Z, lo, hi):
    c = [(a + b) / 2 for a, b in zip(lo, hi)]
    r = [(b - a) / 2 for a, b in zip(lo, hi)]
    return np.maximum(np.maximum(np.abs(X - c[0]) - r[0], np.abs(Y - c[1]) - r[1]), np.abs(Z - c[2]) - r[2])


def _u_shape():
    """Two bars in one block joined by a cross bar in the next block."""
    cells = (16, 16, 16)
    X, Y, Z = inputs.node_coords((0, 0, 0), (1, 1, 1), cells)
    phi = np.minimum(np.minimum(_box_phi(X, Y, Z, (0.1, 0.1, 0.1), (0.8, 0.2, 0.3)),
                                _box_phi(X, Y, Z, (0.1, 0.35, 0.1), (0.8, 0.45, 0.3))),
                     _box_phi(X, Y, Z, (0.6, 0.1, 0.1), (0.8, 0.45, 0.3)))
    f = np.random.default_rng(5).uniform(-1, 1, X.size)
    return inputs.Problem(name="u_shape", box_lo=np.zeros(3), box_hi=np.ones(3), cells=cells, sub_cells=(8, 8, 8),
                          phi=phi, f=f, dirichlet_face_mask=0, pin_node=inputs.PIN_AUTO)


def _slab(eps):
    h = 1.0 / 8
    p = inputs.plane_problem(cells=(8, 8, 8), sub_cells=(4, 4, 4), normal=(1, 0, 0), offset=0.5 + eps * h,
                             dirichlet_face_mask=inputs.FACE_XLO, linear=(0, 0, 0, 0), name="slab")
    p.f = np.random.default_rng(0).uniform(-1, 1, p.n_nodes)
    return p


def nitsche_problems():
    """Weak Dirichlet data (Nitsche, Sect. 2.2) on the unfitted boundary: a sphere whose
    whole boundary carries them, a linear solution below a plane cut (strong data on the
    box faces it reaches), and the bumpy sphere at 32^3 with its forced small cuts."""
    sphere = inputs.sphere_problem(cells=(16, 16, 16), sub_cells=(4, 4, 4), centre=(0.51, 0.49, 0.5), radius=0.4,
                                   dirichlet_face_mask=inputs.ALL_FACES, pin_node=inputs.PIN_NONE, name="ni_sphere")
    plane = inputs.plane_problem(cells=(8, 8, 8), sub_cells=(4, 4, 4), normal=(0.6, 0.8, 0.1), offset=0.61,
                                 dirichlet_face_mask=inputs.ALL_FACES, pin_node=inputs.PIN_NONE, name="ni_plane")
    bumpy = inputs.bumpy_sphere(0, n=32)
    bumpy.name = "ni_bumpy"
    bumpy.pin_node = inputs.PIN_NONE
    bumpy.dirichlet_values = np.random.default_rng(3).uniform(-1, 1, bumpy.n_nodes)
    out = {"ni_sphere": sphere, "ni_plane": plane, "ni_bumpy": bumpy}
    for p in out.values():
        p.q = None
        p.weak_dirichlet = True
    return out


class OracleRun:
    def __init__(self, p):
        self.p = p
        self.mesh = Mesh(p)
        self.integ = Integration(self.mesh, p)
        self.sys = System(self.mesh, self.integ, p)
        self._bddc = {}

    def bddc(self, weighting="stiffness", objects="v1", coarse="cef"):
        key = (weighting, objects, coarse)
        if key not in self._bddc:
            self._bddc[key] = BDDC(self.mesh, self.integ, self.sys, weighting=weighting, objects=objects,
                                   coarse=coarse)
        return self._bddc[key]

    def solve(self, rtol=1e-8, **kw):
        B = self.bddc(**kw)
        return pcg(self.sys.apply, self.sys.b, B.apply, rtol=rtol, maxit=2000)


def _elastic_sphere(cells, sub, centre, radius, box_hi=(1.0, 1.0, 1.0), name="el_sphere"):
    """A sphere crossing the clamped face x = 0 with body force (0, 0, -1)."""
    X, Y, Z = inputs.node_coords((0, 0, 0), box_hi, cells)
    c = np.asarray(centre)
    phi = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) - radius
    f = np.zeros((X.size, 3))
    f[:, 2] = -1.0
    return inputs.Problem(name=name, box_lo=np.zeros(3), box_hi=np.asarray(box_hi, float), cells=cells,
                          sub_cells=sub, phi=phi, f=f, q=None, dirichlet_face_mask=inputs.FACE_XLO,
                          pin_node=inputs.PIN_NONE, dirichlet_values=np.zeros((X.size, 3)), ncomp=3,
                          lame=(1.0, 0.3))


def elastic_problems():
    """Small elasticity cases: several blocks, a ragged block grid, the patch test, a sphere union."""
    return {
        "el_sphere8": _elastic_sphere((8, 8, 8), (4, 4, 4), (0.2, 0.5, 0.5), 0.42),
        "el_ragged": _elastic_sphere((12, 9, 6), (4, 3, 3), (0.25, 0.4, 0.24), 0.3, box_hi=(1.0, 0.75, 0.5),
                                     name="el_ragged"),
        "el_patch": inputs.elastic_patch(),
        "el_spheres16": inputs.elastic_spheres(seed=0, n=16, sub=8),
        "el_wall": _elastic_wall(),
    }


def _elastic_wall():
    """A slab below a wavy surface y = 0.55 + 0.2 sin(pi z), clamped on x = 0, through 4
    z layers of blocks (multi-level coarse cyclic reduction with rotation rows)."""
    cells = (8, 8, 16)
    X, Y, Z = inputs.node_coords((0, 0, 0), (1, 1, 2), cells)
    phi = Y - (0.55 + 0.2 * np.sin(np.pi * Z))
    f = np.zeros((X.size, 3))
    f[:, 2] = -1.0
    return inputs.Problem(name="el_wall", box_lo=np.zeros(3), box_hi=np.array([1.0, 1.0, 2.0]), cells=cells,
                          sub_cells=(4, 4, 4), phi=phi, f=f, q=None, dirichlet_face_mask=inputs.FACE_XLO,
                          pin_node=inputs.PIN_NONE, dirichlet_values=np.zeros((X.size, 3)), ncomp=3,
                          lame=(1.0, 0.3))


class ElasticOracleRun(OracleRun):
    def __init__(self, p):
        self.p = p
        self.mesh = Mesh(p)
        self.integ = EL.ElasticIntegration(self.mesh, p)
        self.sys = EL.ElasticSystem(self.mesh, self.integ, p)
        self._bddc = {}


@functools.lru_cache(maxsize=None)
def oracle_run(name):
    if name == "bumpy64":
        return OracleRun(inputs.bumpy_sphere(0))
    if name.startswith("el_"):
        return ElasticOracleRun(elastic_problems()[name])
    if name.startswith("ni_"):
        return OracleRun(nitsche_problems()[name])
    if name.startswith("lb_"):
        return OracleRun(large_block_problems()[name])
    if name == "ml_box":
        # whole box, 8^3 cells in 2^3-cell blocks (64 subdomains): with groups of 2^3
        # blocks the level-2 objects of the three-level method hold several coarse DOFs
        return OracleRun(inputs.box_problem(cells=(8, 8, 8), sub_cells=(2, 2, 2), dirichlet_face_mask=inputs.ALL_FACES,
                                            name="ml_box"))
    return OracleRun(small_problems()[name])


def object_ids(objs, n_dof):
    """Object id per DOF (-1 off the interface) and kinds, in the oracle's order."""
    ids = -np.ones(n_dof, dtype=np.int64)
    for k, o in enumerate(objs):
        ids[o["dofs"]] = k
    return ids, np.array([o["kind"] for o in objs], dtype=np.int64)


def energy_error(A, x, ref):
    e = x - ref
    den = float(ref @ (A @ ref))
    return float(np.sqrt(max(e @ (A @ e), 0.0) / den)) if den > 0 else float(np.sqrt(max(e @ (A @ e), 0.0)))
