"""Pins for the oracle's integer work: classification, DOFs, subdomains, objects."""
import os

import numpy as np
import pytest

from oracle import mesh as M
from paper_1703_06323_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _grid_phi(cells, sub, fn, lo=(0, 0, 0), hi=(1, 1, 1)):
    X, Y, Z = inputs.node_coords(lo, hi, cells)
    return M.Grid(lo, hi, cells, sub), fn(X, Y, Z)


def test_table1_sphere_counts_match_paper():
    """Table 1, Sphere ids 1-3: subdomains, active cells, DOFs, max DOFs/cells per subdomain."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table1_sphere.txt")) if l[0].isdigit()]
    for row in rows[:3]:
        n, n_sd, n_el, n_sdel, n_dof, n_sddof = (int(x) for x in row[1:7])
        p = inputs.sphere_problem(cells=(n, n, n), sub_cells=(8, 8, 8), centre=(0, 0, 0), radius=0.7,
                                  box_lo=(-1, -1, -1), box_hi=(1, 1, 1), dirichlet_face_mask=0,
                                  pin_node=inputs.PIN_NONE)
        m = M.Mesh(p)
        assert m.n_sub == n_sd
        assert int((m.cell_type != M.EXTERNAL).sum()) == n_el
        assert m.n_dof == n_dof
        # n_sdel / n_sddof are the block capacity (8^3 cells, 9^3 nodes); they are
        # reached by blocks that lie entirely inside the sphere (id 3 has some)
        assert max(len(c) for c in m.sub_cells) <= n_sdel
        assert max(d.size for d in m.sub_dofs) <= n_sddof
        if n >= 64:
            assert max(len(c) for c in m.sub_cells) == n_sdel
            assert max(d.size for d in m.sub_dofs) == n_sddof


def test_table1_sphere_large_meshes_counts():
    """Table 1, Sphere ids 4-5 (classification and DOF count only; vectorised parts)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table1_sphere.txt")) if l[0].isdigit()]
    for row in rows[3:]:
        n, n_sd, n_el, _, n_dof = (int(x) for x in row[1:6])
        g, phi = _grid_phi((n, n, n), (8, 8, 8), lambda X, Y, Z: np.sqrt(X * X + Y * Y + Z * Z) - 0.7,
                           lo=(-1, -1, -1), hi=(1, 1, 1))
        t = M.classify_cells(g, phi)
        assert int((t != M.EXTERNAL).sum()) == n_el
        dof, _, _ = M.number_dofs(g, t, phi, 0, -1)
        assert int((dof >= 0).sum()) == n_dof
        nb = n // 8
        act = (t.reshape(nb, 8, nb, 8, nb, 8) != M.EXTERNAL).any(axis=(1, 3, 5)).sum()
        assert act == n_sd


def test_classification_brute_force():
    rng = np.random.default_rng(3)
    g, _ = _grid_phi((5, 4, 3), (1, 1, 1), lambda X, Y, Z: X, hi=(1.0, 0.8, 0.6))
    phi = rng.uniform(-1, 1, g.n_nodes)
    phi[rng.integers(0, g.n_nodes, 10)] = 0.0          # exact zeros count as outside
    t = M.classify_cells(g, phi)
    for c in range(g.n_cells):
        k = sum(phi[v] < 0 for v in g.cell_nodes(c))
        assert t[c] == (M.EXTERNAL if k == 0 else M.INTERNAL if k == 8 else M.CUT)


def test_dofs_brute_force_and_pin():
    p = inputs.manufactured_sphere(1)
    m = M.Mesh(p)
    g = m.grid
    act = np.zeros(g.n_nodes, bool)
    for c in range(g.n_cells):
        if m.cell_type[c] != M.EXTERNAL:
            act[g.cell_nodes(c)] = True
    # the sphere never reaches the box faces, so exactly one node is pinned
    assert m.constrained.sum() == 1 and m.constrained[m.pin]
    # pinned node: all 8 cells internal, minimal phi
    cand = [v for v in range(g.n_nodes)
            if len(g.cells_of_node(v)) == 8 and all(m.cell_type[c] == M.INTERNAL for c in g.cells_of_node(v))]
    assert m.pin == min(cand, key=lambda v: (p.phi[v], v))
    expect = -np.ones(g.n_nodes, dtype=np.int64)
    k = 0
    for v in range(g.n_nodes):
        if act[v] and v != m.pin:
            expect[v] = k
            k += 1
    assert np.array_equal(expect, m.dof_of_node)


def test_box_face_dirichlet_removes_face_nodes():
    p = inputs.box_problem(cells=(6, 6, 6), sub_cells=(2, 2, 2), dirichlet_face_mask=inputs.ALL_FACES)
    m = M.Mesh(p)
    assert m.n_dof == 5 ** 3 and m.pin == -1


@pytest.mark.parametrize("nb", [2, 3])
def test_uncut_box_object_counts_closed_form(nb):
    """Body-fitted partition of a Dirichlet box into nb^3 blocks: (nb-1)^3 corners,
    3 nb (nb-1)^2 edges, 3 nb^2 (nb-1) faces (Sect. 3.2)."""
    s = 3
    p = inputs.box_problem(cells=(nb * s,) * 3, sub_cells=(s, s, s), dirichlet_face_mask=inputs.ALL_FACES)
    m = M.Mesh(p)
    objs = m.objects("std")
    kinds = [o["kind"] for o in objs]
    assert kinds.count(M.CORNER) == (nb - 1) ** 3
    assert kinds.count(M.EDGE) == 3 * nb * (nb - 1) ** 2
    assert kinds.count(M.FACE) == 3 * nb ** 2 * (nb - 1)
    for o in objs:
        size = {M.CORNER: 1, M.EDGE: s - 1, M.FACE: (s - 1) ** 2}[o["kind"]]
        assert len(o["dofs"]) == size
        assert len(o["neigh"]) == {M.CORNER: 8, M.EDGE: 4, M.FACE: 2}[o["kind"]]
    # uncut: variant 1 changes nothing
    assert [o["dofs"] for o in m.objects("v1")] == [o["dofs"] for o in objs]


def test_plane_cut_objects_hand_counted():
    """x < 0.3 in the unit cube, 8^3 cells, 2^3 blocks of 4^3, Dirichlet on x = 0.

    Active cells have i in {0,1,2}; DOF nodes i in {1,2,3}.  Four subdomains (bx = 0).
    Standard objects: 4 faces of 3 x 4 = 12 DOFs (y = 0.5 or z = 0.5 planes) and one
    edge of 3 DOFs on the line y = z = 0.5.  Variant 1: the FE edge between x = 0.25
    (inside) and x = 0.375 (outside) is cut, so both ends become corners and the
    remaining DOF x = 0.125 is a single-DOF sub-edge, i.e. a corner (Sect. 4.4)."""
    p = inputs.plane_problem(cells=(8, 8, 8), sub_cells=(4, 4, 4), normal=(1, 0, 0), offset=0.3,
                             dirichlet_face_mask=inputs.FACE_XLO)
    m = M.Mesh(p)
    assert m.n_sub == 4
    std = m.objects("std")
    faces = [o for o in std if o["kind"] == M.FACE]
    edges = [o for o in std if o["kind"] == M.EDGE]
    assert len(std) == 5 and len(faces) == 4 and len(edges) == 1
    assert all(len(o["dofs"]) == 12 for o in faces)
    assert len(edges[0]["dofs"]) == 3 and len(edges[0]["neigh"]) == 4
    v1 = m.objects("v1")
    corners = [o for o in v1 if o["kind"] == M.CORNER]
    assert len(v1) == 7 and len(corners) == 3
    xs = sorted(float(m.grid.node_xyz(m.node_of_dof[o["dofs"][0]])[0]) for o in corners)
    assert np.allclose(xs, [0.125, 0.25, 0.375])
    # objects ordered by smallest DOF id
    mins = [o["dofs"][0] for o in v1]
    assert mins == sorted(mins)


def test_two_islands_in_one_block_are_two_subdomains():
    """Reading R5: disconnected active pieces of one block are separate subdomains."""
    def phi(X, Y, Z):
        a = np.sqrt((X - 0.2) ** 2 + (Y - 0.2) ** 2 + (Z - 0.2) ** 2) - 0.12
        b = np.sqrt((X - 0.8) ** 2 + (Y - 0.8) ** 2 + (Z - 0.8) ** 2) - 0.12
        return np.minimum(a, b)
    g, ph = _grid_phi((8, 8, 8), (8, 8, 8), phi)
    p = inputs.Problem(name="islands", box_lo=np.zeros(3), box_hi=np.ones(3), cells=(8, 8, 8),
                       sub_cells=(8, 8, 8), phi=ph, f=np.zeros(g.n_nodes), pin_node=inputs.PIN_NONE)
    m = M.Mesh(p)
    assert m.n_sub == 2
    assert min(m.sub_cells[0]) < min(m.sub_cells[1])
    assert not m.is_gamma.any()


def test_neighbour_sets_brute_force():
    p = inputs.manufactured_sphere(2)
    m = M.Mesh(p)
    g = m.grid
    for d in range(0, m.n_dof, 7):
        v = m.node_of_dof[d]
        s = set()
        for w, cells in enumerate(m.sub_cells):
            if any(v in g.cell_nodes(c) for c in cells):
                s.add(w)
        assert tuple(sorted(s)) == m.neigh[d]


def test_objects_partition_interface():
    p = inputs.manufactured_sphere(0)
    m = M.Mesh(p)
    for variant in ("std", "v1"):
        objs = m.objects(variant)
        seen = np.zeros(m.n_dof, int)
        for o in objs:
            seen[o["dofs"]] += 1
            assert all(m.neigh[d] == o["neigh"] for d in o["dofs"])
        assert np.array_equal(seen, m.is_gamma.astype(int))
    assert len(m.objects("v1")) > len(m.objects("std"))
