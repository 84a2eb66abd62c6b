"""Three-level BDDC (oracle; test infrastructure only: the product never imports it).

The paper's conclusions (Sect. 6) point to multilevel BDDC for problems whose coarse
problem outgrows one factorisation, without defining it.  The reading taken here
(reading R26): the coarse problem of the two-level method (Sect. 3.3),

    A_c = sum_w R_cw^T A_c^w R_cw,    A_c^w = Phi^wT A^w Phi^w,

is itself a sub-assembled problem whose "elements" are the subdomains and whose DOFs
are the coarse DOFs.  The three-level method replaces the exact A_c^-1 in Eq. bddc by
one application of BDDC to that problem, built the way Sect. 3 builds the first level:

  * level-2 subdomains: the subdomains grouped G x G x G blocks at a time; inside a
    group, the connected components under "hold a common coarse DOF" (as Sect. 2.1
    splits a block into the components of its cells), numbered by smallest member;
  * neigh_2(k) of coarse DOF k: the level-2 subdomains holding a subdomain that holds
    k; the level-2 interface is {k : |neigh_2(k)| >= 2};
  * level-2 objects: interface coarse DOFs with equal neigh_2, split into connected
    components under "held by a common subdomain"; FACE when |neigh_2| = 2, else
    CORNER for one coarse DOF and EDGE for more (the rule of Sect. 3.2); Lambda_O
    by 'c' / 'ce' / 'cef'; with level1_corners, every coarse DOF of a first-level
    corner is a level-2 corner of its own (the corner enrichment of Sect. 4.4 is
    not averaged away one level up);
  * level-2 coarse DOFs: the uniform mean over each object (Eq. coarse-dofs);
  * weights: stiffness (Eq. alge-weighting on the diagonals of the level-2 Neumann
    matrices A_2^J = sum_{w in J} A_c^w) or topological (1 / |neigh_2|);
  * level-3 problem: A_3 = sum_J R_3J^T Phi_2^JT A_2^J Phi_2^J R_3J, solved exactly.

For elasticity a first-level object carries several coarse DOFs (reading R20: the
mean of each displacement component, then rotation moments about the kept axes);
the classes are then also split by that type, so that a level-2 coarse DOF is the
mean of one kind of first-level coarse DOF (a displacement component, or a rotation
moment about one axis) over the object.  With M_2 the level-2 BDDC preconditioner of
A_c (Eq. bddc one level up), the three-level preconditioner is Eq. bddc with
u_c = M_2 r_c.

Pinned in tests/test_oracle_multilevel.py: one level-2 subdomain and the all-corner
level-2 space both give M_2 = A_c^-1 (hence the two-level M); the level-2 objects of
a full box counted by hand; C_2 Phi_2 = I; the weights' partition of unity; symmetry
of M_2; lambda_min(M_2 A_c) >= 1 (the Sect. 3.4 argument one level up) and the
eigenvalues of M_3 A bounding those of M A from above in order.
"""
from __future__ import annotations

from collections import deque

import numpy as np
import scipy.linalg as sla

from .bddc import SingularLocal
from .mesh import CORNER, EDGE, FACE, _components


def subdomain_blocks(mesh):
    """Block of each subdomain (every cell of a subdomain lies in one block)."""
    return np.array([mesh.grid.block_of_cell(int(cells[0])) for cells in mesh.sub_cells], dtype=np.int64)


def coarse_dof_types(two):
    """Type of every first-level coarse DOF: its displacement component c (0..2; 0 for
    Poisson), or 3 + k for a rotation moment about axis k (its row involves the two
    components other than k)."""
    out = []
    for row in two.coarse_rows:
        comps = sorted({c for (_, c) in row})
        out.append(comps[0] if len(comps) == 1 else 3 + ({0, 1, 2} - set(comps)).pop())
    return out


def group_of_block(grid, b, G):
    """Group (G x G x G blocks) of block b, groups numbered x fastest."""
    nb = grid.nb
    bi, bj, bk = b % nb[0], (b // nb[0]) % nb[1], b // (nb[0] * nb[1])
    gx, gy = -(-int(nb[0]) // G), -(-int(nb[1]) // G)
    return int(bi // G + gx * (bj // G + gy * (bk // G)))


class CoarseBDDC:
    """BDDC of the coarse problem of a two-level oracle BDDC (level 2 of the method)."""

    def __init__(self, two, group=2, coarse="cef", weighting="stiffness", all_interface_corners=False,
                 level1_corners=False):
        mesh = two.mesh
        self.Ac = two.Ac
        nsub, nc = mesh.n_sub, two.n_coarse
        self.n = nc
        cids = [np.asarray(L["cids"], dtype=np.int64) for L in two.local]
        holders = [[] for _ in range(nc)]
        for w in range(nsub):
            for k in cids[w]:
                holders[int(k)].append(w)
        blocks = subdomain_blocks(mesh)
        grp = [group_of_block(mesh.grid, int(b), group) for b in blocks]
        # level-2 subdomains: components of each group under "hold a common coarse DOF"
        J_of = -np.ones(nsub, dtype=np.int64)
        members = []
        for w0 in range(nsub):
            if J_of[w0] >= 0:
                continue
            J = len(members)
            comp = [w0]
            J_of[w0] = J
            queue = deque([w0])
            while queue:
                w = queue.popleft()
                for k in cids[w]:
                    for w2 in holders[int(k)]:
                        if J_of[w2] < 0 and grp[w2] == grp[w0]:
                            J_of[w2] = J
                            comp.append(w2)
                            queue.append(w2)
            members.append(sorted(comp))
        self.J_of = J_of
        self.members = members
        self.n_sub2 = len(members)
        self.neigh2 = [tuple(sorted({int(J_of[w]) for w in holders[k]})) for k in range(nc)]
        gamma = np.array([len(ns) >= 2 for ns in self.neigh2], dtype=bool)
        self.is_gamma = gamma

        # level-2 objects
        def adjacent(k):
            out = set()
            for w in holders[k]:
                out.update(int(x) for x in cids[w])
            return out

        if all_interface_corners:
            objs = [{"dofs": [int(k)], "neigh": self.neigh2[k], "kind": CORNER} for k in np.flatnonzero(gamma)]
        else:
            classes = {}
            kind1 = [two.objs[o]["kind"] for o in two.coarse_obj]
            types = coarse_dof_types(two)
            for k in np.flatnonzero(gamma):
                if level1_corners and kind1[k] == CORNER:
                    classes.setdefault(("corner", int(k)), []).append(int(k))
                else:
                    classes.setdefault((types[k],) + self.neigh2[k], []).append(int(k))
            objs = []
            for key, ks in classes.items():
                ns = self.neigh2[ks[0]]
                for comp in _components(sorted(ks), adjacent):
                    kind = FACE if len(ns) == 2 else (CORNER if len(comp) == 1 else EDGE)
                    if key[0] == "corner":
                        kind = CORNER
                    objs.append({"dofs": comp, "neigh": ns, "kind": kind})
            keep = {"c": (CORNER,), "ce": (CORNER, EDGE), "cef": (CORNER, EDGE, FACE)}[coarse]
            objs = [o for o in objs if o["kind"] in keep]
        objs.sort(key=lambda o: o["dofs"][0])
        self.objs = objs
        self.n_coarse = len(objs)

        # local level-2 problems
        self.local = []
        for J, mem in enumerate(members):
            dofs = np.array(sorted(set().union(*[set(int(x) for x in cids[w]) for w in mem])), dtype=np.int64)
            pos = {int(k): i for i, k in enumerate(dofs)}
            n = dofs.size
            A = np.zeros((n, n))
            for w in mem:
                p = [pos[int(k)] for k in cids[w]]
                A[np.ix_(p, p)] += two.local[w]["Ac"]
            I = np.flatnonzero(~gamma[dofs])
            G = np.flatnonzero(gamma[dofs])
            oids = [q for q, o in enumerate(objs) if J in o["neigh"]]
            C = np.zeros((len(oids), n))
            for r, q in enumerate(oids):
                for k in objs[q]["dofs"]:
                    C[r, pos[k]] = 1.0 / len(objs[q]["dofs"])
            m = len(oids)
            KKT = np.zeros((n + m, n + m))
            KKT[:n, :n] = A
            KKT[:n, n:] = C.T
            KKT[n:, :n] = C
            if m == 0:
                ev = np.linalg.eigvalsh(A)
                if ev[0] <= 1e-12 * ev[-1]:
                    raise SingularLocal(f"level-2 subdomain {J} floats and has no level-2 coarse DOF")
            kkt_lu = sla.lu_factor(KKT)
            rhs = np.zeros((n + m, m))
            rhs[n:, :] = np.eye(m)
            Phi = sla.lu_solve(kkt_lu, rhs)[:n, :] if m else np.zeros((n, 0))
            aii = sla.cho_factor(A[np.ix_(I, I)]) if I.size else None
            self.local.append(dict(dofs=dofs, A=A, I=I, G=G, C=C, cids=np.array(oids, dtype=np.int64),
                                   kkt_lu=kkt_lu, Phi=Phi, Ac=Phi.T @ A @ Phi, aii=aii, diag=np.diag(A).copy()))
        A3 = np.zeros((self.n_coarse, self.n_coarse))
        for L in self.local:
            A3[np.ix_(L["cids"], L["cids"])] += L["Ac"]
        self.A3 = A3
        self.a3_chol = sla.cho_factor(A3) if self.n_coarse else None
        if weighting == "stiffness":
            denom = np.zeros(nc)
            for L in self.local:
                denom[L["dofs"]] += L["diag"]
            for L in self.local:
                L["w"] = L["diag"] / denom[L["dofs"]]
        elif weighting == "topological":
            for L in self.local:
                L["w"] = np.array([1.0 / len(self.neigh2[k]) for k in L["dofs"]])
        else:
            raise ValueError(weighting)

    # -- Eq. bddc on A_c -----------------------------------------------------------
    def interior_solve(self, r):
        z = np.zeros_like(r)
        for L in self.local:
            if L["I"].size:
                idx = L["dofs"][L["I"]]
                z[idx] = sla.cho_solve(L["aii"], r[idx])
        return z

    def weight_T(self, s):
        return [L["w"] * s[L["dofs"]] for L in self.local]

    def weight(self, u_loc):
        v = np.zeros(self.n)
        for L, u in zip(self.local, u_loc):
            v[L["dofs"]] += L["w"] * u
        return v

    def bddc_solve(self, r_loc):
        out = []
        r3 = np.zeros(self.n_coarse)
        for L, r in zip(self.local, r_loc):
            n, m = L["dofs"].size, L["cids"].size
            out.append(sla.lu_solve(L["kkt_lu"], np.concatenate([r, np.zeros(m)]))[:n])
            if m:
                r3[L["cids"]] += L["Phi"].T @ r
        u3 = sla.cho_solve(self.a3_chol, r3) if self.n_coarse else r3
        for q, L in enumerate(self.local):
            if L["cids"].size:
                out[q] = out[q] + L["Phi"] @ u3[L["cids"]]
        return out

    def apply(self, r):
        """u_c = M_2 r_c = I0 A0^-1 I0^T r_c + E W A~_2^-1 W^T E^T r_c on A_c."""
        z0 = self.interior_solve(r)
        s = r - self.Ac @ z0
        v = self.weight(self.bddc_solve(self.weight_T(s)))
        return z0 + v - self.interior_solve(self.Ac @ v)

    def weight_sums(self):
        tot = np.zeros(self.n)
        for L in self.local:
            tot[L["dofs"]] += L["w"]
        return tot


class ThreeLevelBDDC:
    """Eq. bddc with the exact coarse solve replaced by the level-2 BDDC M_2."""

    def __init__(self, two, **kw):
        self.two = two
        self.level2 = CoarseBDDC(two, **kw)

    def apply(self, r):
        return self.two.apply(r, coarse_solve=self.level2.apply)
