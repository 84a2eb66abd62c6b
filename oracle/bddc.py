"""BDDC preconditioner for unfitted meshes (oracle; test infrastructure only).

Follows Sect. 3 and Sect. 4 in the paper's own terms:

  * sub-assembled space: local Neumann matrices A^w over the active cells of
    each subdomain w (Sect. 3.1);
  * coarse DOFs: mean values alpha_lambda^w(v) = mean of v over the DOFs of
    each object lambda in Lambda_O(w)  (Eq. coarse-dofs; the "integral" is read
    as the uniform nodal mean, reading R10);
  * BDDC operator A~ = Galerkin projection of A onto V~ (functions whose coarse
    DOFs agree across neigh(lambda)); its inverse is applied through the
    standard split into local constrained Neumann problems plus a coarse
    problem on the energy-minimising coarse basis Phi^w, each local problem
    solved as the saddle-point system [A^w C^wT; C^w 0] (reading R11);
  * weighting W: topological (Eq. weighting) or stiffness-based (Eq. alge-weighting);
  * harmonic extension E = I - I0 A0^-1 I0^T A with A0 the interior (bubble)
    problems, and Q = E W (Sect. 3.3);
  * preconditioner M = I0 A0^-1 I0^T + Q A~^-1 Q^T   (Eq. bddc).

Parity: pinned by one-subdomain and all-corner BDDC reproducing A^-1, C Phi = I,
the partition of unity of the weights, symmetry of M, lambda_min(M A) = 1
(Sect. 3.4 proof) from dense eigenvalues, and the same A~^-1 obtained by brute
force from an explicit basis of V~ on tiny meshes (tests/test_oracle_bddc.py).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .mesh import coarse_objects


class SingularLocal(Exception):
    pass


def object_rows(obj, grid, mesh, ncomp):
    """Coarse DOFs of one object as rows over its (node DOF, component) pairs.

    Poisson (ncomp = 1): the uniform nodal mean (Eq. coarse-dofs, reading R10).
    Elasticity (ncomp = 3, reading R20): the mean of each component, and for
    objects of several nodes the mean rotation moments (1/n) sum (y x u)_k, y the
    node position relative to the object's centroid in grid units; row k is
    dropped when every node has the same coordinates k+1 and k+2 (an object on a
    grid line along axis k, for which the row vanishes), so corners carry 3 rows,
    edges 5 and faces 6.  Returns a list of dicts {(node_dof, comp): weight}."""
    nodes = [int(d) for d in obj["dofs"]]
    n = len(nodes)
    rows = []
    for c in range(ncomp):
        rows.append({(d, c): 1.0 / n for d in nodes})
    if ncomp == 1 or n == 1:
        return rows
    ijk = np.array([grid.node_ijk(int(mesh.node_of_dof[d])) for d in nodes], dtype=np.float64)
    y = ijk - ijk.mean(axis=0)
    for k in range(3):
        k1, k2 = (k + 1) % 3, (k + 2) % 3
        if np.all(ijk[:, k1] == ijk[0, k1]) and np.all(ijk[:, k2] == ijk[0, k2]):
            continue
        row = {}
        for t, d in enumerate(nodes):
            # (y x u)_k = y_k1 u_k2 - y_k2 u_k1
            row[(d, k2)] = row.get((d, k2), 0.0) + y[t, k1] / n
            row[(d, k1)] = row.get((d, k1), 0.0) - y[t, k2] / n
        rows.append(row)
    return rows


def stiffness_weights(mesh, integ):
    """Eq. alge-weighting per interface DOF d: {w: A^w_dd / sum_w' A^w'_dd} over neigh(d),
    A^w_dd the diagonal of the local Neumann matrix (sum over the active cells of w that
    contain the node)."""
    g = mesh.grid
    diag = {}
    for w in range(mesh.n_sub):
        for c in mesh.sub_cells[w]:
            Ke = integ.stiffness(c)
            for a, v in enumerate(g.cell_nodes(c)):
                d = int(mesh.dof_of_node[v])
                if d >= 0 and mesh.is_gamma[d]:
                    diag[(d, w)] = diag.get((d, w), 0.0) + Ke[a, a]
    out = {}
    for d in np.flatnonzero(mesh.is_gamma):
        tot = sum(diag[(int(d), w)] for w in mesh.neigh[d])
        out[int(d)] = {w: diag[(int(d), w)] / tot for w in mesh.neigh[d]}
    return out


class BDDC:
    def __init__(self, mesh, integ, system, weighting="stiffness", objects="v1", coarse="cef",
                 all_interface_corners=False):
        self.mesh = mesh
        self.system = system
        nc3 = getattr(system, "ncomp", 1)
        self.ncomp = nc3
        g = mesh.grid
        if all_interface_corners:
            # enlarged coarse space of Sect. 4.2: every interface DOF is a corner
            objs = [{"dofs": [d], "neigh": mesh.neigh[d], "kind": 0}
                    for d in np.flatnonzero(mesh.is_gamma)]
        elif objects == "v2":
            # Sect. 4.5: the edges are split by the stiffness weights of Eq. alge-weighting
            objs = coarse_objects(mesh.objects("v2", weights=stiffness_weights(mesh, integ)), coarse)
        else:
            objs = coarse_objects(mesh.objects(objects), coarse)
        self.objs = objs
        # coarse DOFs: the rows of every object, numbered object by object
        self.coarse_rows = []
        self.coarse_obj = []
        for k, o in enumerate(objs):
            for row in object_rows(o, g, mesh, nc3):
                self.coarse_rows.append(row)
                self.coarse_obj.append(k)
        self.n_coarse = len(self.coarse_rows)
        self.local = []
        constrained_nodes = set(np.flatnonzero(mesh.constrained).tolist())
        for w in range(mesh.n_sub):
            ndofs = mesh.sub_dofs[w]
            dofs = (nc3 * ndofs[:, None] + np.arange(nc3)[None, :]).ravel()
            pos = {int(d): i for i, d in enumerate(dofs)}
            n = dofs.size
            A = np.zeros((n, n))
            touches_constraint = False
            for c in mesh.sub_cells[w]:
                nodes = g.cell_nodes(c)
                Ke = integ.stiffness(c)
                li = []
                for v in nodes:
                    if v in constrained_nodes:
                        touches_constraint = True
                    d = mesh.dof_of_node[v]
                    for cc in range(nc3):
                        li.append(pos.get(int(nc3 * d + cc), -1) if d >= 0 else -1)
                for a in range(8 * nc3):
                    if li[a] < 0:
                        continue
                    for b in range(8 * nc3):
                        if li[b] >= 0:
                            A[li[a], li[b]] += Ke[a, b]
            gam = np.repeat(np.array([mesh.is_gamma[d] for d in ndofs], dtype=bool), nc3)
            I = np.flatnonzero(~gam)
            G = np.flatnonzero(gam)
            # coarse DOFs of this subdomain, in global coarse order
            cids = [k for k, ob in enumerate(self.coarse_obj) if w in objs[ob]["neigh"]]
            C = np.zeros((len(cids), n))
            for r, k in enumerate(cids):
                for (d, cc), val in self.coarse_rows[k].items():
                    C[r, pos[nc3 * d + cc]] = val
            if not touches_constraint and len(cids) == 0:
                raise SingularLocal(f"subdomain {w} floats and has no coarse DOF")
            nc = len(cids)
            KKT = np.zeros((n + nc, n + nc))
            KKT[:n, :n] = A
            KKT[:n, n:] = C.T
            KKT[n:, :n] = C
            kkt_lu = sla.lu_factor(KKT)
            rhs = np.zeros((n + nc, nc))
            rhs[n:, :] = np.eye(nc)
            Phi = sla.lu_solve(kkt_lu, rhs)[:n, :] if nc else np.zeros((n, 0))
            AII = A[np.ix_(I, I)]
            aii_chol = sla.cho_factor(AII) if I.size else None
            self.local.append(dict(dofs=dofs, A=A, I=I, G=G, C=C, cids=np.array(cids, dtype=np.int64),
                                   kkt_lu=kkt_lu, Phi=Phi, Ac=Phi.T @ A @ Phi, aii=aii_chol,
                                   diag=np.diag(A).copy()))
        # coarse matrix  A_c = sum_w R_cw^T (Phi^wT A^w Phi^w) R_cw
        Ac = np.zeros((self.n_coarse, self.n_coarse))
        for L in self.local:
            Ac[np.ix_(L["cids"], L["cids"])] += L["Ac"]
        self.Ac = Ac
        self.ac_chol = sla.cho_factor(Ac) if self.n_coarse else None
        # weights per (subdomain, local DOF)
        self.weighting = weighting
        n_dof = system.n
        if weighting == "stiffness":
            denom = np.zeros(n_dof)
            for L in self.local:
                denom[L["dofs"]] += L["diag"]
            for L in self.local:
                L["w"] = L["diag"] / denom[L["dofs"]]
        elif weighting == "topological":
            for L in self.local:
                L["w"] = np.array([1.0 / len(mesh.neigh[d // nc3]) for d in L["dofs"]])
        else:
            raise ValueError(weighting)

    # -- pieces of Eq. bddc --------------------------------------------------
    def interior_solve(self, r):
        """I0 A0^-1 I0^T r: independent Dirichlet problems on the interior DOFs."""
        z = np.zeros_like(r)
        for L in self.local:
            if L["I"].size:
                idx = L["dofs"][L["I"]]
                z[idx] = sla.cho_solve(L["aii"], r[idx])
        return z

    def weight_T(self, s):
        """W^T: global vector -> sub-assembled (list of local vectors)."""
        return [L["w"] * s[L["dofs"]] for L in self.local]

    def weight(self, u_loc):
        """W: sub-assembled -> global, weighted sum of the local values."""
        v = np.zeros(self.system.n)
        for L, u in zip(self.local, u_loc):
            v[L["dofs"]] += L["w"] * u
        return v

    def bddc_solve(self, r_loc, coarse_solve=None):
        """A~^-1 on the BDDC space: local constrained Neumann + coarse correction.
        coarse_solve (optional) replaces the exact A_c^-1 (a multilevel method)."""
        out = []
        rc = np.zeros(self.n_coarse)
        for L, r in zip(self.local, r_loc):
            n = L["dofs"].size
            nc = L["cids"].size
            rhs = np.concatenate([r, np.zeros(nc)])
            out.append(sla.lu_solve(L["kkt_lu"], rhs)[:n])
            if nc:
                rc[L["cids"]] += L["Phi"].T @ r
        if coarse_solve is not None:
            uc = coarse_solve(rc)
        else:
            uc = sla.cho_solve(self.ac_chol, rc) if self.n_coarse else rc
        for k, L in enumerate(self.local):
            if L["cids"].size:
                out[k] = out[k] + L["Phi"] @ uc[L["cids"]]
        return out

    def harmonic_extension(self, v):
        """E v = v - I0 A0^-1 I0^T A v."""
        return v - self.interior_solve(self.system.apply(v))

    def apply(self, r, coarse_solve=None):
        """z = M r with M = I0 A0^-1 I0^T + E W A~^-1 W^T E^T (Eq. bddc)."""
        z0 = self.interior_solve(r)
        s = r - self.system.apply(z0)                 # E^T r
        u_loc = self.bddc_solve(self.weight_T(s), coarse_solve)
        return z0 + self.harmonic_extension(self.weight(u_loc))

    # -- diagnostics ------------------------------------------------------------
    def weight_sums(self):
        tot = np.zeros(self.system.n)
        for L in self.local:
            tot[L["dofs"]] += L["w"]
        return tot

    def dense_preconditioner(self):
        n = self.system.n
        M = np.zeros((n, n))
        for j in range(n):
            e = np.zeros(n)
            e[j] = 1.0
            M[:, j] = self.apply(e)
        return M
