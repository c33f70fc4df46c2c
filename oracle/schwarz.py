"""Two-level ORAS preconditioner, applied exactly (oracle; test infrastructure).

Sec. "Domain decomposition preconditioner":

* Eq. oras: M1^{-1} = sum_i R_i^T D_i A_i^{-1} R_i, with R_i the Boolean
  restriction to the dofs of the overlapping subdomain Gamma_i, D_i the
  diagonal partition of unity, and A_i the local Helmholtz operator with
  absorbing (Robin) conditions on the subdomain interfaces.
* Eq. 2lvl: M^{-1} = M1^{-1} (I - A Q) + Q, Q = Z E^{-1} Z^T, E = Z^T A Z,
  Z^T the interpolation between the fine P3 space on Gamma and the P3 space
  on a coarse mesh Gamma_H.
* The coarse problem is solved by 10 GMRES iterations preconditioned by
  one-level ORAS on the coarse mesh, with the same spatial partition.

Readings where the text is silent (the library follows the same ones):
overlap = the non-overlapping element set plus every element that shares a
mesh vertex with it (one layer; `overlap` layers repeat the rule); D_i is Boolean ownership by the lowest-index
non-overlapping subdomain whose elements carry the dof; A_i is assembled
over the elements of Gamma_i with -i omega sqrt(m_e) B_f on physical Robin
faces and on faces of the boundary of Gamma_i interior to Omega, and keeps
the physical Dirichlet rows; the coarse space drops coarse Dirichlet dofs;
the coarse element partition is that of the fine element holding the coarse
element's centroid (lowest subdomain on ties); coarse velocity is the
volume-weighted mean of fine squared slowness; the inner coarse GMRES is
right-preconditioned, zero initial guess, one Krylov space per column.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.spatial import cKDTree

from . import assemble as oa
from . import p3


def overlap_elements(tets, part, i, layers=1):
    """Elements of part i grown by `layers` element layers: each layer adds
    every element that shares a vertex with the current set."""
    tets = np.asarray(tets)
    inset = np.asarray(part) == i
    for _ in range(layers):
        verts = np.zeros(tets.max() + 1, dtype=bool)
        verts[tets[inset].ravel()] = True
        inset = verts[tets].any(axis=1)
    return np.nonzero(inset)[0]


def ownership(space, part, nparts):
    """owner[j] = lowest subdomain index whose own elements carry dof j."""
    owner = np.full(space.n, nparts, dtype=np.int64)
    for e in range(len(space.tets)):
        g = space.l2g[e]
        owner[g] = np.minimum(owner[g], part[e])
    return owner


def local_matrix(space, velocity, freq, elems, bfaces, btags, dir_dofs):
    """(dofs, A_i): Robin on physical Robin faces and on interior interface
    faces of the element set, identity rows at the global Dirichlet dofs
    (`dir_dofs`) that the element set carries."""
    omega = 2.0 * np.pi * freq
    m = 1.0 / np.asarray(velocity, dtype=np.float64) ** 2
    dofs = np.unique(space.l2g[elems].ravel())
    loc = -np.ones(space.n, dtype=np.int64)
    loc[dofs] = np.arange(len(dofs))
    inset = np.zeros(len(space.tets), dtype=bool)
    inset[elems] = True
    rows, cols, vals = [], [], []

    def add(e, Mat):
        g = loc[space.l2g[e]]
        rows.append(np.repeat(g, p3.NLOC))
        cols.append(np.tile(g, p3.NLOC))
        vals.append(Mat.ravel().astype(np.complex128))

    for e in elems:
        K, M = p3.element_matrices(space.xyz[space.tets[e]])
        add(e, K - omega ** 2 * m[e] * M)
    # faces of the element set's boundary
    owner = space.face_owner()
    phys = {}
    for f, t in zip(np.asarray(bfaces), btags):
        phys[tuple(sorted(int(x) for x in f))] = int(t)
    for e in elems:
        v = space.tets[e]
        for c in range(4):
            key = tuple(sorted(int(v[a]) for a in range(4) if a != c))
            nb = [ee for ee, _ in owner[key] if ee != e]
            if nb:                                   # interior face of Omega
                if inset[nb[0]]:
                    continue
                tag = oa.ROBIN                       # interface: absorbing
            else:
                tag = phys.get(key, None)            # exterior face
                if tag is None:
                    continue                         # natural (Neumann)
            if tag == oa.ROBIN:
                add(e, -1j * omega * np.sqrt(m[e]) * p3.face_mass(space.xyz[v], c))
    Ai = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(len(dofs), len(dofs))).tocsr()
    dloc = loc[np.asarray(dir_dofs, dtype=np.int64)]
    Ai, _ = oa.apply_dirichlet(Ai, None, dloc[dloc >= 0])
    return dofs, Ai


class OneLevelORAS:
    """Eq. oras with exact local solves (SuperLU)."""

    def __init__(self, space, velocity, freq, bfaces, btags, part, nparts, overlap=1):
        part = np.asarray(part)
        self.n = space.n
        owner = ownership(space, part, nparts)
        dd = space.dirichlet_dofs(bfaces, btags)
        self.subs = []
        for i in range(nparts):
            elems = overlap_elements(space.tets, part, i, overlap)
            dofs, Ai = local_matrix(space, velocity, freq, elems, bfaces, btags, dd)
            Di = (owner[dofs] == i).astype(np.float64)
            self.subs.append((dofs, Di, Ai, spla.splu(Ai.tocsc())))

    def apply(self, v):
        """v [n] or [n, s] -> sum_i R_i^T D_i A_i^{-1} R_i v."""
        v = np.asarray(v, dtype=np.complex128)
        out = np.zeros_like(v)
        for dofs, Di, _, lu in self.subs:
            y = lu.solve(np.ascontiguousarray(v[dofs]))
            out[dofs] += (Di[:, None] * y) if y.ndim == 2 else Di * y
        return out


def locate_points(space_c, pts, tol=1e-9):
    """For each point: (coarse element, barycentrics) of the lowest-index
    coarse element that contains it."""
    xyz, tets = space_c.xyz, space_c.tets
    P = xyz[tets]                                   # [nc,4,3]
    cent = P.mean(axis=1)
    rad = np.linalg.norm(P - cent[:, None, :], axis=2).max(axis=1)
    tree = cKDTree(pts)
    elem = np.full(len(pts), -1, dtype=np.int64)
    lam_out = np.zeros((len(pts), 4))
    for e in range(len(tets)):
        idx = np.array(tree.query_ball_point(cent[e], rad[e] * (1 + 1e-9)), dtype=np.int64)
        if len(idx) == 0:
            continue
        idx = idx[elem[idx] < 0]
        if len(idx) == 0:
            continue
        J = (P[e, 1:] - P[e, 0]).T
        l123 = np.linalg.solve(J, (pts[idx] - P[e, 0]).T).T
        lam = np.concatenate([1.0 - l123.sum(axis=1, keepdims=True), l123], axis=1)
        ok = lam.min(axis=1) >= -tol
        elem[idx[ok]] = e
        lam_out[idx[ok]] = lam[ok]
    if (elem < 0).any():
        raise ValueError("%d points lie outside the coarse mesh" % (elem < 0).sum())
    return elem, lam_out


def interpolation(space_f, space_c, keep_c):
    """Z [n_f, n_keep]: coarse P3 basis (columns = coarse dofs in keep_c)
    evaluated at the fine P3 nodes."""
    elem, lam = locate_points(space_c, space_f.coords)
    phi = p3.basis(lam)                            # [n_f, 20]
    col = -np.ones(space_c.n, dtype=np.int64)
    col[keep_c] = np.arange(len(keep_c))
    rows = np.repeat(np.arange(space_f.n), p3.NLOC)
    cols = col[space_c.l2g[elem]].ravel()
    vals = phi.ravel()
    ok = (cols >= 0) & (np.abs(vals) > 1e-14)
    return sp.csr_matrix((vals[ok], (rows[ok], cols[ok])), shape=(space_f.n, len(keep_c)))


def coarse_partition_and_velocity(space_f, space_c, part_f, velocity_f):
    """Coarse element subdomain (fine part at the coarse centroid, lowest on
    ties) and coarse velocity (volume-weighted mean of fine m = 1/v^2 over
    the fine elements whose centroid lies in the coarse element)."""
    Pc = space_c.xyz[space_c.tets]
    cc = Pc.mean(axis=1)
    # parts of fine elements containing each coarse centroid (ties -> lowest)
    Pf = space_f.xyz[space_f.tets]
    fc = Pf.mean(axis=1)
    rf = np.linalg.norm(Pf - fc[:, None, :], axis=2).max(axis=1)
    tree = cKDTree(fc)
    part_c = np.empty(len(cc), dtype=np.int64)
    for e, x in enumerate(cc):
        best = None
        for f in tree.query_ball_point(x, rf.max() * (1 + 1e-9)):
            lam = oa.barycentric(Pf[f], x)
            if lam.min() >= -1e-9:
                best = part_f[f] if best is None else min(best, part_f[f])
        part_c[e] = best
    m_f = 1.0 / np.asarray(velocity_f) ** 2
    vol_f = np.abs(np.linalg.det(Pf[:, 1:] - Pf[:, :1])) / 6.0
    ef, _ = locate_points(space_c, fc)
    msum = np.bincount(ef, weights=m_f * vol_f, minlength=len(cc))
    vsum = np.bincount(ef, weights=vol_f, minlength=len(cc))
    return part_c, 1.0 / np.sqrt(msum / vsum)


def gmres_fixed(apply_A, apply_M, b, iters):
    """`iters` steps of right-preconditioned GMRES from x0 = 0 for one
    column (Arnoldi with modified Gram-Schmidt, least squares by lstsq);
    stops early at an exact (happy) breakdown."""
    beta = np.linalg.norm(b)
    if beta == 0.0:
        return np.zeros_like(b)
    V = [b / beta]
    Zs = []
    H = np.zeros((iters + 1, iters), dtype=np.complex128)
    k = 0
    for j in range(iters):
        z = apply_M(V[j])
        Zs.append(z)
        w = apply_A(z)
        for i in range(j + 1):
            H[i, j] = np.vdot(V[i], w)
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        k = j + 1
        if H[j + 1, j] <= 1e-14 * beta:
            break
        V.append(w / H[j + 1, j])
    e1 = np.zeros(k + 1, dtype=np.complex128)
    e1[0] = beta
    y = np.linalg.lstsq(H[: k + 1, :k], e1, rcond=None)[0]
    return np.stack(Zs[:k], axis=1) @ y


class TwoLevel:
    """Eq. 2lvl on top of Eq. oras; coarse solve exact ('direct') or by
    `inner_its` GMRES iterations with coarse one-level ORAS ('gmres')."""

    def __init__(self, prob, coarse_mode="gmres", inner_its=10, overlap=1):
        fine, coarse = prob["fine"], prob["coarse"]
        self.space = oa.P3Space(fine["xyz"], fine["tets"])
        A, dd = oa.assemble(self.space, prob["velocity"], prob["freq"], fine["bfaces"], fine["btags"])
        self.A, _ = oa.apply_dirichlet(A, None, dd)
        self.fine_oras = OneLevelORAS(self.space, prob["velocity"], prob["freq"], fine["bfaces"],
                                      fine["btags"], prob["elem_part"], prob["nparts"], overlap)
        self.mode = coarse_mode
        self.inner_its = inner_its
        if coarse_mode == "none":
            return
        self.space_c = oa.P3Space(coarse["xyz"], coarse["tets"])
        dd_c = self.space_c.dirichlet_dofs(coarse["bfaces"], coarse["btags"])
        keep = np.setdiff1d(np.arange(self.space_c.n), dd_c)
        self.keep_c = keep
        self.Z = interpolation(self.space, self.space_c, keep)
        self.E = (self.Z.T @ self.A @ self.Z).tocsc()
        self.E_lu = spla.splu(self.E)
        part_c, vel_c = coarse_partition_and_velocity(self.space, self.space_c, prob["elem_part"],
                                                      prob["velocity"])
        self.part_c, self.vel_c = part_c, vel_c
        oras_c = OneLevelORAS(self.space_c, vel_c, prob["freq"], coarse["bfaces"], coarse["btags"],
                              part_c, prob["nparts"], overlap)
        self.coarse_oras = oras_c

    def coarse_apply_M(self, rH):
        """Coarse one-level ORAS on the kept coarse dofs."""
        full = np.zeros(self.space_c.n, dtype=np.complex128)
        full[self.keep_c] = rH
        return self.coarse_oras.apply(full)[self.keep_c]

    def coarse_solve(self, rH):
        if self.mode == "direct":
            return self.E_lu.solve(rH)
        return gmres_fixed(lambda x: self.E @ x, self.coarse_apply_M, rH, self.inner_its)

    def apply(self, v):
        """M^{-1} v for v [n] (Eq. 2lvl)."""
        v = np.asarray(v, dtype=np.complex128)
        if self.mode == "none":
            return self.fine_oras.apply(v)
        q = self.Z @ self.coarse_solve(self.Z.T @ v)
        return self.fine_oras.apply(v - self.A @ q) + q
