"""Global P3 assembly and direct solve (oracle; test infrastructure only).

Sec. "Tetrahedral finite element method", Eq. eqh and Eq. eq1: the
Helmholtz equation with k = omega / c is written as the sparse system
A u = b. Reading of the sign and time convention (e^{-i omega t}): solve
-Lap u - k^2 u = s with first-order absorbing faces d_n u - i k u = g, so

    A = sum_e (K_e - omega^2 m_e M_e) - i omega sum_{Robin f} sqrt(m_e) B_f,
    F_j = int s phi_j + sum_{Robin f} int_f g phi_j,

with m_e = 1 / c_e^2 per element. Homogeneous Dirichlet nodes (free
surface) get an identity row and column and a zero right-hand side.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import p3

ROBIN = 0
DIRICHLET = 1


class P3Space:
    """Global P3 dofs of a tet mesh.

    A lattice node is identified by the multiset {(vertex, weight)} of its
    barycentric representation; equal keys in neighbouring elements are the
    same global dof.
    """

    def __init__(self, xyz, tets):
        self.xyz = np.asarray(xyz, dtype=np.float64)
        self.tets = np.asarray(tets, dtype=np.int64)
        ne = len(self.tets)
        keys = {}
        l2g = np.empty((ne, p3.NLOC), dtype=np.int64)
        coords = []
        for e in range(ne):
            v = self.tets[e]
            P = self.xyz[v]
            X = p3.node_coords(P)
            for i, al in enumerate(p3.ALPHAS):
                key = tuple(sorted((int(v[a]), int(al[a])) for a in range(4) if al[a] > 0))
                g = keys.get(key)
                if g is None:
                    g = len(keys)
                    keys[key] = g
                    coords.append(X[i])
                l2g[e, i] = g
        self.l2g = l2g
        self.coords = np.array(coords)
        self.n = len(coords)
        self._face_owner = None

    def face_owner(self):
        """sorted vertex triple -> (element, local opposite vertex)."""
        if self._face_owner is None:
            d = {}
            for e, v in enumerate(self.tets):
                for c in range(4):
                    key = tuple(sorted(int(v[a]) for a in range(4) if a != c))
                    d.setdefault(key, []).append((e, c))
            self._face_owner = d
        return self._face_owner

    def locate_faces(self, bfaces):
        owner = self.face_owner()
        out = []
        for f in np.asarray(bfaces):
            lst = owner[tuple(sorted(int(x) for x in f))]
            if len(lst) != 1:
                raise ValueError("face %s is not exterior" % (f,))
            out.append(lst[0])
        return out

    def dirichlet_dofs(self, bfaces, btags):
        dofs = set()
        for (e, c), t in zip(self.locate_faces(bfaces), btags):
            if t == DIRICHLET:
                dofs.update(self.l2g[e, p3.face_nodes(c)].tolist())
        return np.array(sorted(dofs), dtype=np.int64)


def assemble(space, velocity, freq, bfaces, btags):
    """Complex-symmetric CSR matrix A (before Dirichlet elimination) and the
    list of Dirichlet dofs."""
    omega = 2.0 * np.pi * freq
    m = 1.0 / np.asarray(velocity, dtype=np.float64) ** 2
    rows, cols, vals = [], [], []
    for e, v in enumerate(space.tets):
        K, M = p3.element_matrices(space.xyz[v])
        Ae = K - omega ** 2 * m[e] * M
        g = space.l2g[e]
        rows.append(np.repeat(g, p3.NLOC))
        cols.append(np.tile(g, p3.NLOC))
        vals.append(Ae.ravel().astype(np.complex128))
    for (e, c), t in zip(space.locate_faces(bfaces), btags):
        if t != ROBIN:
            continue
        B = p3.face_mass(space.xyz[space.tets[e]], c)
        g = space.l2g[e]
        rows.append(np.repeat(g, p3.NLOC))
        cols.append(np.tile(g, p3.NLOC))
        vals.append((-1j * omega * np.sqrt(m[e]) * B).ravel())
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(space.n, space.n)).tocsr()
    A.sum_duplicates()
    A.eliminate_zeros()
    dir_dofs = space.dirichlet_dofs(bfaces, btags)
    return A, dir_dofs


def apply_dirichlet(A, F, dir_dofs):
    """Identity rows/columns at Dirichlet dofs, zero right-hand side there."""
    n = A.shape[0]
    keep = np.ones(n)
    keep[dir_dofs] = 0.0
    Dk = sp.diags(keep)
    A = (Dk @ A @ Dk + sp.diags(1.0 - keep)).tocsr()
    A.eliminate_zeros()
    if F is not None:
        F = np.array(F, dtype=np.complex128, copy=True)
        F[..., dir_dofs] = 0.0
    return A, F


def barycentric(P, x):
    J = (P[1:] - P[0]).T
    l123 = np.linalg.solve(J, x - P[0])
    return np.concatenate([[1.0 - l123.sum()], l123])


def point_source(space, src_xyz, src_amp, tol=1e-10):
    """F [ns, n]: F_j = a phi_j(x_s), evaluated in the lowest-index element
    that contains x_s (continuity makes the choice immaterial)."""
    src_xyz = np.asarray(src_xyz, dtype=np.float64).reshape(-1, 3)
    src_amp = np.asarray(src_amp, dtype=np.complex128).reshape(-1)
    F = np.zeros((len(src_xyz), space.n), dtype=np.complex128)
    for s, (x, a) in enumerate(zip(src_xyz, src_amp)):
        for e, v in enumerate(space.tets):
            P = space.xyz[v]
            lo, hi = P.min(axis=0), P.max(axis=0)
            span = np.max(hi - lo)
            if np.any(x < lo - tol * span) or np.any(x > hi + tol * span):
                continue
            lam = barycentric(P, x)
            if lam.min() >= -tol:
                phi = p3.basis(lam[None, :])[0]
                np.add.at(F[s], space.l2g[e], a * phi)
                break
        else:
            raise ValueError("source %s outside the mesh" % (x,))
    return F


def volume_load(space, f, n=6):
    """F_j = int f phi_j with f(x [q,3], e) -> complex [q] on element e
    (exact when f phi_j has degree <= 2n-1)."""
    lam, w = p3.tet_rule(n)
    phi = p3.basis(lam)
    F = np.zeros(space.n, dtype=np.complex128)
    for e, v in enumerate(space.tets):
        P = space.xyz[v]
        vol6, _ = p3.geometry(P)
        X = lam @ P
        np.add.at(F, space.l2g[e], vol6 * ((w * f(X, e)) @ phi))
    return F


def robin_load(space, bfaces, btags, g, n=8):
    """F_j = sum over Robin faces of int_f g phi_j with g(x [q,3], normal [3], e)
    on the face of element e."""
    tl, w = p3.tri_rule(n)
    F = np.zeros(space.n, dtype=np.complex128)
    for (e, c), t in zip(space.locate_faces(bfaces), btags):
        if t != ROBIN:
            continue
        P = space.xyz[space.tets[e]]
        area, nrm = p3.face_area_normal(P, c)
        lam = p3.face_lambda(c, tl)
        phi = p3.basis(lam)
        X = lam @ P
        np.add.at(F, space.l2g[e], 2.0 * area * ((w * g(X, nrm, e)) @ phi))
    return F


def solve(A, F):
    """u = A^{-1} F (SuperLU, complex128); F [n] or [ns, n]."""
    lu = spla.splu(A.tocsc())
    F = np.asarray(F, dtype=np.complex128)
    if F.ndim == 1:
        return lu.solve(F)
    return lu.solve(F.T.copy()).T.copy()


def evaluate(space, u, e, lam):
    """u_h at barycentric points lam [q,4] of element e."""
    return p3.basis(lam) @ u[space.l2g[e]]


def l2_error(space, u, exact, n=6):
    """(||u_h - u_ex||_L2, ||u_ex||_L2) by a degree-(2n-1) tet rule."""
    lam, w = p3.tet_rule(n)
    phi = p3.basis(lam)
    err = 0.0
    nrm = 0.0
    for e, v in enumerate(space.tets):
        P = space.xyz[v]
        vol6, _ = p3.geometry(P)
        X = lam @ P
        ue = exact(X)
        uh = phi @ u[space.l2g[e]]
        err += vol6 * np.sum(w * np.abs(uh - ue) ** 2)
        nrm += vol6 * np.sum(w * np.abs(ue) ** 2)
    return np.sqrt(err), np.sqrt(nrm)


def system(mesh, velocity, freq, src_xyz=None, src_amp=None):
    """(space, A, F) for a mesh bundle: assembly, point sources, Dirichlet."""
    space = P3Space(mesh["xyz"], mesh["tets"])
    A, dd = assemble(space, velocity, freq, mesh["bfaces"], mesh["btags"])
    F = None
    if src_xyz is not None:
        amp = np.ones(len(src_xyz)) if src_amp is None else src_amp
        F = point_source(space, src_xyz, amp)
    A, F = apply_dirichlet(A, F, dd)
    return space, A, F


def match_dofs(coords_a, coords_b, scale):
    """Permutation p with coords_a[p] == coords_b, matching nearest points
    within 1e-6 * scale (nodes are h/3 apart, far above that)."""
    from scipy.spatial import cKDTree

    d, p = cKDTree(np.asarray(coords_a)).query(np.asarray(coords_b))
    if len(coords_a) != len(coords_b) or np.max(d, initial=0.0) > 1e-6 * scale \
            or len(np.unique(p)) != len(p):
        raise ValueError("dof coordinate sets differ")
    return p.astype(np.int64)
