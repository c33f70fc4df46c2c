"""P3 Lagrange element on tetrahedra (oracle; test infrastructure only).

Sec. "Tetrahedral finite element method": continuous Lagrange elements of
order 3 on tetrahedra. The 20 nodes of a tet sit at barycentric points
alpha/3 with alpha a multi-index of total degree 3 (4 vertices, 2 per edge,
1 per face). The basis function of node alpha is the lattice Lagrange
polynomial prod_a prod_{j<alpha_a} (3 lambda_a - j) / (j + 1).
"""
from __future__ import annotations

import itertools

import numpy as np
from scipy.special import roots_jacobi, roots_legendre

DEG = 3

# multi-indices |alpha| = 3, fixed order (lexicographic, descending)
ALPHAS = np.array(sorted((a for a in itertools.product(range(4), repeat=4) if sum(a) == DEG),
                         reverse=True), dtype=np.int64)
NLOC = len(ALPHAS)  # 20


def _ell(m, t):
    """1D lattice factor prod_{j<m} (3t - j)/(j+1) and its derivative in t."""
    val = np.ones_like(t)
    der = np.zeros_like(t)
    for j in range(m):
        f = (DEG * t - j) / (j + 1)
        der = der * f + val * (DEG / (j + 1))
        val = val * f
    return val, der


def basis(lam):
    """phi [..., 20] at barycentric points lam [..., 4]."""
    out = np.ones(lam.shape[:-1] + (NLOC,))
    for i, al in enumerate(ALPHAS):
        for a in range(4):
            out[..., i] *= _ell(al[a], lam[..., a])[0]
    return out


def basis_dlam(lam):
    """d phi / d lambda_a [..., 20, 4] (lambda treated as independent)."""
    out = np.ones(lam.shape[:-1] + (NLOC, 4))
    for i, al in enumerate(ALPHAS):
        vals = [_ell(al[a], lam[..., a]) for a in range(4)]
        for a in range(4):
            d = vals[a][1].copy()
            for b in range(4):
                if b != a:
                    d = d * vals[b][0]
            out[..., i, a] = d
    return out


# ----------------------------------------------------------------------------
# Quadrature: Stroud conical-product rules (Gauss-Jacobi x Gauss-Jacobi x
# Gauss-Legendre on the collapsed cube), exact for degree 2n-1.
# ----------------------------------------------------------------------------
def _gj01(n, alpha):
    """n-point Gauss-Jacobi rule on [0,1] for weight (1-u)^alpha."""
    x, w = roots_jacobi(n, alpha, 0.0) if alpha > 0 else roots_legendre(n)
    return (1.0 + x) / 2.0, w / 2.0 ** (alpha + 1)


def tet_rule(n):
    """Barycentric points [q,4] and weights [q] on the reference tet
    (weights sum to its volume 1/6). Collapsed map x1 = u, x2 = v(1-u),
    x3 = w(1-u)(1-v), Jacobian (1-u)^2 (1-v)."""
    u, wu = _gj01(n, 2)
    v, wv = _gj01(n, 1)
    t, wt = _gj01(n, 0)
    U, V, T = np.meshgrid(u, v, t, indexing="ij")
    W = (wu[:, None, None] * wv[None, :, None] * wt[None, None, :]).ravel()
    x1 = U.ravel()
    x2 = (V * (1 - U)).ravel()
    x3 = (T * (1 - U) * (1 - V)).ravel()
    lam = np.stack([1 - x1 - x2 - x3, x1, x2, x3], axis=1)
    return lam, W


def tri_rule(n):
    """Barycentric points [q,3] and weights [q] on the reference triangle
    (weights sum to 1/2). Collapsed map x1 = u, x2 = v(1-u)."""
    u, wu = _gj01(n, 1)
    v, wv = _gj01(n, 0)
    U, V = np.meshgrid(u, v, indexing="ij")
    W = (wu[:, None] * wv[None, :]).ravel()
    x1 = U.ravel()
    x2 = (V * (1 - U)).ravel()
    return np.stack([1 - x1 - x2, x1, x2], axis=1), W


# ----------------------------------------------------------------------------
# Element geometry and matrices
# ----------------------------------------------------------------------------
def geometry(P):
    """P [4,3] vertex coordinates -> (|det J|, grad lambda [4,3])."""
    J = (P[1:] - P[0]).T  # columns P1-P0, P2-P0, P3-P0
    detJ = np.linalg.det(J)
    Jinv = np.linalg.inv(J)
    g = np.zeros((4, 3))
    g[1:] = Jinv  # row a-1 of J^{-1} is grad lambda_a
    g[0] = -g[1:].sum(axis=0)
    return abs(detJ), g


_REF_CACHE = {}


def _ref_tables(n):
    """Quadrature points, weights, basis values and lambda-derivatives on the
    reference tet (computed once per rule size)."""
    if n not in _REF_CACHE:
        lam, w = tet_rule(n)
        _REF_CACHE[n] = (lam, w, basis(lam), basis_dlam(lam))
    return _REF_CACHE[n]


def element_matrices(P, n=4):
    """Stiffness K_e = int grad phi_i . grad phi_j and mass
    M_e = int phi_i phi_j over the tet with vertices P (exact for n >= 4:
    integrands of degree 4 and 6)."""
    vol6, glam = geometry(P)
    lam, w, phi, dl = _ref_tables(n)     # phi [q,20], dl [q,20,4]
    gphi = dl @ glam                     # [q,20,3]
    K = vol6 * np.einsum("q,qid,qjd->ij", w, gphi, gphi)
    M = vol6 * np.einsum("q,qi,qj->ij", w, phi, phi)
    return K, M


def face_nodes(c):
    """Local node indices lying on the face opposite vertex c (alpha_c = 0)."""
    return np.nonzero(ALPHAS[:, c] == 0)[0]


def face_lambda(c, tri_lam):
    """Embed triangle barycentrics [q,3] into tet barycentrics [q,4] for the
    face opposite vertex c (face vertices in increasing local order)."""
    others = [a for a in range(4) if a != c]
    lam = np.zeros((len(tri_lam), 4))
    lam[:, others] = tri_lam
    return lam


def face_area_normal(P, c):
    """Area and outward unit normal of the face opposite local vertex c."""
    others = [a for a in range(4) if a != c]
    A, B, C = P[others]
    nrm = np.cross(B - A, C - A)
    area = 0.5 * np.linalg.norm(nrm)
    nrm = nrm / np.linalg.norm(nrm)
    if np.dot(nrm, P[c] - A) > 0:
        nrm = -nrm
    return area, nrm


def face_mass(P, c, n=4):
    """B_f = int_f phi_i phi_j over the face opposite vertex c, as a 20x20
    matrix on the element's nodes (exact for n >= 4)."""
    area, _ = face_area_normal(P, c)
    tl, w = tri_rule(n)
    phi = basis(face_lambda(c, tl))
    return 2.0 * area * np.einsum("q,qi,qj->ij", w, phi, phi)


def node_coords(P):
    """Physical coordinates [20,3] of the element's lattice nodes."""
    return (ALPHAS / DEG) @ P
