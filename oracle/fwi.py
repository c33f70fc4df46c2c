"""Full-waveform-inversion misfit and its gradient (oracle; test infrastructure).

The paper's solver is the forward engine of frequency-domain FWI
(Sec. "Introduction", abstract) but prints no gradient formula. Reading used
(both sides): per-element squared slowness m_e, receivers sampled by the P3
interpolation P (u at a point = sum_j phi_j(x) u_j), least-squares misfit

    chi(m) = 1/2 sum_s sum_k |(P u_s)_k - d_{s,k}|^2,   A(m) u_s = F_s,

and, since A is complex symmetric (A = A^T), the adjoint state

    A lambda_s = P^T conj(r_s),   r_s = P u_s - d_s,

gives  d chi / d m_e = -Re sum_s lambda_s^T (dA/dm_e) u_s  with, on the
element's dofs, dA/dm_e = -omega^2 M_e - (i omega / (2 sqrt(m_e))) sum over
the element's Robin faces of B_f (Dirichlet rows and columns are constant).
Pinned by central finite differences of chi (forward solves only).
"""
from __future__ import annotations

import numpy as np

from . import assemble as oa
from . import p3


def receiver_matrix(space, xyz):
    """Dense P [nr, n]: row k holds phi_j(x_k) in the lowest-index element
    containing x_k (same rule as the point-source load, so P^T a is the load
    of sources of amplitudes a at the receivers)."""
    return oa.point_source(space, xyz, np.ones(len(xyz))).real


def forward(mesh, m, freq, src_xyz):
    """(space, A, U [ns, n], Dirichlet dofs) for the squared slowness m."""
    space = oa.P3Space(mesh["xyz"], mesh["tets"])
    A, dd = oa.assemble(space, 1.0 / np.sqrt(m), freq, mesh["bfaces"], mesh["btags"])
    F = oa.point_source(space, src_xyz, np.ones(len(src_xyz)))
    A, F = oa.apply_dirichlet(A, F, dd)
    U = oa.solve(A, F)
    return space, A, U, dd


def misfit(mesh, m, freq, src_xyz, P, d_obs):
    _, _, U, _ = forward(mesh, m, freq, src_xyz)
    r = U @ P.T - d_obs
    return 0.5 * float(np.sum(np.abs(r) ** 2))


def gradient(mesh, m, freq, src_xyz, P, d_obs):
    """(chi, g [ne]) by the adjoint-state method."""
    space, A, U, dd = forward(mesh, m, freq, src_xyz)
    r = U @ P.T - d_obs                          # [ns, nr]
    chi = 0.5 * float(np.sum(np.abs(r) ** 2))
    Fa = np.conj(r) @ P                          # [ns, n]: P^T conj(r)
    Fa[:, dd] = 0.0
    Lam = oa.solve(A, Fa)
    omega = 2.0 * np.pi * freq
    keep = np.ones(space.n)
    keep[dd] = 0.0
    g = np.zeros(len(space.tets))
    robin = {}
    for (e, c), t in zip(space.locate_faces(mesh["bfaces"]), mesh["btags"]):
        if t == oa.ROBIN:
            robin.setdefault(e, []).append(c)
    for e, v in enumerate(space.tets):
        P_e = space.xyz[v]
        _, M = p3.element_matrices(P_e)
        dA = (-omega ** 2 * M).astype(np.complex128)
        for c in robin.get(e, []):
            dA += -1j * omega / (2.0 * np.sqrt(m[e])) * p3.face_mass(P_e, c)
        dofs = space.l2g[e]
        mask = keep[dofs]
        dA = dA * mask[:, None] * mask[None, :]
        g[e] = -np.real(np.einsum("si,ij,sj->", Lam[:, dofs], dA, U[:, dofs]))
    return chi, g
