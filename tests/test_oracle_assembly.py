"""Pins for the oracle's global assembly, boundary terms, sources and solve.

* Cubic manufactured solutions lie in the P3 space, so the Galerkin solution
  equals them to rounding (any dropped or mis-signed term of A or F breaks it),
  with all-Robin and with a Dirichlet top, on graded meshes with
  per-element velocity.
* A plane wave exp(i k d.x) with impedance data: L2 error falls as h^4.
* Dense LAPACK solve equals the sparse direct solve on tiny meshes.
* Point-source loads reproduce cubics: sum_j F_j p(x_j) = a p(x_s).
"""
import numpy as np
import pytest

from oracle import assemble as oa
from paper_2004_07930_gb300 import workloads as wl


def _graded(n, L, rng):
    d = rng.uniform(0.6, 1.4, size=n)
    return np.concatenate([[0.0], np.cumsum(d) / d.sum() * L])


def _cubic(c):
    """u(x) = sum c_m x^a y^b z^d (deg <= 3) with gradient and Laplacian, in km."""
    mons = [(a, b, d) for a in range(4) for b in range(4) for d in range(4) if a + b + d <= 3]

    def u(X):
        Y = X / 1000.0
        return sum(cm * Y[:, 0] ** a * Y[:, 1] ** b * Y[:, 2] ** d for cm, (a, b, d) in zip(c, mons))

    def grad(X):
        Y = X / 1000.0
        g = np.zeros(X.shape, dtype=complex)
        for cm, (a, b, d) in zip(c, mons):
            if a:
                g[:, 0] += cm * a * Y[:, 0] ** (a - 1) * Y[:, 1] ** b * Y[:, 2] ** d
            if b:
                g[:, 1] += cm * b * Y[:, 0] ** a * Y[:, 1] ** (b - 1) * Y[:, 2] ** d
            if d:
                g[:, 2] += cm * d * Y[:, 0] ** a * Y[:, 1] ** b * Y[:, 2] ** (d - 1)
        return g / 1000.0

    def lap(X):
        Y = X / 1000.0
        out = np.zeros(len(X), dtype=complex)
        for cm, (a, b, d) in zip(c, mons):
            if a > 1:
                out += cm * a * (a - 1) * Y[:, 0] ** (a - 2) * Y[:, 1] ** b * Y[:, 2] ** d
            if b > 1:
                out += cm * b * (b - 1) * Y[:, 0] ** a * Y[:, 1] ** (b - 2) * Y[:, 2] ** d
            if d > 1:
                out += cm * d * (d - 1) * Y[:, 0] ** a * Y[:, 1] ** b * Y[:, 2] ** (d - 2)
        return out / 1e6

    return mons, u, grad, lap


@pytest.mark.parametrize("top_dirichlet", [False, True])
def test_cubic_manufactured_solution_is_exact(top_dirichlet):
    rng = np.random.default_rng(10 + top_dirichlet)
    xs, ys, zs = _graded(3, 1000.0, rng), _graded(2, 800.0, rng), _graded(3, 700.0, rng)
    xyz, tets, hexes = wl.kuhn_grid(xs, ys, zs)
    bf, bt = wl.boundary_faces(xyz, tets, top_dirichlet)
    vel = rng.uniform(1500.0, 3000.0, size=len(tets))       # per-element wavespeed
    freq = 3.0
    omega = 2 * np.pi * freq
    m = 1.0 / vel ** 2
    nm = 20
    c = rng.standard_normal(nm) + 1j * rng.standard_normal(nm)
    mons, u, grad, lap = _cubic(c)
    if top_dirichlet:          # u = z * q(x,y,z), deg q <= 2: vanishes on z = 0
        mons2 = [(a, b, d) for a in range(3) for b in range(3) for d in range(3) if a + b + d <= 2]
        cz = np.zeros(nm, dtype=complex)
        for cm, (a, b, d) in zip(rng.standard_normal(len(mons2)), mons2):
            cz[mons.index((a, b, d + 1))] = cm
        c = cz
        mons, u, grad, lap = _cubic(c)

    space = oa.P3Space(xyz, tets)
    A, dd = oa.assemble(space, vel, freq, bf, bt)
    f = lambda X, e: -lap(X) - omega ** 2 * m[e] * u(X)
    g = lambda X, nrm, e: grad(X) @ nrm - 1j * omega * np.sqrt(m[e]) * u(X)
    F = oa.volume_load(space, f) + oa.robin_load(space, bf, bt, g)
    A, F = oa.apply_dirichlet(A, F, dd)
    uh = oa.solve(A, F)
    ui = u(space.coords)
    assert np.abs(uh - ui).max() <= 1e-9 * np.abs(ui).max()
    if top_dirichlet:
        assert len(dd) == (3 * 3 + 1) * (3 * 2 + 1)
        assert np.abs(uh[dd]).max() == 0.0


def test_plane_wave_h4_convergence():
    freq, v, L = 2.0, 2000.0, 1000.0
    k = 2 * np.pi * freq / v
    d = np.array([1.0, 2.0, 2.0]) / 3.0
    uex = lambda X: np.exp(1j * k * (X @ d))
    g = lambda X, nrm, e: 1j * k * (d @ nrm - 1.0) * uex(X)
    errs = []
    for nc in (2, 4, 8):
        grid = np.linspace(0.0, L, nc + 1)
        xyz, tets, _ = wl.kuhn_grid(grid, grid, grid)
        bf, bt = wl.boundary_faces(xyz, tets, False)
        space = oa.P3Space(xyz, tets)
        A, dd = oa.assemble(space, np.full(len(tets), v), freq, bf, bt)
        F = oa.robin_load(space, bf, bt, g)
        uh = oa.solve(A, F)
        e, nrm = oa.l2_error(space, uh, uex)
        errs.append(e / nrm)
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    print("relative L2 errors", errs, "ratios", r1, r2)
    assert errs[2] < 1e-3
    assert 13.0 < r2 < 19.0                      # h^4: 16 per halving
    assert r1 > 8.0


def test_dense_bruteforce_equals_sparse_solve():
    for nc in (1, 2):
        p = wl.cube_problem(ncell=nc, freq=2.0, v=2000.0, top_dirichlet=(nc == 2), coarse=False,
                            src=((300.0, 450.0, 600.0),))
        space, A, F = oa.system(p["fine"], p["velocity"], p["freq"], p["src_xyz"])
        assert space.n == (3 * nc + 1) ** 3
        u_sp = oa.solve(A, F)[0]
        u_de = np.linalg.solve(A.toarray(), F[0])
        np.testing.assert_allclose(u_sp, u_de, rtol=0, atol=1e-12 * np.abs(u_de).max())
        assert abs(A - A.T).max() <= 1e-14 * abs(A).max()


def test_point_source_reproduces_cubics():
    p = wl.cube_problem(ncell=3, coarse=False)
    space = oa.P3Space(p["fine"]["xyz"], p["fine"]["tets"])
    rng = np.random.default_rng(5)
    xs = rng.uniform(50.0, 950.0, size=(6, 3))
    xs[0] = [500.0, 500.0, 100.0]
    xs[1] = [1000.0 / 3, 1000.0 / 3, 1000.0 / 3]       # a mesh vertex
    amp = rng.standard_normal(6) + 1j * rng.standard_normal(6)
    F = oa.point_source(space, xs, amp)
    X = space.coords
    for _ in range(3):
        c = rng.standard_normal(20)
        _, u, _, _ = _cubic(c)
        np.testing.assert_allclose(F @ u(X), amp * u(xs), rtol=1e-11, atol=1e-12)
    # at a vertex the load is a unit nodal load
    j = np.argmin(np.linalg.norm(X - xs[1], axis=1))
    assert abs(F[1, j] - amp[1]) < 1e-12 and np.count_nonzero(np.abs(F[1]) > 1e-12) == 1


def test_cube_problem_counts():
    p = wl.cube_problem()
    assert p["fine"]["tets"].shape == (1296, 4)
    space, A, F = oa.system(p["fine"], p["velocity"], p["freq"], p["src_xyz"])
    assert space.n == 6859
    assert A.nnz == 299971
    nnz = np.diff(A.indptr)
    assert nnz.min() == 20 and nnz.max() == 175
    assert abs(A - A.T).max() <= 1e-12 * abs(A).max()
