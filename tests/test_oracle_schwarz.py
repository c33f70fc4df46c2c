"""Pins for the oracle's two-level ORAS operator (Eq. oras, Eq. 2lvl).

* The Boolean partition of unity sums to the identity.
* A_i equals the standalone assembly of the overlapping element set with
  Robin on every exterior face (so interfaces get the absorbing condition).
* One subdomain: M1^{-1} = A^{-1}. Coarse mesh = fine mesh: Q = A^{-1}, so
  M^{-1} = A^{-1}.
* Z reproduces global cubics exactly (nested P3 spaces).
* The fixed-step GMRES equals a brute-force least-squares minimiser over an
  explicitly built Krylov basis.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import assemble as oa
from oracle import schwarz as osw
from paper_2004_07930_gb300 import workloads as wl


def test_partition_of_unity_is_identity():
    p = wl.cube_problem(ncell=4, nparts_xyz=(2, 2, 2), coarse=False)
    sp_ = oa.P3Space(p["fine"]["xyz"], p["fine"]["tets"])
    R = osw.OneLevelORAS(sp_, p["velocity"], p["freq"], p["fine"]["bfaces"], p["fine"]["btags"],
                         p["elem_part"], p["nparts"])
    pu = np.zeros(sp_.n)
    cover = np.zeros(sp_.n)
    for dofs, Di, _, _ in R.subs:
        pu[dofs] += Di
        cover[dofs] += 1
    np.testing.assert_array_equal(pu, 1.0)
    assert cover.max() > 1            # subdomains overlap


@pytest.mark.parametrize("top_dirichlet", [False, True])
def test_local_matrix_is_standalone_robin_assembly(top_dirichlet):
    p = wl.cube_problem(ncell=4, nparts_xyz=(2, 2, 1), top_dirichlet=top_dirichlet, coarse=False)
    f = p["fine"]
    rng = np.random.default_rng(3)
    vel = rng.uniform(1800.0, 2600.0, size=len(f["tets"]))
    sp_ = oa.P3Space(f["xyz"], f["tets"])
    dd = sp_.dirichlet_dofs(f["bfaces"], f["btags"])
    for i in range(p["nparts"]):
        elems = osw.overlap_elements(f["tets"], p["elem_part"], i)
        dofs, Ai = osw.local_matrix(sp_, vel, p["freq"], elems, f["bfaces"], f["btags"], dd)
        # standalone mesh of the element set, every exterior face Robin
        sub_t = f["tets"][elems]
        vs, inv = np.unique(sub_t, return_inverse=True)
        sub_xyz = f["xyz"][vs]
        sub_t = inv.reshape(-1, 4)
        bf, _ = wl.boundary_faces(sub_xyz, sub_t, False)
        sub = oa.P3Space(sub_xyz, sub_t)
        B, _ = oa.assemble(sub, vel[elems], p["freq"], bf, np.zeros(len(bf), dtype=np.int32))
        perm = oa.match_dofs(sub.coords, sp_.coords[dofs], 1000.0)   # sub.coords[perm] == dofs coords
        B = B[perm][:, perm]
        is_dir = np.isin(dofs, dd)
        B, _ = oa.apply_dirichlet(B, None, np.nonzero(is_dir)[0])
        assert abs(Ai - B).max() <= 1e-12 * abs(B).max()
        if top_dirichlet:
            assert is_dir.any()


def test_single_subdomain_oras_is_exact_inverse():
    p = wl.cube_problem(ncell=3, nparts_xyz=(1, 1, 1), top_dirichlet=True, coarse=False)
    f = p["fine"]
    space, A, _ = oa.system(f, p["velocity"], p["freq"])
    M = osw.OneLevelORAS(space, p["velocity"], p["freq"], f["bfaces"], f["btags"], p["elem_part"], 1)
    v = wl.random_rhs(space.n, 2, 1).T
    np.testing.assert_allclose(A @ M.apply(v), v, atol=1e-10 * np.abs(v).max())


def test_coarse_equal_fine_gives_exact_inverse():
    p = wl.cube_problem(ncell=2, nparts_xyz=(2, 1, 1), top_dirichlet=True)
    p["coarse"] = dict(p["fine"])            # Z = I
    for mode in ("direct", "gmres"):
        T = osw.TwoLevel(p, coarse_mode=mode, inner_its=400)
        v = wl.random_rhs(T.space.n, 1, 2)[0]
        dd = T.space.dirichlet_dofs(p["fine"]["bfaces"], p["fine"]["btags"])
        v[dd] = 0.0
        z = T.apply(v)
        np.testing.assert_allclose(T.A @ z, v, atol=1e-8 * np.abs(v).max())


def test_interpolation_reproduces_cubics():
    p = wl.cube_problem(ncell=4, coarse=True)
    sf = oa.P3Space(p["fine"]["xyz"], p["fine"]["tets"])
    sc = oa.P3Space(p["coarse"]["xyz"], p["coarse"]["tets"])
    Z = osw.interpolation(sf, sc, np.arange(sc.n))
    rng = np.random.default_rng(7)
    c = rng.standard_normal(20)

    def cubic(X):
        Y = X / 1000.0
        mons = [Y[:, 0] ** a * Y[:, 1] ** b * Y[:, 2] ** d
                for a in range(4) for b in range(4) for d in range(4) if a + b + d <= 3]
        return np.stack(mons, axis=1) @ c

    np.testing.assert_allclose(Z @ cubic(sc.coords), cubic(sf.coords), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(np.asarray(Z.sum(axis=1)).ravel(), 1.0, atol=1e-13)


def test_gmres_fixed_is_krylov_minimiser():
    rng = np.random.default_rng(11)
    n, k = 40, 6
    A = np.eye(n) * 3 + rng.standard_normal((n, n)) * 0.4 + 1j * rng.standard_normal((n, n)) * 0.3
    Mi = np.eye(n) + 0.1 * rng.standard_normal((n, n))
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x = osw.gmres_fixed(lambda v: A @ v, lambda v: Mi @ v, b, k)
    # brute force: x = Mi y, y in span{b, (A Mi) b, ...}, minimising ||b - A x||
    K = [b]
    for _ in range(k - 1):
        K.append(A @ (Mi @ K[-1]))
    K = np.stack(K, axis=1)
    c = np.linalg.lstsq(A @ Mi @ K, b, rcond=None)[0]
    x_bf = Mi @ (K @ c)
    np.testing.assert_allclose(x, x_bf, rtol=1e-9, atol=1e-11)
    # residual is non-increasing in the step count
    r = [np.linalg.norm(b - A @ osw.gmres_fixed(lambda v: A @ v, lambda v: Mi @ v, b, j)) for j in range(1, 8)]
    assert all(r[j + 1] <= r[j] * (1 + 1e-12) for j in range(len(r) - 1))


def test_two_level_oras_gmres_converges_on_cube():
    """Sanity: the two-level operator is a useful preconditioner (GMRES with
    it needs far fewer steps than without)."""
    p = wl.cube_problem()
    T = osw.TwoLevel(p, coarse_mode="gmres")
    space, A, F = oa.system(p["fine"], p["velocity"], p["freq"], p["src_xyz"])
    b = F[0]
    it = {"n": 0}

    def cb(_):
        it["n"] += 1

    Mop = spla.LinearOperator(A.shape, matvec=T.apply, dtype=np.complex128)
    x, info = spla.gmres(A, b, M=Mop, rtol=1e-8, restart=50, maxiter=50, callback=cb,
                         callback_type="pr_norm")
    assert info == 0 and it["n"] < 25
