"""Block FGMRES (option block_arnoldi = 1): one Krylov space shared by the
right-hand sides of a block, block CGS2 + CholQR2 as tall-skinny products.

* the wavefields converge to the oracle's direct solve;
* the basis of a restart cycle is orthonormal as a whole: ||V^H V - I|| <=
  1e-12 over the kept directions (the per-column form only orthogonalises
  each column's own Krylov vectors);
* duplicated sources: the CholQR deflates the dependent directions, no NaN,
  the duplicated columns agree to rounding and converge;
* the block form needs no more iterations than the per-column form.
"""
import numpy as np
import pytest

from oracle import assemble as oa
from paper_2004_07930_gb300 import hz
from paper_2004_07930_gb300 import workloads as wl

from _gpu_common import dof_perm, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu


def _sources(ns, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(80.0, 920.0, size=(ns, 3))


@pytest.fixture(scope="module")
def cube():
    torch_cuda()
    return wl.cube_problem(ncell=6, nparts_xyz=(2, 2, 1))


@pytest.mark.parametrize("precision", [hz.HZ_PREC_FP64, hz.HZ_PREC_MIXED])
def test_block_wavefields_match_oracle(cube, precision):
    src = _sources(6, 3)
    space, A, F = oa.system(cube["fine"], cube["velocity"], cube["freq"], src)
    u_or = oa.solve(A, F)
    its = {}
    for block in (0, 1):
        with hz.Solver.from_problem(cube, rtol=1e-8, precision=precision, block_arnoldi=block, max_block=16) as S:
            perm = dof_perm(S, space, 1000.0)
            u, st = S.solve(src)
            its[block] = st["iterations"]
            assert st["converged"] == 1 and st["max_rel_residual"] <= 1e-8
            assert rel_l2(u, u_or[:, perm]).max() <= 1e-6
    print("iterations per-column", its[0], "block", its[1])
    assert its[1] <= its[0]


def test_block_basis_is_orthonormal(cube):
    src = _sources(8, 4)
    with hz.Solver.from_problem(cube, rtol=1e-10, block_arnoldi=1, coarse_mode=hz.HZ_COARSE_NONE, restart=12,
                                max_block=16) as S:
        S.solve(src)
        V = S.krylov_basis()
    nb, s, n = V.shape
    assert nb >= 2 and s == 8
    Q = V.reshape(nb * s, n)
    keep = np.linalg.norm(Q, axis=1) > 0.5
    Qk = Q[keep]
    err = np.abs(Qk.conj() @ Qk.T - np.eye(len(Qk))).max()
    print("block basis", nb, "x", s, "kept", keep.sum(), "||V^H V - I||", err)
    assert err <= 1e-12


def test_block_duplicated_sources(cube):
    src = np.array([[500.0, 500.0, 100.0]] * 3 + [[250.0, 700.0, 600.0]])
    space, A, F = oa.system(cube["fine"], cube["velocity"], cube["freq"], src)
    u_or = oa.solve(A, F)
    with hz.Solver.from_problem(cube, rtol=1e-8, block_arnoldi=1, max_block=16) as S:
        u, st = S.solve(src)
        res, its = S.column_stats()
        assert np.isfinite(u).all() and st["converged"] == 1
        assert (res <= 1e-8).all()
        perm = dof_perm(S, space, 1000.0)
        assert rel_l2(u, u_or[:, perm]).max() <= 1e-6
        # the duplicated columns share one Krylov direction; they agree to rounding
        assert rel_l2(u[1], u[0]) <= 1e-12 and rel_l2(u[2], u[0]) <= 1e-12
