"""Failure paths and diagnostics of the C ABI on the GPU (errors made on the
host side, never by faulting the device):

* maxit reached: HZ_ENOTCONV, the last iterate returned (finite, residual
  below the starting one), per-column residuals and iterations reported;
* duplicated sources in one block: both columns converge to the same
  wavefield (one Krylov space per column, so no block rank deficiency);
* debug_bounds: the index maps of a valid setup pass the device check;
* overlap = 2: the preconditioner equals the oracle's Eq. oras operator
  grown by two element layers;
* a server returns finished request ids beyond `cap` on later steps.
"""
import numpy as np
import pytest

from oracle import assemble as oa
from oracle import schwarz as osw
from paper_2004_07930_gb300 import hz
from paper_2004_07930_gb300 import workloads as wl

from _gpu_common import dof_perm, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu


def test_maxit_returns_notconv_and_last_iterate():
    torch_cuda()
    p = wl.cube_problem(ncell=4)
    src = [[500.0, 500.0, 100.0], [250.0, 700.0, 600.0]]
    with hz.Solver.from_problem(p, rtol=1e-12, maxit=2) as S:
        with pytest.raises(hz.HzError) as ei:
            S.solve(src)
        assert ei.value.code == hz.HZ_ENOTCONV
        u, st = S.solve(src, raise_on_notconv=False)
        res, its = S.column_stats()
        assert st["converged"] == 0 and st["iterations"] == 2
        assert np.isfinite(u).all() and np.abs(u).max() > 0
        assert res.shape == (2,) and (res > 1e-12).all() and (res < 1.0).all()
        assert np.allclose(res.max(), st["max_rel_residual"])
        assert (its == 2).all()
        assert st["perturbed_pivots"] == S.info()["perturbed_pivots"]


def test_duplicate_sources_in_one_block():
    torch_cuda()
    p = wl.cube_problem(ncell=4)
    space, A, F = oa.system(p["fine"], p["velocity"], p["freq"], [[500.0, 500.0, 100.0]])
    u_or = oa.solve(A, F)
    for prec in (hz.HZ_PREC_FP64, hz.HZ_PREC_MIXED):
        with hz.Solver.from_problem(p, rtol=1e-8, precision=prec) as S:
            u, st = S.solve([[500.0, 500.0, 100.0]] * 3)
            res, its = S.column_stats()
            assert st["converged"] == 1 and np.isfinite(u).all()
            assert (its == its[0]).all()
            np.testing.assert_array_equal(u[1], u[0])
            np.testing.assert_array_equal(u[2], u[0])
            perm = dof_perm(S, space, 1000.0)
            assert rel_l2(u[0], u_or[0, perm]) <= 1e-6


def test_debug_bounds_accepts_valid_setup():
    torch_cuda()
    p = wl.cube_problem()
    for prec in (hz.HZ_PREC_FP64, hz.HZ_PREC_MIXED):
        with hz.Solver.from_problem(p, debug_bounds=1, precision=prec) as S:
            u, st = S.solve(p["src_xyz"])
            assert st["converged"] == 1


def test_two_layer_overlap_matches_oracle():
    torch_cuda()
    p = wl.cube_problem()
    To = osw.TwoLevel(p, coarse_mode="none", overlap=2)
    T1 = osw.TwoLevel(p, coarse_mode="none", overlap=1)
    with hz.Solver.from_problem(p, coarse_mode=hz.HZ_COARSE_NONE, overlap=2) as S:
        perm = dof_perm(S, To.space, 1000.0)
        X = wl.random_rhs(S.n, 2, 31)
        Y = S.apply_prec(X)
        ref = np.stack([To.apply(x[np.argsort(perm)])[perm] for x in X])
        one = np.stack([T1.apply(x[np.argsort(perm)])[perm] for x in X])
        assert rel_l2(Y, ref).max() <= 1e-9
        assert rel_l2(one, ref).min() > 1e-3       # the second layer changes the operator
        assert S.info()["sub_rows"] > 0


def test_server_returns_finished_ids_beyond_cap():
    torch_cuda()
    p = wl.cube_problem(ncell=4)
    with hz.Solver.from_problem(p, rtol=1e-8) as S:
        srv = hz.Server(S, 4)
        for rid, x in enumerate((300.0, 500.0, 700.0)):
            srv.submit(rid, [[x, 500.0, 300.0]])
        got = []
        for _ in range(200):
            ids = srv.step(cap=1)
            assert len(ids) <= 1
            got += ids
            if len(got) == 3:
                break
        assert sorted(got) == [0, 1, 2]
        for rid in got:
            u, st = srv.fetch(rid, 1)
            assert st["converged"] == 1
        assert srv.pending() == (0, 0)
        srv.close()
