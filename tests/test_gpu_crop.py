"""Wavefield parity on a corner crop of the 5 Hz Overthrust-like workload.

The crop (8 x 8 x 10 graded cells at the workload's 1.3 P3 cells per local
minimum wavelength, 2.8 x 2.8 x 4.65 km, free surface on top, absorbing
faces elsewhere, 19,375 dofs) keeps the workload's velocity field, grading
and boundary conditions; it is split into 4 box subdomains with the nested
2x coarser mesh of the two-level method. The library's wavefields for two
surface sources are compared element by element (dofs matched by
coordinates) with the oracle's direct solve:

* FP64 form: relative L2 <= 1e-6 at GMRES rtol 1e-7, and <= 1e-8 at rtol
  1e-10. The rtol is a residual bound: on this crop the forward error at
  rtol 1e-6 equals the residual to within a few per mille (1.00009e-6 was
  measured for one of the two sources), so the 1e-6 wavefield bound is
  checked one decade tighter, and rtol 1e-6 is held to 2e-6;
* mixed form (complex FP32 local solves) at rtol 1e-6: <= 1e-5, with the
  coarse level in FP64 (default) and in FP32 (coarse_fp32 = 1); at rtol
  1e-8: <= 1e-6 (the outer iteration is flexible GMRES with FP64-accurate
  residuals, so the mixed form reaches any tolerance);
* every mixed case with the products by A and E in double-float arithmetic
  (emulate_fp64 = 1, the default) and in native FP64 (emulate_fp64 = 0).
"""
import numpy as np
import pytest

from oracle import assemble as oa
from paper_2004_07930_gb300 import hz
from paper_2004_07930_gb300 import workloads as wl

from _gpu_common import dof_perm, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu

SOURCES = [[1250.0, 1250.0, 100.0], [2000.0, 1000.0, 100.0]]


@pytest.fixture(scope="module")
def crop():
    torch_cuda()
    p = wl.overthrust_problem(5.0, nparts=4, crop=(0.125, 0.125, 1.0), sources=SOURCES)
    space, A, F = oa.system(p["fine"], p["velocity"], p["freq"], p["src_xyz"])
    return p, space, oa.solve(A, F)


@pytest.mark.parametrize("precision,coarse_fp32,rtol,bound", [
    (hz.HZ_PREC_FP64, 0, 1e-6, 2e-6),
    (hz.HZ_PREC_FP64, 0, 1e-7, 1e-6),
    (hz.HZ_PREC_FP64, 0, 1e-10, 1e-8),
    (hz.HZ_PREC_MIXED, 0, 1e-6, 1e-5),
    (hz.HZ_PREC_MIXED, 1, 1e-6, 1e-5),
    (hz.HZ_PREC_MIXED, 0, 1e-8, 1e-6),
])
@pytest.mark.parametrize("emulate", [1, 0])
def test_crop_wavefield_matches_oracle(crop, precision, coarse_fp32, rtol, bound, emulate):
    p, space, u_or = crop
    assert p["fine"]["ncells"] == (8, 8, 10) and space.n == 19375
    if precision == hz.HZ_PREC_FP64 and emulate == 0:
        pytest.skip("emulate_fp64 applies to the mixed form only")
    with hz.Solver.from_problem(p, precision=precision, coarse_fp32=coarse_fp32, rtol=rtol,
                                emulate_fp64=emulate) as S:
        perm = dof_perm(S, space, 20000.0)
        u, st = S.solve(p["src_xyz"])
        err = rel_l2(u, u_or[:, perm])
        res, its = S.column_stats()
        print("precision", precision, "coarse_fp32", coarse_fp32, "emulate_fp64", emulate, "rtol", rtol,
              "iterations", st["iterations"],
              "per column", its.tolist(), "rel L2", err)
        assert st["converged"] == 1 and st["max_rel_residual"] <= rtol
        assert (res <= rtol).all() and its.max() == st["iterations"]
        assert err.max() <= bound


def test_crop_one_level_wavefield_matches_oracle(crop):
    p, space, u_or = crop
    with hz.Solver.from_problem(p, precision=hz.HZ_PREC_MIXED, coarse_mode=hz.HZ_COARSE_NONE, rtol=1e-6) as S:
        perm = dof_perm(S, space, 20000.0)
        u, st = S.solve(p["src_xyz"])
        assert rel_l2(u, u_or[:, perm]).max() <= 1e-5


@pytest.fixture(scope="module")
def crop10():
    """8 x 8 cells (1.4 x 1.4 km, full depth) of the 10 Hz workload: the
    oracle's share of the mixed-precision-at-scale configuration (a 1/8-volume
    crop, ~0.75M dofs, is beyond a direct solve on the host)."""
    torch_cuda()
    p = wl.overthrust_problem(10.0, nparts=4, crop=(0.07, 0.07, 1.0), sources=[[700.0, 600.0, 100.0]])
    space, A, F = oa.system(p["fine"], p["velocity"], p["freq"], p["src_xyz"])
    return p, space, oa.solve(A, F)


@pytest.mark.parametrize("precision,bound", [(hz.HZ_PREC_FP64, 2e-6), (hz.HZ_PREC_MIXED, 1e-5)])
def test_crop_10hz_wavefield_matches_oracle(crop10, precision, bound):
    p, space, u_or = crop10
    assert p["fine"]["ncells"][:2] == (8, 8)
    with hz.Solver.from_problem(p, precision=precision, rtol=1e-6) as S:
        perm = dof_perm(S, space, 20000.0)
        u, st = S.solve(p["src_xyz"])
        err = rel_l2(u, u_or[:, perm])
        print("10 Hz crop n", space.n, "precision", precision, "iterations", st["iterations"], "rel L2", err)
        assert st["converged"] == 1
        assert err.max() <= bound
