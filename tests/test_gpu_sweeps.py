"""Persistent front sweeps (one launch per sweep direction over every tree
level, persistent_sweeps = 1) against the per-level launches
(persistent_sweeps = 0, the default). Both run the same tiles with the same arithmetic
and sum a row block's partial tiles in the same slot order, so the local
solves must agree bit for bit, whatever order the CTAs take the tiles in; a
second application must repeat the first exactly."""
import numpy as np
import pytest

from paper_2004_07930_gb300 import hz
from paper_2004_07930_gb300 import workloads as wl

from _gpu_common import torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["cube", "crop"])
def prob(request):
    torch_cuda()
    if request.param == "cube":
        return wl.cube_problem(ncell=6, nparts_xyz=(2, 2, 1))
    return wl.overthrust_problem(5.0, nparts=4, crop=(0.125, 0.125, 1.0), sources=[[1250.0, 1250.0, 100.0]])


@pytest.mark.parametrize("precision", [hz.HZ_PREC_FP64, hz.HZ_PREC_MIXED])
@pytest.mark.parametrize("coarse", [hz.HZ_COARSE_NONE, hz.HZ_COARSE_GMRES])
def test_persistent_equals_per_level(prob, precision, coarse):
    opts = dict(precision=precision, coarse_mode=coarse)
    with hz.Solver.from_problem(prob, persistent_sweeps=1, **opts) as Sp, \
            hz.Solver.from_problem(prob, persistent_sweeps=0, **opts) as Sl:
        for s in (1, 5, 16):
            X = wl.random_rhs(Sp.n, s, 40 + s)
            Yp = Sp.apply_prec(X)
            Yp2 = Sp.apply_prec(X)
            Yl = Sl.apply_prec(X)
            assert np.isfinite(Yp).all()
            np.testing.assert_array_equal(Yp, Yp2)
            np.testing.assert_array_equal(Yp, Yl)
