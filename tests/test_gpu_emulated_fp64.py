"""FP64 emulated by FP32 pairs (option emulate_fp64, mixed form).

The mixed form keeps the outer FGMRES in FP64 accuracy; with emulate_fp64 =
1 its products with A and E and its Gram-Schmidt products run in
double-float arithmetic (Dekker's TwoProduct, Knuth's TwoSum; about 47
significant bits). Checked here against the same solver in native FP64
(emulate_fp64 = 0) and against the mathematics:

* each column's Krylov basis of the last restart cycle is orthonormal to
  1e-12 (the bound the block Arnoldi test uses), as in native FP64;
* both variants take the same number of iterations (the Arnoldi
  coefficients differ at the 1e-13 level, far below what changes a
  convergence test at rtol 1e-8), up to one;
* their wavefields agree to 1e-7 relative L2 at rtol 1e-8 (the oracle
  comparisons are in test_gpu_crop.py and test_gpu_parity.py).
"""
import numpy as np
import pytest

from paper_2004_07930_gb300 import hz
from paper_2004_07930_gb300 import workloads as wl

from _gpu_common import rel_l2, torch_cuda

pytestmark = pytest.mark.gpu

SOURCES = [[500.0, 500.0, 100.0], [250.0, 700.0, 600.0], [800.0, 300.0, 400.0]]


@pytest.fixture(scope="module")
def cube():
    torch_cuda()
    return wl.cube_problem(ncell=6)


@pytest.mark.parametrize("coarse", [hz.HZ_COARSE_NONE, hz.HZ_COARSE_GMRES])
def test_emulated_matches_native(cube, coarse):
    out = {}
    for emulate in (1, 0):
        with hz.Solver.from_problem(cube, precision=hz.HZ_PREC_MIXED, coarse_mode=coarse, rtol=1e-8, restart=40,
                                    emulate_fp64=emulate) as S:
            u, st = S.solve(SOURCES)
            res, its = S.column_stats()
            assert st["converged"] == 1 and (res <= 1e-8).all()
            V = S.krylov_basis()
            nb, s, n = V.shape
            worst = 0.0
            for c in range(s):
                Q = V[:, c, :]
                Q = Q[np.linalg.norm(Q, axis=1) > 0.5]
                worst = max(worst, np.abs(Q.conj() @ Q.T - np.eye(len(Q))).max())
            out[emulate] = (u, its, worst)
            print("coarse", coarse, "emulate_fp64", emulate, "iterations", its.tolist(), "||V^H V - I||", worst)
            assert worst <= 1e-12
    (u1, its1, _), (u0, its0, _) = out[1], out[0]
    assert np.abs(its1 - its0).max() <= 1
    assert rel_l2(u1, u0).max() <= 1e-7
