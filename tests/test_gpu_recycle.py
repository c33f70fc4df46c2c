"""Krylov subspace recycling (option `recycle`) on the GPU.

With recycling on, every FGMRES cycle starts from the projection
x += U C^H r, r -= C C^H r and runs its Arnoldi process on
(I - C C^H) A M^{-1}, where C = A U is orthonormal; after each cycle the
harmonic Ritz vectors of smallest magnitude join U. This changes the
iterates but not the system solved, so:

* the wavefields still match the oracle's direct solve to the same bounds as
  without recycling (FP64: relative L2 <= 1e-6 at rtol 1e-8; mixed: <= 1e-5
  at rtol 1e-6), on the 5 Hz corner crop with restart 8 (several cycles per
  solve);
* a second solve on the same context, with new sources, starts with the
  space the first one left and needs no more iterations than the same solve
  on a context without recycling, and strictly fewer in total over the
  columns of the one-level method, whose slow modes are the ones recycling
  targets.
"""
import numpy as np
import pytest

from oracle import assemble as oa
from paper_2004_07930_gb300 import hz
from paper_2004_07930_gb300 import workloads as wl

from _gpu_common import dof_perm, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu

FIRST = [[1250.0, 1250.0, 100.0], [2000.0, 1000.0, 100.0]]
SECOND = [[700.0, 2100.0, 100.0], [1600.0, 1700.0, 100.0]]


@pytest.fixture(scope="module")
def crop():
    torch_cuda()
    p = wl.overthrust_problem(5.0, nparts=4, crop=(0.125, 0.125, 1.0), sources=FIRST + SECOND)
    space, A, F = oa.system(p["fine"], p["velocity"], p["freq"], p["src_xyz"])
    return p, space, oa.solve(A, F)


@pytest.mark.parametrize("coarse", [hz.HZ_COARSE_NONE, hz.HZ_COARSE_GMRES])
@pytest.mark.parametrize("precision,rtol,bound", [
    (hz.HZ_PREC_FP64, 1e-8, 1e-6),
    (hz.HZ_PREC_MIXED, 1e-6, 1e-5),
])
def test_recycling_keeps_parity_and_saves_iterations(crop, coarse, precision, rtol, bound):
    p, space, u_or = crop
    src = np.asarray(p["src_xyz"])
    opts = dict(precision=precision, coarse_mode=coarse, rtol=rtol, restart=8)
    with hz.Solver.from_problem(p, recycle=8, **opts) as Sr, hz.Solver.from_problem(p, recycle=0, **opts) as S0:
        perm = dof_perm(Sr, space, 20000.0)
        runs = {}
        for name, S in (("recycle", Sr), ("plain", S0)):
            its_batches = []
            for b, rows in enumerate((slice(0, 2), slice(2, 4))):
                u, st = S.solve(src[rows])
                res, its = S.column_stats()
                assert st["converged"] == 1 and (res <= rtol).all()
                err = rel_l2(u, u_or[rows][:, perm])
                assert err.max() <= bound, (name, b, err)
                its_batches.append(its.copy())
            runs[name] = its_batches
        print("coarse", coarse, "precision", precision, "iterations per column",
              {k: [v.tolist() for v in vs] for k, vs in runs.items()})
        # the first batch starts from an empty recycled space in both contexts
        assert runs["recycle"][1].max() <= runs["plain"][1].max()
        if coarse == hz.HZ_COARSE_NONE:
            assert runs["recycle"][1].sum() < runs["plain"][1].sum()
