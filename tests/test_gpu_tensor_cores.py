"""Tensor-core front sweeps (mixed form, tensor_cores = 1): the local solves
run as tcgen05 MMAs on a three-term TF32 split of the FP32 factors and
inputs (hi*hi + hi*lo + lo*hi, FP32 accumulation), so the preconditioner
keeps FP32 accuracy: within 1e-5 of the exact Eq. oras operator (the plain
SIMT FP32 sweeps: ~3e-7; a single TF32 product: ~3e-4), and FGMRES needs the
same iterations as with the SIMT sweeps. Blocks of 9-16 columns run the
tensor-core kernels; narrower and wider blocks keep the SIMT sweeps."""
import numpy as np
import pytest

from oracle import assemble as oa
from oracle import schwarz as osw
from paper_2004_07930_gb300 import hz
from paper_2004_07930_gb300 import workloads as wl

from _gpu_common import dof_perm, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cube():
    torch_cuda()
    return wl.cube_problem(ncell=6, nparts_xyz=(2, 2, 1))


def _sources(ns, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(80.0, 920.0, size=(ns, 3))


@pytest.mark.parametrize("s", [16, 12])
def test_preconditioner_close_to_oracle(cube, s):
    T = osw.TwoLevel(cube, coarse_mode="none")
    opts = dict(precision=hz.HZ_PREC_MIXED, coarse_mode=hz.HZ_COARSE_NONE)
    with hz.Solver.from_problem(cube, tensor_cores=1, **opts) as St, \
            hz.Solver.from_problem(cube, tensor_cores=0, **opts) as Ss:
        perm = dof_perm(St, T.space, 1000.0)
        X = wl.random_rhs(St.n, s, 21)
        Yt = St.apply_prec(X)
        Yt2 = St.apply_prec(X)
        Ys = Ss.apply_prec(X)
    ref = np.stack([T.apply(x[np.argsort(perm)])[perm] for x in X])   # exact Eq. oras (FP64)
    np.testing.assert_array_equal(Yt, Yt2)                 # deterministic
    d = rel_l2(Yt, Ys)
    e_tc, e_s = rel_l2(Yt, ref).max(), rel_l2(Ys, ref).max()
    print("s", s, "tensor-core vs SIMT FP32: %.3e; vs exact: tensor cores %.3e, SIMT %.3e" % (d.max(), e_tc, e_s))
    assert d.max() > 1e-8                                   # the tensor-core tiles did run
    assert e_s <= 1e-5
    assert e_tc <= 1e-5


@pytest.mark.parametrize("coarse", [hz.HZ_COARSE_NONE, hz.HZ_COARSE_GMRES])
def test_wavefields_match_oracle(cube, coarse):
    src = _sources(16, 5)
    space, A, F = oa.system(cube["fine"], cube["velocity"], cube["freq"], src)
    u_or = oa.solve(A, F)
    its = {}
    for tc in (0, 1):
        with hz.Solver.from_problem(cube, rtol=1e-8, precision=hz.HZ_PREC_MIXED, coarse_mode=coarse,
                                    tensor_cores=tc) as S:
            perm = dof_perm(S, space, 1000.0)
            u, st = S.solve(src)
            its[tc] = st["iterations"]
            assert st["converged"] == 1
            assert rel_l2(u, u_or[:, perm]).max() <= 1e-6
    print("coarse", coarse, "iterations SIMT", its[0], "tensor cores", its[1])
    assert its[1] <= its[0] + 1


@pytest.mark.parametrize("s", [4, 24])
def test_other_widths_keep_simt(cube, s):
    """Blocks of at most 8 or more than 16 columns run the SIMT sweeps even
    with tensor_cores = 1: identical preconditioner to tensor_cores = 0."""
    opts = dict(precision=hz.HZ_PREC_MIXED, coarse_mode=hz.HZ_COARSE_NONE)
    with hz.Solver.from_problem(cube, tensor_cores=1, **opts) as St, \
            hz.Solver.from_problem(cube, tensor_cores=0, **opts) as Ss:
        X = wl.random_rhs(St.n, s, 8)
        np.testing.assert_array_equal(St.apply_prec(X), Ss.apply_prec(X))
