"""GPU parity: every step of the path through the C ABI against the oracle.

Inputs are seeded (workloads module); expected values come from the oracle
(SciPy SuperLU and the exact two-level operator). Tolerances: the products
and preconditioner applications are exact algorithms, so they agree to a few
hundred units of rounding relative to the local conditioning (1e-9); the
wavefields must agree to relative L2 <= 1e-6 (FP64 form) at GMRES rtol 1e-6
and <= 1e-5 in the mixed form.
"""
import numpy as np
import pytest

from oracle import assemble as oa
from oracle import schwarz as osw
from paper_2004_07930_gb300 import workloads as wl
from paper_2004_07930_gb300 import hz

from _gpu_common import dof_perm, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cube():
    torch_cuda()
    p = wl.cube_problem()
    T = osw.TwoLevel(p, coarse_mode="gmres")
    return p, T


@pytest.mark.parametrize("precision,emulate", [(hz.HZ_PREC_FP64, 1), (hz.HZ_PREC_MIXED, 1), (hz.HZ_PREC_MIXED, 0)])
def test_matrix_and_spmm_match_oracle(cube, precision, emulate):
    """Native FP64 product (FP64 form, or mixed with emulate_fp64 = 0) and
    the double-float product of the mixed form: both within 1e-13 of the
    largest entry of the SciPy product."""
    p, T = cube
    with hz.Solver.from_problem(p, coarse_mode=hz.HZ_COARSE_NONE, precision=precision, emulate_fp64=emulate) as S:
        perm = dof_perm(S, T.space, 1000.0)
        A = S.matrix_csr()
        Ao = T.A[perm][:, perm]
        assert abs(A - Ao).max() <= 1e-13 * abs(Ao).max()
        X = wl.random_rhs(S.n, 5, 3)
        Y = S.apply_A(X)
        ref = (Ao @ X.T).T
        print("precision", precision, "emulate_fp64", emulate, "max err / max |ref|",
              np.abs(Y - ref).max() / np.abs(ref).max())
        assert np.abs(Y - ref).max() <= 1e-13 * np.abs(ref).max()
        info = S.info()
        assert info["n"] == 6859 and info["nnz"] == 299971


@pytest.mark.parametrize("mode", ["none", "direct", "gmres"])
def test_preconditioner_matches_oracle(cube, mode):
    p, T = cube
    code = {"none": hz.HZ_COARSE_NONE, "direct": hz.HZ_COARSE_DIRECT, "gmres": hz.HZ_COARSE_GMRES}[mode]
    To = T if mode == "gmres" else osw.TwoLevel(p, coarse_mode=mode)
    with hz.Solver.from_problem(p, coarse_mode=code) as S:
        perm = dof_perm(S, To.space, 1000.0)
        X = wl.random_rhs(S.n, 3, 4)
        Y = S.apply_prec(X)
        ref = np.stack([To.apply(x[np.argsort(perm)])[perm] for x in X])
        err = rel_l2(Y, ref)
        print(mode, "rel err", err)
        assert err.max() <= 1e-9


def test_device_buffers_equal_host_buffers(cube):
    torch = torch_cuda()
    p, _ = cube
    with hz.Solver.from_problem(p) as S:
        X = wl.random_rhs(S.n, 2, 5)
        Yh = S.apply_prec(X)
        Yd = S.apply_prec(torch.from_numpy(X).cuda()).cpu().numpy()
        np.testing.assert_array_equal(Yh, Yd)


@pytest.mark.parametrize("rtol,bound", [(1e-10, 1e-8), (1e-8, 1e-7), (1e-6, 1e-6)])
def test_cube_wavefield_matches_oracle(cube, rtol, bound):
    p, T = cube
    space, A, F = oa.system(p["fine"], p["velocity"], p["freq"], p["src_xyz"])
    u_or = oa.solve(A, F)
    with hz.Solver.from_problem(p, rtol=rtol) as S:
        perm = dof_perm(S, space, 1000.0)
        u, st = S.solve(p["src_xyz"])
        err = rel_l2(u, u_or[:, perm])
        print("rtol", rtol, "iterations", st["iterations"], "rel L2", err, "residual", st["max_rel_residual"])
        assert st["converged"] == 1 and st["max_rel_residual"] <= rtol
        assert err.max() <= bound


def test_single_subdomain_converges_in_one_iteration():
    torch_cuda()
    p = wl.cube_problem(ncell=4, nparts_xyz=(1, 1, 1), top_dirichlet=True, coarse=False)
    space, A, F = oa.system(p["fine"], p["velocity"], p["freq"], p["src_xyz"])
    with hz.Solver.from_problem(p, coarse_mode=hz.HZ_COARSE_NONE, rtol=1e-10) as S:
        u, st = S.solve(p["src_xyz"])
        assert S.info()["perturbed_pivots"] == 0
        assert st["iterations"] == 1
        perm = dof_perm(S, space, 1000.0)
        assert rel_l2(u, oa.solve(A, F)[:, perm]).max() <= 1e-9


def test_dirichlet_top_heterogeneous_and_ragged_blocks():
    torch_cuda()
    rng = np.random.default_rng(8)
    p = wl.cube_problem(ncell=4, nparts_xyz=(2, 1, 2), top_dirichlet=True)
    p["velocity"] = rng.uniform(1500.0, 2500.0, len(p["velocity"]))
    src = np.column_stack([rng.uniform(100, 900, 7), rng.uniform(100, 900, 7), rng.uniform(50, 900, 7)])
    amp = rng.standard_normal(7) + 1j * rng.standard_normal(7)
    space, A, F = oa.system(p["fine"], p["velocity"], p["freq"], src, amp)
    u_or = oa.solve(A, F)
    with hz.Solver.from_problem(p, rtol=1e-10, max_block=3) as S:     # blocks 3 + 3 + 1
        perm = dof_perm(S, space, 1000.0)
        u, st = S.solve(src, amp)
        assert rel_l2(u, u_or[:, perm]).max() <= 1e-8
        # the same sources one at a time
        for q in (0, 6):
            u1, _ = S.solve(src[q:q + 1], amp[q:q + 1])
            assert rel_l2(u1[0], u[q]) <= 1e-9


def test_solve_rhs_plane_wave_data():
    """Impedance data of an exact plane wave: the GPU solution equals the
    oracle's discrete solution (and so approximates exp(i k d.x))."""
    torch_cuda()
    p = wl.cube_problem(ncell=4)
    k = 2 * np.pi * p["freq"] / 2000.0
    d = np.array([1.0, 2.0, 2.0]) / 3.0
    g = lambda X, nrm, e: 1j * k * (d @ nrm - 1.0) * np.exp(1j * k * (X @ d))
    space = oa.P3Space(p["fine"]["xyz"], p["fine"]["tets"])
    A, _ = oa.assemble(space, p["velocity"], p["freq"], p["fine"]["bfaces"], p["fine"]["btags"])
    F = oa.robin_load(space, p["fine"]["bfaces"], p["fine"]["btags"], g)
    u_or = oa.solve(A, F)
    with hz.Solver.from_problem(p, rtol=1e-11) as S:
        perm = dof_perm(S, space, 1000.0)
        u, st = S.solve_rhs(F[perm][None, :])
        assert rel_l2(u[0], u_or[perm]) <= 1e-8


@pytest.mark.parametrize("coarse", [hz.HZ_COARSE_NONE, hz.HZ_COARSE_GMRES])
def test_mixed_form_wavefield_matches_oracle(cube, coarse):
    """Mixed form (complex FP32 local solves inside FP64 FGMRES): the
    wavefield still converges to the FP64 oracle's discrete solution; at
    rtol 1e-6 the error bound of the mixed form is 1e-5."""
    p, T = cube
    space, A, F = oa.system(p["fine"], p["velocity"], p["freq"], p["src_xyz"])
    u_or = oa.solve(A, F)
    for rtol, bound in ((1e-6, 1e-5), (1e-10, 1e-8)):
        with hz.Solver.from_problem(p, rtol=rtol, precision=hz.HZ_PREC_MIXED, coarse_mode=coarse) as S:
            perm = dof_perm(S, space, 1000.0)
            u, st = S.solve(p["src_xyz"])
            err = rel_l2(u, u_or[:, perm])
            print("mixed rtol", rtol, "iterations", st["iterations"], "rel L2", err)
            assert st["converged"] == 1
            assert err.max() <= bound


def test_graphs_and_eager_agree(cube):
    """The captured-graph replay of the local and coarse solves gives the
    same preconditioner as eager launches."""
    p, _ = cube
    X = wl.random_rhs(6859, 3, 9)
    with hz.Solver.from_problem(p, use_graphs=1) as S1, hz.Solver.from_problem(p, use_graphs=0) as S0:
        Y1 = S1.apply_prec(X)
        Y1b = S1.apply_prec(X)
        Y0 = S0.apply_prec(X)
    np.testing.assert_array_equal(Y1, Y1b)
    np.testing.assert_array_equal(Y1, Y0)
