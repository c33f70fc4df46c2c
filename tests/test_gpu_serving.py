"""Serving loop (continuous batching): a request's wavefields are the same
alone and in a mix with requests that arrive before and after it, and they
match the oracle's direct solution."""
import numpy as np
import pytest

from oracle import assemble as oa
from paper_2004_07930_gb300 import hz
from paper_2004_07930_gb300 import workloads as wl
from paper_2004_07930_gb300.serve import ServingLoop

from _gpu_common import dof_perm, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu

SRC_A = [[300.0, 400.0, 200.0], [700.0, 650.0, 500.0]]
SRC_B = [[500.0, 500.0, 100.0], [250.0, 750.0, 800.0], [820.0, 180.0, 350.0]]
SRC_C = [[600.0, 300.0, 650.0], [150.0, 150.0, 150.0]]


def _drain(srv, ids_ns):
    out = {}
    for _ in range(200):
        for rid in srv.step():
            out[rid] = srv.fetch(rid, ids_ns[rid])
        if len(out) == len(ids_ns):
            return out
    raise AssertionError("server did not finish")


def _oracle_wavefields(p, S, src):
    space, A, _ = oa.system(p["fine"], p["velocity"], p["freq"])
    perm = dof_perm(S, space, 1000.0)
    F = oa.point_source(space, src, np.ones(len(src)))
    F[:, space.dirichlet_dofs(p["fine"]["bfaces"], p["fine"]["btags"])] = 0.0
    return oa.solve(A, F)[:, perm]


@pytest.mark.parametrize("precision", [hz.HZ_PREC_MIXED, hz.HZ_PREC_FP64])
def test_request_same_alone_and_in_mix(precision):
    torch_cuda()
    p = wl.cube_problem(ncell=4, nparts_xyz=(2, 2, 1))
    with hz.Solver.from_problem(p, rtol=1e-8, precision=precision, restart=3) as S:
        alone = hz.Server(S, 4)
        alone.submit(7, SRC_A)
        uA, stA = _drain(alone, {7: 2})[7]
        alone.close()
        mix = hz.Server(S, 4)
        mix.submit(1, SRC_B)
        assert mix.step() == []                 # B is on the device when A and C arrive
        mix.submit(7, SRC_A)
        mix.submit(3, SRC_C)
        assert mix.pending()[0] > 0             # more columns than free slots: queued
        res = _drain(mix, {1: 3, 7: 2, 3: 2})
        assert mix.pending() == (0, 0)
        mix.close()
        uA_mix, st = res[7]
        assert st["converged"] == 1 and stA["converged"] == 1
        assert st["iterations"] == stA["iterations"]
        assert np.abs(uA_mix - uA).max() <= 1e-12 * np.abs(uA).max()
        for rid, src in ((1, SRC_B), (7, SRC_A), (3, SRC_C)):
            assert rel_l2(res[rid][0], _oracle_wavefields(p, S, src)).max() <= 1e-6
            assert res[rid][1]["max_rel_residual"] <= 1e-8


def test_serving_loop_two_frequencies():
    torch_cuda()
    p2 = wl.cube_problem(ncell=4, freq=2.0)
    p3 = wl.cube_problem(ncell=4, freq=3.0)
    solvers = {2.0: hz.Solver.from_problem(p2, rtol=1e-8), 3.0: hz.Solver.from_problem(p3, rtol=1e-8)}
    try:
        loop = ServingLoop(solvers, 4)
        reqs = [(0.0, 1, 2.0, SRC_A), (0.0, 2, 3.0, SRC_B), (0.01, 3, 2.0, SRC_C), (0.02, 4, 3.0, SRC_A)]
        summ = loop.run_stream(reqs, keep_wavefields=True)
        loop.close()
        assert summ["requests"] == 4 and summ["rhs"] == 9 and summ["converged"]
        assert summ["latency_p99_s"] >= summ["latency_p50_s"] > 0
        for off, rid, f, src in reqs:
            p = p2 if f == 2.0 else p3
            ref = _oracle_wavefields(p, solvers[f], src)
            assert rel_l2(loop.results[rid][0], ref).max() <= 1e-6
    finally:
        for S in solvers.values():
            S.close()


def test_server_rejects_bad_requests():
    torch_cuda()
    p = wl.cube_problem(ncell=4)
    with hz.Solver.from_problem(p, rtol=1e-8) as S:
        srv = hz.Server(S, 2)
        with pytest.raises(hz.HzError):
            srv.submit(1, [[5000.0, 0.0, 0.0]])   # outside the mesh
        srv.submit(1, SRC_A)
        with pytest.raises(hz.HzError):
            srv.submit(1, SRC_C)                 # id in use
        with pytest.raises(hz.HzError):
            srv.fetch(1, 2)                      # not finished
        _drain(srv, {1: 2})
        srv.close()
        with pytest.raises(hz.HzError):
            hz.Server(S, 65)                     # more slots than max_block


def test_admission_by_device_budget():
    """A budget of 2.5 columns' worth of device bytes gives the server 2
    slots (the power of two below 2.5): a third source waits in the queue and is admitted when a slot (and
    its memory) frees; every request still matches the oracle."""
    torch_cuda()
    p = wl.cube_problem(ncell=4)
    with hz.Solver.from_problem(p, rtol=1e-8, restart=3) as S:
        loop = ServingLoop({2.0: S}, device_budget=2.5 * S.column_bytes())
        assert loop.slots == {2.0: 2}
        loop.submit(1, 2.0, SRC_A)
        loop.submit(2, 2.0, [SRC_C[0]])
        loop.step(2.0)
        assert loop.servers[2.0].pending() == (1, 2)     # one source held back by the budget
        while loop.busy():
            loop.step(2.0)
        loop.close()
        for rid, src in ((1, SRC_A), (2, [SRC_C[0]])):
            u, st, _ = loop.results[rid]
            assert st["converged"] == 1
            assert rel_l2(u, _oracle_wavefields(p, S, src)).max() <= 1e-6
