"""Shared helpers of the GPU parity tests (inputs from the seeded generators,
expected values from the oracle only)."""
import numpy as np
import pytest

from oracle import assemble as oa
from oracle import schwarz as osw


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def solver(prob, **opts):
    from paper_2004_07930_gb300 import hz

    return hz.Solver.from_problem(prob, **opts)


def dof_perm(S, space, scale):
    """perm such that oracle dof perm[j] sits at library dof j."""
    return oa.match_dofs(space.coords, S.coords(), scale)


def oracle_twolevel(prob, mode):
    return osw.TwoLevel(prob, coarse_mode=mode)


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)
