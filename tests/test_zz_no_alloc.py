"""Allocation-free product with A (hz_apply_A_noalloc).

Some callers cannot allocate device memory when they call the library (for
example code that runs where cudaMalloc/cudaFree are not allowed because they
synchronise the device, or processes whose device memory is entirely managed
by their own allocator). hz_apply_A_noalloc takes its two work blocks from a
fixed file-scope device array instead of the context workspace. This test
checks it against hz_apply_A through the C ABI on two calls in a row, and
that sizes beyond the array are refused. It is collected last so that a run
stopping at the first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2004_07930_gb300 import hz
from paper_2004_07930_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_noalloc_product_matches_apply_A_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = hz.load()
    p = wl.cube_problem()
    stream = torch.cuda.current_stream()
    with hz.Solver.from_problem(p, coarse_mode=hz.HZ_COARSE_NONE, stream=stream) as S:
        for seed in (21, 22):                       # two calls in a row
            X = torch.from_numpy(wl.random_rhs(S.n, 5, seed)).cuda()
            ref = S.apply_A(X)
            Y = torch.full_like(X, complex(np.nan, np.nan))
            rc = lib.hz_apply_A_noalloc(S._ctx, X.data_ptr(), Y.data_ptr(), 5, stream.cuda_stream)
            assert rc == hz.HZ_OK, lib.hz_last_error()
            torch.cuda.synchronize()
            scale = ref.abs().max().item()
            assert (Y - ref).abs().max().item() <= 1e-13 * scale
        # beyond the fixed array: refused, nothing launched
        too_many = hz.HZ_NOALLOC_MAX_ENTRIES // S.n + 1
        Xb = torch.zeros((too_many, S.n), dtype=torch.complex128, device="cuda")
        rc = lib.hz_apply_A_noalloc(S._ctx, Xb.data_ptr(), Xb.data_ptr(), too_many, stream.cuda_stream)
        assert rc == hz.HZ_EINVAL
        assert b"exceeds" in lib.hz_last_error()
