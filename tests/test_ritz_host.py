"""Harmonic Ritz pairs used by the recycling option (host code of the
library, no GPU): against NumPy's dense eigen-decomposition of the same
matrix Hm + h^2 Hm^{-H} e_m e_m^T, and the defining property that the
residual A p - theta p is orthogonal to A's image (checked through the
equivalent small problem)."""
import ctypes as C
import os

import numpy as np
import pytest

from paper_2004_07930_gb300 import build as hzbuild
from paper_2004_07930_gb300 import hz


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(hzbuild.LIB):
        hzbuild.build()
    L = hz.load()
    L.hz_internal_harmonic_ritz.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p]
    return L


def _hessenberg(m, seed):
    rng = np.random.default_rng(seed)
    H = rng.standard_normal((m + 1, m)) + 1j * rng.standard_normal((m + 1, m))
    H = np.triu(H, -1)
    H[np.arange(1, m + 1), np.arange(m)] = np.abs(H[np.arange(1, m + 1), np.arange(m)]) + 0.1
    return H


@pytest.mark.parametrize("m,k,seed", [(6, 2, 0), (20, 5, 1), (30, 10, 2)])
def test_harmonic_ritz_matches_dense_eig(lib, m, k, seed):
    Hb = _hessenberg(m, seed)
    Hc = np.asfortranarray(Hb)
    P = np.zeros((k, m), dtype=np.complex128)          # column-major m x k == row-major k x m
    th = np.zeros(k, dtype=np.complex128)
    rc = lib.hz_internal_harmonic_ritz(Hc.ctypes.data, m, k, P.ctypes.data, th.ctypes.data)
    assert rc == 0
    Hm, h = Hb[:m], Hb[m, m - 1]
    em = np.zeros(m)
    em[-1] = 1.0
    G = Hm + abs(h) ** 2 * np.outer(np.linalg.solve(Hm.conj().T, em), em)
    lam, _ = np.linalg.eig(G)
    want = lam[np.argsort(np.abs(lam))][:k]
    np.testing.assert_allclose(np.sort_complex(th), np.sort_complex(want), rtol=1e-8, atol=1e-10)
    for q in range(k):
        p = P[q]
        assert abs(np.linalg.norm(p) - 1.0) < 1e-12
        assert np.linalg.norm(G @ p - th[q] * p) <= 1e-8 * np.linalg.norm(G, 2)
        # harmonic Ritz property: Hbar p - theta [p; 0] is orthogonal to the range of Hbar
        r = Hb @ p - th[q] * np.concatenate([p, [0.0]])
        assert np.linalg.norm(Hb.conj().T @ r) <= 1e-8 * np.linalg.norm(Hb, 2) ** 2
    assert np.all(np.diff(np.abs(th)) >= -1e-12)
