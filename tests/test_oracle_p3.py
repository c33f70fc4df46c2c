"""Pins for the oracle's P3 element (basis, quadrature, element matrices).

Each check is fixed by mathematics, not by re-running the oracle's formula:
the Lagrange property, polynomial reproduction, exact monomial integrals over
the simplex, finite-difference derivatives, and closed forms for constant and
linear fields.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import p3


def _rand_tet(rng):
    while True:
        P = rng.uniform(-1.0, 2.0, size=(4, 3))
        if abs(np.linalg.det(P[1:] - P[0])) > 0.3:
            return P


def test_twenty_nodes_lagrange_property():
    assert p3.NLOC == 20
    lam_nodes = p3.ALPHAS / 3.0
    V = p3.basis(lam_nodes)               # V[j, i] = phi_i(node_j)
    np.testing.assert_allclose(V, np.eye(20), atol=1e-13)


def test_partition_of_unity_and_cubic_reproduction():
    rng = np.random.default_rng(1)
    lam = rng.dirichlet(np.ones(4), size=50)
    phi = p3.basis(lam)
    np.testing.assert_allclose(phi.sum(axis=1), 1.0, atol=1e-13)
    P = _rand_tet(rng)
    X = p3.node_coords(P)
    x = lam @ P
    c = rng.standard_normal(20)

    def cubic(y):
        mons = [y[:, 0] ** a * y[:, 1] ** b * y[:, 2] ** d
                for a in range(4) for b in range(4) for d in range(4) if a + b + d <= 3]
        return np.stack(mons, axis=1) @ c

    np.testing.assert_allclose(phi @ cubic(X), cubic(x), rtol=1e-11, atol=1e-11)


def test_basis_derivative_matches_finite_difference():
    rng = np.random.default_rng(2)
    lam = rng.dirichlet(np.ones(4), size=10)
    d = p3.basis_dlam(lam)
    h = 1e-6
    for a in range(4):
        lp, lm = lam.copy(), lam.copy()
        lp[:, a] += h
        lm[:, a] -= h
        fd = (p3.basis(lp) - p3.basis(lm)) / (2 * h)
        np.testing.assert_allclose(d[:, :, a], fd, atol=1e-7)


@pytest.mark.parametrize("n", [4, 6, 8])
def test_tet_rule_exact_monomials(n):
    # int over a simplex of lambda^alpha = |T| * 3! * alpha! / (|alpha| + 3)!
    lam, w = p3.tet_rule(n)
    assert w.sum() == pytest.approx(1.0 / 6.0, rel=1e-14)
    for al in itertools.product(range(2 * n), repeat=4):
        if sum(al) > 2 * n - 1:
            continue
        exact = (1.0 / 6.0) * 6.0 * np.prod([math.factorial(a) for a in al]) / math.factorial(sum(al) + 3)
        got = np.sum(w * np.prod(lam ** np.array(al), axis=1))
        assert got == pytest.approx(exact, rel=1e-12, abs=1e-16), al


@pytest.mark.parametrize("n", [4, 8])
def test_tri_rule_exact_monomials(n):
    lam, w = p3.tri_rule(n)
    assert w.sum() == pytest.approx(0.5, rel=1e-14)
    for al in itertools.product(range(2 * n), repeat=3):
        if sum(al) > 2 * n - 1:
            continue
        exact = 0.5 * 2.0 * np.prod([math.factorial(a) for a in al]) / math.factorial(sum(al) + 2)
        got = np.sum(w * np.prod(lam ** np.array(al), axis=1))
        assert got == pytest.approx(exact, rel=1e-12, abs=1e-16), al


def test_stiffness_constants_and_linear_energy():
    rng = np.random.default_rng(3)
    for _ in range(5):
        P = _rand_tet(rng)
        vol = abs(np.linalg.det(P[1:] - P[0])) / 6.0
        K, M = p3.element_matrices(P)
        np.testing.assert_allclose(K, K.T, atol=1e-12)
        np.testing.assert_allclose(K @ np.ones(20), 0.0, atol=1e-10 * np.abs(K).max())
        # u = c . x is reproduced exactly: u^T K u = |c|^2 |T|
        c = rng.standard_normal(3)
        u = p3.node_coords(P) @ c
        assert u @ K @ u == pytest.approx(vol * c @ c, rel=1e-11)
        # mass: 1^T M 1 = |T|, 1^T M u = int c.x = |T| c.centroid
        one = np.ones(20)
        assert one @ M @ one == pytest.approx(vol, rel=1e-12)
        assert one @ M @ u == pytest.approx(vol * c @ P.mean(axis=0), rel=1e-11, abs=1e-12)
        # int (c.x)^2 over a simplex = |T|/20 (sum_a y_a^2 + (sum_a y_a)^2), y_a = c.P_a
        y = P @ c
        assert u @ M @ u == pytest.approx(vol / 20.0 * (y @ y + y.sum() ** 2), rel=1e-11)
        w = np.linalg.eigvalsh(K)
        assert w.min() > -1e-10 * w.max()


def test_face_mass_area_and_support():
    rng = np.random.default_rng(4)
    P = _rand_tet(rng)
    for c in range(4):
        B = p3.face_mass(P, c)
        area, nrm = p3.face_area_normal(P, c)
        others = [a for a in range(4) if a != c]
        A_, B_, C_ = P[others]
        assert area == pytest.approx(0.5 * np.linalg.norm(np.cross(B_ - A_, C_ - A_)))
        assert np.dot(nrm, P[c] - A_) < 0       # outward
        one = np.ones(20)
        assert one @ B @ one == pytest.approx(area, rel=1e-12)
        off = np.setdiff1d(np.arange(20), p3.face_nodes(c))
        assert len(p3.face_nodes(c)) == 10
        assert np.abs(B[off]).max() < 1e-14 and np.abs(B[:, off]).max() < 1e-14
        # int_f (c.x) = area * (c . face centroid)
        cc = rng.standard_normal(3)
        u = p3.node_coords(P) @ cc
        assert one @ B @ u == pytest.approx(area * cc @ P[others].mean(axis=0), rel=1e-11, abs=1e-12)
