"""Pin of the oracle's FWI gradient: central finite differences of the
misfit (an independent route: forward solves only) on a small cube with a
Dirichlet top, so that the mass term, the Robin term and the Dirichlet
masking all enter."""
import numpy as np

from oracle import assemble as oa
from oracle import fwi
from paper_2004_07930_gb300 import workloads as wl


def test_adjoint_gradient_matches_central_differences():
    p = wl.cube_problem(ncell=2, freq=2.0, top_dirichlet=True, coarse=False)
    mesh = p["fine"]
    rng = np.random.default_rng(4)
    ne = len(mesh["tets"])
    m0 = (1.0 / 2000.0 ** 2) * (1.0 + 0.1 * rng.standard_normal(ne))
    src = np.array([[300.0, 400.0, 300.0], [650.0, 600.0, 500.0]])
    rec = rng.uniform(100.0, 900.0, size=(5, 3))
    space = oa.P3Space(mesh["xyz"], mesh["tets"])
    P = fwi.receiver_matrix(space, rec)
    m_true = m0 * (1.0 + 0.05 * rng.standard_normal(ne))
    _, _, U_true, _ = fwi.forward(mesh, m_true, p["freq"], src)
    d_obs = U_true @ P.T
    chi, g = fwi.gradient(mesh, m0, p["freq"], src, P, d_obs)
    assert chi > 0
    # elements touching the absorbing faces and interior ones alike
    for e in rng.choice(ne, 6, replace=False):
        h = 1e-4 * m0[e]
        mp, mm = m0.copy(), m0.copy()
        mp[e] += h
        mm[e] -= h
        fd = (fwi.misfit(mesh, mp, p["freq"], src, P, d_obs) - fwi.misfit(mesh, mm, p["freq"], src, P, d_obs)) / (2 * h)
        assert abs(fd - g[e]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(g).max()), (e, fd, g[e])


def test_gradient_vanishes_at_the_true_model():
    p = wl.cube_problem(ncell=2, freq=2.0, top_dirichlet=False, coarse=False)
    mesh = p["fine"]
    ne = len(mesh["tets"])
    m = np.full(ne, 1.0 / 2000.0 ** 2)
    src = np.array([[500.0, 500.0, 300.0]])
    rec = np.array([[200.0, 300.0, 700.0], [800.0, 600.0, 200.0]])
    space = oa.P3Space(mesh["xyz"], mesh["tets"])
    P = fwi.receiver_matrix(space, rec)
    _, _, U, _ = fwi.forward(mesh, m, p["freq"], src)
    chi, g = fwi.gradient(mesh, m, p["freq"], src, P, U @ P.T)
    assert chi == 0.0 and np.all(g == 0.0)
