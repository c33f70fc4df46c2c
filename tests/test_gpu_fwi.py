"""FWI misfit and adjoint-state gradient on the device: against the oracle's
gradient on the 6^3-cell cube and against central finite differences of the
library's own misfit (per element on the cube; along a seeded direction on
the 5 Hz Overthrust-like workload)."""
import numpy as np
import pytest

from oracle import assemble as oa
from oracle import fwi as ofwi
from paper_2004_07930_gb300 import fwi, hz
from paper_2004_07930_gb300 import workloads as wl

from _gpu_common import torch_cuda

pytestmark = pytest.mark.gpu


def _cube_case(top_dirichlet):
    p = wl.cube_problem(ncell=6, freq=2.0, top_dirichlet=top_dirichlet, coarse=True)
    src, rec = wl.fwi_acquisition(p, nsrc_xy=(2, 2), nrec_xy=(4, 4), depth=150.0, margin=0.2)
    m0 = 1.0 / p["velocity"] ** 2
    m_true = 1.0 / wl.gaussian_anomaly(p, amp=0.03, seed=5) ** 2
    return p, src, rec, m0, m_true


@pytest.mark.parametrize("top_dirichlet", [False, True])
def test_gradient_matches_oracle(top_dirichlet):
    torch_cuda()
    p, src, rec, m0, m_true = _cube_case(top_dirichlet)
    mesh = p["fine"]
    space = oa.P3Space(mesh["xyz"], mesh["tets"])
    P = ofwi.receiver_matrix(space, rec)
    _, _, U_true, _ = ofwi.forward(mesh, m_true, p["freq"], src)
    d_obs = U_true @ P.T
    chi_o, g_o = ofwi.gradient(mesh, m0, p["freq"], src, P, d_obs)
    opt = hz.default_options(rtol=1e-11, maxit=400)
    chi, g, dsyn, st = fwi.misfit_and_gradient(p, m0, src, rec, d_obs, options=opt)
    assert st["converged"] == 1 and st["ncols"] == 2 * len(src)
    assert abs(chi - chi_o) <= 1e-8 * chi_o
    assert np.abs(g - g_o).max() <= 1e-7 * np.abs(g_o).max()
    _, _, U0, _ = ofwi.forward(mesh, m0, p["freq"], src)
    ref = U0 @ P.T
    assert np.abs(dsyn - ref).max() <= 1e-9 * np.abs(ref).max()


def test_receiver_operator_matches_oracle():
    torch_cuda()
    p, src, rec, m0, _ = _cube_case(True)
    space = oa.P3Space(p["fine"]["xyz"], p["fine"]["tets"])
    P = ofwi.receiver_matrix(space, rec)
    P[:, space.dirichlet_dofs(p["fine"]["bfaces"], p["fine"]["btags"])] = 0.0
    with hz.Solver.from_problem(p) as S:
        idx, w = S.receiver_operator(rec)
        perm = oa.match_dofs(space.coords, S.coords(), 1000.0)
    lib = np.zeros((len(rec), len(perm)))
    for k in range(len(rec)):
        for i in range(20):
            if idx[k, i] >= 0:
                lib[k, idx[k, i]] += w[k, i]
    assert np.abs(lib - P[:, perm]).max() <= 1e-13


def test_gradient_matches_central_differences_per_element():
    torch_cuda()
    p, src, rec, m0, m_true = _cube_case(True)
    opt = hz.default_options(rtol=1e-12, maxit=600)
    d_obs = fwi.synthetic_data(p, m_true, src, rec, options=opt)
    chi, g, _, _ = fwi.misfit_and_gradient(p, m0, src, rec, d_obs, options=opt)
    rng = np.random.Generator(np.random.PCG64(11))
    for e in rng.choice(len(m0), 20, replace=False):
        h = 1e-4 * m0[e]
        mp, mm = m0.copy(), m0.copy()
        mp[e] += h
        mm[e] -= h
        fd = (fwi.misfit_and_gradient(p, mp, src, rec, d_obs, options=opt)[0]
              - fwi.misfit_and_gradient(p, mm, src, rec, d_obs, options=opt)[0]) / (2 * h)
        assert abs(fd - g[e]) <= 1e-4 * max(abs(fd), 1e-2 * np.abs(g).max()), (e, fd, g[e])


def test_autograd_function():
    torch = torch_cuda()
    p, src, rec, m0, m_true = _cube_case(True)
    opt = hz.default_options(rtol=1e-11, maxit=400)
    d_obs = fwi.synthetic_data(p, m_true, src, rec, options=opt)
    m = torch.tensor(m0, dtype=torch.float64, device="cuda", requires_grad=True)
    chi = fwi.Misfit.apply(m, p, src, rec, d_obs, opt)
    (2.0 * chi).backward()
    _, g, _, _ = fwi.misfit_and_gradient(p, m0, src, rec, d_obs, options=opt)
    assert torch.equal(m.grad.cpu(), torch.from_numpy(2.0 * g))


@pytest.mark.slow
def test_gradient_directional_fd_full_size():
    """5 Hz Overthrust-like model (0.95M dofs, 64 subdomains), 32 sources,
    400 receivers at 100 m depth, data of a +-3% Gaussian anomaly of 1 km
    radius, solves at rtol 1e-10 (mixed form: FP32 local solves inside FP64
    FGMRES): the directional derivative g . dm matches central differences
    of chi. dm = m0 sign(g) u with u seeded in [0.5, 1.5]: a direction along
    which the derivative is large against the solver noise, and which exposes
    a wrong scale or a wrong sign on any subset of elements. Per-element
    differences at this size would need two factorisations per element."""
    torch_cuda()
    p = wl.overthrust_problem(5.0)
    src, rec = wl.fwi_acquisition(p)
    m0 = 1.0 / p["velocity"] ** 2
    m_true = 1.0 / wl.gaussian_anomaly(p, amp=0.03, radius=1000.0, seed=1) ** 2
    opt = hz.default_options(rtol=1e-10, maxit=3000, coarse_mode=hz.HZ_COARSE_NONE, precision=hz.HZ_PREC_MIXED)
    d_obs = fwi.synthetic_data(p, m_true, src, rec, options=opt)
    chi, g, _, st = fwi.misfit_and_gradient(p, m0, src, rec, d_obs, options=opt)
    assert st["converged"] == 1 and chi > 0
    rng = np.random.Generator(np.random.PCG64(2))
    dm = m0 * np.sign(g) * rng.uniform(0.5, 1.5, len(m0))
    h = 1e-4  # the +-h dm models change chi by ~35%: central differences still O(h^2) accurate
    cp = fwi.misfit_and_gradient(p, m0 + h * dm, src, rec, d_obs, options=opt)[0]
    cm = fwi.misfit_and_gradient(p, m0 - h * dm, src, rec, d_obs, options=opt)[0]
    fd = (cp - cm) / (2 * h)
    print("chi %.6e  fd %.6e  g.dm %.6e" % (chi, fd, g @ dm))
    assert abs(fd - g @ dm) <= 1e-3 * abs(fd), (chi, fd, g @ dm)
