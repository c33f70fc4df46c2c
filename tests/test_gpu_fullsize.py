"""Full-size checks on the 5 Hz Overthrust-like workload (the bench
configuration): the oracle cannot solve a 0.95M-dof P3 system, so it checks
what holds at any size.

* Sampled rows of A: around 40 random elements, the oracle assembles the
  patch of every element sharing a vertex with them (with the global
  boundary faces of the patch); the rows of the sampled elements' nodes are
  complete there and must equal the library's rows (matched by coordinates).
* Point-source right-hand sides from the oracle on the source's element.
* The GPU wavefields (FP64 and mixed forms, 16 sources, the launch
  configuration bench.py times) satisfy ||F - A u|| / ||F|| <= rtol with the
  library's A, which the sampled rows tie to the oracle.
"""
import numpy as np
import pytest

from oracle import assemble as oa
from paper_2004_07930_gb300 import hz
from paper_2004_07930_gb300 import workloads as wl

from _gpu_common import torch_cuda

pytestmark = pytest.mark.gpu


def _patch(prob, elems):
    f = prob["fine"]
    tets = f["tets"]
    vmark = np.zeros(len(f["xyz"]), dtype=bool)
    vmark[tets[elems].ravel()] = True
    patch = np.nonzero(vmark[tets].any(axis=1))[0]
    sub_t = tets[patch]
    vs, inv = np.unique(sub_t, return_inverse=True)
    sub_xyz = f["xyz"][vs]
    sub_t = inv.reshape(-1, 4)
    # global boundary faces whose three vertices are in the patch and that belong to a patch element
    gmap = -np.ones(len(f["xyz"]), dtype=np.int64)
    gmap[vs] = np.arange(len(vs))
    bf = f["bfaces"]
    inside = (gmap[bf] >= 0).all(axis=1)
    bfl = gmap[bf[inside]]
    keys = {tuple(sorted(r)) for r in bfl.tolist()}
    own = set()
    for t in sub_t.tolist():
        for c in range(4):
            own.add(tuple(sorted(t[:c] + t[c + 1:])))
    keep = np.array([tuple(sorted(r)) in own for r in bfl.tolist()], dtype=bool)
    return patch, sub_xyz, sub_t, bfl[keep].astype(np.int32), f["btags"][inside][keep]


@pytest.fixture(scope="module")
def big():
    torch_cuda()
    return wl.overthrust_problem(5.0)


def test_sampled_rows_of_A_match_oracle(big):
    p = big
    with hz.Solver.from_problem(p, coarse_mode=hz.HZ_COARSE_NONE, precision=hz.HZ_PREC_MIXED) as S:
        A = S.matrix_csr()
        X = S.coords()
    rng = np.random.default_rng(0)
    elems = rng.choice(len(p["fine"]["tets"]), 40, replace=False)
    elems = np.concatenate([elems, [0, len(p["fine"]["tets"]) - 1]])     # include boundary corners
    patch, sxyz, st_, bf, bt = _patch(p, elems)
    space = oa.P3Space(sxyz, st_)
    Ao, dd = oa.assemble(space, p["velocity"][patch], p["freq"], bf, bt)
    from scipy.spatial import cKDTree

    tree = cKDTree(X)
    dist, lib_of = tree.query(space.coords)
    assert dist.max() < 1e-6 * 20000.0
    # rows = nodes of the sampled elements (complete inside the patch)
    loc = {e: i for i, e in enumerate(patch)}
    rows = np.unique(space.l2g[[loc[e] for e in elems]].ravel())
    dirset = set(dd.tolist())
    checked = 0
    scale = abs(A).max()
    for r in rows:
        lr = lib_of[r]
        lib_row = A.getrow(lr)
        if r in dirset:
            assert lib_row.nnz == 1 and lib_row[0, lr] == 1.0
            continue
        orow = Ao.getrow(r)
        cols = orow.indices
        keepc = ~np.isin(cols, dd)
        ref = dict(zip(lib_of[cols[keepc]], orow.data[keepc]))
        got = dict(zip(lib_row.indices, lib_row.data))
        assert set(ref) == set(got)
        for c in ref:
            assert abs(ref[c] - got[c]) <= 1e-12 * scale
        checked += 1
    assert checked > 200


@pytest.mark.parametrize("precision", [hz.HZ_PREC_MIXED, hz.HZ_PREC_FP64])
def test_wavefields_satisfy_the_system(big, precision):
    torch = torch_cuda()
    p = big
    rtol = 1e-6
    with hz.Solver.from_problem(p, precision=precision, rtol=rtol, stream=torch.cuda.current_stream()) as S:
        A = S.matrix_csr()
        X = S.coords()
        out = torch.empty((len(p["src_xyz"]), S.n), dtype=torch.complex128, device="cuda")
        u, st = S.solve(p["src_xyz"], out=out)
        torch.cuda.synchronize()
        u = u.cpu().numpy()
        info = S.info()
    assert st["converged"] == 1 and st["max_rel_residual"] <= rtol
    assert info["perturbed_pivots"] == 0
    from scipy.spatial import cKDTree

    tree = cKDTree(X)
    for q, xs in enumerate(p["src_xyz"]):
        # oracle load on the element patch around the source
        c = wl.centroids(p["fine"]["xyz"], p["fine"]["tets"])
        near = np.argsort(np.linalg.norm(c - xs, axis=1))[:48]
        patch, sxyz, st_, bf, bt = _patch(p, near)
        space = oa.P3Space(sxyz, st_)
        F = oa.point_source(space, xs[None, :], [1.0])[0]
        dd = space.dirichlet_dofs(bf, bt)
        F[dd] = 0.0
        Fl = np.zeros(S.n, dtype=np.complex128)
        nz = np.nonzero(F)[0]
        d, li = tree.query(space.coords[nz])
        assert d.max() < 1e-3
        Fl[li] = F[nz]
        r = Fl - A @ u[q]
        assert np.linalg.norm(r) <= rtol * (1 + 1e-6) * np.linalg.norm(Fl)
