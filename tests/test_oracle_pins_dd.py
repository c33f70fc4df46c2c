"""Hand-derived pins for the domain-decomposition rules of the oracle.

The paper leaves three rules of Eq. oras / Eq. 2lvl unstated; the oracle and
the library take the same readings, so each one is pinned here against an
answer worked out by hand on a tiny Kuhn grid (not recomputed by the rule):

* overlap_elements: one layer = every element sharing a VERTEX with the
  non-overlapping set (a face-sharing rule gives a different, smaller set);
* ownership: a dof belongs to the LOWEST-index subdomain whose own elements
  carry it (not the subdomain of the first element met, not the highest);
* coarse_partition_and_velocity: a coarse element takes the squared slowness
  m = 1/v^2 averaged over the fine elements inside it by volume (not the
  mean of v), and the subdomain of the fine element holding its centroid
  (lowest index when the centroid lies on a subdomain boundary).

Each pin is a predicate on a candidate rule; every test also checks that a
planted wrong rule (the plausible alternative reading) fails the same pin.
"""
import itertools

import numpy as np

from oracle import assemble as oa
from oracle import schwarz as osw
from paper_2004_07930_gb300 import workloads as wl

KUHN = list(itertools.permutations(range(3)))  # the 6 tets of a hex, in kuhn_grid order


# ---------------------------------------------------------------------------
# overlap: 3 x 1 x 1 unit hexes, hex 0 -> part 0, hexes 1, 2 -> part 1.
# Every Kuhn tet of the hex [1,2]x[0,1]^2 has the vertex (1,0,0) (its v0),
# so all 6 touch hex 0; none of hex [2,3] does. Every Kuhn tet of hex 0 has
# the vertex (1,1,1) (its v3), so all 6 touch hex 1.
#   part 0: hexes 0, 1 -> elements 0..11   (face rule: 6 + the 2 tets of hex 1
#           whose permutation puts x last, i.e. a face on x = 1)
#   part 1: all 18 elements                 (face rule: 12 + the 2 tets of
#           hex 0 whose permutation puts x first)
# ---------------------------------------------------------------------------
def _strip3():
    xyz, tets, hexes = wl.kuhn_grid([0.0, 1.0, 2.0, 3.0], [0.0, 1.0], [0.0, 1.0])
    part = np.where(hexes[:, 0] == 0, 0, 1)
    return xyz, tets, hexes, part


def overlap_pin_holds(rule):
    _, tets, _, part = _strip3()
    ok0 = np.array_equal(np.sort(rule(tets, part, 0)), np.arange(12))
    ok1 = np.array_equal(np.sort(rule(tets, part, 1)), np.arange(18))
    return ok0 and ok1


def _face_sharing_overlap(tets, part, i):
    """Planted wrong reading: grow by elements sharing a FACE."""
    tets = np.asarray(tets)
    own = set(np.nonzero(part == i)[0].tolist())
    faces = set()
    for e in own:
        for c in range(4):
            faces.add(tuple(sorted(int(tets[e][a]) for a in range(4) if a != c)))
    out = set(own)
    for e in range(len(tets)):
        for c in range(4):
            if tuple(sorted(int(tets[e][a]) for a in range(4) if a != c)) in faces:
                out.add(e)
    return np.array(sorted(out))


def test_overlap_is_vertex_sharing():
    assert overlap_pin_holds(osw.overlap_elements)
    assert not overlap_pin_holds(_face_sharing_overlap)
    # the face rule's own sets, derived above by hand
    _, tets, _, part = _strip3()
    assert len(_face_sharing_overlap(tets, part, 0)) == 8
    assert len(_face_sharing_overlap(tets, part, 1)) == 14


def test_second_overlap_layer():
    """Two layers from hex 0 reach every tet of hex 2 that touches the plane
    x = 2 (all 6: their v0 = (2,0,0)) -> all 18 elements; one layer from
    hex 2 (part 2) reaches hex 1 only."""
    _, tets, hexes, _ = _strip3()
    part = hexes[:, 0].astype(np.int64)
    assert np.array_equal(osw.overlap_elements(tets, part, 0, 2), np.arange(18))
    assert np.array_equal(osw.overlap_elements(tets, part, 2, 1), np.arange(6, 18))


# ---------------------------------------------------------------------------
# ownership: same strip, hex 0 -> part 1, hexes 1, 2 -> part 0. The P3 nodes
# on the plane x = 1 are carried by both parts; the lowest index is 0, so
#   owner = 1 for x < 1, owner = 0 for x >= 1.
# A "first element met" rule gives 1 on the plane (element 0 is part 1), a
# "highest index" rule also gives 1 there.
# ---------------------------------------------------------------------------
def ownership_pin_holds(rule):
    xyz, tets, hexes, _ = _strip3()
    part = np.where(hexes[:, 0] == 0, 1, 0)
    space = oa.P3Space(xyz, tets)
    owner = np.asarray(rule(space, part, 2))
    x = space.coords[:, 0]
    want = np.where(x < 1.0 - 1e-9, 1, 0)
    return np.array_equal(owner, want)


def _first_element_owner(space, part, nparts):
    owner = np.full(space.n, -1, dtype=np.int64)
    for e in range(len(space.tets)):
        g = space.l2g[e]
        owner[g] = np.where(owner[g] < 0, part[e], owner[g])
    return owner


def _highest_owner(space, part, nparts):
    owner = np.full(space.n, -1, dtype=np.int64)
    for e in range(len(space.tets)):
        g = space.l2g[e]
        owner[g] = np.maximum(owner[g], part[e])
    return owner


def test_ownership_is_lowest_index():
    assert ownership_pin_holds(osw.ownership)
    assert not ownership_pin_holds(_first_element_owner)
    assert not ownership_pin_holds(_highest_owner)


# ---------------------------------------------------------------------------
# coarse element data: fine grid 4 x 2 x 2 unit hexes, coarse grid its 2x
# coarsening (2 x 1 x 1 hexes of side 2). Fine v = 1000 m/s for x < 1, else
# 2000 m/s; fine part = 1 for x < 1, else 0.
# A coarse Kuhn tet of the hex [0,2]^3 is {x_p0 >= x_p1 >= x_p2} (p its
# permutation). The fraction of its volume with x < 1 is 1/8, 1/2 or 7/8
# when x is p0, p1 or p2 (largest, median or smallest of three ordered
# coordinates: P(all < 1), P(median < 1), 1 - P(all >= 1)); the region is a
# union of fine tets (x = 1 is a fine grid plane), so
#   m_c = f / 1000^2 + (1 - f) / 2000^2,  f in {1/8, 1/2, 7/8}.
# Its centroid has x = 1.5, 1.0 or 0.5 for the same three cases, so its part
# is 0, 0 (centroid on the plane x = 1: parts 1 and 0 touch -> lowest, 0) or
# 1. Coarse tets of the hex [2,4] x [0,2]^2: m = 1/2000^2, part 0.
# ---------------------------------------------------------------------------
def _coarse_case():
    fine = wl._mesh_bundle(np.arange(5.0), np.arange(3.0), np.arange(3.0), False)
    coarse = wl._mesh_bundle(np.arange(0.0, 5.0, 2.0), np.arange(0.0, 3.0, 2.0), np.arange(0.0, 3.0, 2.0), False)
    sf = oa.P3Space(fine["xyz"], fine["tets"])
    sc = oa.P3Space(coarse["xyz"], coarse["tets"])
    left = fine["hex_ijk"][:, 0] == 0
    vel = np.where(left, 1000.0, 2000.0)
    part = np.where(left, 1, 0)
    return sf, sc, coarse, part, vel


def _expected_coarse(coarse):
    m1, m2 = 1.0 / 1000.0 ** 2, 1.0 / 2000.0 ** 2
    frac = {0: 1.0 / 8.0, 1: 0.5, 2: 7.0 / 8.0}      # by the rank of x in the permutation
    part_of_rank = {0: 0, 1: 0, 2: 1}
    part_c, m_c = [], []
    for h, p in zip(coarse["hex_ijk"], itertools.cycle(KUHN)):
        if h[0] == 0:
            r = p.index(0)
            part_c.append(part_of_rank[r])
            m_c.append(frac[r] * m1 + (1.0 - frac[r]) * m2)
        else:
            part_c.append(0)
            m_c.append(m2)
    return np.array(part_c), 1.0 / np.sqrt(np.array(m_c))


def coarse_pin_holds(rule):
    sf, sc, coarse, part, vel = _coarse_case()
    part_c, vel_c = rule(sf, sc, part, vel)
    want_part, want_vel = _expected_coarse(coarse)
    return np.array_equal(np.asarray(part_c), want_part) and np.allclose(vel_c, want_vel, rtol=1e-12, atol=0.0)


def _mean_velocity_rule(space_f, space_c, part_f, velocity_f):
    """Planted wrong reading: coarse v = volume-weighted mean of fine v."""
    part_c, _ = osw.coarse_partition_and_velocity(space_f, space_c, part_f, velocity_f)
    Pf = space_f.xyz[space_f.tets]
    vol = np.abs(np.linalg.det(Pf[:, 1:] - Pf[:, :1])) / 6.0
    ef, _ = osw.locate_points(space_c, Pf.mean(axis=1))
    vs = np.bincount(ef, weights=vol * velocity_f, minlength=len(space_c.tets))
    w = np.bincount(ef, weights=vol, minlength=len(space_c.tets))
    return part_c, vs / w


def _highest_part_rule(space_f, space_c, part_f, velocity_f):
    """Planted wrong reading: the highest subdomain on a tie."""
    _, vel_c = osw.coarse_partition_and_velocity(space_f, space_c, part_f, velocity_f)
    pc, _ = osw.coarse_partition_and_velocity(space_f, space_c, -np.asarray(part_f), velocity_f)
    return -pc, vel_c


def test_coarse_partition_and_velocity():
    assert coarse_pin_holds(osw.coarse_partition_and_velocity)
    assert not coarse_pin_holds(_mean_velocity_rule)
    assert not coarse_pin_holds(_highest_part_rule)
