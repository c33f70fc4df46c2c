"""Seeded synthetic inputs: graded Kuhn tensor-grid meshes, velocity models,
boundary tags, box partitions and source sets.

This module holds input generation only (no discretisation, no solver
arithmetic). Both the CUDA path and the CPU oracle take their inputs from it.

Problem setting (Sec. "Tetrahedral finite element method"): Helmholtz on a
box Omega with a free surface (homogeneous Dirichlet) on top and first-order
absorbing faces elsewhere; sources near the surface; P3 elements whose size
follows the local wavelength (h-adaptivity, five nodes per local wavelength,
half that on the coarse mesh of the two-level method, Sec. "Numerical
results").

Conventions: metres, m/s, Hz; z is depth, positive downwards, z = 0 the
surface.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

ROBIN = 0
DIRICHLET = 1


# ----------------------------------------------------------------------------
# Kuhn tensor grid
# ----------------------------------------------------------------------------
_KUHN_PERMS = list(itertools.permutations(range(3)))


def kuhn_grid(xs, ys, zs):
    """Tensor grid with node planes xs, ys, zs; every hex split into 6 Kuhn
    tetrahedra (one per permutation p: v0 = (0,0,0), v_{k+1} = v_k + e_p(k)).

    The same main diagonal in every hex keeps the mesh conforming and nested
    under 2x refinement. Returns (xyz [nv,3] float64, tets [ne,4] int32,
    hex_ijk [ne,3] int32).
    """
    xs, ys, zs = (np.asarray(a, dtype=np.float64) for a in (xs, ys, zs))
    nx, ny, nz = len(xs) - 1, len(ys) - 1, len(zs) - 1
    X, Y, Z = np.meshgrid(xs, ys, zs, indexing="ij")
    # vertex id = i + (nx+1) * (j + (ny+1) * k)
    xyz = np.stack([X.transpose(2, 1, 0).ravel(), Y.transpose(2, 1, 0).ravel(),
                    Z.transpose(2, 1, 0).ravel()], axis=1)

    def vid(i, j, k):
        return i + (nx + 1) * (j + (ny + 1) * k)

    I, J, K = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    I, J, K = (a.transpose(2, 1, 0).ravel() for a in (I, J, K))  # hex order: i fastest
    tets = []
    hexes = []
    for p in _KUHN_PERMS:
        off = np.zeros(3, dtype=np.int64)
        verts = [vid(I, J, K)]
        for a in p:
            off[a] += 1
            verts.append(vid(I + off[0], J + off[1], K + off[2]))
        tets.append(np.stack(verts, axis=1))
        hexes.append(np.stack([I, J, K], axis=1))
    # order: hex-major, the 6 Kuhn tets of one hex contiguous
    tets = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    hexes = np.stack(hexes, axis=1).reshape(-1, 3).astype(np.int32)
    return xyz, tets, hexes


def boundary_faces(xyz, tets, top_dirichlet):
    """Exterior triangles of a tet mesh with their boundary tags.

    A triangle on the plane z = min(z) is DIRICHLET when `top_dirichlet`
    (free surface), every other exterior triangle ROBIN (first-order
    absorbing). Returns (bfaces [nbf,3] int32, tags [nbf] int32).
    """
    tets = np.asarray(tets)
    faces = np.concatenate([tets[:, [1, 2, 3]], tets[:, [0, 2, 3]],
                            tets[:, [0, 1, 3]], tets[:, [0, 1, 2]]], axis=0)
    key = np.sort(faces, axis=1)
    uniq, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    ext = uniq[cnt == 1]
    z = xyz[:, 2]
    ztop = z.min()
    on_top = np.all(np.abs(z[ext] - ztop) <= 1e-9 * max(1.0, abs(z.max() - ztop)), axis=1)
    tags = np.full(len(ext), ROBIN, dtype=np.int32)
    if top_dirichlet:
        tags[on_top] = DIRICHLET
    return ext.astype(np.int32), tags


def box_partition(hex_ijk, ncells, nparts_xyz):
    """Element -> subdomain map of a box partition of the hex-cell grid.

    Cell index range [0, n) along each axis is cut into p contiguous slabs
    (slab of cell i = floor(i * p / n)); subdomain id = px-fastest.
    """
    hex_ijk = np.asarray(hex_ijk)
    parts = np.zeros(len(hex_ijk), dtype=np.int64)
    stride = 1
    for a in range(3):
        n, p = ncells[a], nparts_xyz[a]
        parts += stride * ((hex_ijk[:, a].astype(np.int64) * p) // n)
        stride *= p
    return parts.astype(np.int32)


def best_box_layout(ncells, nparts):
    """px*py*pz = nparts minimising the count of interface cell faces; ties
    go to larger px, then larger py."""
    best = None
    for px in range(1, nparts + 1):
        if nparts % px:
            continue
        for py in range(1, nparts // px + 1):
            if (nparts // px) % py:
                continue
            pz = nparts // (px * py)
            if px > ncells[0] or py > ncells[1] or pz > ncells[2]:
                continue
            nx, ny, nz = ncells
            faces = (px - 1) * ny * nz + (py - 1) * nx * nz + (pz - 1) * nx * ny
            key = (faces, -px, -py)
            if best is None or key < best[0]:
                best = (key, (px, py, pz))
    if best is None:
        raise ValueError("no box layout with %d parts fits %s cells" % (nparts, ncells))
    return best[1]


def centroids(xyz, tets):
    return xyz[np.asarray(tets)].mean(axis=1)


# ----------------------------------------------------------------------------
# Overthrust-like velocity model (synthetic stand-in for SEG/EAGE Overthrust)
# ----------------------------------------------------------------------------
class OverthrustLike:
    """v(x,y,z) on the 20 x 20 x 4.65 km box.

    Background 2300 + 3700 (z/4650)^0.8 m/s; six folded interfaces
    z_k = 4650 k/7 + 300 sin(2 pi x/7000 + phi_k) cos(2 pi y/9000);
    offset dv = 400 (-1)^(L+1) with L the number of interfaces above the
    point; times (1 + 0.05 g) with g a unit-variance Gaussian random field of
    500 m correlation length (white noise on a 100 m grid smoothed by a
    Gaussian kernel); clipped to [2300, 6000]. NumPy PCG64(seed): phi_k are
    the first six draws, then the noise.
    """

    LX, LY, LZ = 20000.0, 20000.0, 4650.0

    def __init__(self, seed=0, dx_noise=100.0, corr=500.0):
        from scipy import ndimage

        rng = np.random.Generator(np.random.PCG64(seed))
        self.phi = rng.uniform(0.0, 2.0 * math.pi, size=6)
        self.dx = dx_noise
        shape = (int(round(self.LX / dx_noise)) + 1, int(round(self.LY / dx_noise)) + 1,
                 int(math.ceil(self.LZ / dx_noise)) + 1)
        w = rng.standard_normal(shape)
        # smoothing white noise with a Gaussian of std s gives covariance
        # exp(-r^2 / (4 s^2)); s = corr / sqrt(2) gives exp(-r^2 / (2 corr^2))
        s = corr / math.sqrt(2.0) / dx_noise
        g = ndimage.gaussian_filter(w, sigma=s, mode="reflect")
        g = (g - g.mean()) / g.std()
        self.g = g

    def interfaces(self, x, y):
        k = np.arange(1, 7)
        z0 = self.LZ * k / 7.0
        return z0[None, :] + 300.0 * np.sin(2 * math.pi * x[:, None] / 7000.0 + self.phi[None, :]) \
            * np.cos(2 * math.pi * y[:, None] / 9000.0)

    def background(self, x, y, z):
        x, y, z = (np.atleast_1d(np.asarray(a, dtype=np.float64)) for a in (x, y, z))
        zi = self.interfaces(x, y)
        L = (zi < z[:, None]).sum(axis=1)
        dv = 400.0 * np.where((L + 1) % 2 == 0, 1.0, -1.0)
        return 2300.0 + 3700.0 * (np.clip(z, 0, None) / self.LZ) ** 0.8 + dv

    def noise(self, x, y, z):
        p = np.stack([x, y, z], axis=1) / self.dx
        hi = np.array(self.g.shape) - 1
        p = np.clip(p, 0, hi - 1e-9)
        i0 = np.floor(p).astype(np.int64)
        t = p - i0
        out = np.zeros(len(p))
        for c in itertools.product((0, 1), repeat=3):
            wgt = np.ones(len(p))
            for a in range(3):
                wgt *= t[:, a] if c[a] else (1.0 - t[:, a])
            out += wgt * self.g[i0[:, 0] + c[0], i0[:, 1] + c[1], i0[:, 2] + c[2]]
        return out

    def __call__(self, x, y, z):
        x, y, z = (np.atleast_1d(np.asarray(a, dtype=np.float64)) for a in (x, y, z))
        v = self.background(x, y, z) * (1.0 + 0.05 * self.noise(x, y, z))
        return np.clip(v, 2300.0, 6000.0)


def _even_up(n):
    n = max(2, int(n))
    return n + (n % 2)


def graded_axis_z(model_vmin_of_z, depth, freq, cells_per_wavelength=1.3, nsamp=2000):
    """Vertical node planes with dz(z) = vmin(z) / (cpw f), fitted to `depth`.

    The coarse planes (every other node) are uniform in
    tau(z) = integral of cpw f / vmin(z') dz'; the fine cell count is
    ceil(tau(depth)) rounded up to even, and every fine cell is one half of a
    coarse cell (midpoint split), so that the Kuhn split of the 2x coarser
    grid is nested in the fine one.
    """
    z = np.linspace(0.0, depth, nsamp + 1)
    dens = cells_per_wavelength * freq / model_vmin_of_z(z)
    tau = np.concatenate([[0.0], np.cumsum(0.5 * (dens[1:] + dens[:-1]) * np.diff(z))])
    nz = _even_up(math.ceil(tau[-1] - 1e-9))
    targets = np.linspace(0.0, tau[-1], nz // 2 + 1)
    zc = np.interp(targets, tau, z)
    zc[0], zc[-1] = 0.0, depth
    zs = np.empty(nz + 1)
    zs[0::2] = zc
    zs[1::2] = 0.5 * (zc[1:] + zc[:-1])
    return zs


def overthrust_grid(freq, model=None, cells_per_wavelength=1.3, vmin_h=2300.0):
    """Graded tensor grid for the Overthrust-like box at frequency `freq`:
    horizontal spacing vmin_h / (cpw f) (uniform, counts even), vertical
    spacing graded on the horizontal minimum of the background velocity."""
    m = model if model is not None else OverthrustLike(0)
    h = vmin_h / (cells_per_wavelength * freq)
    nx = _even_up(math.ceil(m.LX / h - 1e-9))
    ny = _even_up(math.ceil(m.LY / h - 1e-9))
    xs = np.linspace(0.0, m.LX, nx + 1)
    ys = np.linspace(0.0, m.LY, ny + 1)
    gx, gy = np.meshgrid(np.linspace(0, m.LX, 81), np.linspace(0, m.LY, 81), indexing="ij")
    gx, gy = gx.ravel(), gy.ravel()

    def vmin(zz):
        out = np.empty_like(zz)
        for i, zv in enumerate(zz):
            out[i] = np.clip(m.background(gx, gy, np.full_like(gx, zv)), 2300.0, 6000.0).min()
        return out

    zs = graded_axis_z(vmin, m.LZ, freq, cells_per_wavelength, nsamp=400)
    return xs, ys, zs


# ----------------------------------------------------------------------------
# Problem bundles
# ----------------------------------------------------------------------------
def _mesh_bundle(xs, ys, zs, top_dirichlet):
    xyz, tets, hexes = kuhn_grid(xs, ys, zs)
    bf, bt = boundary_faces(xyz, tets, top_dirichlet)
    return dict(xs=np.asarray(xs, float), ys=np.asarray(ys, float), zs=np.asarray(zs, float),
                xyz=xyz, tets=tets, hex_ijk=hexes, bfaces=bf, btags=bt,
                ncells=(len(xs) - 1, len(ys) - 1, len(zs) - 1))


def make_problem(xs, ys, zs, velocity_fn, freq, nparts_xyz, src_xyz, src_amp=None,
                 top_dirichlet=True, coarse=True):
    """Fine mesh + optional nested 2x-coarser mesh + partition + sources.

    velocity per element = velocity_fn at the element centroid.
    """
    fine = _mesh_bundle(xs, ys, zs, top_dirichlet)
    c = centroids(fine["xyz"], fine["tets"])
    vel = np.asarray(velocity_fn(c[:, 0], c[:, 1], c[:, 2]), dtype=np.float64)
    part = box_partition(fine["hex_ijk"], fine["ncells"], nparts_xyz)
    src_xyz = np.asarray(src_xyz, dtype=np.float64).reshape(-1, 3)
    if src_amp is None:
        src_amp = np.ones(len(src_xyz), dtype=np.complex128)
    prob = dict(fine=fine, velocity=vel, freq=float(freq), elem_part=part,
                nparts=int(np.prod(nparts_xyz)), nparts_xyz=tuple(nparts_xyz),
                src_xyz=src_xyz, src_amp=np.asarray(src_amp, dtype=np.complex128))
    if coarse:
        if any((len(a) - 1) % 2 for a in (xs, ys, zs)):
            raise ValueError("nested coarse grid needs even cell counts")
        prob["coarse"] = _mesh_bundle(xs[::2], ys[::2], zs[::2], top_dirichlet)
    return prob


def cube_problem(ncell=6, freq=2.0, v=2000.0, L=1000.0, nparts_xyz=(2, 2, 1),
                 src=((500.0, 500.0, 100.0),), top_dirichlet=False, coarse=True):
    """Homogeneous cube [0,L]^3, ncell^3 hexes x 6 Kuhn tets, all faces Robin
    unless `top_dirichlet`. Default: 6^3 cells, 2 Hz, 2000 m/s, 4 boxes."""
    g = np.linspace(0.0, L, ncell + 1)
    return make_problem(g, g, g, lambda x, y, z: np.full(len(x), float(v)), freq,
                        nparts_xyz, src, top_dirichlet=top_dirichlet,
                        coarse=coarse and ncell % 2 == 0)


def surface_source_grid(nx, ny, x0, x1, depth=100.0):
    xs = np.linspace(x0, x1, nx)
    ys = np.linspace(x0, x1, ny)
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), np.full(X.size, depth)], axis=1)


def overthrust_problem(freq=5.0, nparts=64, seed=0, sources=None, crop=None,
                       cells_per_wavelength=1.3):
    """Overthrust-like graded problem: Dirichlet top, Robin elsewhere.

    sources default: 4x4 surface grid at x, y in {2.5, 7.5, 12.5, 17.5} km,
    z = 100 m. `crop=(fx, fy, fz)` keeps the leading fraction of cells along
    each axis (rounded to even counts) with its own boundary faces.
    """
    model = OverthrustLike(seed)
    xs, ys, zs = overthrust_grid(freq, model, cells_per_wavelength)
    if crop is not None:
        def cut(a, f):
            n = _even_up(round((len(a) - 1) * f))
            return a[: n + 1]
        xs, ys, zs = cut(xs, crop[0]), cut(ys, crop[1]), cut(zs, crop[2])
    ncells = (len(xs) - 1, len(ys) - 1, len(zs) - 1)
    layout = best_box_layout(ncells, nparts)
    if sources is None:
        s = np.array([2500.0, 7500.0, 12500.0, 17500.0])
        X, Y = np.meshgrid(s, s, indexing="ij")
        sources = np.stack([X.ravel(), Y.ravel(), np.full(16, 100.0)], axis=1)
        if crop is not None:
            keep = (sources[:, 0] < xs[-1]) & (sources[:, 1] < ys[-1])
            sources = sources[keep]
    prob = make_problem(xs, ys, zs, model, freq, layout, sources, top_dirichlet=True)
    prob["model_seed"] = seed
    return prob


def random_rhs(n, ns, seed):
    """Seeded complex normal block [ns, n] (test right-hand sides)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((ns, n)) + 1j * rng.standard_normal((ns, n))


# ----------------------------------------------------------------------------
# FWI inputs: acquisition and a perturbed "true" model
# ----------------------------------------------------------------------------
def gaussian_anomaly(prob, amp=0.03, radius=None, seed=0):
    """Per-element velocity of `prob` times (1 + sign * amp * exp(-|x-c|^2 /
    (2 radius^2))): one Gaussian anomaly of +-amp (sign and centre c drawn
    from PCG64(seed); c uniform in the middle half of the box); radius
    defaults to 1/8 of the smallest box side."""
    rng = np.random.Generator(np.random.PCG64(seed))
    fine = prob["fine"]
    lo = np.array([fine["xs"][0], fine["ys"][0], fine["zs"][0]])
    hi = np.array([fine["xs"][-1], fine["ys"][-1], fine["zs"][-1]])
    sign = 1.0 if rng.uniform() < 0.5 else -1.0
    c = lo + (hi - lo) * rng.uniform(0.25, 0.75, size=3)
    r = (hi - lo).min() / 8.0 if radius is None else radius
    x = centroids(fine["xyz"], fine["tets"])
    return prob["velocity"] * (1.0 + sign * amp * np.exp(-((x - c) ** 2).sum(axis=1) / (2.0 * r * r)))


def fwi_acquisition(prob, nsrc_xy=(8, 4), nrec_xy=(20, 20), depth=100.0, margin=0.05):
    """Sources on a regular nsrc_xy grid and receivers on a regular nrec_xy
    grid, both at `depth` below the top face, inset by `margin` of the box."""
    fine = prob["fine"]
    x0, x1 = fine["xs"][0], fine["xs"][-1]
    y0, y1 = fine["ys"][0], fine["ys"][-1]
    z = fine["zs"][0] + depth

    def grid(nx, ny):
        xs = np.linspace(x0 + margin * (x1 - x0), x1 - margin * (x1 - x0), nx)
        ys = np.linspace(y0 + margin * (y1 - y0), y1 - margin * (y1 - y0), ny)
        X, Y = np.meshgrid(xs, ys, indexing="ij")
        return np.stack([X.ravel(), Y.ravel(), np.full(X.size, z)], axis=1)

    return grid(*nsrc_xy), grid(*nrec_xy)
