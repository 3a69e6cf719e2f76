"""Synthetic adaptive Cartesian grids (input data only).

Layout shared by the CUDA library and the oracle
------------------------------------------------
The model volume is a lattice of ``nroot = (nx, ny, nz)`` cubic root cells of
side ``root_size`` whose lower corner is ``root_lo``.  Each root is the top of
an octree.  Nodes are numbered so that the roots come first (x fastest, then y,
then z); a refined node's 8 children are stored contiguously starting at
``first_child[node]`` in the order ``child = bx + 2*by + 4*bz`` (b = 1 for the
upper half along that axis).  ``first_child[node] == -1`` marks a leaf, and
``leaf_of_node[node]`` gives its leaf id (leaves are numbered in node order).
Per-leaf arrays are indexed ``[leaf, lambda]``.

Seeds: a workload ``i`` uses ``numpy.random.default_rng(1709 * 100 + i)`` for
anything random.  Config 1 and config 2 contain nothing random.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 1709 * 100


@dataclasses.dataclass
class Grid:
    nroot: tuple
    root_lo: tuple
    root_size: float
    first_child: np.ndarray          # int32 [n_nodes]
    leaf_of_node: np.ndarray         # int32 [n_nodes]
    leaf_lo: np.ndarray              # float64 [n_leaf, 3] (exact dyadic values)
    leaf_size: np.ndarray            # float64 [n_leaf]
    kappa_rho: np.ndarray            # float32 [n_leaf, n_lambda]  extinction per length
    emissivity: np.ndarray           # float32 [n_leaf, n_lambda]  luminosity / volume / sr
    albedo: np.ndarray               # float32 [n_lambda]
    g: np.ndarray                    # float32 [n_lambda]
    point_xyz: np.ndarray = None     # float32 [n_point, 3]
    point_lum: np.ndarray = None     # float32 [n_point, n_lambda] total luminosity
    name: str = ""

    def __post_init__(self):
        if self.point_xyz is None:
            self.point_xyz = np.zeros((0, 3), np.float32)
        if self.point_lum is None:
            self.point_lum = np.zeros((0, self.n_lambda), np.float32)

    @property
    def n_nodes(self):
        return int(self.first_child.shape[0])

    @property
    def n_leaf(self):
        return int(self.leaf_size.shape[0])

    @property
    def n_lambda(self):
        return int(self.kappa_rho.shape[1])

    @property
    def leaf_centre(self):
        return self.leaf_lo + 0.5 * self.leaf_size[:, None]

    @property
    def model_size(self):
        """Largest linear extent of the model volume."""
        return float(max(self.nroot) * self.root_size)

    def with_lambda(self, kappa_rho, emissivity, albedo, g, name=None):
        return dataclasses.replace(
            self, kappa_rho=np.ascontiguousarray(kappa_rho, np.float32),
            emissivity=np.ascontiguousarray(emissivity, np.float32),
            albedo=np.ascontiguousarray(albedo, np.float32),
            g=np.ascontiguousarray(g, np.float32),
            point_lum=np.zeros((self.point_xyz.shape[0], np.asarray(albedo).size), np.float32)
            if self.point_lum.shape[1] != np.asarray(albedo).size else self.point_lum,
            name=name or self.name)

    def leaf_containing(self, x):
        """Leaf id whose closed box contains point x (first match)."""
        x = np.asarray(x, np.float64)
        inside = np.all((self.leaf_lo <= x) & (x <= self.leaf_lo + self.leaf_size[:, None]), axis=1)
        ids = np.nonzero(inside)[0]
        return int(ids[0]) if ids.size else -1


def refine_tree(nroot, root_lo, root_size, max_level, refine):
    """Build the flattened forest.

    ``refine(lo[N,3], size[N], level) -> bool[N]`` decides which nodes of a
    level get 8 children (never beyond ``max_level``).  Returns
    (first_child, leaf_of_node, leaf_lo, leaf_size).
    """
    nx, ny, nz = nroot
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    lo = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64) * root_size
    lo += np.asarray(root_lo, np.float64)
    size = np.full(lo.shape[0], float(root_size))
    level_lo, level_size = [lo], [size]
    first_child_levels = []
    offset = lo.shape[0]
    level = 0
    while True:
        cur_lo, cur_size = level_lo[-1], level_size[-1]
        if level < max_level:
            mask = np.asarray(refine(cur_lo, cur_size, level), bool)
        else:
            mask = np.zeros(cur_lo.shape[0], bool)
        fc = np.full(cur_lo.shape[0], -1, np.int64)
        nref = int(mask.sum())
        fc[mask] = offset + 8 * np.arange(nref)
        first_child_levels.append(fc)
        if nref == 0:
            break
        half = cur_size[mask] * 0.5
        plo = cur_lo[mask]
        bits = np.array([[b & 1, (b >> 1) & 1, (b >> 2) & 1] for b in range(8)], np.float64)
        clo = (plo[:, None, :] + bits[None, :, :] * half[:, None, None]).reshape(-1, 3)
        csize = np.repeat(half, 8)
        level_lo.append(clo)
        level_size.append(csize)
        offset += 8 * nref
        level += 1
    first_child = np.concatenate(first_child_levels).astype(np.int32)
    all_lo = np.concatenate(level_lo)
    all_size = np.concatenate(level_size)
    is_leaf = first_child < 0
    leaf_of_node = np.full(first_child.shape[0], -1, np.int32)
    leaf_of_node[is_leaf] = np.arange(int(is_leaf.sum()), dtype=np.int32)
    return first_child, leaf_of_node, all_lo[is_leaf].copy(), all_size[is_leaf].copy()


def lattice_grid(n, box_lo=-1.0, box_size=2.0, as_tree=False):
    """Uniform n^3 grid: either an n^3 root lattice, or (n a power of two) one
    root refined uniformly."""
    if as_tree:
        levels = int(round(math.log2(n)))
        assert 2 ** levels == n
        fc, lon, llo, lsz = refine_tree((1, 1, 1), (box_lo,) * 3, box_size, levels,
                                        lambda lo, s, lev: np.ones(lo.shape[0], bool))
        return (1, 1, 1), (box_lo,) * 3, box_size, fc, lon, llo, lsz
    fc, lon, llo, lsz = refine_tree((n, n, n), (box_lo,) * 3, box_size / n, 0,
                                    lambda lo, s, lev: np.zeros(lo.shape[0], bool))
    return (n, n, n), (box_lo,) * 3, box_size / n, fc, lon, llo, lsz


def _assemble(topo, kappa_rho, emissivity, albedo, g, name, point_xyz=None, point_lum=None):
    nroot, root_lo, root_size, fc, lon, llo, lsz = topo
    return Grid(nroot=tuple(int(v) for v in nroot), root_lo=tuple(float(v) for v in root_lo),
                root_size=float(root_size), first_child=fc, leaf_of_node=lon,
                leaf_lo=llo, leaf_size=lsz,
                kappa_rho=np.ascontiguousarray(kappa_rho, np.float32),
                emissivity=np.ascontiguousarray(emissivity, np.float32),
                albedo=np.ascontiguousarray(albedo, np.float32),
                g=np.ascontiguousarray(g, np.float32),
                point_xyz=None if point_xyz is None else np.ascontiguousarray(point_xyz, np.float32),
                point_lum=None if point_lum is None else np.ascontiguousarray(point_lum, np.float32),
                name=name)


def sphere_cube(n, radius=0.8, tau_radial=1.0, source_at=(0.0625, 0.0625, 0.0625),
                albedo=0.6, g=0.6, as_tree=False, box_lo=-1.0, box_size=2.0, lum=1.0,
                name=None):
    """Homogeneous dust sphere in a uniform n^3 box, one emitting cell.

    Dust: kappa*rho = tau_radial / radius in every cell whose centre lies within
    ``radius`` of the origin (centre-in voxelisation), 0 elsewhere.  The cell
    containing ``source_at`` emits total luminosity ``lum`` isotropically
    (emissivity = lum / (4 pi V))."""
    topo = lattice_grid(n, box_lo, box_size, as_tree)
    llo, lsz = topo[5], topo[6]
    centre = llo + 0.5 * lsz[:, None]
    r = np.sqrt((centre ** 2).sum(1))
    kr = np.where(r <= radius, tau_radial / radius, 0.0)[:, None]
    inside = np.all((llo <= np.asarray(source_at)) & (np.asarray(source_at) < llo + lsz[:, None]), axis=1)
    src = int(np.nonzero(inside)[0][0])
    emis = np.zeros((llo.shape[0], 1))
    emis[src, 0] = lum / (4.0 * math.pi * lsz[src] ** 3)
    return _assemble(topo, kr, emis, [albedo], [g], name or f"sphere{n}")


def config1(as_tree=False):
    """16^3 uniform grid, box side 2 kpc, homogeneous dust sphere of radius
    0.8 kpc with radial tau_V = 1, one emitting cell with L = 1 (the 16^3 grid
    has no central cell: the source is the cell whose centre is
    (0.0625, 0.0625, 0.0625) kpc), albedo 0.6, g = 0.6."""
    return sphere_cube(16, as_tree=as_tree, name="sphere16")


def small_sphere(n=9, cell=0.25, **kw):
    """Odd-n variant with an exact central source cell (for symmetry pins).
    Cells have the dyadic side ``cell`` so every face coordinate is exact."""
    return sphere_cube(n, source_at=(0.0, 0.0, 0.0), box_lo=-0.5 * n * cell,
                       box_size=n * cell, **kw)


# --------------------------------------------------------------------------- galaxy
def _disk_bulge_emissivity(c, h_s, z_s, r_e, bt):
    R = np.sqrt(c[:, 0] ** 2 + c[:, 1] ** 2)
    r = np.sqrt((c ** 2).sum(1))
    disk = np.exp(-R / h_s - np.abs(c[:, 2]) / z_s)
    b4 = 7.669
    bulge = np.exp(-b4 * (r / r_e) ** 0.25)
    return disk, bulge


def galaxy_disk(max_level=6, tau_b=2.0, h_d=4.5, z_d=0.2, h_s=3.0, z_s=0.3, r_e=1.0,
                bt=0.3, threshold=0.1, nroot=(9, 9, 1), root_size=4.0,
                albedo=0.6, g=0.6, n_lambda=1, name="galaxy"):
    """Exponential-disk galaxy on an adaptive grid.

    Root cubes of ``root_size`` kpc tile the box; a node is refined (up to
    ``max_level`` times) where max(kappa*rho) over the node times its side
    exceeds ``threshold`` (the cell optical depth).  Dust:
    kappa*rho = tau_b / (2 z_d) * exp(-R/h_d - |z|/z_d).  Stars: exponential
    disk exp(-R/h_s - |z|/z_s) plus a Sersic n=4 bulge
    exp(-7.669 (r/r_e)^(1/4)), bulge-to-total ``bt``, total luminosity 1.
    Values are taken at cell centres."""
    k0 = tau_b / (2.0 * z_d)
    root_lo = (-0.5 * nroot[0] * root_size, -0.5 * nroot[1] * root_size, -0.5 * nroot[2] * root_size)

    def refine(lo, size, level):
        hi = lo + size[:, None]
        # closest point of the box to the z axis and to the mid plane
        cx = np.clip(0.0, lo[:, 0], hi[:, 0])
        cy = np.clip(0.0, lo[:, 1], hi[:, 1])
        cz = np.clip(0.0, lo[:, 2], hi[:, 2])
        kmax = k0 * np.exp(-np.sqrt(cx ** 2 + cy ** 2) / h_d - np.abs(cz) / z_d)
        return kmax * size > threshold

    topo = (nroot, root_lo, root_size) + refine_tree(nroot, root_lo, root_size, max_level, refine)
    llo, lsz = topo[5], topo[6]
    c = llo + 0.5 * lsz[:, None]
    R = np.sqrt(c[:, 0] ** 2 + c[:, 1] ** 2)
    kr = k0 * np.exp(-R / h_d - np.abs(c[:, 2]) / z_d)
    disk, bulge = _disk_bulge_emissivity(c, h_s, z_s, r_e, bt)
    V = lsz ** 3
    emis = ((1.0 - bt) * disk / (4 * math.pi * (disk * V).sum())
            + bt * bulge / (4 * math.pi * (bulge * V).sum()))
    if n_lambda == 1:
        return _assemble(topo, kr[:, None], emis[:, None], [albedo], [g], name)
    raise ValueError("use with_lambda() for multi-wavelength variants")


def config2():
    """~3e5-leaf exponential-disk galaxy (4 kpc roots refined up to 6 levels
    where the cell optical depth exceeds the threshold), B band, albedo 0.6,
    g = 0.6.  The threshold 0.145 gives 297,840 leaves."""
    return galaxy_disk(threshold=0.145, name="galaxy3e5")


# --------------------------------------------------------------------------- clumpy cubes
def lognormal_cube(n, seed_index, tau_mean=2.0, sigma_ln=1.0, smooth_cells=2.0, n_src=16,
                   box_size=2.0, albedo=0.6, g=0.6, name=None):
    """n^3 lattice with a lognormal density: ln(rho) is white noise smoothed by
    a Gaussian of ``smooth_cells`` cells, renormalised to std ``sigma_ln``;
    kappa*rho is scaled so the mean edge-to-edge optical depth is
    ``tau_mean``.  ``n_src`` cells drawn with probability proportional to rho
    emit a total luminosity 1."""
    rng = np.random.default_rng(SEED_BASE + seed_index)
    noise = rng.standard_normal((n, n, n))
    k = np.fft.fftfreq(n)
    kk = k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2
    field = np.real(np.fft.ifftn(np.fft.fftn(noise) * np.exp(-2 * math.pi ** 2 * smooth_cells ** 2 * kk)))
    field = (field - field.mean()) / field.std() * sigma_ln
    rho = np.exp(field)
    topo = lattice_grid(n, -0.5 * box_size, box_size)
    # lattice leaves are ordered x fastest: leaf id = ix + n*(iy + n*iz); field index [iz, iy, ix]
    rho_leaf = rho.reshape(-1)
    kr = rho_leaf / rho_leaf.mean() * tau_mean / box_size
    p = rho_leaf / rho_leaf.sum()
    src = rng.choice(rho_leaf.size, size=n_src, replace=False, p=p)
    V = (box_size / n) ** 3
    emis = np.zeros(rho_leaf.size)
    emis[src] = 1.0 / (n_src * 4 * math.pi * V)
    return _assemble(topo, kr[:, None], emis[:, None], [albedo], [g], name or f"lognormal{n}")


# --------------------------------------------------------------------------- particle galaxy
def spiral_factor(x, y, amplitude=0.3, pitch_deg=15.0):
    """Two-arm logarithmic spiral modulation 1 + A cos(2 (phi - ln R / tan(pitch)))."""
    R = np.maximum(np.sqrt(x * x + y * y), 1e-6)
    phi = np.arctan2(y, x)
    return 1.0 + amplitude * np.cos(2.0 * (phi - np.log(R) / math.tan(math.radians(pitch_deg))))


def galaxy_particles(n, seed_index=5, h_s=3.0, z_s=0.3, r_e=1.0, bt=0.3, r_max=18.0, z_max=2.0,
                     amplitude=0.3):
    """n star particles: an exponential disk (h_s, z_s) with the two-arm
    spiral modulation (by rejection) and a Sersic n=4 bulge (r_e) holding
    the fraction bt, within |x|, |y| < r_max and |z| < z_max (kpc)."""
    rng = np.random.default_rng(SEED_BASE + seed_index)
    nb = int(round(bt * n))
    nd = n - nb
    out = []
    # disk: R from the Gamma(2, h_s) radial law of an exponential surface density
    got = 0
    while got < nd:
        m = 2 * (nd - got) + 1024
        R = rng.gamma(2.0, h_s, m)
        phi = rng.uniform(-math.pi, math.pi, m)
        z = rng.laplace(0.0, z_s, m)
        x, y = R * np.cos(phi), R * np.sin(phi)
        keep = rng.uniform(0.0, 1.0 + amplitude, m) < spiral_factor(x, y, amplitude)
        keep &= (np.abs(x) < r_max) & (np.abs(y) < r_max) & (np.abs(z) < z_max)
        p = np.stack([x[keep], y[keep], z[keep]], 1)[: nd - got]
        out.append(p)
        got += p.shape[0]
    # bulge: r by inverting the enclosed-light curve of exp(-7.669 (r/r_e)^(1/4)) on a grid
    rr = np.geomspace(1e-4, r_max, 4096)
    dens = np.exp(-7.669 * (rr / r_e) ** 0.25) * rr ** 2
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (dens[1:] + dens[:-1]) * np.diff(rr))])
    cdf /= cdf[-1]
    got = 0
    while got < nb:
        m = 2 * (nb - got) + 1024
        r = np.interp(rng.uniform(0.0, 1.0, m), cdf, rr)
        u = rng.normal(size=(m, 3))
        p = u / np.linalg.norm(u, axis=1)[:, None] * r[:, None]
        keep = (np.abs(p[:, 0]) < r_max) & (np.abs(p[:, 1]) < r_max) & (np.abs(p[:, 2]) < z_max)
        p = p[keep][: nb - got]
        out.append(p)
        got += p.shape[0]
    return np.concatenate(out)


def particle_galaxy(n_particles=4_000_000, max_per_leaf=2, max_level=10, tau_b=2.0, h_d=4.5, z_d=0.2,
                    threshold=0.1, nroot=(9, 9, 1), root_size=4.0, lambdas_um=None, seed_index=5,
                    name="particle_galaxy"):
    """The large SPH-like galaxy: star particles (galaxy_particles) deposited
    on an adaptive tree of root cubes refined, up to max_level times, where a
    node holds more than max_per_leaf particles or its dust optical depth
    (max kappa*rho over the node, spiral crest included, times its side)
    exceeds threshold.  Dust: tau_b/(2 z_d) exp(-R/h_d - |z|/z_d) times the
    spiral modulation at the cell centre.  Emissivity: the leaf's particles,
    of equal luminosity (total 1), per volume and sr.  lambdas_um: the
    wavelengths, kappa ~ lambda^-1.3 normalised at 0.443 um, albedo 0.7 -> 0.4
    and g 0.75 -> 0.4 linear in log lambda from the first to the last; default
    one B-band wavelength with albedo 0.6, g 0.6."""
    p = galaxy_particles(n_particles, seed_index)
    root_lo = np.array([-0.5 * nroot[0] * root_size, -0.5 * nroot[1] * root_size, -0.5 * nroot[2] * root_size])
    k0 = tau_b / (2.0 * z_d)
    rel = p - root_lo[None, :]

    def refine(lo, size, level):
        s = float(size[0])  # every node of a level has the same side
        dims = np.array(nroot, np.int64) << level
        ip = np.floor(rel / s).astype(np.int64)
        keys = ip[:, 0] + dims[0] * (ip[:, 1] + dims[1] * ip[:, 2])
        ukeys, counts = np.unique(keys, return_counts=True)
        il = np.rint((lo - root_lo[None, :]) / s).astype(np.int64)
        nkeys = il[:, 0] + dims[0] * (il[:, 1] + dims[1] * il[:, 2])
        pos = np.clip(np.searchsorted(ukeys, nkeys), 0, max(ukeys.size - 1, 0))
        cnt = np.where(ukeys[pos] == nkeys, counts[pos], 0)
        hi = lo + size[:, None]
        cx, cy, cz = (np.clip(0.0, lo[:, a], hi[:, a]) for a in range(3))
        kmax = k0 * (1.0 + 0.3) * np.exp(-np.sqrt(cx ** 2 + cy ** 2) / h_d - np.abs(cz) / z_d)
        return (cnt > max_per_leaf) | (kmax * size > threshold)

    topo = (tuple(nroot), tuple(root_lo), root_size) + refine_tree(nroot, root_lo, root_size, max_level, refine)
    llo, lsz = topo[5], topo[6]
    c = llo + 0.5 * lsz[:, None]
    R = np.sqrt(c[:, 0] ** 2 + c[:, 1] ** 2)
    kr = k0 * np.exp(-R / h_d - np.abs(c[:, 2]) / z_d) * spiral_factor(c[:, 0], c[:, 1])
    # particles -> leaves by descent, level by level
    fc = topo[3]
    lon = topo[4]
    dims0 = np.array(nroot, np.int64)
    ip = np.floor(rel / root_size).astype(np.int64)
    node = ip[:, 0] + dims0[0] * (ip[:, 1] + dims0[1] * ip[:, 2])
    s = root_size
    off = rel - ip * root_size
    while True:
        child = fc[node]
        inner = child >= 0
        if not inner.any():
            break
        s *= 0.5
        b = (off[inner] >= s).astype(np.int64)
        node[inner] = child[inner] + b[:, 0] + 2 * b[:, 1] + 4 * b[:, 2]
        off[inner] -= b * s
    leaf = lon[node]
    n_leaf = llo.shape[0]
    counts = np.bincount(leaf, minlength=n_leaf).astype(np.float64)
    emis = counts / (n_particles * 4 * math.pi * lsz ** 3)
    if lambdas_um is None:
        return _assemble(topo, kr[:, None], emis[:, None], [0.6], [0.6], name)
    lam = np.asarray(lambdas_um, np.float64)
    t = np.log(lam / lam[0]) / np.log(lam[-1] / lam[0]) if lam.size > 1 else np.zeros(1)
    krl = kr[:, None] * (lam[None, :] / 0.443) ** -1.3
    return _assemble(topo, krl, np.repeat(emis[:, None], lam.size, axis=1), 0.7 - 0.3 * t, 0.75 - 0.35 * t, name)


def config5(n_lambda=16, **kw):
    """The large particle galaxy: 4e6 star particles, an adaptive tree of
    10 levels, 16 wavelengths log-spaced 0.15-2.2 um."""
    lam = np.geomspace(0.15, 2.2, n_lambda) if n_lambda > 1 else None
    return particle_galaxy(lambdas_um=lam, name="galaxy_particles", **kw)
