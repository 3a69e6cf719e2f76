"""Pins of the oracle's grid traversal (the ray-cell intersections every
step of Sect. 2 is built on) by brute force: point location against a scan
of all leaf boxes, and segment lists against dense sampling along the ray."""
import numpy as np
import pytest

import oracle
import synth
from synth.grids import refine_tree, _assemble


def random_tree(seed, nroot=(3, 2, 2), levels=3):
    rng = np.random.default_rng(seed)
    topo = (nroot, (-1.5, -1.0, -1.0), 1.0) + refine_tree(
        nroot, (-1.5, -1.0, -1.0), 1.0, levels, lambda lo, s, lev: rng.random(lo.shape[0]) < 0.45)
    n = topo[5].shape[0]
    return _assemble(topo, np.ones((n, 1)), np.zeros((n, 1)), [0.5], [0.5], "random")


def brute_leaf(grid, p):
    hi = grid.leaf_lo + grid.leaf_size[:, None]
    inside = np.all((grid.leaf_lo <= p) & (p < hi), axis=1)
    ids = np.nonzero(inside)[0]
    assert ids.size <= 1
    return int(ids[0]) if ids.size else -1


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_locate_matches_scan(seed):
    grid = random_tree(seed)
    rng = np.random.default_rng(100 + seed)
    up = np.ones(3)
    for _ in range(400):
        p = rng.uniform([-1.5, -1, -1], [1.5, 1, 1])
        leaf, box = oracle.locate(grid, p, up)
        assert leaf == brute_leaf(grid, p)
        assert np.allclose(box[:3], grid.leaf_lo[leaf]) and box[3] == grid.leaf_size[leaf]


def test_locate_face_convention():
    grid = synth.sphere_cube(4)  # cells of side 0.5, faces at -1, -0.5, 0, 0.5, 1
    p = np.array([0.0, 0.25, 0.25])
    lp, bp = oracle.locate(grid, p, np.array([1.0, 0, 0]))
    lm, bm = oracle.locate(grid, p, np.array([-1.0, 0, 0]))
    assert bp[0] == 0.0 and bm[0] == -0.5
    assert oracle.locate(grid, np.array([1.0, 0.1, 0.1]), np.array([1.0, 0, 0]))[0] == -1
    assert oracle.locate(grid, np.array([1.0, 0.1, 0.1]), np.array([-1.0, 0, 0]))[0] >= 0


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_segments_match_dense_sampling(seed):
    grid = random_tree(seed)
    rng = np.random.default_rng(200 + seed)
    for _ in range(25):
        xs = rng.uniform([-1.4, -0.9, -0.9], [1.4, 0.9, 0.9])
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        leaves, tin, tout = oracle.trace(grid, xs, n)
        assert np.all(np.diff(tin) >= 0) and np.allclose(tin[1:], tout[:-1])
        # dense sampling: per-leaf path length
        h = 1e-4
        t = np.arange(0, tout[-1], h) + h / 2
        pts = xs[None, :] + t[:, None] * n[None, :]
        lo, hi = grid.leaf_lo, grid.leaf_lo + grid.leaf_size[:, None]
        ids = np.empty(t.size, int)
        for i0 in range(0, t.size, 2000):
            blk = pts[i0:i0 + 2000]
            ins = np.all((lo[None] <= blk[:, None]) & (blk[:, None] < hi[None]), axis=2)
            ids[i0:i0 + 2000] = np.where(ins.any(1), ins.argmax(1), -1)
        ids = ids[ids >= 0]
        samp = np.bincount(ids, minlength=grid.n_leaf) * h
        seg = np.bincount(leaves, weights=tout - tin, minlength=grid.n_leaf)
        assert np.abs(samp - seg).max() < 3 * h
        # order of visited leaves with non-negligible segments
        long = leaves[(tout - tin) > 5 * h]
        dedup = ids[np.r_[True, ids[1:] != ids[:-1]]]
        counts = np.bincount(ids, minlength=grid.n_leaf)
        dedup = dedup[counts[dedup] > 5]
        assert list(long) == list(dedup)


def test_diagonal_ray_moves_through_edges():
    """A ray along a cube diagonal from a cell centre crosses edges and
    corners exactly; it must move diagonally and visit only cells on the
    diagonal (every segment has positive length)."""
    grid = synth.small_sphere(9)
    xs = np.zeros(3)
    n = np.ones(3) / np.sqrt(3.0)
    leaves, tin, tout = oracle.trace(grid, xs, n)
    assert len(leaves) == 5
    c = grid.leaf_centre[leaves]
    assert np.allclose(c[:, 0], c[:, 1]) and np.allclose(c[:, 1], c[:, 2])
    assert np.all(tout - tin > 0)


def test_tau_between_homogeneous():
    grid = synth.sphere_cube(8, radius=10.0, tau_radial=10.0)  # kappa*rho = 1 everywhere
    a = np.array([-0.9, 0.1, 0.3])
    b = np.array([0.7, -0.2, 0.15])
    assert abs(oracle.tau_between(grid, a, b) - np.linalg.norm(b - a)) < 1e-12
