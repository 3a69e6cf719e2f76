"""Pins of the oracle's HEALPix functions (ray directions, Sect. 3.1.1; j_sca
sampling, Sect. 3.1.2) against the published definition of the scheme
(Gorski et al. 2005) and properties it fixes."""
import math

import numpy as np
import pytest

import oracle
from oracle.oracle import pix2vec_all


def ring_centres(k):
    """Pixel centres of the RING scheme written directly from its definition:
    cap ring i < nside: z = 1 - i^2/(3 nside^2), 4i pixels at
    phi = pi/(2i) (j - 1/2); belt ring nside <= i <= 3 nside:
    z = 4/3 - 2i/(3 nside), 4 nside pixels at phi = pi/(2 nside)(j - s/2),
    s = (i - nside + 1) mod 2; southern caps mirror the northern ones."""
    ns = 2 ** k
    out = []
    for i in range(1, 4 * ns):
        if i < ns:
            z = 1 - i * i / (3 * ns * ns)
            phis = [math.pi / (2 * i) * (j - 0.5) for j in range(1, 4 * i + 1)]
        elif i <= 3 * ns:
            z = 4 / 3 - 2 * i / (3 * ns)
            s = (i - ns + 1) % 2
            phis = [math.pi / (2 * ns) * (j - s / 2) for j in range(1, 4 * ns + 1)]
        else:
            ii = 4 * ns - i
            z = -(1 - ii * ii / (3 * ns * ns))
            phis = [math.pi / (2 * ii) * (j - 0.5) for j in range(1, 4 * ii + 1)]
        st = math.sqrt(max(0.0, 1 - z * z))
        out += [(st * math.cos(p), st * math.sin(p), z) for p in phis]
    return np.array(out)


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4])
def test_nested_centres_are_the_ring_centres(k):
    nest = pix2vec_all(k)
    ring = ring_centres(k)
    assert nest.shape == ring.shape == (12 * 4 ** k, 3)
    # every nested centre coincides with exactly one ring centre
    d = np.linalg.norm(nest[:, None, :] - ring[None, :, :], axis=2)
    nearest = d.argmin(1)
    assert np.all(d.min(1) < 1e-12)
    assert np.unique(nearest).size == nest.shape[0]


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4, 5, 6])
def test_roundtrip_and_unit_norm(k):
    v = pix2vec_all(k) if k <= 5 else None
    npix = 12 * 4 ** k
    ps = range(npix) if k <= 5 else np.random.default_rng(k).integers(0, npix, 3000)
    for p in ps:
        c = v[p] if v is not None else oracle.pix2vec(k, p)
        assert abs(np.linalg.norm(c) - 1) < 1e-14
        assert oracle.vec2pix(k, c) == p


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4])
def test_children_lie_in_parent(k):
    """Nested quad-tree: the 4 children 4p..4p+3 at level k+1 lie in pixel p."""
    for p in range(12 * 4 ** k):
        for c in range(4):
            assert oracle.vec2pix(k, oracle.pix2vec(k + 1, 4 * p + c)) == p


def test_vec2pix_levels_are_nested():
    rng = np.random.default_rng(5)
    v = rng.standard_normal((4000, 3))
    for x in v:
        p6 = oracle.vec2pix(6, x)
        for k in (0, 2, 4, 5):
            assert oracle.vec2pix(k, x) == p6 >> (2 * (6 - k))


def test_equal_area_monte_carlo():
    """All 48 pixels of level 1 have area 4 pi/48: counts of uniform random
    directions are multinomial with equal probabilities."""
    rng = np.random.default_rng(11)
    n = 240000
    v = rng.standard_normal((n, 3))
    counts = np.bincount([oracle.vec2pix(1, x) for x in v], minlength=48)
    expect = n / 48
    chi2 = ((counts - expect) ** 2 / expect).sum()
    assert chi2 < 100  # 47 dof: p(chi2 > 100) ~ 1e-5
    assert np.all(np.abs(counts - expect) < 5 * np.sqrt(expect))  # 5 sigma per pixel


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4])
def test_exact_symmetries(k):
    """The centre set is exactly (bitwise) invariant under the rotation
    (x, y, z) -> (-y, x, z), the mirror x <-> y and z -> -z, and sums to 0."""
    c = pix2vec_all(k)
    keys = {tuple(r) for r in c}
    for t in (lambda r: (-r[1], r[0], r[2]), lambda r: (r[1], r[0], r[2]),
              lambda r: (r[0], r[1], -r[2]), lambda r: (-r[0], r[1], r[2])):
        assert {t(r) for r in c} == keys
    assert np.abs(c.sum(0)).max() < 1e-12


def test_pixel_counts_per_ring():
    for k in range(0, 5):
        ns = 2 ** k
        z = np.round(pix2vec_all(k)[:, 2], 12)
        vals, cnt = np.unique(z, return_counts=True)
        assert vals.size == 4 * ns - 1
        # caps: 4i pixels on ring i; belt: 4 nside
        expect = sorted([4 * min(i, ns, 4 * ns - i) for i in range(1, 4 * ns)])
        assert sorted(cnt.tolist()) == expect
