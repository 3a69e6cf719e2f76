"""Pins of the oracle's octant mode (Sect. 3.6.4: for symmetric models only
the sources of the first octant are traced and the contributions in the
other octants follow from the symmetry).

For a model symmetric under the reflections about the planes through its
centre, the field of a source's image is the image of the source's field
whenever every decision along a ray has a mirror image.  On a uniform
lattice that holds exactly, so the octant mode must reproduce the full mode
to rounding: RFED, scattering source function and the ledger of the whole
model.  Sources on k mirror planes are their own images under 2^k
reflections and carry weight 1/2^k.  Mistakes planted in the octant branch
(the weight dropped, N_s counting the traced sources only, the j_sca pixels
not reflected with their cell) each fail the pin.

On adaptive grids a ray can run exactly along a cell face (a zero direction
component while the source's coordinate equals a face coordinate); the face
convention gives it the upper cell, its mirror image the lower one, so the
two modes differ there (measured below on a two-level galaxy: 7e-4 per cell
in the median, at most 0.9%, the absorbed total 3e-6)."""
import numpy as np
import pytest

import oracle
import synth


def symmetric_lattice():
    """9^3 dusty lattice with the central cell (on all three mirror planes,
    weight 1/8), its neighbours along the axes (on two planes) and a
    symmetric set of eight off-plane cells emitting."""
    g = synth.small_sphere(9, cell=0.25, radius=0.8, tau_radial=1.0)
    c = g.leaf_centre
    em = np.zeros_like(g.emissivity)
    for pos, lum in [((0, 0, 0), 1.0), ((0.5, 0, 0), 0.4), ((-0.5, 0, 0), 0.4)]:
        em[np.nonzero(np.all(np.isclose(c, pos), axis=1))[0][0], 0] = lum
    off = np.all(np.isclose(np.abs(c), [0.25, 0.5, 0.75]), axis=1)
    assert off.sum() == 8
    em[off, 0] = 0.3
    return g.with_lambda(g.kappa_rho, em, g.albedo, g.g)


def run(grid, octant, lib_path=None, n_iter=1, **kw):
    o = oracle.Oracle(grid, oracle.OracleParams(a_rt=0.05, r_pre=0.5, octant=octant, **kw), lib_path=lib_path)
    o.direct()
    out = [(o.rfed()[0].copy(), o.stats()[0], o.f_u)]
    for _ in range(n_iter):
        o.scatter_iter()
        out.append((o.rfed()[0].copy(), o.stats()[0], o.f_u))
    return out, o.jsca_total.copy()


def pin_octant(lib_path=None):
    grid = symmetric_lattice()
    full, jf = run(grid, 0)
    octa, jo = run(grid, 1, lib_path)
    for (Uf, lf, ff), (Uo, lo, fo) in zip(full, octa):
        assert fo == ff
        assert np.abs(Uo - Uf).max() <= 1e-12 * Uf.max()
        for k in ("emitted", "absorbed", "scattered", "escaped", "blocked", "cut"):
            assert abs(lo[k][0] - lf[k][0]) <= 1e-12 * lf["emitted"][0], k
    assert np.abs(jo - jf).max() <= 1e-12 * jf.max()


def test_octant_equals_full_mode_on_a_uniform_lattice():
    pin_octant()


def test_octant_rejects_an_asymmetric_model():
    with pytest.raises(oracle.OracleError):
        run(synth.config1(), 1)


def test_octant_on_an_adaptive_grid_differs_only_by_face_grazing_rays():
    grid = synth.galaxy_disk(max_level=3, threshold=0.3, nroot=(2, 2, 1), root_size=4.0)
    (f,), _ = run(grid, 0, n_iter=0)
    (o,), _ = run(grid, 1, n_iter=0)
    rel = np.abs(o[0] / f[0] - 1)
    assert np.median(rel) < 2e-3 and rel.max() < 0.02
    assert abs(o[1]["absorbed"][0] / f[1]["absorbed"][0] - 1) < 1e-4


PLANTED = {
    "source weight dropped": [("C.wsrc = ldexp(1.0, -k);", "C.wsrc = 1.0;")],
    "N_s counts the traced sources": [("            ++ns;  /* N_s counts every source of the model */\n", ""),
                                      ("            is_src[s] = (char)on;\n", "            is_src[s] = (char)on;\n            ns += on;\n")],
    "pixels not reflected": [("v += dep_P[S->off_lam[l] + cm * npx + mpix[m - 1][kl][q]];",
                              "v += dep_P[S->off_lam[l] + cm * npx + q];")],
}


@pytest.mark.parametrize("name", sorted(PLANTED))
def test_planted_mistakes_fail(name, tmp_path):
    path = oracle.build_variant(PLANTED[name], str(tmp_path))
    with pytest.raises(AssertionError):
        pin_octant(lib_path=path)
