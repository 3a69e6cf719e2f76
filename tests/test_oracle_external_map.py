"""Pins of the oracle's map for a distant observer and of its gradient with
respect to kappa*rho (the source held fixed).

- A homogeneous cube with a uniform source: every line of sight gives
  eta (1 - e^{-kr D}) / kr with D its chord through the cube (slab
  intersection), and eta D without dust.
- The vector-Jacobian product equals central finite differences of the
  same map (double precision) on random cells of a clumpy cube.
- A mistake planted in the gradient (the attenuation of the cells behind
  dropped) fails it."""
import numpy as np
import pytest

import oracle
import synth


def homogeneous(kr, n=8):
    g = synth.lognormal_cube(n, 7, tau_mean=1.0, n_src=1)
    g.kappa_rho[:] = kr
    g.emissivity[:] = 0.25
    return g


def chord(p0, d, lo, hi):
    with np.errstate(divide="ignore"):
        ta, tb = (lo - p0) / d, (hi - p0) / d
    t0 = np.max(np.where(d != 0, np.minimum(ta, tb), -np.inf))
    t1 = np.min(np.where(d != 0, np.maximum(ta, tb), np.inf))
    return max(0.0, t1 - t0)


@pytest.mark.parametrize("kr", [0.0, 0.7])
def test_homogeneous_cube_closed_form(kr):
    g = homogeneous(kr)
    o = oracle.Oracle(g, oracle.OracleParams())
    view, up = np.array([0.3, -0.8, 0.52]), np.array([0.0, 0.0, 1.0])
    m = oracle.ExternalMapOracle(o, view, up, (-1.6, -1.6), 0.2, 16, 16, use_jsca=False)
    img = m.map()
    for j in range(16):
        for i in range(16):
            p0 = (m.origin[0] + (i + 0.5) * m.px) * m.r + (m.origin[1] + (j + 0.5) * m.px) * m.u
            D = chord(p0, -m.w, m.lo, m.hi)
            k = float(g.kappa_rho[0, 0])  # kr as stored (float32)
            ref = 0.25 * D if kr == 0 else 0.25 * -np.expm1(-k * D) / k
            assert abs(img[0, j, i] - ref) <= 1e-12 * max(ref, 1e-30) + 1e-15
    assert np.count_nonzero(img) > 100


def fd_check(lib_path=None, plant=False):
    g = synth.lognormal_cube(8, 8, tau_mean=2.0, n_src=4)
    o = oracle.Oracle(g, oracle.OracleParams(a_rt=0.05, r_pre=0.5))
    o.direct()
    o.scatter_iter()
    m = oracle.ExternalMapOracle(o, (0.0, -1.0, 0.0), (0.0, 0.0, 1.0), (-1.0, -1.0), 0.125, 16, 16)
    kr = m.kappa()
    rng = np.random.default_rng(1709 * 100 + 40)
    target = m.map() * (1 + 0.3 * rng.standard_normal((1, 16, 16)))
    dmap = m.map(kr) - target  # d/dmap of 1/2 |map - target|^2
    grad = m.vjp(dmap, kr)
    if plant:  # the attenuation of what lies behind a cell, dropped
        grad = np.zeros_like(kr)
        for jj in range(16):
            for ii in range(16):
                leaf, ds = m.segments(ii, jj)
                E, dE = oracle.oracle._cell_emission(m.eta[leaf, 0], kr[leaf, 0], ds)
                Tf = np.concatenate([[1.0], np.cumprod(np.exp(-kr[leaf, 0] * ds))[:-1]])
                np.add.at(grad[:, 0], leaf, dmap[0, jj, ii] * Tf * dE)
    cells = rng.choice(g.n_leaf, 24, replace=False)
    for c in cells:
        h = 1e-5 * max(kr[c, 0], 1e-3)
        kp, km = kr.copy(), kr.copy()
        kp[c, 0] += h
        km[c, 0] -= h
        Lp = 0.5 * ((m.map(kp) - target) ** 2).sum()
        Lm = 0.5 * ((m.map(km) - target) ** 2).sum()
        fd = (Lp - Lm) / (2 * h)
        assert abs(grad[c, 0] - fd) <= 1e-5 * np.abs(grad).max() + 1e-6 * abs(fd), (c, grad[c, 0], fd)


def test_gradient_matches_central_differences():
    fd_check()


def test_planted_gradient_mistake_fails():
    with pytest.raises(AssertionError):
        fd_check(plant=True)


def test_albedo_gradient_matches_direct_light_sweeps():
    """After step 2 alone, j_sca is the albedo times a quantity of the direct
    light, which the albedo does not change: central differences of the map
    over two oracle sweeps at albedo (1 +- eps) give the albedo gradient."""
    def sweep(alb):
        g = synth.lognormal_cube(8, 8, tau_mean=2.0, n_src=4)
        g.albedo[:] = alb
        o = oracle.Oracle(g, oracle.OracleParams(a_rt=0.05, r_pre=0.5))
        o.direct()
        return oracle.ExternalMapOracle(o, (0.3, -0.8, 0.52), (0.0, 0.0, 1.0), (-1.6, -1.6), 0.2, 16, 16)
    a0, eps = 0.6, 1e-3
    m = sweep(a0)
    dmap = np.random.default_rng(7).standard_normal((1, 16, 16))
    ga = m.vjp_albedo(dmap)
    mp, mm = sweep(a0 * (1 + eps)), sweep(a0 * (1 - eps))
    # the albedos as stored (float32)
    fd = ((dmap * mp.map()).sum() - (dmap * mm.map()).sum()) / (float(mp.g.albedo[0]) - float(mm.g.albedo[0]))
    assert abs(ga[0] - fd) <= 1e-8 * abs(fd)
    assert np.count_nonzero(m.eta_sca) > 0


def _g_sweep(gval, lib_path=None, view=(0.3, -0.8, 0.52)):
    g = synth.lognormal_cube(8, 8, tau_mean=2.0, n_src=4)
    g.g[:] = gval
    o = oracle.Oracle(g, oracle.OracleParams(a_rt=0.05, r_pre=0.5), lib_path=lib_path)
    o.dg_arm(view)
    o.direct()
    return o


def g_tally_pin(lib_path=None):
    """After step 2 alone the deposited luminosities do not depend on g
    (nothing scattered has been traced yet), so central differences of the
    total j_sca pixel holding the view over sweeps at g +- eps give the
    tally of d j_sca / d g, cell by cell."""
    view = np.array([0.3, -0.8, 0.52])
    g0, eps = 0.6, 1e-3
    o = _g_sweep(g0, lib_path)
    op, om = _g_sweep(g0 + eps, lib_path), _g_sweep(g0 - eps, lib_path)
    assert op.k_lam == o.k_lam == om.k_lam  # the same j_sca level (Eq. 5)
    q = oracle.oracle.vec2pix(o.k_lam[0], view / np.linalg.norm(view))
    h = float(op.grid.g[0]) - float(om.grid.g[0])  # the step as stored (float32)
    fd = (op.jsca(0, "total")[:, q] - om.jsca(0, "total")[:, q]) / h
    dg = o.dg()[:, 0]
    assert np.count_nonzero(dg) > 0.3 * dg.size
    assert np.all(np.abs(dg - fd) <= 1e-5 * np.abs(fd).max() + 1e-4 * np.abs(fd))
    return o, op, om, h


def test_g_tally_matches_central_differences():
    g_tally_pin()


def test_g_gradient_of_the_map():
    o, op, om, h = g_tally_pin()
    frame = ((0.3, -0.8, 0.52), (0.0, 0.0, 1.0), (-1.6, -1.6), 0.2, 16, 16)
    m = oracle.ExternalMapOracle(o, *frame)
    dmap = np.random.default_rng(9).standard_normal((1, 16, 16))
    gg = m.vjp_g(dmap, o.dg())
    fd = ((dmap * oracle.ExternalMapOracle(op, *frame).map()).sum() -
          (dmap * oracle.ExternalMapOracle(om, *frame).map()).sum()) / h
    assert abs(gg[0] - fd) <= 1e-4 * abs(fd)


@pytest.mark.parametrize("name", ["normalisation_dropped", "sign_of_mu"])
def test_planted_g_tally_mistakes_fail(tmp_path, name):
    repl = {
        # the derivative of the normalisation Z left out
        "normalisation_dropped": [("sca * (or_hg_dg(G->g[l], mu) - or_hg(G->g[l], mu) * Zg[l] / Z[l]) / Z[l];",
                                   "sca * or_hg_dg(G->g[l], mu) / Z[l];")],
        # dx/dg taken as 2g + 2mu
        "sign_of_mu": [("1.5 * (1.0 - g * g) * (2.0 * g - 2.0 * mu)", "1.5 * (1.0 - g * g) * (2.0 * g + 2.0 * mu)")],
    }[name]
    path = oracle.build_variant(repl, str(tmp_path))
    with pytest.raises(AssertionError):
        g_tally_pin(lib_path=path)
