"""Pins of the oracle's forward mode: the derivative of the RFED and of the
absorbed luminosity with respect to the albedo, carried as extra wavelengths
through the sweep (same extinction, no emission of their own, the scattered
light lost x d(albedo) of their wavelength as an extra source; blocking,
splitting and merging decided by the wavelengths themselves).

- Without blocking (a_RT = 0) no decision depends on the albedo, so central
  differences over two sweeps at albedo (1 +- eps) give the derivative of
  every cell's U and L_abs (to the truncation of the differences).
- The forward mode leaves the wavelengths themselves bit for bit unchanged,
  blocking included.
- Two mistakes planted in the derivative's source fail the first pin."""
import numpy as np
import pytest

import oracle
import synth


def two_lambda_cube():
    g = synth.lognormal_cube(6, 8, tau_mean=2.0, n_src=3, box_size=1.5)
    kr = g.kappa_rho * np.array([1.0, 0.4], np.float32)[None, :]
    return g.with_lambda(kr, np.repeat(g.emissivity, 2, axis=1), [0.6, 0.45], [0.6, 0.35])


def sweep(grid, lib_path=None, n_iter=2, **kw):
    o = oracle.Oracle(grid, oracle.OracleParams(r_pre=0.5, **kw), lib_path=lib_path)
    o.direct()
    for _ in range(n_iter):
        o.scatter_iter()
    return o


def fd_pin(lib_path=None):
    g = two_lambda_cube()
    t = sweep(g, lib_path, a_rt=0.0, tangent_albedo=1)
    dU, dL = t.rfed_tangent()
    eps = 1e-3
    for l in range(2):
        res = []
        for sgn in (1, -1):
            a = g.albedo.copy()
            a[l] *= 1 + sgn * eps
            gp = g.with_lambda(g.kappa_rho, g.emissivity, a, g.g)
            o = sweep(gp, a_rt=0.0)
            res.append((o.rfed(), float(gp.albedo[l]), o.stats()[1]))
        (Up, Lp), ap, cp = res[0]
        (Um, Lm), am, cm = res[1]
        assert cp == cm  # no decision depends on the albedo without blocking
        fdU = (Up[:, l] - Um[:, l]) / (ap - am)
        fdL = (Lp[:, l] - Lm[:, l]) / (ap - am)
        for a_, b_ in ((dU[:, l], fdU), (dL[:, l], fdL)):
            assert np.abs(b_).max() > 0
            assert np.all(np.abs(a_ - b_) <= 1e-5 * np.abs(b_).max() + 1e-4 * np.abs(b_)), l
    return t


def test_tangent_matches_central_differences():
    fd_pin()


def test_tangent_leaves_the_wavelengths_unchanged():
    g = two_lambda_cube()
    a = sweep(g, a_rt=0.05)
    b = sweep(g, a_rt=0.05, tangent_albedo=1)
    assert np.array_equal(a.rfed()[0], b.rfed()[0])
    la, ca = a.stats()
    lb, cb = b.stats()
    assert ca["blocks"] > 0 and ca["blocks"] == cb["blocks"] and ca["crossings"] == cb["crossings"]
    for k in la:
        assert np.array_equal(la[k], lb[k]), k
    dU, dL = b.rfed_tangent()
    assert np.all(dU >= 0) and dU.max() > 0  # more albedo, more scattered light everywhere


@pytest.mark.parametrize("name", ["cross_term_dropped", "cross_term_after_attenuation"])
def test_planted_tangent_mistakes_fail(tmp_path, name):
    target = "? w * lost + I_in[l - P->tangent] * P_in_unit * kr * ds * fac[l]"
    repl = {"cross_term_dropped": "? w * lost",
            # the wavelength's intensity after the segment instead of entering it
            "cross_term_after_attenuation": "? w * lost + ray->I[l - P->tangent] * P_in_unit * kr * ds * fac[l]"}[name]
    path = oracle.build_variant([(target, repl)], str(tmp_path))
    with pytest.raises(AssertionError):
        fd_pin(lib_path=path)
