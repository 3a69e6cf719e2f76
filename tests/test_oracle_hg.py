"""Pins of the phase function (Eq. 4), the j_sca resolution rule (Eq. 5),
the accuracy threshold (Eq. 10) and the paper's memory example (Sect. 3.1.2)."""
import math
import os

import numpy as np
import pytest
from scipy import integrate
from scipy.optimize import brentq

import oracle
import synth
from oracle.oracle import pix2vec_all

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("g", [0.0, 0.1, 0.4, 0.6, 0.75, -0.3])
def test_hg_normalised_and_mean_cosine(g):
    norm = integrate.quad(lambda mu: 2 * math.pi * oracle.hg(g, mu), -1, 1, epsabs=1e-13)[0]
    mean = integrate.quad(lambda mu: 2 * math.pi * mu * oracle.hg(g, mu), -1, 1, epsabs=1e-13)[0]
    assert abs(norm - 1) < 1e-10
    assert abs(mean - g) < 1e-10


def test_hg_isotropic_limit():
    for mu in (-1, -0.3, 0.2, 1):
        assert abs(oracle.hg(0.0, mu) - 1 / (4 * math.pi)) < 1e-15


def _table():
    rows = []
    with open(os.path.join(GOLDEN, "k_hp_table.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([float(x) for x in line.split()])
    return rows


def test_k_hp_golden_table():
    for g, fwhm_deg, k_real, k_floor, npix in _table():
        kr = oracle.k_hp_real(g, 5)
        assert abs(kr - k_real) < 0.006, (g, kr)
        k = oracle.k_hp(g, 5, 3)
        assert k == int(k_floor)
        assert 12 * 4 ** k == int(npix)
        # FWHM from the unrounded k: theta_min^2 = 4 pi / (12 4^k)
        th = math.sqrt(4 * math.pi / (12 * 4 ** kr))
        assert abs(math.degrees(5 * th) - fwhm_deg) < 0.06


@pytest.mark.parametrize("g", [0.15, 0.35, 0.55, 0.65])
def test_k_hp_fwhm_by_root_finding(g):
    """Half maximum of Phi - Phi(pi) found numerically from Eq. 4."""
    f = lambda t: oracle.hg(g, math.cos(t))
    half = 0.5 * (f(0) + f(math.pi))
    th = brentq(lambda t: f(t) - half, 1e-9, math.pi - 1e-9, xtol=1e-14)
    tmin = 2 * th / 5
    assert abs(oracle.k_hp_real(g, 5) - 0.5 * math.log2(4 * math.pi / (12 * tmin ** 2))) < 1e-9


def test_k_hp_cap_and_isotropic():
    assert oracle.k_hp(0.0, 5, 3) == 0
    assert oracle.k_hp(0.9, 5, 3) == 3
    assert oracle.k_hp(0.9, 5, 2) == 2


def test_memory_example():
    """Sect. 3.1.2: 31 wavelengths, ~700,000 cells, k = 2 everywhere -> ~33 GB
    of j_sca at 8 bytes per value."""
    k = 2
    gb = 7e5 * 31 * 12 * 4 ** k * 8 / 1e9
    assert 32.5 < gb < 34.0


@pytest.mark.parametrize("k,g", [(1, 0.3), (2, 0.6), (3, 0.75)])
def test_discrete_rows_converge_to_g(k, g):
    """Normalised HG rows on HEALPix(k): weights sum to 1 by construction and
    their mean cosine approaches g as k grows (checked for the ray along a
    pixel centre and along an arbitrary direction)."""
    c = pix2vec_all(k)
    for n in (c[3], np.array([0.3, -0.5, 0.81]) / np.linalg.norm([0.3, -0.5, 0.81])):
        w = np.array([oracle.hg(g, float(q @ n)) for q in c])
        w /= w.sum()
        mc = float((w * (c @ n)).sum())
        assert abs(mc - g) < {1: 0.25, 2: 0.08, 3: 0.03}[k]


def test_f_u_and_sources():
    """Eq. 10: f_U = 4 a_RT / N_s with N_s the number of sources of the phase."""
    grid = synth.lognormal_cube(8, 3, n_src=5)
    o = oracle.Oracle(grid, oracle.OracleParams(a_rt=0.05, r_pre=0.4))
    o.direct()
    assert o.n_src == 5
    assert abs(o.f_u - 4 * 0.05 / 5) < 1e-15
    o.scatter_iter()
    dusty = int((grid.kappa_rho[:, 0] > 0).sum())
    assert o.n_src == dusty
    assert abs(o.f_u - 4 * 0.05 / dusty) < 1e-15
