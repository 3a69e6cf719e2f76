"""Pins of the oracle's multi-wavelength branch (Sect. 3.2) and of its point
sources (Sect. 3.6.1), recomputed from the definitions in plain Python.

Multi-wavelength rays carry one intensity per wavelength.  At every crossing
each wavelength is tested with Eq. 1 on its own; a ray is blocked only when
every wavelength is negligible, and a negligible wavelength is still
attenuated but deposits nothing (its loss is booked as "skipped").  The
scattering source function of wavelength l is sampled on HEALPix(k_l) with
k_l from Eq. 5, its block of the j_sca array following the blocks of the
wavelengths before it; scattering rays start at the level
max(k0, max_l k_l), and each wavelength re-emits the pending luminosity of
the ray's nested parent pixel at its own level.

Each pin is also run against copies of the oracle with a mistake planted in
that branch (tests/test_oracle_multilambda.py::test_planted_mistakes_fail):
blocking on any negligible wavelength, U_LL of the first wavelength used for
all, scattering rows of every wavelength written into the first
wavelength's block, scattering rays started at the smallest k_l, the 4 pi
of a point source's per-sr luminosity dropped, and a point source placed
with two coordinates swapped.  Each planted mistake fails its pin."""
import math

import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss

import oracle
import synth
from test_oracle_physics import _cells_along, _chord, _hg_weights, cell_integral

# ----------------------------------------------------------------- helpers


def _three_lambda(grid, kr, emis_scale, albedo, g):
    nl = len(albedo)
    kr = np.ascontiguousarray(kr, np.float32)
    em = np.repeat(grid.emissivity, nl, axis=1) * np.asarray(emis_scale, np.float32)[None, :]
    return grid.with_lambda(kr, em, albedo, g)


LAMBDA_G = [0.75, 0.5, 0.2]          # k_l = 3, 2, 1 by Eq. 5 (n_FWHM 5, cap 3)
LAMBDA_ALBEDO = [0.7, 0.5, 0.3]


def _expected_offsets(n_leaf, k_lam):
    """Block l of the j_sca array starts after the blocks of the wavelengths
    before it, each n_leaf rows of 12 4^k pixels (Sect. 3.1.2)."""
    off, out = 0, []
    for k in k_lam:
        out.append(off)
        off += n_leaf * 12 * 4 ** k
    return out, off


def _paths(grid, xs, src, k):
    """Every ray of level k from xs: (pixel, direction, [(leaf, t_in, ds)])."""
    out = []
    for p in range(12 * 4 ** k):
        v = oracle.pix2vec(k, p)
        segs, t = [], 0.0
        for leaf, ds in _cells_along(grid, xs, v, src):
            segs.append((leaf, t, ds))
            t += ds
        out.append((p, v, segs))
    return out


def _fac(dtau):
    return -math.expm1(-dtau) / dtau if dtau > 0 else 1.0


# ------------------------------------------------------- the direct light pin


def _direct_setup():
    base = synth.small_sphere(9, cell=0.25, radius=100.0, tau_radial=0.0, albedo=0.6, g=0.6)
    kr = np.zeros((base.n_leaf, 3))
    kr[:] = [0.4, 1.0, 2.2]  # homogeneous, different per wavelength
    return _three_lambda(base, kr, [1.0, 0.6, 1.5], LAMBDA_ALBEDO, LAMBDA_G)


def pin_multilambda_direct(lib_path=None):
    """Steps 1 and 2 of one central source, 3 wavelengths, homogeneous dust,
    fixed angular density (no split, no merge): the step-1 U_LL with the R_pre
    cut, then every Eq. 1 decision per wavelength and crossing with
    f_U = 4 a_RT / N_s, the blocking of rays where all wavelengths are
    negligible, the direct-light U, the skipped and blocked luminosity and
    the pending scattering rows of every wavelength (Eq. 4 at its own k_l,
    rows normalised) -- all recomputed here."""
    grid = _direct_setup()
    nl, k0, R = 3, 4, 0.55
    src = int(np.nonzero(grid.emissivity[:, 0])[0][0])
    xs = grid.leaf_centre[src]
    cell = 0.25
    V = cell ** 3
    S = grid.emissivity[src].astype(np.float64) * V  # per-sr luminosity per wavelength
    kr = grid.kappa_rho.astype(np.float64)
    alb = grid.albedo.astype(np.float64)
    gg = grid.g.astype(np.float64)
    om = 4 * math.pi / (12 * 4 ** k0)
    paths = _paths(grid, xs, src, k0)

    # step 1: U_LL within R_pre
    U_LL = np.zeros((grid.n_leaf, nl))
    entries = []
    for p, v, segs in paths:
        I = S.copy()
        for leaf, t_in, ds in segs:
            if leaf != src:
                entries.append(abs(t_in - R))
                if t_in >= R:
                    break
            dtau = kr[leaf] * ds
            for l in range(nl):
                U_LL[leaf, l] += I[l] * om * ds * _fac(dtau[l]) / V
            I *= np.exp(-dtau)
    assert min(entries) > 1e-9  # no entry distance sits on R_pre

    # ratios dU / U_LL along the unblocked rays choose f_U: a value well
    # away from every ratio, near their 30th percentile, where most rays are
    # blocked somewhere but many crossings have some wavelengths negligible
    # and others not
    ratios = []
    for p, v, segs in paths:
        I = S.copy()
        for leaf, t_in, ds in segs:
            dtau = kr[leaf] * ds
            if leaf != src and np.all(U_LL[leaf] > 0):
                r2 = float(((grid.leaf_centre[leaf] - xs) ** 2).sum())
                fac = np.array([_fac(x) for x in dtau])
                ratios += list(I * fac / r2 / U_LL[leaf])
            I *= np.exp(-dtau)
    target = np.quantile(np.array(ratios), 0.3)
    ratios = np.unique(np.array(ratios))
    mids = np.sqrt(ratios[1:] * ratios[:-1])
    gaps = ratios[1:] / ratios[:-1] - 1
    ok = gaps > 2e-4
    f_u = float(mids[ok][np.argmin(np.abs(np.log(mids[ok] / target)))])
    f_u = float(np.float64(4.0 * (f_u / 4.0)))

    o = oracle.Oracle(grid, oracle.OracleParams(k0=k0, a_rt=f_u / 4.0, r_pre=R, n_rays_min=0, merge=0),
                      lib_path=lib_path)
    o.run_phase(0)
    assert np.abs(o.U_LL.reshape(-1, nl) - U_LL).max() <= 1e-9 * U_LL.max()
    o.direct()
    led, cnt = o.stats()
    assert o.f_u == f_u and o.n_src == 1

    # step 2, recomputed
    U = np.zeros((grid.n_leaf, nl))
    k_lam = [oracle.k_hp(x) for x in gg]
    assert k_lam == [3, 2, 1]
    nq = {k: oracle.pix2vec_all(k) for k in set(k_lam)}
    rows = [np.zeros((grid.n_leaf, 12 * 4 ** k)) for k in k_lam]
    blocked, mixed, skipped, blocked_lum = 0, 0, np.zeros(nl), np.zeros(nl)
    for p, v, segs in paths:
        I = S.copy()
        for leaf, t_in, ds in segs:
            dtau = kr[leaf] * ds
            fac = np.array([_fac(x) for x in dtau])
            neg = np.zeros(nl, bool)
            if leaf != src:
                r2 = float(((grid.leaf_centre[leaf] - xs) ** 2).sum())
                neg = I * fac / r2 < f_u * U_LL[leaf]
                if neg.all():
                    blocked += 1
                    blocked_lum += I * om
                    break
                mixed += int(neg.any())
            for l in range(nl):
                lost = I[l] * om * (1.0 - math.exp(-dtau[l]))
                if neg[l]:
                    skipped[l] += lost
                    continue
                U[leaf, l] += I[l] * om * ds * fac[l] / V
                if lost > 0:
                    rows[l][leaf] += alb[l] * lost * _hg_weights(gg[l], nq[k_lam[l]], v)
            I *= np.exp(-dtau)
    assert blocked >= 100 and mixed >= 100 and np.all(skipped > 0)
    assert cnt["blocks"] == blocked  # the call's counters cover both phases; step 1 blocks nothing
    U_o = o.rfed()[0]
    for l in range(nl):
        assert np.abs(U_o[:, l] - U[:, l]).max() <= 1e-9 * U[:, l].max(), f"U, lambda {l}"
        assert abs(led["skipped"][l] / skipped[l] - 1) < 1e-9, f"skipped, lambda {l}"
        assert abs(led["blocked"][l] / blocked_lum[l] - 1) < 1e-9, f"blocked, lambda {l}"
        got = o.jsca(l, "pending")
        assert np.abs(got - rows[l]).max() <= 1e-9 * rows[l].max(), f"j_sca rows, lambda {l}"


# ------------------------------------------- the scattering rows and re-emission


def _scatterer_setup():
    base = synth.small_sphere(9, cell=0.25, radius=100.0, tau_radial=0.0, albedo=0.6, g=0.6)
    scat = int(np.nonzero(np.all(np.isclose(base.leaf_centre, [0.25, 0.0, 0.0]), axis=1))[0][0])
    kr = np.zeros((base.n_leaf, 3))
    kr[scat] = [0.04, 0.08, 0.02]  # optically thin scatterer next to the source
    return _three_lambda(base, kr, [1.0, 0.5, 2.0], LAMBDA_ALBEDO, LAMBDA_G), scat


def pin_multilambda_scattering(lib_path=None):
    """One thin scatterer beside the source, 3 wavelengths with k_l = 3, 2, 1
    and initial ray level k0 = 2, no split, merge or blocking.  The pending
    rows of every wavelength (Eq. 4 at its own level, rows normalised) and, in
    the next scattering iteration, the RFED that three detector cells receive
    from rays that start at level max(k0, max k_l) = 3 and carry, per
    wavelength, the pending luminosity of their nested parent pixel at level
    k_l per its solid angle -- recomputed here."""
    grid, scat = _scatterer_setup()
    nl, k0, cell = 3, 2, 0.25
    V = cell ** 3
    o = oracle.Oracle(grid, oracle.OracleParams(k0=k0, a_rt=0.0, r_pre=100.0, n_rays_min=0, merge=0),
                      lib_path=lib_path)
    offsets, total = _expected_offsets(grid.n_leaf, [3, 2, 1])
    assert list(o.k_lam) == [3, 2, 1]
    assert list(o.off_lam) == offsets and o.pend_a.size == total
    o.direct()
    U1 = o.rfed()[0].copy()

    src = int(np.nonzero(grid.emissivity[:, 0])[0][0])
    S = grid.emissivity[src].astype(np.float64) * V
    kr = grid.kappa_rho[scat].astype(np.float64)
    alb = grid.albedo.astype(np.float64)
    gg = grid.g.astype(np.float64)
    lo, hi = grid.leaf_lo[scat], grid.leaf_lo[scat] + cell
    om0 = 4 * math.pi / (12 * 4 ** k0)
    rows = []
    for l, k in enumerate([3, 2, 1]):
        nq = oracle.pix2vec_all(k)
        row = np.zeros(12 * 4 ** k)
        for v in oracle.pix2vec_all(k0):
            ds = _chord(np.zeros(3), v, lo, hi)
            if ds > 0:
                row += alb[l] * S[l] * om0 * -math.expm1(-kr[l] * ds) * _hg_weights(gg[l], nq, v)
        got = o.jsca(l, "pending")
        assert np.abs(np.delete(got, scat, axis=0)).max() == 0.0, f"rows outside the scatterer, lambda {l}"
        assert np.abs(got[scat] - row).max() <= 1e-9 * row.max(), f"pending row, lambda {l}"
        rows.append(row)

    o.scatter_iter()
    dU = o.rfed()[0] - U1
    xs = grid.leaf_centre[scat]
    kstart = 3
    omk = 4 * math.pi / (12 * 4 ** kstart)
    detectors = {name: int(np.nonzero(np.all(np.isclose(grid.leaf_centre, c), axis=1))[0][0])
                 for name, c in (("forward", [1.0, 0.0, 0.0]), ("backward", [0.0, 0.0, 0.0]),
                                 ("side", [0.25, 0.5, 0.0]))}
    for l, k in enumerate([3, 2, 1]):
        om_l = 4 * math.pi / (12 * 4 ** k)
        ref = dict.fromkeys(detectors, 0.0)
        for p in range(12 * 4 ** kstart):
            v = oracle.pix2vec(kstart, p)
            P = rows[l][p >> (2 * (kstart - k))] / om_l * omk
            T = math.exp(-kr[l] * _chord(xs, v, lo, hi))
            for name, d in detectors.items():
                ds = _chord(xs, v, grid.leaf_lo[d], grid.leaf_lo[d] + cell)
                if ds > 0:
                    ref[name] += P * T * ds / V
        for name, d in detectors.items():
            assert ref[name] > 0
            assert abs(dU[d, l] / ref[name] - 1) < 1e-7, (l, name, dU[d, l], ref[name])
    # g = 0.75 scatters forward strongly
    assert dU[detectors["forward"], 0] > 5 * dU[detectors["backward"], 0]


# ------------------------------------------------------------ the point source


def _box_integral(lo, L, xp, kr, ng=48):
    """int_box exp(-kr r)/r^2 dV around a point xp strictly inside the box:
    over the six faces, dOmega = h dA / rho^3 and the radial integral runs
    from the point to the face (h: distance of the face plane, rho: distance
    to the face point)."""
    x, w = leggauss(ng)
    tot = 0.0
    for a in range(3):
        b, c = [i for i in range(3) if i != a]
        ub = lo[b] + 0.5 * L * (x + 1) - xp[b]
        uc = lo[c] + 0.5 * L * (x + 1) - xp[c]
        B, Cc = np.meshgrid(ub, uc, indexing="ij")
        W = (w[:, None] * w[None, :]) * (0.5 * L) ** 2
        for face in (lo[a], lo[a] + L):
            h = abs(face - xp[a])
            rho = np.sqrt(B * B + Cc * Cc + h * h)
            radial = rho if kr == 0 else -np.expm1(-kr * rho) / kr
            tot += float((W * h / rho ** 3 * radial).sum())
    return tot


def _point_setup():
    base = synth.small_sphere(5, cell=0.25, radius=100.0, tau_radial=0.0, albedo=0.0, g=0.0)
    kr = np.zeros((base.n_leaf, 2))
    kr[:, 1] = 1.5
    grid = base.with_lambda(kr, np.zeros((base.n_leaf, 2)), [0.0, 0.0], [0.0, 0.0])
    grid.point_xyz = np.array([[0.0625, -0.1875, 0.03125]], np.float32)
    grid.point_lum = np.array([[0.7, 0.3]], np.float32)
    return grid


def pin_point_source(lib_path=None):
    """A point source off every cell centre (Sect. 3.6.1), two wavelengths
    (empty and homogeneous medium), at brute-force angular density: the RFED
    of every cell is L/(4 pi V c) int_cell e^{-kr r}/r^2 dV, with r measured
    from the point (the per-sr luminosity is L/(4 pi))."""
    grid = _point_setup()
    o = oracle.Oracle(grid, oracle.OracleParams(k0=8, a_rt=0.0, r_pre=100.0, n_rays_min=0, merge=0),
                      lib_path=lib_path)
    o.direct()
    U = o.rfed()[0]
    xp = grid.point_xyz[0].astype(np.float64)
    L = 0.25
    V = L ** 3
    home = grid.leaf_containing(xp)
    assert not np.allclose(grid.leaf_centre[home], xp)
    for l, krl in enumerate((0.0, 1.5)):
        lum = float(grid.point_lum[0, l])
        for leaf in range(grid.n_leaf):
            lo = grid.leaf_lo[leaf]
            ref = _box_integral(lo, L, xp, krl) if leaf == home else cell_integral(lo, L, xp, krl)
            ref *= lum / (4 * math.pi * V)
            assert abs(U[leaf, l] / ref - 1) < 1.5e-3, (l, leaf, U[leaf, l], ref)


# ------------------------------------------------------------------ the tests


def test_jsca_layout_follows_eq5():
    """k_l from Eq. 5 per wavelength and the j_sca blocks one after another,
    n_leaf rows of 12 4^k_l pixels each (the GPU layout is compared with the
    same definition in the GPU tests)."""
    grid, _ = _scatterer_setup()
    o = oracle.Oracle(grid, oracle.OracleParams())
    offsets, total = _expected_offsets(grid.n_leaf, [3, 2, 1])
    assert list(o.k_lam) == [3, 2, 1] and list(o.off_lam) == offsets
    assert o.jsca_total.size == total


def test_multilambda_direct_light_recomputed():
    pin_multilambda_direct()


def test_multilambda_scattering_rows_and_reemission():
    pin_multilambda_scattering()


def test_point_source_rfed_matches_cell_integrals():
    pin_point_source()


def test_point_sources_count_in_n_s():
    """Eq. 10 with N_s the sources of the phase: emitting cells plus point
    sources."""
    grid = _point_setup()
    em = np.zeros((grid.n_leaf, 2), np.float32)
    em[[0, 7, 20], 0] = 1.0
    grid = grid.with_lambda(grid.kappa_rho, em, grid.albedo, grid.g)
    grid.point_xyz = np.array([[0.0625, -0.1875, 0.03125], [-0.3125, 0.1875, 0.0625]], np.float32)
    grid.point_lum = np.array([[0.7, 0.3], [0.0, 0.2]], np.float32)
    o = oracle.Oracle(grid, oracle.OracleParams(a_rt=0.05, r_pre=0.3))
    o.direct()
    assert o.n_src == 5 and o.f_u == 4 * 0.05 / 5


PLANTED = {
    "block on any negligible wavelength": (
        pin_multilambda_direct,
        [("int all = 1;", "int all = 0;"), ("all &= neg[l];", "all |= neg[l];")]),
    "U_LL of the first wavelength for all": (
        pin_multilambda_direct,
        [("neg[l] = dU < C->f_u * S->U_LL[(int64_t)leaf * nl + l];",
          "neg[l] = dU < C->f_u * S->U_LL[(int64_t)leaf * nl + 0];")]),
    "rows of every wavelength in the first block": (
        pin_multilambda_scattering,
        [("double *row = C->pend_dst + S->off_lam[l] + (int64_t)leaf * npx;",
          "double *row = C->pend_dst + S->off_lam[0] + (int64_t)leaf * npx;")]),
    "scattering rays start at the smallest k": (
        pin_multilambda_scattering,
        [("int kmax_lam = 0;\n    for (int l = 0; l < nl; ++l) if (S->k_lam[l] > kmax_lam) kmax_lam = S->k_lam[l];",
          "int kmax_lam = 99;\n    for (int l = 0; l < nl; ++l) if (S->k_lam[l] < kmax_lam) kmax_lam = S->k_lam[l];")]),
    "point source without the 4 pi": (
        pin_point_source,
        [("Il = G->point_lum[(s - G->n_leaf) * nl + l] / (4.0 * OR_PI);",
          "Il = G->point_lum[(s - G->n_leaf) * nl + l];")]),
    "point source with swapped coordinates": (
        pin_point_source,
        [("C.xs[1] = G->point_xyz[3 * ip + 1];\n            C.xs[2] = G->point_xyz[3 * ip + 2];",
          "C.xs[1] = G->point_xyz[3 * ip + 2];\n            C.xs[2] = G->point_xyz[3 * ip + 1];")]),
}


@pytest.mark.parametrize("name", sorted(PLANTED))
def test_planted_mistakes_fail(name, tmp_path):
    """Each mistake planted in a copy of the oracle fails the pin of its
    branch (while the unchanged oracle passes it, above)."""
    pin, repl = PLANTED[name]
    path = oracle.build_variant(repl, str(tmp_path))
    with pytest.raises(AssertionError):
        pin(lib_path=path)
