"""Parity of the CUDA sweep (through the C ABI) with the FP64 oracle on the
same seeded inputs.

Tolerances (floating point, float32 GPU vs float64 oracle): per-cell RFED
<= 1e-3 relative for cells above 1e-6 of the maximum; total absorbed,
scattered and escaped luminosity <= 1e-4 relative; crossing, split, block and
merge counts within 1e-4 relative (at least 2 events, for small counts: a
float32 distance can flip one decision that sits on its threshold)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1709_03802_gb300 import DartRay, DartRayError  # noqa: E402

REL_CELL = 1e-3
REL_TOTAL = 1e-4


def close_counts(a, b, rel=1e-4, floor=2):
    return abs(a - b) <= max(rel * max(a, b), floor)


def check_rfed(gpu, ref, tag=""):
    """Per-cell U within REL_CELL above 1e-6 of the maximum, the floor taken
    per wavelength (a weak wavelength is checked against its own maximum),
    and the absorbed luminosity per wavelength within REL_TOTAL."""
    U, L_abs = gpu.rfed()
    Ur, Lr = ref.rfed()
    worst = 0.0
    for l in range(Ur.shape[1]):
        u, ur = U[:, l], Ur[:, l]
        if ur.max() <= 0:
            assert np.all(u == 0), f"{tag} lambda {l}: U where the oracle has none"
            continue
        big = ur > 1e-6 * ur.max()
        rel = np.abs(u[big] / ur[big] - 1)
        assert rel.max() <= REL_CELL, f"{tag} lambda {l}: per-cell U rel {rel.max():.3e}"
        # cells below the floor are still small on both sides
        assert np.all(np.abs(u[~big]) <= 2e-6 * ur.max() + 1e-30), f"{tag} lambda {l}: floor"
        if Lr[:, l].sum() > 0:
            assert abs(L_abs[:, l].sum() / Lr[:, l].sum() - 1) <= REL_TOTAL, f"{tag} lambda {l}: L_abs"
        worst = max(worst, rel.max())
    return worst


def check_ledger(st, ref, tag="", count_rel=1e-4):
    led, cnt = ref.stats()
    for k in ("emitted", "absorbed", "scattered", "escaped", "blocked", "cut"):
        a, b = np.asarray(st[k]), led[k]
        tot = led["emitted"].sum()
        assert np.all(np.abs(a - b) <= REL_TOTAL * max(tot, 1e-300)), f"{tag} ledger {k}: {a} vs {b}"
    bad = {k: (st[k], cnt[k]) for k in ("crossings", "rays", "splits", "blocks", "escapes", "cuts", "lows", "merges")
           if not close_counts(st[k], cnt[k], rel=count_rel)}
    assert not bad, f"{tag} counts (gpu, oracle): {bad}"


ORACLE_KEYS = set(oracle.OracleParams.__dataclass_fields__)


def run_pair(grid, n_iter, count_rel=1e-4, **params):
    gpu = DartRay(grid, **params)
    ref = oracle.Oracle(grid, oracle.OracleParams(**{k: v for k, v in params.items() if k in ORACLE_KEYS}))
    st = gpu.direct()
    gpu.direct_stats = st
    ref.direct()
    check_ledger(st, ref, "direct", count_rel)
    check_rfed(gpu, ref, "direct")
    assert abs(st["f_u"] - ref.f_u) <= 1e-12 * max(ref.f_u, 1e-300)
    for it in range(n_iter):
        rem, st = gpu.scatter_iter()
        rem_ref = ref.scatter_iter()
        check_ledger(st, ref, f"iter{it}", count_rel)
        check_rfed(gpu, ref, f"iter{it}")
        assert abs(rem - rem_ref) <= REL_TOTAL * max(rem_ref, 1e-12)
    return gpu, ref


def test_sphere_direct_and_scattering():
    grid = synth.small_sphere(9, cell=0.25, radius=0.8, tau_radial=1.0)
    gpu, ref = run_pair(grid, 2, a_rt=0.05, r_pre=0.5)
    # scattering source function, per pixel
    for which in ("total", "pending"):
        a = gpu.jsca_block(0, which)
        b = ref.jsca(0, which)
        big = b > 1e-6 * b.max()
        assert np.abs(a[big] / b[big] - 1).max() <= REL_CELL


def test_config1_full():
    """16^3 sphere, one source, direct light + 3 scattering iterations."""
    grid = synth.config1()
    run_pair(grid, 3, a_rt=0.05, r_pre=0.3)


def test_tree_representation():
    grid = synth.config1(as_tree=True)
    run_pair(grid, 1, a_rt=0.05, r_pre=0.3)


@pytest.mark.parametrize("merge", [0, 1])
def test_adaptive_galaxy(merge):
    grid = synth.galaxy_disk(max_level=3, threshold=0.3, nroot=(3, 3, 1), root_size=4.0)
    gpu, ref = run_pair(grid, 1, a_rt=0.05, r_pre=2.0, merge=merge, src_stride=23)
    if merge:
        # Eq. 3 fires on this grid, on both sides (the counts were compared)
        assert ref.stats()[1]["merges"] > 0 and gpu.last_stats["merges"] > 0
    else:
        assert ref.stats()[1]["merges"] == 0 and gpu.last_stats["merges"] == 0


def test_multi_lambda():
    g1 = synth.small_sphere(7, cell=0.25, radius=0.7, tau_radial=1.0)
    nl = 4
    kr = g1.kappa_rho * np.array([1.6, 1.0, 0.6, 0.3], np.float32)[None, :]
    em = np.repeat(g1.emissivity, nl, axis=1) * np.array([0.5, 1.0, 1.0, 0.7], np.float32)[None, :]
    grid = g1.with_lambda(kr, em, [0.7, 0.6, 0.5, 0.4], [0.75, 0.6, 0.5, 0.4])
    run_pair(grid, 1, a_rt=0.05, r_pre=0.4)


def _to_device(grid):
    """The grid with every input array on the GPU (inputs_on_device)."""
    import dataclasses
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    return dataclasses.replace(
        grid, first_child=t(grid.first_child), leaf_of_node=t(grid.leaf_of_node), kappa_rho=t(grid.kappa_rho),
        emissivity=t(grid.emissivity), albedo=t(grid.albedo), g=t(grid.g),
        point_xyz=torch.zeros((0, 3), device="cuda"), point_lum=torch.zeros((0, grid.n_lambda), device="cuda"))


@pytest.mark.parametrize("nl", [3, 5])
def test_wavelength_counts_between_marcher_widths(nl, tmp_path):
    """3 and 5 wavelengths, which the library pads to rays of 4 and 8: the
    ledger, RFED and j_sca of every wavelength, the internal and the
    distant-observer maps, device inputs and outputs and the state file,
    all in the caller's layout, against the oracle."""
    g1 = synth.small_sphere(7, cell=0.25, radius=0.7, tau_radial=1.0)
    f = np.array([1.6, 1.0, 0.6, 0.3, 0.2], np.float32)[:nl]
    kr = g1.kappa_rho * f[None, :]
    em = np.repeat(g1.emissivity, nl, axis=1) * np.array([0.5, 1.0, 1.0, 0.7, 0.9], np.float32)[None, :nl]
    grid = g1.with_lambda(kr, em, [0.7, 0.6, 0.5, 0.45, 0.4][:nl], [0.75, 0.6, 0.5, 0.45, 0.3][:nl])
    gpu, ref = run_pair(grid, 1, a_rt=0.05, r_pre=0.4)
    assert list(gpu.k_lam) == list(ref.k_lam) and list(gpu.off_lam) == list(ref.off_lam)
    assert gpu.sca_len == ref.jsca_total.size
    for l in range(nl):
        a, b = gpu.jsca_block(l), ref.jsca(l)
        big = b > 1e-6 * b.max()
        assert np.abs(a[big] / b[big] - 1).max() <= REL_CELL, l
    obs = [0.3, -0.2, 0.1]
    a, b = gpu.map(obs, 3, max_sub=3), ref.map(obs, 3, max_sub=3)
    assert a.shape == b.shape == (nl, 12 * 4 ** 3)
    big = b > 1e-6 * b.max()
    assert np.abs(a[big] / b[big] - 1).max() <= REL_CELL
    frame = ((0.3, -0.8, 0.52), (0.0, 0.0, 1.0), (-1.4, -1.4), 0.1, 28, 28)
    e = gpu.map_external(*frame)
    r = oracle.ExternalMapOracle(ref, *frame).map()
    big = r > 1e-6 * r.max()
    assert e.shape == (nl, 28, 28) and np.abs(e[big] / r[big] - 1).max() <= REL_CELL
    dm = np.random.default_rng(5).standard_normal((nl, 28, 28)).astype(np.float32)
    gk_host = gpu.map_external_vjp(*frame, dm)
    gk_dev = gpu.map_external_vjp(*frame, torch.tensor(dm, device="cuda"))
    assert gk_host.shape == (grid.n_leaf, nl)
    assert np.allclose(gk_dev.cpu().numpy(), gk_host, rtol=1e-5, atol=1e-6 * np.abs(gk_host).max())
    U_dev = torch.empty((grid.n_leaf, nl), dtype=torch.float32, device="cuda")
    gpu.rfed(U=U_dev)
    U_host, L_host = gpu.rfed()
    assert np.array_equal(U_dev.cpu().numpy(), U_host)
    path = str(tmp_path / "state.bin")
    gpu.save(path)
    other = DartRay(grid, r_pre=0.4)
    other.load(path)
    assert np.array_equal(other.rfed()[0], U_host)
    assert np.array_equal(other.jsca(), gpu.jsca())
    on_dev = DartRay(_to_device(grid), r_pre=0.4)
    on_dev.direct()
    Ud, _ = on_dev.rfed()
    st_ref = DartRay(grid, r_pre=0.4)
    st_ref.direct()
    assert np.abs(Ud - st_ref.rfed()[0]).max() <= 1e-5 * Ud.max()


def test_point_sources():
    g = synth.lognormal_cube(8, 4, n_src=3, tau_mean=1.5)
    pts = np.array([[0.13, -0.27, 0.41], [-0.6, 0.2, -0.05]], np.float32)
    grid = synth.Grid(nroot=g.nroot, root_lo=g.root_lo, root_size=g.root_size, first_child=g.first_child,
                      leaf_of_node=g.leaf_of_node, leaf_lo=g.leaf_lo, leaf_size=g.leaf_size,
                      kappa_rho=g.kappa_rho, emissivity=g.emissivity, albedo=g.albedo, g=g.g,
                      point_xyz=pts, point_lum=np.array([[0.5], [0.25]], np.float32))
    # Point sources sit at non-dyadic positions: ray-face distances are no
    # longer exact in float32, so a few rays that graze an edge visit a
    # zero-length cell in one precision and not in the other (each such
    # crossing deposits nothing) and a few R_pre cuts flip; counts are
    # compared to 5e-3 here.
    run_pair(grid, 1, count_rel=5e-3, a_rt=0.02, r_pre=0.6)


def test_no_sources_gives_zero():
    grid = synth.config1()
    grid.emissivity[:] = 0
    gpu = DartRay(grid)
    st = gpu.direct()
    U, L = gpu.rfed()
    assert st["sources"] == 0 and st["crossings"] == 0 and np.all(U == 0)
    rem, st = gpu.scatter_iter()
    assert rem == 0 and st["crossings"] == 0


def test_single_cell_model():
    grid = synth.sphere_cube(1, radius=10.0, tau_radial=5.0)
    run_pair(grid, 1, a_rt=0.05, r_pre=1.0)


def test_scatter_before_direct_is_an_error():
    gpu = DartRay(synth.config1())
    with pytest.raises(DartRayError) as e:
        gpu.scatter_iter()
    assert e.value.code == -6


def test_crossing_cap_reports_limit():
    gpu = DartRay(synth.config1(), max_cross=3)
    with pytest.raises(DartRayError) as e:
        gpu.direct()
    assert e.value.code == -5
    # the grid stays usable
    gpu2 = DartRay(synth.config1())
    gpu2.direct()


def test_small_queues_recover_by_batching():
    grid = synth.galaxy_disk(max_level=2, threshold=0.3, nroot=(3, 3, 1), root_size=4.0)
    a = DartRay(grid, queue_rays=1 << 16, r_pre=2.0)
    b = DartRay(grid, r_pre=2.0)
    sa, sb = a.direct(), b.direct()
    Ua, Ub = a.rfed()[0], b.rfed()[0]
    assert sa["crossings"] == sb["crossings"]
    assert np.abs(Ua - Ub).max() <= 1e-5 * Ub.max()
    # a second call sizes its batches from the first call's heaviest batch:
    # no more restarts than the first call, the same result
    sa2 = a.direct()
    assert sa2["restarts"] <= sa["restarts"]
    assert sa2["crossings"] == sa["crossings"]
    assert np.abs(a.rfed()[0] - Ua).max() <= 1e-5 * Ub.max()


def test_device_buffers_and_state_roundtrip(tmp_path):
    grid = synth.small_sphere(7, cell=0.25, radius=0.6, tau_radial=1.0)
    gpu = DartRay(grid, r_pre=0.4)
    gpu.direct()
    gpu.scatter_iter()
    U_dev = torch.empty((grid.n_leaf, 1), dtype=torch.float32, device="cuda")
    gpu.rfed(U=U_dev)
    U_host, _ = gpu.rfed()
    assert np.array_equal(U_dev.cpu().numpy(), U_host)
    path = str(tmp_path / "state.bin")
    gpu.save(path)
    m1 = gpu.map([0.05, -0.1, 0.02], 3)
    other = DartRay(grid, r_pre=0.4)
    other.load(path)
    assert np.array_equal(other.rfed()[0], U_host)
    m2 = other.map([0.05, -0.1, 0.02], 3)
    assert np.abs(m2 - m1).max() <= 1e-6 * m1.max()  # float atomics: order may differ


def test_inputs_on_device():
    grid = synth.small_sphere(7, cell=0.25, radius=0.6, tau_radial=1.0)
    import dataclasses
    dgrid = dataclasses.replace(
        grid, first_child=torch.from_numpy(grid.first_child).cuda(),
        leaf_of_node=torch.from_numpy(grid.leaf_of_node).cuda(),
        kappa_rho=torch.from_numpy(grid.kappa_rho).cuda(), emissivity=torch.from_numpy(grid.emissivity).cuda(),
        albedo=torch.from_numpy(grid.albedo).cuda(), g=torch.from_numpy(grid.g).cuda(),
        point_xyz=torch.zeros((0, 3), device="cuda"), point_lum=torch.zeros((0, 1), device="cuda"))
    a = DartRay(dgrid, r_pre=0.4)
    b = DartRay(grid, r_pre=0.4)
    a.direct()
    b.direct()
    assert np.array_equal(a.rfed()[0], b.rfed()[0]) or np.abs(a.rfed()[0] - b.rfed()[0]).max() < 1e-6 * b.rfed()[0].max()


@pytest.mark.parametrize("use_jsca", [0, 1])
def test_map_parity(use_jsca):
    grid = synth.small_sphere(9, cell=0.25, radius=0.8, tau_radial=1.0)
    params = dict(a_rt=0.05, r_pre=0.5)
    gpu = DartRay(grid, **params)
    ref = oracle.Oracle(grid, oracle.OracleParams(**params))
    gpu.direct()
    ref.direct()
    gpu.scatter_iter()
    ref.scatter_iter()
    obs = [0.3, -0.2, 0.1]
    a = gpu.map(obs, 3, max_sub=3, use_jsca=bool(use_jsca))
    b = ref.map(obs, 3, max_sub=3, use_jsca=bool(use_jsca))
    big = b > 1e-6 * b.max()
    assert np.abs(a[big] / b[big] - 1).max() <= REL_CELL
    assert abs(a.sum() / b.sum() - 1) <= REL_TOTAL


@pytest.mark.parametrize("records", [0, 5000])
def test_deferred_deposit_matches_direct_atomics(records):
    """The deferred per-cell accumulation of crossing records (and its
    mix with direct atomics when the record buffer is small) gives the same
    scattering source function as per-pixel atomic deposits."""
    grid = synth.config1()
    a = DartRay(grid, r_pre=0.3, deposit_direct=1)
    b = DartRay(grid, r_pre=0.3, deposit_records=records)
    for g in (a, b):
        g.direct()
        g.scatter_iter()
    ja, jb = a.jsca("total"), b.jsca("total")
    big = ja > 1e-6 * ja.max()
    assert np.abs(jb[big] / ja[big] - 1).max() <= 1e-5
    Ua, Ub = a.rfed()[0], b.rfed()[0]
    # U is summed with float atomics in a run-dependent order; a blocking test
    # that sits on its threshold can flip: 1e-4
    assert np.abs(Ub / np.maximum(Ua, 1e-30) - 1)[Ua > 1e-6 * Ua.max()].max() <= 1e-4


def test_galaxy_full_size_sampled_sources():
    """The 297,840-leaf galaxy at full size, in the launch configuration the
    benchmark uses (all pipelines, automatic queues, 2^30 deposit records per
    pipeline), on a sample the oracle finishes in seconds: every 30000th
    source of steps 1-2 and of one scattering iteration."""
    grid = synth.config2()
    params = dict(a_rt=0.05, r_pre=0.15 * grid.model_size, src_stride=30000, deposit_records=1 << 30)
    gpu, ref = run_pair(grid, 1, **params)
    led, cnt = ref.stats()
    assert cnt["crossings"] > 1_000_000 and cnt["sources"] > 0


def test_sixteen_wavelengths():
    """16 wavelengths (the widest ray record): differing kappa*rho,
    emissivity, albedo and g, so that k_lambda runs over 0..3, negligible
    wavelengths are skipped while others deposit (Sect. 3.2), and the
    scattering rays start at the largest k_lambda."""
    g1 = synth.small_sphere(7, cell=0.25, radius=0.7, tau_radial=1.0)
    nl = 16
    t = np.linspace(0.0, 1.0, nl)
    kr = g1.kappa_rho * (2.0 - 1.8 * t).astype(np.float32)[None, :]
    em = np.repeat(g1.emissivity, nl, axis=1) * (0.3 + t).astype(np.float32)[None, :]
    albedo = (0.75 - 0.4 * t).astype(np.float32)
    gg = (0.78 - 0.72 * t).astype(np.float32)
    grid = g1.with_lambda(kr, em, albedo, gg)
    gpu, ref = run_pair(grid, 1, a_rt=0.05, r_pre=0.4)
    assert sorted(set(ref.k_lam)) == [0, 1, 2, 3] and list(gpu.k_lam) == list(ref.k_lam)
    assert ref.stats()[0]["skipped"].sum() > 0  # some wavelengths were negligible on their own


def _write_state(path, grid, U, U_LL, pend_cur, pend_next, jtot, l_sca2, have_direct=True):
    """A restart file in the library's format (the header's state layout:
    magic, n_leaf, n_lambda, j_sca length, direct flag, L_sca2, then U, U_LL,
    the pending buffer to emit, the pending buffer deposited last, j_sca
    total, all float32)."""
    with open(path, "wb") as f:
        f.write(b"DRTSTAT1")
        f.write(np.array([grid.n_leaf, grid.n_lambda, jtot.size, int(have_direct)], np.int64).tobytes())
        f.write(np.array([l_sca2], np.float64).tobytes())
        for a in (U, U_LL, pend_cur, pend_next, jtot):
            f.write(np.ascontiguousarray(a, np.float32).tobytes())


def _map_pair(grid, params, observer, nside_k, max_sub, tmp_path):
    """Oracle sweep (sampled sources), its state loaded into the library, and
    both maps: the map kernel sees the oracle's j_sca (rounded to float32)."""
    ref = oracle.Oracle(grid, oracle.OracleParams(**{k: v for k, v in params.items() if k in ORACLE_KEYS}))
    ref.direct()
    ref.scatter_iter()
    gpu = DartRay(grid, **params)
    path = str(tmp_path / "oracle_state.bin")
    _write_state(path, grid, ref.U, ref.U_LL, ref.pend_a, ref.pend_b, ref.jsca_total, ref.L_sca2)
    gpu.load(path)
    out = {}
    for use in (False, True):
        a = gpu.map(observer, nside_k, max_sub=max_sub, use_jsca=use)
        b = ref.map(observer, nside_k, max_sub=max_sub, use_jsca=use)
        for l in range(grid.n_lambda):
            big = b[l] > 1e-6 * b[l].max()
            assert np.abs(a[l][big] / b[l][big] - 1).max() <= REL_CELL, (use, l)
            assert np.all(a[l][~big] <= 2e-6 * b[l].max())
            assert abs(a[l].sum() / b[l].sum() - 1) <= REL_TOTAL, (use, l)
        out[use] = (a, b)
    return out


def test_map_parity_adaptive_galaxy(tmp_path):
    """Internal-observer map on an adaptive grid (cell sides 0.5 and 1 kpc),
    the observer in a fine cell next to coarse ones, nside 16, subdivision
    up to three levels."""
    grid = synth.galaxy_disk(max_level=3, threshold=0.3, nroot=(3, 3, 1), root_size=4.0)
    obs = (1.8125, 0.3125, 0.9375)
    lf = grid.leaf_containing(obs)
    above = grid.leaf_containing((1.8125, 0.3125, 1.0625))
    assert grid.leaf_size[lf] == 0.5 and grid.leaf_size[above] == 1.0
    _map_pair(grid, dict(a_rt=0.05, r_pre=2.0, src_stride=23), obs, 4, 3, tmp_path)


def test_map_parity_galaxy_full_size(tmp_path):
    """The map the benchmark makes: the 297,840-leaf galaxy (6 refinement
    levels), nside 64, subdivision up to three levels, the observer at
    (8, 0, 0) kpc in the mid-plane; j_sca from the oracle's sweep of every
    30000th source."""
    grid = synth.config2()
    params = dict(a_rt=0.05, r_pre=0.15 * grid.model_size, src_stride=30000)
    out = _map_pair(grid, params, (8.0, 0.0, 0.0), 6, 3, tmp_path)
    a, b = out[True]
    assert np.count_nonzero(b) > 0.5 * b.size  # most of the sky sees some cell


def test_galaxy_full_size_small_buffers():
    """The 297,840-leaf galaxy on sampled sources with ray queues and a
    record buffer small enough that a phase restarts after a queue overflow,
    records are flushed in mid-phase, and batches run on both pipelines --
    all against the oracle."""
    grid = synth.config2()
    params = dict(a_rt=0.05, r_pre=0.15 * grid.model_size, src_stride=30000)
    chosen = None
    for q in (1 << 16, 1 << 17, 1 << 18, 1 << 19):
        try:
            probe = DartRay(grid, queue_rays=q, deposit_records=1 << 18, **params)
            st = probe.direct()
        except DartRayError as e:
            if e.code == -4:  # a single source's wave does not fit: try a larger queue
                continue
            raise
        probe.close()
        if st["restarts"] > 0:
            chosen = q
            break
    assert chosen is not None, "no queue size both fits one source and forces a restart"
    gpu, ref = run_pair(grid, 1, queue_rays=chosen, deposit_records=1 << 18, **params)
    st = gpu.direct_stats
    assert st["restarts"] > 0 and st["flushes"] > 1 and st["batches"] > 1, st
    assert gpu.last_stats["flushes"] > 1


def test_deterministic_mode_bit_identical_and_within_tolerance():
    """deterministic=1 sums U, the j_sca rows and the ledger in 64-bit fixed
    point: two runs give bit-identical RFED, scattering source function,
    ledger and counters, and both match the oracle at the usual tolerances.
    The galaxy (merges, splits, blocking, several batches) is run on sampled
    sources."""
    grid = synth.galaxy_disk(max_level=3, threshold=0.3, nroot=(3, 3, 1), root_size=4.0)
    params = dict(a_rt=0.05, r_pre=2.0, src_stride=23, deterministic=1)
    gpu, ref = run_pair(grid, 1, **params)
    again = DartRay(grid, **params)
    s1 = again.direct()
    for k in ("crossings", "rays", "splits", "merges", "blocks", "escapes", "records", "emitted", "absorbed",
              "scattered", "escaped", "blocked", "skipped"):
        assert np.array_equal(np.asarray(s1[k]), np.asarray(gpu.direct_stats[k])), k
    rem_a, s2 = again.scatter_iter()
    for k in ("crossings", "rays", "splits", "merges", "blocks", "escapes", "absorbed", "scattered", "escaped"):
        assert np.array_equal(np.asarray(s2[k]), np.asarray(gpu.last_stats[k])), k
    assert np.array_equal(again.rfed()[0], gpu.rfed()[0])
    assert np.array_equal(again.jsca("total"), gpu.jsca("total"))
    assert np.array_equal(again.jsca("pending"), gpu.jsca("pending"))


def test_deterministic_mode_galaxy_full_size():
    """The 297,840-leaf galaxy in the deterministic mode on sampled sources,
    against the oracle, with the benchmark's launch configuration."""
    grid = synth.config2()
    params = dict(a_rt=0.05, r_pre=0.15 * grid.model_size, src_stride=30000, deterministic=1)
    run_pair(grid, 1, **params)
