"""The map for a distant observer and its reverse march (gradients with
respect to kappa*rho and the albedo), through the C ABI and
torch.autograd, against the FP64 oracle and against central finite
differences of the library's own map.

Readings: the lines of sight are parallel (orthographic); the source of a
cell is its emissivity plus the total j_sca of the pixel holding the
direction toward the observer, per solid angle and volume; the gradient
holds the radiation field of the last sweep fixed (j_sca then scales with
the albedo and does not depend on kappa*rho)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1709_03802_gb300 import DartRay, DartRayError, external_map  # noqa: E402
from test_gpu_parity import ORACLE_KEYS, _write_state  # noqa: E402

EDGE_ON = ((0.0, -1.0, 0.0), (0.0, 0.0, 1.0))
OBLIQUE = ((0.3, -0.8, 0.52), (0.0, 0.0, 1.0))


def _swept_pair(tmp_path, n=16):
    """Oracle sweep (steps 1-2 and one scattering iteration) of a clumpy
    cube, its state loaded into the library so both maps see the same j_sca."""
    grid = synth.lognormal_cube(n, 4, tau_mean=2.0, n_src=8)
    params = dict(a_rt=0.05, r_pre=0.5)
    ref = oracle.Oracle(grid, oracle.OracleParams(**{k: v for k, v in params.items() if k in ORACLE_KEYS}))
    ref.direct()
    ref.scatter_iter()
    gpu = DartRay(grid, **params)
    path = str(tmp_path / "oracle_state.bin")
    _write_state(path, grid, ref.U, ref.U_LL, ref.pend_a, ref.pend_b, ref.jsca_total, ref.L_sca2)
    gpu.load(path)
    return grid, gpu, ref


@pytest.mark.parametrize("view", [EDGE_ON, OBLIQUE], ids=["edge-on", "oblique"])
def test_external_map_and_gradients_match_oracle(tmp_path, view):
    grid, gpu, ref = _swept_pair(tmp_path)
    nx = ny = 50
    # edge-on, no line of sight within 0.004 of a cell face (cell side 0.125)
    px, org = (0.048, (-1.2, -1.2)) if view is EDGE_ON else (0.072, (-1.8, -1.8))
    rng = np.random.default_rng(1709 * 100 + 41)
    for use in (False, True):
        m = oracle.ExternalMapOracle(ref, view[0], view[1], org, px, nx, ny, use_jsca=use)
        b = m.map()
        a = gpu.map_external(view[0], view[1], org, px, nx, ny, use_jsca=use)
        big = b > 1e-6 * b.max()
        # the 8 emitting cells alone light few lines of sight; j_sca all that
        # cross the cube (the oblique image is larger than the cube)
        assert big.sum() > (0.3 * b.size if use else 10)
        assert np.abs(a[big] / b[big] - 1).max() <= 1e-4, use
        assert np.all(np.abs(a[~big]) <= 2e-6 * b.max())
        dmap = rng.standard_normal(b.shape)
        gk, ga = gpu.map_external_vjp(view[0], view[1], org, px, nx, ny, dmap.astype(np.float32), use_jsca=use,
                                      with_albedo=True)
        rk = m.vjp(dmap.astype(np.float32).astype(np.float64))
        ra = m.vjp_albedo(dmap.astype(np.float32).astype(np.float64))
        scale = np.abs(rk).max()
        assert scale > 0
        assert np.all(np.abs(gk - rk) <= 1e-4 * scale + 1e-3 * np.abs(rk)), use
        if use:
            assert abs(ga[0] - ra[0]) <= 1e-4 * abs(ra[0])
        else:
            assert ga[0] == 0.0
    gpu.close()


def test_external_map_device_buffers_and_kappa_rho_update(tmp_path):
    """Device in/out buffers give the host results; set_kappa_rho changes
    the map as the oracle's map of the changed medium."""
    grid, gpu, ref = _swept_pair(tmp_path, n=8)
    view, up = OBLIQUE
    a = gpu.map_external(view, up, (-1.8, -1.8), 0.1, 36, 36)
    d = torch.empty((1, 36, 36), dtype=torch.float32, device="cuda")
    gpu.map_external(view, up, (-1.8, -1.8), 0.1, 36, 36, out=d)
    assert np.array_equal(a, d.cpu().numpy())
    dm = torch.ones_like(d)
    g1 = gpu.map_external_vjp(view, up, (-1.8, -1.8), 0.1, 36, 36, dm)
    g2 = gpu.map_external_vjp(view, up, (-1.8, -1.8), 0.1, 36, 36, np.ones((1, 36, 36), np.float32))
    assert np.allclose(g1.cpu().numpy(), g2, rtol=1e-5, atol=1e-7 * np.abs(g2).max())
    kr2 = (grid.kappa_rho * 1.5).astype(np.float32)
    gpu.set_kappa_rho(kr2)
    m = oracle.ExternalMapOracle(ref, view, up, (-1.8, -1.8), 0.1, 36, 36)
    b = m.map(kr2.astype(np.float64))
    a2 = gpu.map_external(view, up, (-1.8, -1.8), 0.1, 36, 36)
    big = b > 1e-6 * b.max()
    assert np.abs(a2[big] / b[big] - 1).max() <= 1e-4
    with pytest.raises(DartRayError):
        gpu.map_external(view, view, (-1.8, -1.8), 0.1, 36, 36)  # up parallel to the view
    gpu.close()


def _config4(emission_everywhere=False):
    grid = synth.lognormal_cube(64, 4, tau_mean=2.0)
    if emission_everywhere:  # a diffuse source: every line of sight carries light
        grid.emissivity[:] = (grid.kappa_rho / grid.kappa_rho.mean() * 0.01).astype(np.float32)
    return grid


def test_config4_gradient_against_oracle_full_size():
    """The 64^3 clumpy cube (mean tau_V = 2), the 256x256 edge-on map of a
    diffuse source, a seeded upstream gradient: every cell's gradient
    against the oracle's."""
    grid = _config4(emission_everywhere=True)
    gpu = DartRay(grid, a_rt=0.05, r_pre=0.3)
    ref = oracle.Oracle(grid, oracle.OracleParams(a_rt=0.05, r_pre=0.3))
    view, up = EDGE_ON
    m = oracle.ExternalMapOracle(ref, view, up, (-1.0, -1.0), 2.0 / 256, 256, 256, use_jsca=False)
    b = m.map()
    a = gpu.map_external(view, up, (-1.0, -1.0), 2.0 / 256, 256, 256, use_jsca=False)
    assert np.abs(a / b - 1).max() <= 1e-4
    dmap = np.random.default_rng(1709 * 100 + 42).standard_normal(b.shape).astype(np.float32)
    gk = gpu.map_external_vjp(view, up, (-1.0, -1.0), 2.0 / 256, 256, 256, dmap, use_jsca=False)
    rk = m.vjp(dmap.astype(np.float64))
    assert np.all(np.abs(gk - rk) <= 1e-4 * np.abs(rk).max() + 1e-3 * np.abs(rk))
    gpu.close()


def test_config4_autograd_against_central_differences():
    """Config 4 end to end: the library's sweep of the 64^3 clumpy cube
    (steps 1-2 and two scattering iterations), the 256x256 edge-on map
    through torch.autograd, an L2 loss against a seeded target map; the
    gradient on 64 seeded cells against central differences of the same
    loss to 1e-3."""
    grid = _config4()
    gpu = DartRay(grid, a_rt=0.05, r_pre=0.3)
    gpu.direct()
    for _ in range(2):
        gpu.scatter_iter()
    view, up = EDGE_ON
    frame = (view, up, (-1.0, -1.0), 2.0 / 256, 256, 256)
    kr = torch.tensor(grid.kappa_rho, device="cuda", requires_grad=True)
    img = external_map(gpu, kr, *frame)
    rng = np.random.default_rng(1709 * 100 + 43)
    target = (img.detach() * torch.tensor(1 + 0.2 * rng.standard_normal((1, 256, 256)), device="cuda")).double()
    loss = 0.5 * ((img.double() - target) ** 2).sum()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    loss.backward()
    t1.record()
    torch.cuda.synchronize()
    grad = kr.grad[:, 0].cpu().numpy().astype(np.float64)
    assert np.count_nonzero(grad) > 0.5 * grad.size
    cells = rng.choice(grid.n_leaf, 64, replace=False)
    base = kr.detach().clone()

    def loss_at(k):
        with torch.no_grad():
            im = external_map(gpu, k, *frame)
            return float(0.5 * ((im.double() - target) ** 2).sum())

    worst = 0.0
    for c in cells:
        h = 0.05 * float(base[c, 0])
        kp, km = base.clone(), base.clone()
        kp[c, 0] += h
        km[c, 0] -= h
        h2 = float(kp[c, 0]) - float(km[c, 0])  # the step as stored (float32)
        fd = (loss_at(kp) - loss_at(km)) / h2
        err = abs(grad[c] - fd) / max(abs(fd), 1e-3 * np.abs(grad).max())
        worst = max(worst, err)
    print(f"config 4: reverse march {t0.elapsed_time(t1):.2f} ms; worst FD difference {worst:.2e}")
    assert worst <= 1e-3
    gpu.close()


@pytest.mark.parametrize("records", [None, 0], ids=["deferred", "atomic"])
def test_g_tally_and_gradient_match_oracle(records):
    """The tally of d j_sca / d g for the view pixel (both deposit
    schedules: flushed records and per-crossing row atomics) and the map's
    g gradient, each side on its own sweep (steps 1-2 and one scattering
    iteration) of a clumpy cube."""
    grid = synth.lognormal_cube(16, 4, tau_mean=2.0, n_src=8)
    params = dict(a_rt=0.05, r_pre=0.5)
    view, up = OBLIQUE
    extra = {} if records is None else dict(deposit_records=records)
    gpu = DartRay(grid, **params, **extra)
    ref = oracle.Oracle(grid, oracle.OracleParams(**params))
    gpu.dg_arm(view)
    ref.dg_arm(view)
    gpu.direct()
    ref.direct()
    gpu.scatter_iter()
    ref.scatter_iter()
    a, b = gpu.dg()[:, 0], ref.dg()[:, 0]
    scale = np.abs(b).max()
    assert np.count_nonzero(b) > 0.5 * b.size
    assert np.all(np.abs(a - b) <= 1e-4 * scale + 3e-3 * np.abs(b))
    frame = (view, up, (-1.8, -1.8), 0.072, 50, 50)
    dmap = np.random.default_rng(1709 * 100 + 44).standard_normal((1, 50, 50))
    _, gg = gpu.map_external_vjp(*frame, dmap.astype(np.float32), with_g=True)
    rg = oracle.ExternalMapOracle(ref, *frame).vjp_g(dmap.astype(np.float32).astype(np.float64), ref.dg())
    assert abs(gg[0] - rg[0]) <= 3e-3 * abs(rg[0])
    with pytest.raises(DartRayError):  # another view than the armed one
        gpu.map_external_vjp(EDGE_ON[0], up, (-1.8, -1.8), 0.072, 50, 50, dmap.astype(np.float32), with_g=True)
    gpu.close()


def test_albedo_and_g_gradients_through_autograd_against_central_differences():
    """Config 4's cube and map with the albedo and g as autograd inputs,
    after step 2 (whose deposited luminosities depend on neither): central
    differences over deterministic sweeps at albedo +- eps and g +- eps."""
    grid = _config4()
    view, up = EDGE_ON
    frame = (view, up, (-1.0, -1.0), 2.0 / 256, 256, 256)
    rng = np.random.default_rng(1709 * 100 + 45)
    target = None

    def sweep(alb, gv):
        gr = grid.with_lambda(grid.kappa_rho, grid.emissivity, [alb], [gv])
        m = DartRay(gr, a_rt=0.05, r_pre=0.3, deterministic=1)
        m.dg_arm(view)
        m.direct()
        return m, gr

    def loss(img):
        return float(0.5 * ((img.double() - target) ** 2).sum())

    m, gr = sweep(0.6, 0.6)
    kr = torch.tensor(gr.kappa_rho, device="cuda", requires_grad=True)
    alb = torch.tensor(gr.albedo, device="cuda", requires_grad=True)
    gg = torch.tensor(gr.g, device="cuda", requires_grad=True)
    img = external_map(m, kr, *frame, albedo=alb, g=gg)
    target = (img.detach() * torch.tensor(1 + 0.2 * rng.standard_normal((1, 256, 256)), device="cuda")).double()
    L = 0.5 * ((img.double() - target) ** 2).sum()
    L.backward()
    m.close()
    for name, base, grad in (("albedo", 0.6, alb.grad), ("g", 0.6, gg.grad)):
        vals = []
        for sgn in (1, -1):
            a, gv = (base * (1 + sgn * 1e-2), 0.6) if name == "albedo" else (0.6, base * (1 + sgn * 1e-2))
            mm, g2 = sweep(a, gv)
            k2 = torch.tensor(g2.kappa_rho, device="cuda")
            with torch.no_grad():
                vals.append((loss(external_map(mm, k2, *frame)),
                             float(g2.albedo[0] if name == "albedo" else g2.g[0])))
            mm.close()
        fd = (vals[0][0] - vals[1][0]) / (vals[0][1] - vals[1][1])
        print(f"d loss / d {name}: autograd {float(grad[0]):.6e}, central differences {fd:.6e}")
        assert abs(float(grad[0]) - fd) <= 1e-3 * abs(fd), name
