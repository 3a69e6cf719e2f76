"""Forward mode (tangent_albedo): the derivative of U and L_abs with respect
to each wavelength's albedo, carried through the sweep as extra wavelengths
with the decisions of their own wavelength, against the oracle's forward
mode and against central differences of the library's own sweeps."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1709_03802_gb300 import DartRay, DartRayError  # noqa: E402
from test_gpu_parity import REL_CELL, run_pair  # noqa: E402
from test_oracle_tangent import two_lambda_cube  # noqa: E402


def check_tangent(gpu, ref):
    dU, dL = gpu.rfed_tangent()
    rU, rL = ref.rfed_tangent()
    for l in range(rU.shape[1]):
        big = rU[:, l] > 1e-6 * rU[:, l].max()
        assert rU[:, l].max() > 0
        assert np.abs(dU[big, l] / rU[big, l] - 1).max() <= REL_CELL, l
        assert np.all(np.abs(dL[:, l] - rL[:, l]) <= REL_CELL * (np.abs(rL[:, l]).max() + np.abs(rL[:, l]))), l


def test_tangent_clumpy_cube_two_wavelengths_with_blocking():
    """Two wavelengths (the forward mode pads them to rays of 4), blocking
    on, steps 1-2 and two scattering iterations."""
    gpu, ref = run_pair(two_lambda_cube(), 2, a_rt=0.05, r_pre=0.5, tangent_albedo=1)
    assert ref.stats()[1]["blocks"] > 0
    check_tangent(gpu, ref)
    # the wavelengths themselves are those of a plain sweep
    plain = DartRay(two_lambda_cube(), a_rt=0.05, r_pre=0.5)
    plain.direct()
    for _ in range(2):
        plain.scatter_iter()
    U0, U1 = plain.rfed()[0], gpu.rfed()[0]
    assert np.abs(U1 - U0).max() <= 1e-5 * U0.max()


def test_tangent_adaptive_galaxy_with_merges():
    grid = synth.galaxy_disk(max_level=3, threshold=0.3, nroot=(3, 3, 1), root_size=4.0)
    gpu, ref = run_pair(grid, 1, a_rt=0.05, r_pre=2.0, src_stride=23, tangent_albedo=1)
    assert ref.stats()[1]["merges"] > 0
    check_tangent(gpu, ref)
    dU = torch.empty((grid.n_leaf, 1), dtype=torch.float32, device="cuda")
    dL = torch.empty_like(dU)
    gpu.rfed_tangent(dU, dL)
    assert np.array_equal(dU.cpu().numpy(), gpu.rfed_tangent()[0])


def test_tangent_against_central_differences():
    """Without blocking no decision depends on the albedo, and U after step
    2 and two iterations is a quadratic in it: central differences of two
    deterministic sweeps at albedo (1 +- 1e-2) give the derivative."""
    g = two_lambda_cube()
    t = DartRay(g, a_rt=0.0, r_pre=0.5, tangent_albedo=1)
    t.direct()
    for _ in range(2):
        t.scatter_iter()
    dU = t.rfed_tangent()[0]
    for l in range(2):
        U, a = [], []
        for sgn in (1, -1):
            alb = g.albedo.copy()
            alb[l] *= 1 + sgn * 1e-2
            gp = g.with_lambda(g.kappa_rho, g.emissivity, alb, g.g)
            m = DartRay(gp, a_rt=0.0, r_pre=0.5, deterministic=1)
            m.direct()
            for _ in range(2):
                m.scatter_iter()
            U.append(m.rfed()[0][:, l].astype(np.float64))
            a.append(float(gp.albedo[l]))
        fd = (U[0] - U[1]) / (a[0] - a[1])
        big = fd > 1e-6 * fd.max()
        rel = np.abs(dU[big, l] / fd[big] - 1)
        print(f"forward mode vs central differences, lambda {l}: max {rel.max():.2e}")
        assert rel.max() <= REL_CELL


def test_tangent_rejections(tmp_path):
    g = two_lambda_cube()
    for kw in (dict(deterministic=1), ):
        with pytest.raises(DartRayError):
            DartRay(g, tangent_albedo=1, **kw)
    t = DartRay(g, tangent_albedo=1, r_pre=0.5)
    with pytest.raises(DartRayError):
        t.save(str(tmp_path / "state.bin"))
    p = DartRay(g, r_pre=0.5)
    with pytest.raises(DartRayError):
        p.rfed_tangent()


def test_rfed_albedo_autograd_against_central_differences():
    """A loss of U and L_abs through torch.autograd (rfed_albedo) against
    central differences of the same loss over deterministic sweeps at
    albedo (1 +- 1e-2), no blocking."""
    from paper_1709_03802_gb300 import rfed_albedo
    g = two_lambda_cube()

    def sweep(grid, **kw):
        m = DartRay(grid, a_rt=0.0, r_pre=0.5, **kw)
        m.direct()
        for _ in range(2):
            m.scatter_iter()
        return m

    rng = np.random.default_rng(1709 * 100 + 46)
    w = torch.tensor(rng.uniform(0.5, 1.5, (g.n_leaf, 2)), device="cuda")

    t = sweep(g, tangent_albedo=1)
    alb = torch.tensor(g.albedo, device="cuda", requires_grad=True)
    U, L = rfed_albedo(t, alb)
    S = float(U.detach().max())  # a fixed scale

    def loss(U, L):
        return (w * U.double() ** 2).sum() / S + L.double().sum()

    loss(U, L).backward()
    for l in range(2):
        vals = []
        for sgn in (1, -1):
            a = g.albedo.copy()
            a[l] *= 1 + sgn * 1e-2
            gp = g.with_lambda(g.kappa_rho, g.emissivity, a, g.g)
            m = sweep(gp, deterministic=1)
            Up, Lp = m.rfed()
            val = loss(torch.tensor(Up, device="cuda"), torch.tensor(Lp, device="cuda"))
            vals.append((float(val), float(gp.albedo[l])))
        fd = (vals[0][0] - vals[1][0]) / (vals[0][1] - vals[1][1])
        print(f"d loss / d albedo[{l}]: autograd {float(alb.grad[l]):.6e}, central differences {fd:.6e}")
        assert abs(float(alb.grad[l]) - fd) <= REL_CELL * abs(fd)


def test_tangent_three_wavelengths_padded():
    """Three wavelengths in the forward mode: rays of 8 (3 wavelengths, one
    padding, their 3 derivatives, one padding)."""
    g1 = two_lambda_cube()
    kr = g1.kappa_rho[:, :1] * np.array([1.0, 0.6, 0.3], np.float32)[None, :]
    g = g1.with_lambda(kr, np.repeat(g1.emissivity[:, :1], 3, axis=1), [0.65, 0.55, 0.4], [0.7, 0.5, 0.3])
    gpu, ref = run_pair(g, 1, a_rt=0.05, r_pre=0.5, tangent_albedo=1)
    check_tangent(gpu, ref)
