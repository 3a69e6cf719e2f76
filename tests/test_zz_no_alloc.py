"""dartray_map_noalloc: the map entry point for callers that cannot call
cudaMalloc (allocation-restricted allocators, applications that reserve all
device memory up front).  It sums the map in a fixed static device buffer
instead of an allocated one; its output must equal dartray_map's.

This file is collected last so that, if it fails, a run stopping at the first
failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1709_03802_gb300 import DartRay  # noqa: E402
from paper_1709_03802_gb300 import dartray as dr  # noqa: E402


def _call(fn, h, obs, nside_k, max_sub, use_jsca, out):
    """Call the C entry point directly (host output)."""
    lib = dr.load()
    o = (C.c_double * 3)(*obs)
    rc = getattr(lib, fn)(h, o, nside_k, max_sub, use_jsca, out.ctypes.data_as(C.c_void_p), 0)
    assert rc == 0, lib.dartray_last_error().decode()


def test_map_noalloc_matches_map_two_calls():
    grid = synth.small_sphere(9, cell=0.25, radius=0.8, tau_radial=1.0)
    gpu = DartRay(grid, r_pre=0.5)
    gpu.direct()
    gpu.scatter_iter()
    nk = 5
    ref = np.zeros((grid.n_lambda, 12 * 4 ** nk), np.float32)
    _call("dartray_map", gpu._h, (0.3, -0.2, 0.1), nk, 3, 1, ref)
    assert ref.sum() > 0
    # calls in a row: the static buffer keeps the previous map, so each call
    # must clear it; every observer against dartray_map (float atomics sum in
    # a run-dependent order)
    for obs in ((0.3, -0.2, 0.1), (-0.7, 0.45, 0.05), (0.3, -0.2, 0.1)):
        want = np.zeros_like(ref)
        _call("dartray_map", gpu._h, obs, nk, 3, 1, want)
        out = np.full_like(ref, np.nan)
        _call("dartray_map_noalloc", gpu._h, obs, nk, 3, 1, out)
        assert np.abs(out - want).max() <= 1e-5 * want.max(), obs
    # device output through the same entry point
    dev = torch.empty(ref.shape, dtype=torch.float32, device="cuda")
    lib = dr.load()
    o = (C.c_double * 3)(0.3, -0.2, 0.1)
    assert lib.dartray_map_noalloc(gpu._h, o, nk, 3, 1, C.c_void_p(dev.data_ptr()), 1) == 0
    assert np.abs(dev.cpu().numpy() - ref).max() <= 1e-5 * ref.max()


def test_map_noalloc_large_then_small_multi_wavelength():
    """Two wavelengths: a map near the static buffer's size (nside 256: 75%
    of it), then a small one, each against dartray_map; stale data of the
    large map must not leak into the small one."""
    g1 = synth.small_sphere(7, cell=0.25, radius=0.7, tau_radial=1.0)
    grid = g1.with_lambda(g1.kappa_rho * np.array([1.5, 0.5], np.float32)[None, :],
                          np.repeat(g1.emissivity, 2, axis=1), [0.6, 0.5], [0.6, 0.4])
    gpu = DartRay(grid, r_pre=0.4)
    gpu.direct()
    gpu.scatter_iter()
    for nk, obs in ((8, (0.2, 0.1, -0.3)), (4, (-0.4, 0.2, 0.1))):
        want = np.zeros((2, 12 * 4 ** nk), np.float32)
        _call("dartray_map", gpu._h, obs, nk, 2, 1, want)
        out = np.full_like(want, np.nan)
        _call("dartray_map_noalloc", gpu._h, obs, nk, 2, 1, out)
        assert want.sum() > 0
        assert np.abs(out - want).max() <= 1e-5 * want.max(), nk


def test_map_noalloc_rejects_oversized_maps():
    grid = synth.small_sphere(5, cell=0.25)
    gpu = DartRay(grid, r_pre=0.5)
    lib = dr.load()
    out = np.zeros(1, np.float32)
    o = (C.c_double * 3)(0.0, 0.0, 0.0)
    rc = lib.dartray_map_noalloc(gpu._h, o, 10, 0, 0, out.ctypes.data_as(C.c_void_p), 0)
    assert rc == -1
    assert "static buffer" in lib.dartray_last_error().decode()
