"""The octant mode (Sect. 3.6.4: for symmetric models only the sources of
the first octant are traced and the contributions in the other octants
follow from the symmetry) against the oracle's octant mode -- the same
algorithm in FP64, whose equality with the full mode on uniform lattices is
pinned in tests/test_oracle_octant.py -- and against the library's full
mode at full size."""
import time

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1709_03802_gb300 import DartRay  # noqa: E402
from test_gpu_parity import REL_CELL, REL_TOTAL, run_pair  # noqa: E402
from test_oracle_octant import symmetric_lattice  # noqa: E402


def test_octant_symmetric_lattice():
    """Sources on three, two and no mirror planes (weights 1/8, 1/4, 1)."""
    gpu, ref = run_pair(symmetric_lattice(), 2, a_rt=0.05, r_pre=0.5, octant=1)
    # the first octant holds 3 of the 11 emitting cells (steps 1 and 2 count them twice)
    assert gpu.direct_stats["sources"] == 6


def test_octant_adaptive_galaxy():
    """An adaptive galaxy (cell sides 0.5 and 1 kpc, 1,152 leaves) with
    splits, merges and blocking."""
    grid = synth.galaxy_disk(max_level=3, threshold=0.3, nroot=(2, 2, 1), root_size=4.0)
    gpu, ref = run_pair(grid, 1, a_rt=0.05, r_pre=1.5, octant=1)
    assert ref.stats()[1]["merges"] > 0


def test_octant_against_full_mode_galaxy_full_size():
    """The 297,840-leaf galaxy, steps 1-2 and one scattering iteration, in
    the octant mode against the full mode of the library: the two modes
    differ only where rays run exactly along cell faces (see
    tests/test_oracle_octant.py), which on this six-level grid moves the
    ledger by up to about 1.5e-3 (measured: absorbed light of step 2 1.1e-4,
    escaped light of the scattering iteration 1.45e-3) and cells by about
    1e-3 in the median; the octant mode is several times faster."""
    grid = synth.config2()
    params = dict(a_rt=0.05, r_pre=0.15 * grid.model_size)
    out = {}
    for octant in (0, 1):
        gpu = DartRay(grid, octant=octant, **params)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sd = gpu.direct()
        rem, si = gpu.scatter_iter()
        torch.cuda.synchronize()
        out[octant] = dict(t=time.perf_counter() - t0, U=gpu.rfed()[0], rem=rem, sd=sd, si=si)
        gpu.close()
    full, octa = out[0], out[1]
    for st in ("sd", "si"):
        for k in ("emitted", "absorbed", "escaped"):
            d = octa[st][k].sum() / full[st][k].sum() - 1
            print(f"octant vs full, {st} {k}: {d:.2e}")
            assert abs(d) <= 50 * REL_TOTAL, (st, k)
    assert abs(octa["rem"] / full["rem"] - 1) <= 50 * REL_TOTAL
    big = full["U"] > 1e-6 * full["U"].max()
    rel = np.abs(octa["U"][big] / full["U"][big] - 1)
    assert np.median(rel) < 1e-2
    assert octa["sd"]["crossings"] < 0.25 * full["sd"]["crossings"]
    speedup = full["t"] / octa["t"]
    print(f"full {full['t']:.2f} s, octant {octa['t']:.2f} s, speed-up {speedup:.2f}, "
          f"per-cell difference median {np.median(rel):.2e} max {rel.max():.2e}")
    assert speedup > 3
