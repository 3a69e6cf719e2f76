"""The large particle galaxy at full size: 4e6 star particles (disk with a
two-arm logarithmic spiral, Sersic bulge) on a 10-level tree of 7,618,867
leaves, 16 wavelengths from 0.15 to 2.2 um.

A full sweep is far beyond one test's time: one source of this grid sends
about 2.5e7 rays and 2e8 crossings in steps 1-2 (the finest cells are 3.9 pc
across, so Eq. 2 splits rays to HEALPix level 12 and beyond), and the grid has
3.2e6 emitting cells.  Both tests therefore trace sampled sources:

- a spot check of steps 1-2 at 0.44 um against the oracle on two sources
  (j_sca at level 1 to keep the oracle's memory small);
- the 16 wavelengths in blocks that fit the GPU's memory (the three j_sca
  arrays of all 16 at once would take 0.46 TB), steps 1-2, one scattering
  iteration and the nside-64 internal-observer map at (8, 0, 0) kpc per
  block, with the energy ledger of every wavelength checked."""
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1709_03802_gb300 import DartRay  # noqa: E402
from test_gpu_parity import ORACLE_KEYS, REL_CELL, REL_TOTAL, check_ledger  # noqa: E402

BLOCKS = [[0], [1], [2], [3], [4, 5, 6, 7], [8, 9, 10, 11], [12, 13, 14, 15]]


@pytest.fixture(scope="module")
def galaxy():
    g = synth.config5()
    lv = np.round(np.log2(g.root_size / g.leaf_size)).astype(int)
    assert g.n_leaf == 7_618_867 and lv.max() == 10
    return g


def block(g, ls):
    return g.with_lambda(g.kappa_rho[:, ls], g.emissivity[:, ls], g.albedo[ls], g.g[ls])


def test_spot_check_against_oracle(galaxy):
    g1 = block(galaxy, [6])  # 0.439 um
    params = dict(a_rt=0.05, r_pre=0.15 * g1.model_size, k_sca_cap=1, src_stride=1_600_000, src_offset=7)
    gpu = DartRay(g1, **params)
    ref = oracle.Oracle(g1, oracle.OracleParams(**{k: v for k, v in params.items() if k in ORACLE_KEYS}))
    st = gpu.direct()
    ref.direct()
    check_ledger(st, ref, "config 5")
    assert st["sources"] == 2
    # per cell: the bulk of the cells agrees to ~1e-5 (median 2e-6, 99.9% at
    # 2.5e-5 measured); about 1.4e-4 of them differ by more than 1e-3 (up to
    # 9e-2 measured): rays up to 30 kpc from their source pass within float32
    # rounding of the corners and edges of 3.9 pc cells and cross them in one
    # precision but not the other
    U, L_abs = gpu.rfed()
    Ur, Lr = ref.rfed()
    big = Ur[:, 0] > 1e-6 * Ur[:, 0].max()
    rel = np.abs(U[big, 0] / Ur[big, 0] - 1)
    q = np.quantile(rel, [0.5, 0.99, 0.999])
    print(f"config 5 spot check: {big.sum()} cells above the floor; per-cell U rel median {q[0]:.2e}, "
          f"99% {q[1]:.2e}, 99.9% {q[2]:.2e}, max {rel.max():.2e}; above 1e-3: {(rel > 1e-3).mean():.2e} of them")
    assert abs(L_abs.sum() / Lr.sum() - 1) <= REL_TOTAL
    assert q[0] <= 1e-4 and q[2] <= REL_CELL and (rel > REL_CELL).mean() <= 1e-3
    print(f"config 5 spot check: {st['crossings']:.3e} crossings, {st['rays']:.3e} rays, "
          f"{st['gpu_ms'] / 1e3:.2f} s on the GPU")
    gpu.close()


def test_sixteen_wavelengths_and_map(galaxy):
    stride = 100_000
    maps, lines = [], []
    for ls in BLOCKS:
        gb = block(galaxy, ls)
        gpu = DartRay(gb, a_rt=0.05, r_pre=0.15 * gb.model_size, src_stride=stride, src_offset=3,
                      queue_rays=1 << 26, deposit_records=1 << 25)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sd = gpu.direct()
        rem, si = gpu.scatter_iter()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        m = gpu.map((8.0, 0.0, 0.0), 6, max_sub=3)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        for st in (sd, si):
            # every emitted unit ends absorbed, scattered, escaped, blocked or skipped
            out = st["absorbed"] + st["scattered"] + st["escaped"] + st["blocked"] + st["skipped"]
            assert np.all(np.abs(out / st["emitted"] - 1) <= 1e-4), (ls, out, st["emitted"])
        assert np.all(np.isfinite(m)) and np.all(m >= 0) and np.all(m.sum(axis=1) > 0)
        maps.append(m)
        cross = sd["crossings"] + si["crossings"]
        lines.append(f"lambda {ls}: {cross:.3e} crossings in {t1 - t0:.2f} s ({cross / (t1 - t0):.3e}/s), "
                     f"map {t2 - t1:.2f} s")
        gpu.close()
    sky = np.concatenate(maps)
    assert sky.shape == (16, 12 * 4 ** 6)
    print("config 5, every 100000th source:\n  " + "\n  ".join(lines))
