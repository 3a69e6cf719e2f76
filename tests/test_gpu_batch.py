"""Batched grids: several independent models traced together in one grid
(dartray_grid_create_batch), against FP64 oracle runs of each model alone
and against the library's single-model grids.

The method is additive over sources and no ray leaves its model, so a model
in a batch has the same RFED, scattering source function and ledger as the
same model alone; N_s (Eq. 10), R_pre and the stop of the scattering
iterations (f_L) are each model's own."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1709_03802_gb300 import DartRay, DartRayBatch, DartRayError  # noqa: E402
from test_gpu_parity import REL_CELL, REL_TOTAL, ORACLE_KEYS, close_counts  # noqa: E402


def models():
    """Uneven models of one dust model: three clumpy cubes of different
    sizes and optical depths, a small adaptive galaxy, and a cube lit by two
    point sources."""
    out = [synth.lognormal_cube(4, 3, tau_mean=0.5, n_src=3), synth.lognormal_cube(8, 4, tau_mean=2.0, n_src=4),
           synth.lognormal_cube(16, 5, tau_mean=4.0, n_src=5),
           synth.galaxy_disk(max_level=2, threshold=0.3, nroot=(2, 2, 1), root_size=4.0)]
    c = synth.lognormal_cube(8, 6, tau_mean=1.0, n_src=1)
    c.emissivity[:] = 0
    c.point_xyz = np.array([[0.13, -0.27, 0.41], [-0.6, 0.2, -0.05]], np.float32)
    c.point_lum = np.array([[0.5], [0.25]], np.float32)
    out.append(c)
    return out


def check_model(gpu, m, ref, tag):
    U = gpu.model_rfed(m)[0][:, 0]
    Ur = ref.rfed()[0][:, 0]
    big = Ur > 1e-6 * Ur.max()
    rel = np.abs(U[big] / Ur[big] - 1).max()
    assert rel <= REL_CELL, f"{tag} model {m}: per-cell U rel {rel:.2e}"
    st = gpu.model_stats(m)
    led, _ = ref.stats()
    tot = led["emitted"].sum()
    for k in ("emitted", "absorbed", "scattered", "escaped", "blocked", "cut"):
        assert abs(st[k][0] - led[k][0]) <= REL_TOTAL * tot, f"{tag} model {m} ledger {k}: {st[k][0]} vs {led[k][0]}"
    assert abs(st["f_u"] - ref.f_u) <= 1e-12 * max(ref.f_u, 1e-300)
    j = gpu.model_jsca_block(m, 0, "total")
    jr = ref.jsca(0, "total")
    jb = jr > 1e-6 * jr.max()
    if jb.any():
        assert np.abs(j[jb] / jr[jb] - 1).max() <= REL_CELL, f"{tag} model {m}: j_sca"


def test_batch_matches_oracle_per_model():
    """Steps 1-2 and two scattering iterations of five uneven models in one
    batch, each against its own oracle run (point sources included)."""
    grids = models()
    params = dict(a_rt=0.05, r_pre=0.6, f_l=1e-12)
    gpu = DartRayBatch(grids, **params)
    refs = [oracle.Oracle(g, oracle.OracleParams(**{k: v for k, v in params.items() if k in ORACLE_KEYS}))
            for g in grids]
    st = gpu.direct()
    for r in refs:
        r.direct()
    for m, r in enumerate(refs):
        check_model(gpu, m, r, "direct")
    assert close_counts(st["crossings"], sum(r.stats()[1]["crossings"] for r in refs), rel=5e-3)
    for it in range(2):
        rem, st = gpu.scatter_iter()
        rems = [r.scatter_iter() for r in refs]
        for m, r in enumerate(refs):
            check_model(gpu, m, r, f"iter{it}")
            assert abs(gpu.model_info(m)["remaining"] - rems[m]) <= REL_TOTAL * max(rems[m], 1e-12)
        assert abs(rem - max(rems)) <= REL_TOTAL * max(rems)


def test_batch_stops_models_one_by_one():
    """With f_L = 5%, models reach it after different numbers of
    iterations; a model that has reached it stops emitting, exactly as a
    loop over the models alone would stop it."""
    grids = models()[:4]
    f_l = 0.05
    params = dict(a_rt=0.05, r_pre=0.6, f_l=f_l)
    gpu = DartRayBatch(grids, **params)
    gpu.direct()
    n_iter = []
    refs = []
    for g in grids:
        r = oracle.Oracle(g, oracle.OracleParams(**{k: v for k, v in params.items() if k in ORACLE_KEYS}))
        r.direct()
        n = 0
        while True:
            n += 1
            if r.scatter_iter() < f_l or n >= 12:
                break
        n_iter.append(n)
        refs.append(r)
    assert len(set(n_iter)) > 1, n_iter  # the models stop at different iterations
    for it in range(max(n_iter)):
        rem, _ = gpu.scatter_iter()
        active = [gpu.model_info(m)["active"] for m in range(len(grids))]
        assert active == [it + 1 < n for n in n_iter], (it, active, n_iter)
    assert rem < f_l
    for m, r in enumerate(refs):
        U = gpu.model_rfed(m)[0][:, 0]
        Ur = r.rfed()[0][:, 0]
        big = Ur > 1e-6 * Ur.max()
        assert np.abs(U[big] / Ur[big] - 1).max() <= REL_CELL, m
        j, jr = gpu.model_jsca_block(m, 0), r.jsca(0, "total")
        jb = jr > 1e-6 * jr.max()
        assert np.abs(j[jb] / jr[jb] - 1).max() <= REL_CELL, m


def test_batch_equals_single_model_grids():
    """The batch against the library's single-model grids, model by model."""
    grids = models()
    params = dict(a_rt=0.05, r_pre=0.6, f_l=1e-12)
    gpu = DartRayBatch(grids, **params)
    gpu.direct()
    gpu.scatter_iter()
    for m, g in enumerate(grids):
        one = DartRay(g, **params)
        one.direct()
        one.scatter_iter()
        U, U1 = gpu.model_rfed(m)[0], one.rfed()[0]
        big = U1 > 1e-6 * U1.max()
        assert np.abs(U[big] / U1[big] - 1).max() <= 1e-4, m
        one.close()


def test_batch_rejects_mixed_dust_models():
    a = synth.lognormal_cube(4, 3)
    b = synth.lognormal_cube(4, 4, albedo=0.5)
    with pytest.raises(DartRayError) as e:
        DartRayBatch([a, b])
    assert e.value.code == -1
