"""Dust emission and self-heating (Sect. 3.3) on the GPU -- the emission
kernel, the emissivity update and the incremental step 2 of the library --
against the oracle's loop on the same models (tests/test_oracle_dust.py
pins the oracle's)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1709_03802_gb300 import DartRay, dust_self_heating  # noqa: E402
from test_gpu_parity import REL_CELL  # noqa: E402
from test_oracle_dust import DLAM_IR, DLAM_ST, LAM_IR, SCALE, models  # noqa: E402


def run_both(ir_kappa_scale):
    st, dust = models(ir_kappa_scale)
    p = dict(a_rt=0.05, r_pre=0.5)
    g_st = DartRay(st, **p)
    g_st.direct()
    for _ in range(12):
        if g_st.scatter_iter()[0] < 0.01:
            break
    g_d = DartRay(dust, **p)
    T, j, hist = dust_self_heating(g_st, g_d, LAM_IR, DLAM_IR, DLAM_ST, SCALE)
    o_st = oracle.Oracle(st, oracle.OracleParams(**p))
    o_st.direct()
    for _ in range(12):
        if o_st.scatter_iter() < 0.01:
            break
    o_d = oracle.Oracle(dust, oracle.OracleParams(**p))
    To, jo, ho = oracle.dust_self_heating(o_st, o_d, LAM_IR, DLAM_IR, DLAM_ST, SCALE)
    return (g_d, T, j, hist), (o_d, To, jo, ho)


@pytest.mark.parametrize("ir_kappa_scale", [1.0, 1e-6], ids=["thick", "thin"])
def test_self_heating_matches_oracle(ir_kappa_scale):
    (g_d, T, j, hist), (o_d, To, jo, ho) = run_both(ir_kappa_scale)
    assert len(hist) == len(ho), (hist, ho)
    hot = To > 0
    assert np.array_equal(T > 0, hot)
    assert np.abs(T[hot] / To[hot] - 1).max() <= REL_CELL
    big = jo > 1e-6 * jo.max(axis=0, keepdims=True)
    assert np.abs(j[big] / jo[big] - 1).max() <= REL_CELL
    U, Uo = g_d.rfed()[0], o_d.rfed()[0]
    for l in range(U.shape[1]):
        b = Uo[:, l] > 1e-6 * Uo[:, l].max()
        assert np.abs(U[b, l] / Uo[b, l] - 1).max() <= REL_CELL, l
