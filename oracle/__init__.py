"""FP64 CPU oracle of the DART-Ray V2 ray-propagation sweep.

Test infrastructure only: tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of bench.py use it.  The CUDA
library never imports, links or calls anything here.
"""
from .oracle import (build, build_variant, OracleParams, Oracle, OracleError, pix2vec, pix2vec_all, vec2pix, hg, k_hp_real, k_hp,
                     locate, trace, tau_between, LEDGER_NAMES, COUNTER_NAMES, planck_lambda, dust_emission,
                     absorbed_power, dust_self_heating, external_frame, ExternalMapOracle)

__all__ = ["build", "build_variant", "OracleParams", "Oracle", "OracleError", "pix2vec", "pix2vec_all", "vec2pix", "hg", "k_hp_real", "k_hp",
           "locate", "trace", "tau_between", "LEDGER_NAMES", "COUNTER_NAMES", "planck_lambda", "dust_emission",
           "absorbed_power", "dust_self_heating", "external_frame", "ExternalMapOracle"]
