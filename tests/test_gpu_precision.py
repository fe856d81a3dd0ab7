"""FP32 against the oracle's FP64 chain near the Curie point (T_C = 1.443):
the ensemble averages the paper's FP32 GPU runs report (Sec. 3, Fig. 1)
must match the serial FP64 oracle's within |d<|m|>| <= 2e-3 and 3 sigma of
the sampling error.

The oracle side is stored in tests/golden/batched_mt_oracle.json, written by
tests/golden/make_batched_mt_oracle.py, which calls only the oracle: for each
case many independent chains (all +z, n_eq + n_meas sweeps, the cone adapting
in every sweep) and the mean and spread of their per-chain averages.  The GPU
side runs chains of the same protocol with seeds of a disjoint range, enough
of them that its own standard error is about 2e-4 on <|m|>.  sigma is the
standard error of the difference from the spreads between chains (not a
single run's blocking error, which understates it near T_C).

Cases: the lattices of the batched temperature sweep nearest T_C (128^3 at
T = 1.40, 16^3 at 1.45, 32^3 at 1.50, 64^3 at 1.55) and 16^3 at 1.40 and
1.50, so that 16^3 is covered on both sides of T_C."""
import json
import math
import os

import numpy as np
import pytest

import workloads
from paper_2103_03517_gb300 import studies

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "batched_mt_oracle.json")
NEAR_TC = ["mT_27", "mT_28", "mT_29", "mT_30", "extra_16c_T1.40", "extra_16c_T1.50"]
SIGMA_GPU = 2e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2103_03517_gb300 import build as libbuild
    libbuild.build()


@pytest.fixture(scope="module")
def gpu_vs_oracle():
    with open(GOLDEN) as f:
        golden = json.load(f)["cases"]
    cases = workloads.precision_cases()
    chosen = {name: cases[name] for name in NEAR_TC}
    n_chains = {name: min(20000, max(8, math.ceil((golden[name]["obs"]["ml"]["sd"] / SIGMA_GPU) ** 2)))
                for name in chosen}
    res = studies.chain_ensembles(
        chosen, n_chains, lambda name, k: workloads.precision_seed(workloads.PRECISION_GPU_SEED0, cases[name], k),
        lambda name: workloads.PRECISION_SWEEPS[cases[name].dims[0]])
    return golden, res


@pytest.mark.parametrize("name", NEAR_TC)
def test_fp32_near_tc_matches_oracle(gpu_vs_oracle, name):
    golden, res = gpu_vs_oracle
    g, r = golden[name], res[name]
    assert g["sweeps"] == list(workloads.PRECISION_SWEEPS[g["L"]])
    for key in ("ml", "ml2", "mabs_z", "e"):
        a = r[key]
        o = g["obs"][key]
        diff = float(a.mean()) - o["mean"]
        sigma = math.sqrt(a.var(ddof=1) / a.size + o["sd"] ** 2 / g["chains"])
        assert abs(diff) <= 3 * sigma, (name, key, diff, sigma)
        if key == "ml":  # the benchmark spec's bound on <|m|>
            assert abs(diff) <= 2e-3, (name, diff, sigma)
            assert sigma < 6.7e-4, (name, sigma)  # 2e-3 is then at least 3 sigma
