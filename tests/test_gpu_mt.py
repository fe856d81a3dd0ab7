"""The magnetisation-curve study (Sec. 3, Fig. 1) through the public API: a
small batch of uneven lattices over a temperature sweep, checked against the
harmonic spin-wave law at low temperature, the paramagnet above T_C, the cone
adaptation and the same lattice run alone."""
import math

import numpy as np
import pytest

import paper_2103_03517_gb300 as mc
from paper_2103_03517_gb300 import studies as st

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2103_03517_gb300 import build as libbuild
    libbuild.build()


def test_magnetization_curve_small_batch():
    dims = [(16, 16, 16), (32, 16, 16), (16, 16, 16), (16, 16, 16)]
    temps = [0.3, 0.8, 1.2, 2.5]
    n_eq, n_meas, seed = 300, 700, 5
    r = st.magnetization_curve(dims, temps, K_u=0.01, n_eq=n_eq, n_meas=n_meas, seed=seed)
    m = r["m"]
    assert m[0] > m[1] > m[2] > m[3]
    # harmonic spin waves on the simple cubic lattice: 1 - m = W T / 6, W = 1.516386
    assert abs(m[0] - (1.0 - 1.516386 / 6.0 * 0.3)) < 0.03
    assert m[3] < 0.15                          # paramagnet, |m| of order N^(-1/2)
    assert all(0.0 < e < 0.05 for e in r["m_err"])
    assert all(c > 0.0 for c in r["chi_par"] + r["chi_perp"] + r["chi_l"])
    assert r["k"][0] > r["k"][1] > r["k"][2]     # Eq. 4 scaling falls with T
    # the cone adapts to 50% acceptance below T_C (above it even the whole
    # sphere may accept more than half, and the cone stops at 180 degrees)
    assert all(0.4 < a < 0.6 for a in r["accept"][:3])
    assert r["e"][0] < r["e"][1] < r["e"][2] < r["e"][3]
    # lattice 1 alone: the same chain and observables, bit for bit
    h = mc.mc_create_ex(mc.make_desc(dims[1], K_u=0.01, T=temps[1], seed=seed + 1, ring_capacity=n_meas,
                                     sample_torque=0))
    try:
        mc.mc_sweep(h, n_eq)
        mc.mc_reset_stats(h)
        mc.mc_sweep(h, n_meas, measure=True)
        o = mc.mc_measure(h)
    finally:
        mc.mc_destroy(h)
    N = math.prod(dims[1])
    assert o.ml == m[1] and o.e == r["e"][1]
    assert N * (o.m2[2] - o.m_abs[2] ** 2) / temps[1] == r["chi_par"][1]
    assert r["updates"] == float(sum(math.prod(d) for d in dims)) * (n_eq + n_meas)
