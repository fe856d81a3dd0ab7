"""Eq. 4 (Sec. 3) on the GPU: the anisotropy scaling from the standard
algorithm's easy-axis energy equals the oracle's in FP64, agrees with FP64
in FP32, and agrees with the constrained algorithm's torque and hard - easy
energy difference at low temperature, as the paper reports."""
import math

import numpy as np
import pytest

import oracle
import paper_2103_03517_gb300 as mc
from _stats import blocking_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2103_03517_gb300 import build as libbuild
    libbuild.build()


def test_eq4_fp64_matches_oracle():
    dims, axis = (16, 8, 6), (0.3, 0.2, 0.9)
    kw = dict(T=0.7, seed=5)
    o = oracle.Lattice(dims, J=1.0, Ku=0.05, axis=axis, Kc=0.02, ring_cap=1, **kw)
    h = mc.mc_create_ex(mc.make_desc(dims, K_u=0.05, axis=axis, K_c=0.02, precision=mc.MC_FP64,
                                     ring_capacity=8, **kw))
    try:
        o.sweep(30)
        o.sweep(40, measure=True)
        mc.mc_sweep(h, 30)
        mc.mc_sweep(h, 40, measure=True)
        got, expect = mc.mc_anisotropy_scaling(h), o.anisotropy_scaling()
        np.testing.assert_allclose(got, expect, rtol=0, atol=1e-9)
        assert 0.0 < got[0] < 1.0 and 0.0 < got[1] < 1.0
    finally:
        mc.mc_destroy(h)


def test_eq4_without_samples_or_constant():
    h = mc.mc_create_ex(mc.make_desc((8, 8, 8), K_u=0.05, T=0.5))
    try:
        with pytest.raises(mc.MCError) as e:
            mc.mc_anisotropy_scaling(h)
        assert e.value.code == mc.MC_ERR_STATE
        mc.mc_sweep(h, 5, measure=True)
        k_u, k_c = mc.mc_anisotropy_scaling(h)
        assert 0.0 < k_u <= 1.0 and math.isnan(k_c)
    finally:
        mc.mc_destroy(h)


def _eq4_series(h, K, n):
    s = mc.mc_samples(h, n)
    return 1 - 3 * (s["e_parts"][:, 1] + K) / (2 * K)


def test_eq4_fp32_agrees_with_fp64():
    """k_u of Eq. 4 (16^3, T = 0.9) from eight independent runs per
    precision: the FP32 and FP64 means agree within the 3-sigma-equivalent
    bound (t3) of the spread between runs."""
    from _stats import diff_within_t3
    K, n, runs = 0.05, 3000, 8
    k = {}
    for p in (mc.MC_FP32, mc.MC_FP64):
        hs = [mc.mc_create_ex(mc.make_desc((16, 16, 16), K_u=K, T=0.9, seed=1 + 2 * r + p, precision=p,
                                           ring_capacity=16)) for r in range(runs)]
        g = mc.mc_group_create(hs)
        try:
            mc.mc_group_sweep(g, 500)
            mc.mc_group_sweep(g, n, measure=True)
            mc.mc_group_sync(g)
            k[p] = np.array([mc.mc_anisotropy_scaling(h)[0] for h in hs])
        finally:
            mc.mc_group_destroy(g)
            for h in hs:
                mc.mc_destroy(h)
    d, se, bound = diff_within_t3(k[mc.MC_FP32], k[mc.MC_FP64])
    assert abs(d) <= bound, (k, d, se)


@pytest.mark.parametrize("T", [0.2, 0.4])
def test_eq4_agrees_with_constrained_routes(T):
    """Uniaxial K_u = 0.05 on 16^3 (T_C = 1.44): k_u from Eq. 4 (standard
    sweeps) against K(T)/K_u from the constrained torque at theta_c = 45 deg
    (tau_theta / N = -K(T) sin 2 theta) and from the hard - easy difference of
    the mean anisotropy energy (constrained at 90 and 0 deg)."""
    K, n_eq, n = 0.05, 1000, 4000
    dims = (16, 16, 16)
    std = mc.mc_create_ex(mc.make_desc(dims, K_u=K, T=T, seed=11, ring_capacity=n))
    cons = {}
    try:
        mc.mc_sweep(std, n_eq)
        mc.mc_sweep(std, n, measure=True)
        k_eq4 = mc.mc_anisotropy_scaling(std)[0]
        err = blocking_error(_eq4_series(std, K, n))
        for th in (0.0, 45.0, 90.0):
            t = math.radians(th)
            h = mc.mc_create_ex(mc.make_desc(dims, K_u=K, T=T, seed=12 + int(th), ring_capacity=n,
                                             init_dir=(math.sin(t), 0.0, math.cos(t))))
            cons[th] = h
            mc.mc_constrained_sweep(h, th, 0.0, n_eq)
            mc.mc_constrained_sweep(h, th, 0.0, n, measure=True)
        k_torque = -mc.mc_measure(cons[45.0]).torque[1] / K
        k_diff = (mc.mc_measure(cons[90.0]).e_parts[1] - mc.mc_measure(cons[0.0]).e_parts[1]) / K
        assert abs(k_eq4 - k_torque) < max(5 * err, 0.02), (T, k_eq4, k_torque, k_diff)
        assert abs(k_eq4 - k_diff) < max(5 * err, 0.02), (T, k_eq4, k_torque, k_diff)
    finally:
        mc.mc_destroy(std)
        for h in cons.values():
            mc.mc_destroy(h)
