"""Per-grain magnetisation of films (Sec. 4, the terms of Eq. 8) through the
C ABI against the oracle's chain, FP64, and its checkpoint round trip."""
import numpy as np
import pytest

import oracle
import paper_2103_03517_gb300 as mc
import workloads
from test_gpu_parity import make_pair

pytestmark = pytest.mark.gpu


def test_fp64_grain_samples_match_oracle():
    """Three grain samples of an FP64 film, taken after 10, 15 and 25 sweeps
    on both sides (bit-identical chains): <m_g> agrees with the oracle's
    per-grain lengths of the same states to the fixed-point rounding."""
    dims = (32, 32, 4)
    gid, mask, axes = workloads.voronoi_film(*dims, 8.0, seed=3)
    ng = int(gid.max()) + 1
    h, o = make_pair(dims, J=1.0, Ku=0.05, T=0.6, seed=11, bc=(0, 0, 1), film=(gid, mask, axes), ring=64)
    try:
        ref = np.zeros(ng)
        for n in (10, 5, 10):
            mc.mc_sweep(h, n)
            o.sweep(n)
            mc.mc_grain_sample(h)
            ref += oracle.grain_magnetization(o.spins(), gid, ng)
        got, count = mc.mc_grain_magnetization(h, ng)
        assert count == 3
        np.testing.assert_allclose(got, ref / 3, rtol=0, atol=1e-8)
        assert got.min() > 0.2  # grains are ordered at T = 0.6
        mc.mc_reset_stats(h)
        assert mc.mc_grain_magnetization(h, ng)[1] == 0
    finally:
        mc.mc_destroy(h)


def test_grain_samples_survive_checkpoint(tmp_path):
    dims = (32, 32, 4)
    gid, mask, axes = workloads.voronoi_film(*dims, 8.0, seed=4)
    ng = int(gid.max()) + 1
    d = mc.make_desc(dims, K_u=0.05, T=0.7, seed=2, boundary=(0, 0, 1), bond_mask=mask, grain_id=gid,
                     grain_axis=axes, ring_capacity=16)
    h = mc.mc_create_ex(d)
    try:
        for _ in range(4):
            mc.mc_sweep(h, 5)
            mc.mc_grain_sample(h)
        path = str(tmp_path / "film.ck")
        mc.mc_save(h, path)
        c = mc.mc_load(path)
        try:
            a, na = mc.mc_grain_magnetization(h, ng)
            b, nb = mc.mc_grain_magnetization(c, ng)
            assert na == nb == 4 and np.array_equal(a, b)
        finally:
            mc.mc_destroy(c)
        with pytest.raises(Exception):
            mc.mc_grain_magnetization(h, ng - 1)
    finally:
        mc.mc_destroy(h)


def test_film_curie_study_small():
    """Sec. 4 in miniature: a 64 x 64 x 4 film with grains of mean diameter
    12 and the continuous film of the same thickness.  The grains start
    ordered and disorder with T; Eq. 8 fits their m(T) closely; the
    continuous film's T_C (Eq. 3) lies below the bulk 1.443.  (Grains this
    small keep a finite-size tail of m above T_C, which the series fits with
    high-T_C terms, so their average is not compared with the film's.)"""
    from paper_2103_03517_gb300.studies import film_curie_study
    dims = (64, 64, 4)
    temps = [round(0.1 * i, 2) for i in range(1, 16)]
    cont = film_curie_study(dims, None, None, None, temps, n_eq=400, n_meas=800)
    gid, mask, axes = workloads.voronoi_film(*dims, 12.0, seed=1)
    gr = film_curie_study(dims, gid, mask, axes, temps, n_eq=400, n_meas=800)
    tc_c, tc_g = cont["fit"]["T_C"], gr["fit"]["T_C_mean"]
    assert 0.8 < tc_c < 1.443, cont
    assert 0.8 < tc_g < 1.8, (tc_g, gr["m"])
    m = gr["m"]
    assert m[0] > 0.9 and m[-1] < 0.3 and all(a > b - 0.02 for a, b in zip(m, m[1:])), m
    assert gr["fit"]["rms"] < 0.02, gr["fit"]
