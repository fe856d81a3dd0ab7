"""K_u(T) and K_c(T) by Asselin's torque method (Sec. 3, Fig. 1(a)) through
studies.anisotropy_torque_study, on a reduced grid of constraint directions.
FP64 on the GPU runs the oracle's constrained chain bit for bit, so its
torques, and the constants fitted from them, equal the oracle's to rounding
of the sums; FP32 agrees with FP64 within the statistical error."""
import math

import numpy as np
import pytest

import oracle
from paper_2103_03517_gb300 import analysis as an
from paper_2103_03517_gb300 import studies

pytestmark = pytest.mark.gpu

GRID = dict(thetas=(20.0, 45.0, 70.0), phis=(0.0, 45.0))


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2103_03517_gb300 import build as libbuild
    libbuild.build()


def test_torque_fit_fp64_equals_the_oracle():
    dims, Ku, Kc, T, n_eq, n_meas = (12, 12, 12), 0.05, 0.02, 0.2, 30, 60
    gpu = studies.anisotropy_torque_study(dims, K_u=Ku, K_c=Kc, temps=(T,), n_eq=n_eq, n_meas=n_meas, seed=3,
                                          precision=1, **GRID)
    taus = []
    for i, r in enumerate(gpu["runs"]):
        th, ph = r["theta"], r["phi"]
        # the study starts each lattice along init_dir = e_C, normalised as
        # mc_create_ex does (sqrt of x x + y y + z z, then a division)
        v = studies._unit(th, ph)
        n = math.sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2])
        o = oracle.Lattice(dims, J=1.0, Ku=Ku, Kc=Kc, T=T, seed=3 + i, ring_cap=1)
        o.set_spins(np.tile(np.array([v[0] / n, v[1] / n, v[2] / n]), (int(np.prod(dims)), 1)))
        o.constrained_sweep(th, ph, n_eq)
        o.reset_stats()
        o.constrained_sweep(th, ph, n_meas, measure=True)
        s = o.stats()
        taus.append(float(an.torque_theta(np.array([s["tqx"], s["tqy"], s["tqz"]]) / s["n"], ph)))
        assert abs(r["tau"] - taus[-1]) < 1e-9, (th, ph, r["tau"], taus[-1])
    f_or = an.torque_fit([r["theta"] for r in gpu["runs"]], [r["phi"] for r in gpu["runs"]], taus)
    f_gpu = an.torque_fit([r["theta"] for r in gpu["runs"]], [r["phi"] for r in gpu["runs"]],
                          [r["tau"] for r in gpu["runs"]])
    assert abs(f_gpu["K_u"] - f_or["K_u"]) < 1e-9 and abs(f_gpu["K_c"] - f_or["K_c"]) < 1e-9


def test_torque_fit_fp32_agrees_with_fp64():
    """16^3, T = 0.6: the constants fitted from FP32 and FP64 chains differ
    by less than 3 standard errors of the difference; both are below their
    T = 0 values (thermal softening) and positive."""
    kw = dict(K_u=0.05, K_c=0.02, temps=(0.6,), n_eq=300, n_meas=1500, **GRID)
    f32 = studies.anisotropy_torque_study((16, 16, 16), precision=0, seed=100, **kw)["fits"][0.6]
    f64 = studies.anisotropy_torque_study((16, 16, 16), precision=1, seed=200, **kw)["fits"][0.6]
    for k in ("K_u", "K_c"):
        err = math.hypot(f32[k + "_err"], f64[k + "_err"])
        assert abs(f32[k] - f64[k]) < 3 * err, (k, f32, f64)
    assert 0.0 < f64["K_u"] < 0.05 and 0.0 < f64["K_c"] < 0.02
