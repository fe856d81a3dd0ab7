"""Serving (continuous batching): a job's result is the same alone, inside a
mixed stream of jobs, and through direct mc_sweep calls; admission refuses
jobs that can never fit the memory budget; jobs overlap on the device."""
import time

import numpy as np
import pytest

import paper_2103_03517_gb300 as mc
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2103_03517_gb300 import build as libbuild
    libbuild.build()


def _wait(server, ids, timeout=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(ids):
        for i in ids:
            if i in out:
                continue
            rc, res = mc.mc_poll(server, i)
            if rc == mc.MC_OK:
                out[i] = res
        assert time.time() - t0 < timeout, "jobs did not finish"
        time.sleep(0.005)
    return out


def _probe_job():
    d = mc.make_desc((16, 16, 16), K_u=0.01, T=0.8, seed=77, ring_capacity=64)
    return mc.make_job(d, mc.MC_JOB_SWEEP, n_equilibrate=37, n_measure=53)


def _mixed_jobs():
    film = workloads.voronoi_film(32, 32, 4, 6.0, seed=1)
    jobs = []
    jobs.append(mc.make_job(mc.make_desc((32, 32, 32), K_u=0.01, T=1.2, seed=1), mc.MC_JOB_SWEEP,
                            n_equilibrate=20, n_measure=120))
    jobs.append(mc.make_job(mc.make_desc((8, 8, 8), K_u=0.05, K_c=0.02, T=0.5, seed=2,
                                         init_dir=(np.sin(np.radians(30)), 0, np.cos(np.radians(30)))),
                            mc.MC_JOB_CONSTRAINED, theta_c_deg=30.0, phi_c_deg=0.0, n_equilibrate=15, n_measure=25))
    gid, mask, axes = film
    jobs.append(mc.make_job(mc.make_desc((32, 32, 4), K_u=0.02, T=0.6, seed=3, boundary=(0, 0, 1),
                                         bond_mask=mask, grain_id=gid, grain_axis=axes),
                            mc.MC_JOB_SWEEP, n_equilibrate=10, n_measure=70))
    jobs.append(mc.make_job(mc.make_desc((64, 16, 8), K_u=0.01, T=0.3, seed=4, precision=mc.MC_FP64),
                            mc.MC_JOB_SWEEP, n_equilibrate=5, n_measure=33))
    jobs.append(mc.make_job(mc.make_desc((128, 8, 8), K_u=0.01, T=0.9, seed=5), mc.MC_JOB_SWEEP,
                            n_equilibrate=60, n_measure=11))
    return jobs


def test_job_result_is_the_same_alone_in_a_mix_and_direct():
    # alone
    s = mc.mc_server_create(max_epoch_sweeps=16)
    try:
        jid = mc.mc_submit(s, _probe_job())
        alone = _wait(s, [jid])[jid]
    finally:
        mc.mc_server_destroy(s)
    assert alone.status == mc.MC_OK and alone.obs.n_samples == 53
    # in a mix: probe submitted between other jobs of every kind
    s = mc.mc_server_create(max_epoch_sweeps=16)
    try:
        others = _mixed_jobs()
        ids = [mc.mc_submit(s, j) for j in others[:3]]
        pid = mc.mc_submit(s, _probe_job())
        ids += [mc.mc_submit(s, j) for j in others[3:]]
        res = _wait(s, ids + [pid])
    finally:
        mc.mc_server_destroy(s)
    assert all(r.status == mc.MC_OK for r in res.values())
    mixed = res[pid]
    assert mixed.obs.asdict() == alone.obs.asdict()
    # direct calls through the lattice API
    h = mc.mc_create_ex(mc.make_desc((16, 16, 16), K_u=0.01, T=0.8, seed=77, ring_capacity=64))
    try:
        mc.mc_sweep(h, 37)
        mc.mc_reset_stats(h)
        mc.mc_sweep(h, 53, measure=True)
        direct = mc.mc_measure(h)
    finally:
        mc.mc_destroy(h)
    assert direct.asdict() == alone.obs.asdict()
    # the constrained job in the mix sampled torques and kept M along e_C
    cres = res[ids[1]].obs
    assert cres.n_samples == 25 and abs(cres.m[1]) < 1e-6


def test_admission_refuses_a_job_that_can_never_fit():
    s = mc.mc_server_create(memory_budget=1 << 20)
    try:
        with pytest.raises(mc.MCError) as e:
            mc.mc_submit(s, mc.make_job(mc.make_desc((64, 64, 64)), n_measure=1))
        assert e.value.code == mc.MC_ERR_NOMEM
        jid = mc.mc_submit(s, mc.make_job(mc.make_desc((8, 8, 8)), n_measure=3))
        assert _wait(s, [jid])[jid].status == mc.MC_OK
    finally:
        mc.mc_server_destroy(s)


def test_jobs_overlap_and_memory_is_returned():
    s = mc.mc_server_create(max_epoch_sweeps=8)
    try:
        ids = [mc.mc_submit(s, mc.make_job(mc.make_desc((32, 32, 32), T=0.5 + 0.1 * k, seed=k), n_equilibrate=50,
                                           n_measure=150)) for k in range(6)]
        seen = 0
        t0 = time.time()
        while time.time() - t0 < 60:
            _, queued, resident, used = mc.mc_server_stats(s)
            seen = max(seen, resident)
            if queued == 0 and resident == 0:
                break
            time.sleep(0.002)
        res = _wait(s, ids)
        assert seen >= 2
        assert all(r.t_submit <= r.t_admit <= r.t_finish for r in res.values())
        assert mc.mc_server_stats(s)[3] == 0
        with pytest.raises(mc.MCError):
            mc.mc_poll(s, 999999)
    finally:
        mc.mc_server_destroy(s)


def test_cancel_queued_resident_and_finished_jobs():
    """Host-side fault injection: a queued job is dropped at once, a
    resident one is retired after its epoch with its memory returned, and
    the server carries on with later jobs."""
    s = mc.mc_server_create(max_resident=1, max_epoch_sweeps=8)
    try:
        long_job = mc.make_job(mc.make_desc((64, 64, 64), T=0.7, seed=1), n_equilibrate=100000, n_measure=10)
        a = mc.mc_submit(s, long_job)
        b = mc.mc_submit(s, mc.make_job(mc.make_desc((16, 16, 16), seed=2), n_measure=5))
        t0 = time.time()
        while mc.mc_server_stats(s)[2] < 1:  # a is resident, b queued behind it
            assert time.time() - t0 < 30
            time.sleep(0.002)
        mc.mc_cancel(s, b)
        rc, res = mc.mc_poll(s, b)
        assert rc == mc.MC_OK and res.status == mc.MC_ERR_CANCELLED
        mc.mc_cancel(s, a)
        res = _wait(s, [a])[a]
        assert res.status == mc.MC_ERR_CANCELLED and res.t_finish >= res.t_admit > 0
        with pytest.raises(mc.MCError) as e:
            mc.mc_cancel(s, a)
        assert e.value.code == mc.MC_ERR_STATE
        with pytest.raises(mc.MCError) as e:
            mc.mc_cancel(s, 987654)
        assert e.value.code == mc.MC_ERR_ARG
        c = mc.mc_submit(s, _probe_job())
        assert _wait(s, [c])[c].status == mc.MC_OK
        t0 = time.time()
        while mc.mc_server_stats(s)[3] != 0:
            assert time.time() - t0 < 30
            time.sleep(0.002)
    finally:
        mc.mc_server_destroy(s)


def test_forget_drops_finished_records_only():
    """A finished job's record goes with mc_forget (its id is then unknown);
    a job still queued or running cannot be forgotten."""
    s = mc.mc_server_create(max_resident=1, max_epoch_sweeps=8)
    try:
        long_job = mc.make_job(mc.make_desc((64, 64, 64), T=0.7, seed=1), n_equilibrate=100000, n_measure=10)
        a = mc.mc_submit(s, long_job)
        with pytest.raises(mc.MCError) as e:
            mc.mc_forget(s, a)
        assert e.value.code == mc.MC_ERR_STATE
        mc.mc_cancel(s, a)
        _wait(s, [a])
        mc.mc_forget(s, a)
        with pytest.raises(mc.MCError) as e:
            mc.mc_poll(s, a)
        assert e.value.code == mc.MC_ERR_ARG
        c = mc.mc_submit(s, _probe_job())
        assert _wait(s, [c])[c].status == mc.MC_OK
        mc.mc_forget(s, c)
        with pytest.raises(mc.MCError) as e:
            mc.mc_forget(s, c)
        assert e.value.code == mc.MC_ERR_ARG
    finally:
        mc.mc_server_destroy(s)
