"""The JSON-lines request loop in front of the server (host logic only):
job parsing into mc_job, rejection of malformed jobs, and the loop's
submit / poll / write order against a fake server."""
import json

import pytest

import paper_2103_03517_gb300 as mc
from paper_2103_03517_gb300 import build as libbuild
from paper_2103_03517_gb300 import serve


@pytest.fixture(scope="module", autouse=True)
def _built():
    libbuild.build()


def test_job_from_dict_fills_the_job():
    j = serve.job_from_dict({"dims": [32, 16, 8], "T": 0.7, "K_u": 0.05, "K_c": 0.02, "seed": 9,
                             "precision": "fp64", "boundary": ["pinned", "periodic", "open"],
                             "lattice": "sc", "theta0_deg": 45, "kind": "constrained", "theta_c_deg": 30,
                             "phi_c_deg": 45, "n_equilibrate": 100, "n_measure": 200, "id": "a"})
    d = j.lattice
    assert list(d.dims) == [32, 16, 8] and d.T == 0.7 and d.K_u == 0.05 and d.K_c == 0.02 and d.seed == 9
    assert d.precision == mc.MC_FP64 and list(d.boundary) == [mc.MC_PINNED, mc.MC_PERIODIC, mc.MC_OPEN]
    assert d.theta0_deg == 45 and d.lattice == mc.MC_SC
    assert j.kind == mc.MC_JOB_CONSTRAINED and j.theta_c_deg == 30 and j.phi_c_deg == 45
    assert j.n_equilibrate == 100 and j.n_measure == 200
    k = serve.job_from_dict({"dims": [16, 16, 16]})
    assert k.kind == mc.MC_JOB_SWEEP and k.lattice.precision == mc.MC_FP32 and k.lattice.J == 1.0


@pytest.mark.parametrize("bad", [
    {"T": 0.5},                                       # no dims
    {"dims": [16, 16]},                               # two sizes
    {"dims": [16, 16, 16], "temperature": 0.5},       # unknown key
    {"dims": [16, 16, 16], "boundary": ["periodic", "open"]},
    {"dims": [16, 16, 16], "boundary": ["periodic", "open", "wrap"]},
    {"dims": [16, 16, 16], "precision": "fp16"},
    {"dims": [16, 16, 16], "kind": "anneal"},
    {"dims": [16, 16, 16], "H": [0.0, 1.0]},
    {"dims": [16, 16, 16], "n_measure": -1},
])
def test_job_from_dict_rejects_malformed_jobs(bad):
    with pytest.raises(ValueError):
        serve.job_from_dict(bad)


class FakeServer:
    """Ids in submission order; job i finishes after i + 1 polls."""

    def __init__(self):
        self.jobs, self.polls = [], {}

    def submit(self, job):
        if job.lattice.T <= 0:
            raise mc.MCError(mc.MC_ERR_ARG, "T must be > 0")
        self.jobs.append(job)
        jid = 100 + len(self.jobs) - 1
        self.polls[jid] = 0
        return jid

    def poll(self, jid):
        self.polls[jid] += 1
        i = jid - 100
        if self.polls[jid] <= i:
            return mc.MC_PENDING, None
        r = mc.mc_result()
        r.status = 0
        r.t_submit, r.t_admit, r.t_finish = 1.0 + i, 1.5 + i, 2.0 + 2 * i
        r.obs.ml = 0.5 + 0.1 * i
        return mc.MC_OK, r


def test_serve_loop_submits_as_lines_arrive_and_writes_every_result():
    lines = [json.dumps({"dims": [16, 16, 16], "T": 0.5, "id": "first"}), "",
             "{not json", json.dumps({"dims": [16, 16, 16], "T": -1.0}),
             json.dumps({"dims": [8, 8, 8], "T": 1.0, "n_measure": 10, "id": 7}),
             json.dumps({"dims": [8, 8, 8], "T": 1.2}), json.dumps([1, 2, 3])]
    srv, out = FakeServer(), []
    n = serve.serve(iter(lines), out.append, srv.submit, srv.poll, poll_interval=0.0)
    assert n == len(out) == 6
    errors = [r for r in out if "error" in r]
    assert [r["line"] for r in errors] == [3, 4, 7]
    results = {r["job"]: r for r in out if "job" in r}
    assert sorted(results) == [100, 101, 102]
    assert results[100]["id"] == "first" and results[101]["id"] == 7 and "id" not in results[102]
    assert results[101]["obs"]["ml"] == pytest.approx(0.6)
    assert results[102]["latency_s"] == pytest.approx(3.0)
    assert [j.lattice.dims[0] for j in srv.jobs] == [16, 8, 8]
    assert all(json.dumps(r) for r in out)   # every record is JSON-ready


def test_serve_loop_forgets_each_job_once_its_result_is_written():
    lines = [json.dumps({"dims": [16, 16, 16], "T": 0.5}), json.dumps({"dims": [8, 8, 8], "T": 1.0}),
             json.dumps({"dims": [8, 8, 8], "T": 1.2})]
    srv, out, forgotten = FakeServer(), [], []

    def forget(jid):
        assert any(r.get("job") == jid for r in out), "forgotten before its result was written"
        forgotten.append(jid)

    serve.serve(iter(lines), out.append, srv.submit, srv.poll, poll_interval=0.0, forget=forget)
    assert sorted(forgotten) == [100, 101, 102]
