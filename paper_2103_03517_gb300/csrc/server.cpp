// server.cpp -- continuous-batching request loop.  Jobs (temperature / field
// points of the unconstrained or constrained algorithm, any lattice size,
// granular films) are admitted while the device-memory budget and the
// resident-slot limit allow; their state stays resident; every epoch advances
// all resident lattices with batched launches (one group per kind and phase);
// finished jobs are retired and their memory freed between epochs.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "runtime.h"

using namespace mcgb;

namespace {

struct Job {
    uint64_t id = 0;
    mc_job job;
    std::vector<uint8_t> bonds;
    std::vector<int32_t> grain;
    std::vector<double> axes;
    size_t bytes = 0;
    double t_submit = 0, t_admit = 0, t_finish = 0;
    int status = MC_PENDING;
    mc_observables obs;
    mc_handle h = nullptr;
    bool measuring = false;
    bool cancel = false;  // retire at the end of the current epoch
    int remaining = 0;    // sweeps left in the current phase
};

}  // namespace

struct mc_server {
    mc_server_desc d;
    cudaStream_t stream = nullptr;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Job*> queue;
    std::vector<Job*> resident;
    std::map<uint64_t, std::unique_ptr<Job>> jobs;
    size_t budget = 0, used = 0;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread worker;
    std::chrono::steady_clock::time_point t0;

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    void loop();
    void run_epoch(std::vector<Job*>& res);
};

// The film tables are needed only until create_lattice has taken its own
// device copy; a served film holds about 5 B of them per site.
static void release_tables(Job* j) {
    std::vector<uint8_t>().swap(j->bonds);
    std::vector<int32_t>().swap(j->grain);
    std::vector<double>().swap(j->axes);
}

static void finish(mc_server* s, Job* j, int status) {
    release_tables(j);
    if (j->h) {
        if (status == MC_OK) {
            int rc = mc_measure(j->h, &j->obs);
            if (rc) status = rc;
        }
        mc_destroy(j->h);
        j->h = nullptr;
        s->used -= j->bytes;
    }
    j->t_finish = s->now();
    j->status = status;
}

void mc_server::run_epoch(std::vector<Job*>& res) {
    NvtxRange range("mc server epoch");
    int n = d.max_epoch_sweeps;
    for (Job* j : res) n = std::min(n, j->remaining);
    if (n < 1) n = 1;
    // one group per (kind, phase); lattices of a group share precision
    for (int kind = 0; kind < 2; ++kind)
        for (int meas = 0; meas < 2; ++meas)
            for (int prec = 0; prec < 2; ++prec) {
                std::vector<mc_handle> hs;
                std::vector<double> th, ph;
                for (Job* j : res)
                    if (j->job.kind == kind && int(j->measuring) == meas && j->h->hp.precision == prec) {
                        hs.push_back(j->h);
                        th.push_back(j->job.theta_c_deg);
                        ph.push_back(j->job.phi_c_deg);
                    }
                if (hs.empty()) continue;
                mc_group_handle g = nullptr;
                int rc = mc_group_create(hs.data(), int(hs.size()), &g);
                if (rc == MC_OK) {
                    rc = kind == MC_JOB_CONSTRAINED ? mc_group_constrained_sweep(g, th.data(), ph.data(), n, meas)
                                                    : mc_group_sweep(g, n, meas);
                    int rc2 = mc_group_sync(g);
                    if (!rc) rc = rc2;
                    mc_group_destroy(g);
                }
                if (rc) {
                    for (Job* j : res)
                        if (std::find(hs.begin(), hs.end(), j->h) != hs.end()) {
                            std::lock_guard<std::mutex> lk(mu);
                            finish(this, j, rc);
                        }
                }
            }
    std::lock_guard<std::mutex> lk(mu);
    std::vector<Job*> keep;
    for (Job* j : res) {
        if (j->status != MC_PENDING) continue;
        if (j->cancel) {
            finish(this, j, MC_ERR_CANCELLED);
            continue;
        }
        j->remaining -= n;
        if (j->remaining <= 0) {
            if (!j->measuring && j->job.n_measure > 0) {
                j->measuring = true;
                j->remaining = j->job.n_measure;
                mc_reset_stats(j->h);
            } else {
                finish(this, j, MC_OK);
                continue;
            }
        }
        keep.push_back(j);
    }
    resident.swap(keep);
    cv.notify_all();
}

void mc_server::loop() {
    cudaSetDevice(d.device);
    for (;;) {
        std::vector<Job*> res;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv.wait(lk, [&] { return stop || !queue.empty() || !resident.empty(); });
            if (stop) return;
            // admission: FIFO while memory and slots allow
            NvtxRange range("mc server admission");
            while (!queue.empty() && int(resident.size()) < d.max_resident) {
                Job* j = queue.front();
                if (used + j->bytes > budget) break;
                mc_desc desc = j->job.lattice;
                desc.device = d.device;
                desc.stream = stream;
                desc.bond_mask = j->bonds.empty() ? nullptr : j->bonds.data();
                desc.grain_id = j->grain.empty() ? nullptr : j->grain.data();
                desc.grain_axis = j->axes.empty() ? nullptr : j->axes.data();
                queue.pop_front();
                int rc = create_lattice(&desc, &j->h);
                release_tables(j);
                if (rc) { j->h = nullptr; j->t_finish = now(); j->status = rc; continue; }
                used += j->bytes;
                j->t_admit = now();
                j->measuring = j->job.n_equilibrate <= 0;
                j->remaining = j->measuring ? j->job.n_measure : j->job.n_equilibrate;
                if (j->remaining <= 0) { finish(this, j, MC_OK); continue; }
                resident.push_back(j);
            }
            res = resident;
        }
        if (!res.empty()) run_epoch(res);
    }
}

extern "C" {

MC_API int mc_server_create(const mc_server_desc* d, mc_server** out) {
    if (!d || !out) return fail(MC_ERR_ARG, "null argument");
    mc_server* s = new mc_server();
    s->d = *d;
    if (s->d.max_resident <= 0) s->d.max_resident = 256;
    if (s->d.max_epoch_sweeps <= 0) s->d.max_epoch_sweeps = 50;
    if (cudaSetDevice(d->device) != cudaSuccess) { delete s; return fail(MC_ERR_CUDA, "cudaSetDevice failed"); }
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) { delete s; return fail(MC_ERR_CUDA, "cudaMemGetInfo failed"); }
    s->budget = d->memory_budget ? std::min(d->memory_budget, free_b) : size_t(0.9 * double(free_b));
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete s;
        return fail(MC_ERR_CUDA, "cudaStreamCreate failed");
    }
    s->t0 = std::chrono::steady_clock::now();
    s->worker = std::thread([s] { s->loop(); });
    *out = s;
    return MC_OK;
}

MC_API int mc_server_destroy(mc_server* s) {
    if (!s) return MC_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->d.device);
    for (auto& kv : s->jobs)
        if (kv.second->h) mc_destroy(kv.second->h);
    cudaStreamDestroy(s->stream);
    delete s;
    return MC_OK;
}

MC_API int mc_submit(mc_server* s, const mc_job* job, uint64_t* job_id) {
    if (!s || !job || !job_id) return fail(MC_ERR_ARG, "null argument");
    if (job->kind != MC_JOB_SWEEP && job->kind != MC_JOB_CONSTRAINED) return fail(MC_ERR_ARG, "job kind invalid");
    if (job->n_equilibrate < 0 || job->n_measure < 0) return fail(MC_ERR_ARG, "negative sweep count");
    int rc = validate_desc(&job->lattice);
    if (rc) return rc;
    if (job->kind == MC_JOB_CONSTRAINED) {
        if (!(job->theta_c_deg >= 0.0 && job->theta_c_deg <= 180.0)) return fail(MC_ERR_ARG, "theta_c outside [0, 180]");
        for (int a = 0; a < 3; ++a)
            if (job->lattice.boundary[a] == MC_PINNED) return fail(MC_ERR_ARG, "constrained jobs need no pinned boundary");
    }
    if (job->lattice.lattice != MC_SC) return fail(MC_ERR_ARG, "served jobs need a simple cubic lattice");
    auto j = std::make_unique<Job>();
    j->job = *job;
    const mc_desc& d = job->lattice;
    const size_t N = size_t(d.dims[0]) * d.dims[1] * d.dims[2];
    if (d.bond_mask) j->bonds.assign(d.bond_mask, d.bond_mask + N);
    if (d.grain_id) {
        j->grain.assign(d.grain_id, d.grain_id + N);
        j->axes.assign(d.grain_axis, d.grain_axis + 3 * size_t(d.n_grains));
    }
    j->job.lattice.bond_mask = nullptr;
    j->job.lattice.grain_id = nullptr;
    j->job.lattice.grain_axis = nullptr;
    j->bytes = lattice_bytes(&d) + (job->kind == MC_JOB_CONSTRAINED ? aos_bytes(&d) : 0);
    std::lock_guard<std::mutex> lk(s->mu);
    if (j->bytes > s->budget) return fail(MC_ERR_NOMEM, "job needs %zu bytes, budget is %zu", j->bytes, s->budget);
    j->id = s->next_id++;
    j->t_submit = s->now();
    *job_id = j->id;
    s->queue.push_back(j.get());
    s->jobs[j->id] = std::move(j);
    s->cv.notify_all();
    return MC_OK;
}

MC_API int mc_poll(mc_server* s, uint64_t job_id, mc_result* out) {
    if (!s) return fail(MC_ERR_ARG, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return fail(MC_ERR_ARG, "unknown job id %llu", (unsigned long long)job_id);
    Job* j = it->second.get();
    if (j->status == MC_PENDING) return MC_PENDING;
    if (out) {
        out->obs = j->obs;
        out->t_submit = j->t_submit;
        out->t_admit = j->t_admit;
        out->t_finish = j->t_finish;
        out->status = j->status;
    }
    return MC_OK;
}

MC_API int mc_cancel(mc_server* s, uint64_t job_id) {
    if (!s) return fail(MC_ERR_ARG, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return fail(MC_ERR_ARG, "unknown job id %llu", (unsigned long long)job_id);
    Job* j = it->second.get();
    if (j->status != MC_PENDING) return fail(MC_ERR_STATE, "job %llu has finished", (unsigned long long)job_id);
    auto q = std::find(s->queue.begin(), s->queue.end(), j);
    if (q != s->queue.end()) {  // not admitted: drop it now
        s->queue.erase(q);
        release_tables(j);
        j->t_finish = s->now();
        j->status = MC_ERR_CANCELLED;
    } else {
        j->cancel = true;  // resident: the worker retires it after the epoch
    }
    s->cv.notify_all();
    return MC_OK;
}

MC_API int mc_forget(mc_server* s, uint64_t job_id) {
    if (!s) return fail(MC_ERR_ARG, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return fail(MC_ERR_ARG, "unknown job id %llu", (unsigned long long)job_id);
    if (it->second->status == MC_PENDING)
        return fail(MC_ERR_STATE, "job %llu has not finished", (unsigned long long)job_id);
    s->jobs.erase(it);
    return MC_OK;
}

MC_API int mc_server_stats(mc_server* s, double* now, int* queued, int* resident, size_t* bytes) {
    if (!s) return fail(MC_ERR_ARG, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    if (now) *now = s->now();
    if (queued) *queued = int(s->queue.size());
    if (resident) *resident = int(s->resident.size());
    if (bytes) *bytes = s->used;
    return MC_OK;
}

}  // extern "C"
