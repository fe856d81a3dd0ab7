// tune.cpp -- launch-shape autotuner of the batched sweeps: for each knob of
// LaunchShape in turn, every candidate is timed with CUDA events over a few
// sweeps of the real lattices, from the same saved state each time, and the
// fastest is kept.  The lattices' spins and device state are restored after
// every trial, so the Markov chains are left exactly as they were (the draws
// are keyed by site and sweep, and every result is independent of the launch
// shape).
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "runtime.h"

namespace mcgb {

namespace {

constexpr double kTuneMargin = 0.01;  // relative gain a candidate needs over the default

// Device copy of the spins and LatState of every lattice, for restoring.
struct Snapshot {
    void* mem = nullptr;
    std::vector<size_t> off;
    ~Snapshot() {
        if (mem) cudaFree(mem);
    }
};

size_t spin_bytes(const mc_lattice* h) {
    return size_t(h->hp.nsub) * 6 * size_t(h->hp.stride) * (h->hp.precision == MC_FP64 ? 8 : 4);
}

size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

int copy_state(const std::vector<mc_lattice*>& lats, Snapshot& snap, bool save, cudaStream_t s) {
    char* base = static_cast<char*>(snap.mem);
    for (size_t i = 0; i < lats.size(); ++i) {
        mc_lattice* h = lats[i];
        char* spins = base + snap.off[i];
        char* st = spins + al256(spin_bytes(h));
        cudaError_t e;
        if (save) {
            e = cudaMemcpyAsync(spins, h->hp.spins, spin_bytes(h), cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(st, &h->d_lat->st, sizeof(LatState), cudaMemcpyDeviceToDevice, s);
        } else {
            e = cudaMemcpyAsync(h->hp.spins, spins, spin_bytes(h), cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(&h->d_lat->st, st, sizeof(LatState), cudaMemcpyDeviceToDevice, s);
        }
        if (e != cudaSuccess) return cuda_fail(e, "autotune state copy");
    }
    return MC_OK;
}

}  // namespace

int autotune(int precision, LaunchSet& ls, const std::vector<mc_lattice*>& lats, const void* cone, int sweeps,
             int what, cudaStream_t s, mc_tune_report* out) {
    if (sweeps < 1 || !(what & (MC_TUNE_SWEEP | MC_TUNE_CONSTRAINED))) return fail(MC_ERR_ARG, "invalid argument");
    const bool tune_free = (what & MC_TUNE_SWEEP) && (ls.nt_row || ls.nt_rowx);
    const bool tune_cons = (what & MC_TUNE_CONSTRAINED) && (ls.nt_pairs || ls.nt_pairs_lead);
    for (mc_lattice* h : lats) {
        if (h->hp.nsub > 1) return fail(MC_ERR_ARG, "crystal lattices have no tunable launch shape");
        if (tune_cons) {
            for (int a = 0; a < 3; ++a)
                if (h->hp.bc[a] == MC_PINNED) return fail(MC_ERR_ARG, "constrained sweeps need no pinned boundary");
            if (!h->d_aos) {  // the packed copy and field of constrained sweeps
                int rc = ensure_aos(h);
                if (!rc) rc = upload_params(h);
                if (rc) return rc;
            }
        }
    }
    mc_tune_report rep;
    std::memset(&rep, 0, sizeof rep);
    rep.row = ls.shape.row;
    rep.field = ls.shape.field;
    rep.pair = ls.shape.pair;
    if (tune_free || tune_cons) {
        Snapshot snap;
        size_t total = 0;
        for (mc_lattice* h : lats) {
            snap.off.push_back(total);
            total += al256(spin_bytes(h)) + al256(sizeof(LatState));
        }
        cudaError_t e = cudaMalloc(&snap.mem, total);
        if (e != cudaSuccess) {
            snap.mem = nullptr;
            return fail(MC_ERR_NOMEM, "no room for the autotuner's saved state (%zu bytes)", total);
        }
        int rc = copy_state(lats, snap, true, s);
        if (rc) return rc;
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        const KernelSet& k = kernel_set(precision);
        // mean ms per sweep of `sweeps` sweeps after one untimed, then restore
        auto trial = [&](bool constrained, double& ms) -> int {
            int r = enqueue_sweeps(k, ls, cone, 1, 0, constrained, s, nullptr);
            if (!r) {
                cudaEventRecord(a, s);
                r = enqueue_sweeps(k, ls, cone, sweeps, 0, constrained, s, nullptr);
                cudaEventRecord(b, s);
            }
            if (!r) {
                const cudaError_t ee = cudaEventSynchronize(b);
                if (ee != cudaSuccess) r = cuda_fail(ee, "autotune trial");
            }
            float t = 0.f;
            if (!r) cudaEventElapsedTime(&t, a, b);
            ms = double(t) / sweeps;
            const int rr = copy_state(lats, snap, false, s);
            return r ? r : rr;
        };
        // one knob: time every candidate, keep the fastest; another candidate
        // replaces the default (candidate 0) only if it is faster by more than
        // kTuneMargin, so that timing noise between near-equal shapes does not
        // decide
        auto knob = [&](int& choice, int n, double* ms, bool constrained) -> int {
            double best = 0.0;
            int pick = choice;
            for (int c = 0; c < n; ++c) {
                choice = c;
                const int r = trial(constrained, ms[c]);
                if (r) return r;
                if (c == 0 || ms[c] < best * (pick == 0 ? 1.0 - kTuneMargin : 1.0)) {
                    best = ms[c];
                    pick = c;
                }
            }
            choice = pick;
            return MC_OK;
        };
        if (!rc && tune_free) rc = knob(ls.shape.row, kRowShapes, rep.row_ms, false);
        if (!rc && tune_cons) rc = knob(ls.shape.field, kFieldShapes, rep.field_ms, true);
        if (!rc && tune_cons) rc = knob(ls.shape.pair, kPairShapes, rep.pair_ms, true);
        const cudaError_t es = cudaStreamSynchronize(s);
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        if (rc) return rc;
        if (es != cudaSuccess) return cuda_fail(es, "autotune sync");
        rep.row = ls.shape.row;
        rep.field = ls.shape.field;
        rep.pair = ls.shape.pair;
    }
    if (out) *out = rep;
    return MC_OK;
}

}  // namespace mcgb

using namespace mcgb;

extern "C" {

MC_API int mc_autotune(mc_handle h, int sweeps, int what, mc_tune_report* out) {
    if (!h) return fail(MC_ERR_ARG, "null handle");
    if (h->hp.nsub > 1) return fail(MC_ERR_ARG, "crystal lattices have no tunable launch shape");
    cudaSetDevice(h->device);
    NvtxRange range("mc_autotune");
    LaunchSet ls = single_launch_set(h);
    const int rc = autotune(h->hp.precision, ls, std::vector<mc_lattice*>{h}, h->cone, sweeps, what, h->stream, out);
    if (rc) return rc;
    h->shape = ls.shape;
    destroy_graphs(h->graphs);  // captured with the old shapes
    return MC_OK;
}

}  // extern "C"
