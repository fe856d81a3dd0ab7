// groups.cpp -- batched advance of many independent lattices: one launch per
// colour pass for the whole group, replayed from captured CUDA graphs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "runtime.h"

using namespace mcgb;


struct mc_group {
    std::vector<mc_handle> lats;
    std::vector<cudaStream_t> member_streams;  // restored at destroy
    int device = 0;
    int precision = 0;
    cudaStream_t stream = nullptr;
    void* d_mem = nullptr;
    void* d_wave = nullptr;  // wavefront plan of the group's wavefront lattices
    LaunchSet ls;
    const void* cone = nullptr;
    SweepGraphs graphs;  // captured sweeps of the whole group
    LatState* h_states = nullptr;  // pinned staging of mc_group_measure, one per member
    std::vector<ResidentPlan*> res_plans;  // members' resident plans (LaunchSet::res)
};

static int group_run(mc_group* g, int n, int measure, bool constrained) {
    NvtxRange range(constrained ? "mc_group_constrained_sweep" : "mc_group_sweep");
    cudaSetDevice(g->device);
    return run_sweeps(g->graphs, g->precision, g->ls, g->cone, n, measure, constrained, g->stream);
}

extern "C" {

MC_API int mc_group_create(const mc_handle* lattices, int n, mc_group_handle* out) {
    if (!lattices || n < 1 || !out) return fail(MC_ERR_ARG, "invalid argument");
    mc_group* g = new mc_group();
    g->lats.assign(lattices, lattices + n);
    g->device = lattices[0]->device;
    g->precision = lattices[0]->hp.precision;
    g->stream = lattices[0]->stream;
    g->cone = lattices[0]->cone;
    for (int i = 0; i < n; ++i) {
        if (!lattices[i] || lattices[i]->device != g->device || lattices[i]->hp.precision != g->precision) {
            delete g;
            return fail(MC_ERR_ARG, "group members must share device and precision");
        }
        if (lattices[i]->hp.nsub > 1) {
            delete g;
            return fail(MC_ERR_ARG, "group members must be simple cubic lattices");
        }
        if (lattices[i]->slab_nz) {
            delete g;
            return fail(MC_ERR_ARG, "a slab sweeps with its lattice's other slabs (mc_slab_sweep), not in a group");
        }
    }
    // launch tables: the lattices in launch order (general-path and small
    // lattices first, so their few tiles start early and overlap the rest),
    // with their site-tile and pair-tile starts
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const LatParams &pa = lattices[a]->hp, &pb = lattices[b]->hp;
        if ((pa.colour_kernel == kColourGeneral) != (pb.colour_kernel == kColourGeneral))
            return pa.colour_kernel == kColourGeneral;
        return pa.N < pb.N;
    });
    std::vector<LatDev*> all(n);
    std::vector<uint32_t> sa(n + 1, 0);
    for (int j = 0; j < n; ++j) {
        const LatParams& hp = lattices[order[j]]->hp;
        all[j] = lattices[order[j]]->d_lat;
        sa[j + 1] = sa[j] + hp.nblocks_site;
    }
    // colour passes: one list per colour-pass kernel (LatParams::colour_kernel);
    // constrained pair passes: one list per pair order (LatParams::pair_leader);
    // each list with its tile starts, in launch order
    // general, row, row with films; pairs in pair order, in site order; row
    // lattices other than the wavefront ones
    constexpr int kLists = 6;
    std::vector<LatDev*> sub[kLists];
    std::vector<uint32_t> st[kLists];
    for (int c = 0; c < kLists; ++c) st[c].assign(1, 0);
    std::vector<const LatParams*> wave_hp;
    std::vector<LatDev*> wave_dev;
    for (int j = 0; j < n; ++j) {
        const LatParams& hp = lattices[order[j]]->hp;
        const int c = hp.colour_kernel, q = 3 + (hp.pair_leader ? 1 : 0);
        sub[c].push_back(all[j]);
        st[c].push_back(st[c].back() + hp.nblocks_site);
        sub[q].push_back(all[j]);
        st[q].push_back(st[q].back() + hp.nblocks_pair);
        if (hp.wave) {
            wave_hp.push_back(&hp);
            wave_dev.push_back(all[j]);
        } else if (c == kColourRow) {
            sub[5].push_back(all[j]);
            st[5].push_back(st[5].back() + hp.nblocks_site);
        }
    }
    cudaSetDevice(g->device);
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t b_ptr = al(sizeof(LatDev*) * n);
    const size_t b_idx = al(sizeof(uint32_t) * (n + 1));
    const size_t total = (1 + kLists) * b_ptr + (1 + kLists) * b_idx;  // all + lists; site starts + list starts
    cudaError_t e = cudaMalloc(&g->d_mem, total);
    if (e != cudaSuccess) { delete g; return cuda_fail(e, "cudaMalloc(group)"); }
    std::vector<char> host(total, 0);
    char* hb = host.data();
    char* db = static_cast<char*>(g->d_mem);
    const size_t o0 = (1 + kLists) * b_ptr;
    std::copy(all.begin(), all.end(), reinterpret_cast<LatDev**>(hb));
    std::copy(sa.begin(), sa.end(), reinterpret_cast<uint32_t*>(hb + o0));
    g->ls.all = GroupArgs{reinterpret_cast<LatDev**>(db), reinterpret_cast<uint32_t*>(db + o0), n};
    g->ls.nt_all = sa.back();
    GroupArgs* lists[kLists] = {&g->ls.rest, &g->ls.row, &g->ls.rowx, &g->ls.pairs, &g->ls.pairs_lead,
                                &g->ls.row_rest};
    uint32_t* counts[kLists] = {&g->ls.nt_rest,  &g->ls.nt_row,        &g->ls.nt_rowx,
                                &g->ls.nt_pairs, &g->ls.nt_pairs_lead, &g->ls.nt_row_rest};
    for (int c = 0; c < kLists; ++c) {
        const size_t op = size_t(1 + c) * b_ptr, oi = o0 + size_t(1 + c) * b_idx;
        std::copy(sub[c].begin(), sub[c].end(), reinterpret_cast<LatDev**>(hb + op));
        std::copy(st[c].begin(), st[c].end(), reinterpret_cast<uint32_t*>(hb + oi));
        *lists[c] = GroupArgs{reinterpret_cast<LatDev**>(db + op), reinterpret_cast<uint32_t*>(db + oi),
                              int(sub[c].size())};
        *counts[c] = st[c].back();
    }
    // resident lattices: alone, or a group made only of large ones (swept one
    // after another, each held in shared memory)
    bool all_res = true;
    for (int i = 0; i < n; ++i)
        all_res = all_res && lattices[i]->res && (n == 1 || lattices[i]->hp.N >= kResGroupMinSpins);
    if (all_res) {
        for (int i = 0; i < n; ++i) g->res_plans.push_back(lattices[i]->res);
        g->ls.res = g->res_plans.data();
        g->ls.n_res = n;
    }
    g->ls.sample_level = 1;
    for (int i = 0; i < n; ++i)
        if (lattices[i]->hp.sample_torque) g->ls.sample_level = 2;
    // the members' queued work must be complete before the group uses them;
    // from now on every member runs on the group stream, so that calls on a
    // member order after the group's work
    for (int i = 0; i < n; ++i) {
        cudaStreamSynchronize(lattices[i]->stream);
        g->member_streams.push_back(lattices[i]->stream);
        lattices[i]->stream = g->stream;
    }
    if (cudaMemcpy(g->d_mem, host.data(), host.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        for (int i = 0; i < n; ++i) lattices[i]->stream = g->member_streams[i];
        cudaFree(g->d_mem);
        delete g;
        return fail(MC_ERR_CUDA, "group table upload failed");
    }
    if (!wave_hp.empty()) {  // one wavefront plan over all the group's wavefront lattices
        const uint32_t blocks = kernels_f32().wave_blocks();
        const WavePlan pl = plan_wave(wave_hp, blocks);
        const int rc = upload_wave_plan(pl, wave_dev, g->stream, &g->d_wave, &g->ls.wave);
        if (rc) {
            for (int i = 0; i < n; ++i) lattices[i]->stream = g->member_streams[i];
            cudaFree(g->d_mem);
            delete g;
            return rc;
        }
        g->ls.nb_wave = uint32_t(pl.off.size() - 1);
    }
    *out = g;
    return MC_OK;
}

MC_API int mc_group_destroy(mc_group_handle g) {
    if (!g) return MC_OK;
    cudaSetDevice(g->device);
    cudaStreamSynchronize(g->stream);
    destroy_graphs(g->graphs);
    cudaFree(g->d_mem);
    if (g->d_wave) cudaFree(g->d_wave);
    if (g->h_states) cudaFreeHost(g->h_states);
    for (size_t i = 0; i < g->lats.size(); ++i) g->lats[i]->stream = g->member_streams[i];
    delete g;
    return MC_OK;
}

MC_API int mc_group_sweep(mc_group_handle g, int n_sweeps, int measure) {
    if (!g || n_sweeps < 0) return fail(MC_ERR_ARG, "invalid argument");
    return group_run(g, n_sweeps, measure ? 1 : 0, false);
}

MC_API int mc_group_constrained_sweep(mc_group_handle g, const double* theta_c_deg, const double* phi_c_deg,
                                      int n_sweeps, int measure) {
    if (!g || !theta_c_deg || !phi_c_deg || n_sweeps < 0) return fail(MC_ERR_ARG, "invalid argument");
    cudaSetDevice(g->device);
    for (size_t i = 0; i < g->lats.size(); ++i) {
        mc_handle h = g->lats[i];
        if (!(theta_c_deg[i] >= 0.0 && theta_c_deg[i] <= 180.0) || !std::isfinite(phi_c_deg[i]))
            return fail(MC_ERR_ARG, "constraint angle %zu invalid", i);
        for (int a = 0; a < 3; ++a)
            if (h->hp.bc[a] == MC_PINNED) return fail(MC_ERR_ARG, "constrained sweeps need no pinned boundary");
        int rc = ensure_aos(h);
        if (rc) return rc;
        constraint_frame(theta_c_deg[i], phi_c_deg[i], h->hp.R);
        rc = upload_params(h);  // on the group stream (members adopt it)
        if (rc) return rc;
    }
    return group_run(g, n_sweeps, measure ? 1 : 0, true);
}

// n_sweeps sweeps of the group with events around every launch that moves
// spins; per kind (TimedLaunch) the summed milliseconds and the count.
static int time_kinds(mc_group* g, int n_sweeps, int measure, bool constrained, double ms[kTimedKinds],
                      int count[kTimedKinds]) {
    cudaSetDevice(g->device);
    std::vector<TimedLaunch> ev;
    int rc = enqueue_sweeps(kernel_set(g->precision), g->ls, g->cone, n_sweeps, measure ? 1 : 0, constrained, g->stream,
                            &ev);
    cudaError_t e = cudaStreamSynchronize(g->stream);
    for (int k = 0; k < kTimedKinds; ++k) {
        ms[k] = 0.0;
        count[k] = 0;
    }
    for (auto& t : ev) {
        float x = 0.f;
        cudaEventElapsedTime(&x, t.a, t.b);
        ms[t.kind] += x;
        count[t.kind] += 1;
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "time_passes sync");
    return MC_OK;
}

MC_API int mc_group_time_passes(mc_group_handle g, int n_sweeps, int measure, double* avg_ms, int* launches) {
    if (!g || n_sweeps < 1 || !avg_ms || !launches) return fail(MC_ERR_ARG, "invalid argument");
    double ms[kTimedKinds];
    int count[kTimedKinds];
    const int rc = time_kinds(g, n_sweeps, measure, false, ms, count);
    if (rc) return rc;
    double total = 0.0;
    int n = 0;
    for (int k = 0; k < kTimedKinds; ++k) {
        total += ms[k];
        n += count[k];
    }
    *launches = n;
    *avg_ms = n ? total / double(n) : 0.0;
    return MC_OK;
}

MC_API int mc_group_time_kernels(mc_group_handle g, int n_sweeps, int measure, int constrained, double avg_ms[4],
                                 int launches[4]) {
    if (!g || n_sweeps < 1 || !avg_ms || !launches) return fail(MC_ERR_ARG, "invalid argument");
    for (mc_handle h : g->lats)
        if (constrained && !h->d_aos) return fail(MC_ERR_STATE, "no constrained sweep has set the constraint yet");
    double ms[kTimedKinds];
    int count[kTimedKinds];
    const int rc = time_kinds(g, n_sweeps, measure, constrained != 0, ms, count);
    if (rc) return rc;
    for (int k = 0; k < kTimedKinds; ++k) {
        launches[k] = count[k];
        avg_ms[k] = count[k] ? ms[k] / double(count[k]) : 0.0;
    }
    return MC_OK;
}

MC_API int mc_group_autotune(mc_group_handle g, int sweeps, int what, mc_tune_report* out) {
    if (!g) return fail(MC_ERR_ARG, "null group");
    cudaSetDevice(g->device);
    NvtxRange range("mc_group_autotune");
    const int rc = autotune(g->precision, g->ls, g->lats, g->cone, sweeps, what, g->stream, out);
    if (rc) return rc;
    destroy_graphs(g->graphs);  // captured with the old shapes
    return MC_OK;
}

MC_API int mc_group_set_shapes(mc_group_handle g, int row, int field, int pair) {
    if (!g) return fail(MC_ERR_ARG, "null group");
    if (row < 0 || row >= kRowShapes || field < 0 || field >= kFieldShapes || pair < 0 || pair >= kPairShapes)
        return fail(MC_ERR_ARG, "launch shape out of range");
    g->ls.shape.row = row;
    g->ls.shape.field = field;
    g->ls.shape.pair = pair;
    destroy_graphs(g->graphs);  // captured with the old shapes
    return MC_OK;
}

MC_API int mc_group_measure(mc_group_handle g, mc_observables* out, int n) {
    if (!g || !out || n != int(g->lats.size())) return fail(MC_ERR_ARG, "invalid argument");
    cudaSetDevice(g->device);
    if (!g->h_states) {
        cudaError_t e = cudaMallocHost(reinterpret_cast<void**>(&g->h_states), sizeof(LatState) * size_t(n));
        if (e != cudaSuccess) {
            g->h_states = nullptr;
            return cuda_fail(e, "cudaMallocHost(group measure)");
        }
    }
    // every member runs on the group stream: one copy each, one wait
    for (int i = 0; i < n; ++i) {
        const cudaError_t e = cudaMemcpyAsync(&g->h_states[i], &g->lats[i]->d_lat->st, sizeof(LatState),
                                              cudaMemcpyDeviceToHost, g->stream);
        if (e != cudaSuccess) return cuda_fail(e, "group measure copy");
    }
    const cudaError_t e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return cuda_fail(e, "group measure sync");
    int first = MC_OK;
    for (int i = 0; i < n; ++i) {
        const int rc = observables_from(g->lats[i], g->h_states[i], &out[i]);
        if (rc && first == MC_OK) first = rc;
    }
    if (first != MC_OK) return fail(first, "device reported error %d", first);
    return MC_OK;
}

MC_API int mc_group_sync(mc_group_handle g) {
    if (!g) return fail(MC_ERR_ARG, "null group");
    cudaSetDevice(g->device);
    cudaError_t e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return cuda_fail(e, "group sync");
    for (mc_handle h : g->lats) {
        LatState st;
        int rc = read_state(h, &st);
        if (rc) return rc;
        if (st.error) return fail(st.error, "device reported error %d", st.error);
    }
    return MC_OK;
}

}  // extern "C"
