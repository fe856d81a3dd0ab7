// runtime.h -- host-side objects shared by the runtime, groups and server.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <utility>
#include <vector>

#include "kernels.h"
#include "mc.h"
#include "mc_internal.h"

namespace mcgb {
// An NVTX range for the scope of the object (a no-op without a profiler).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Captured CUDA graphs of kGraphSweeps sweeps of one launch set, by
// [constrained][measure]; built on first use and replayed.
constexpr int kGraphSweeps = 16;
// A resident lattice (LatParams::rctl) sweeps held in shared memory in calls
// of at least this many sweeps; shorter calls, which would not pay for the
// lattice's load and store, take the row passes (the same chain).
constexpr int kResMinSweeps = 3;
// A group sweeps its lattices resident one after another only when every
// member is resident and holds at least this many spins (a 128^3 lattice:
// held in shared memory it sweeps faster than its share of a batched row
// pass; smaller lattices sweep faster batched).
constexpr long long kResGroupMinSpins = 1ll << 21;
struct SweepGraphs {
    cudaGraphExec_t exec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
};
}  // namespace mcgb

struct mc_lattice {
    mc_desc desc;                 // copy (film pointers cleared)
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t owned_stream = nullptr;   // created by the library, destroyed with it
    mcgb::LatParams hp;           // host copy of the device parameters
    void* d_base = nullptr;       // the lattice's single device allocation
    size_t bytes = 0;
    mcgb::LatDev* d_lat = nullptr;
    mcgb::LatDev** d_group_lats = nullptr;   // launch tables of the lattice alone
    uint32_t* d_group_start = nullptr;
    uint32_t* d_group_start_pair = nullptr;
    void* d_aos = nullptr;        // packed spin copy of constrained sweeps (LatParams::aos)
    void* d_wave = nullptr;       // wavefront plan of the lattice alone (LatParams::wave)
    mcgb::WaveArgs wave_args = {};
    uint32_t wave_nblocks = 0;
    mcgb::ResidentPlan* res = nullptr;  // resident sweeps of the lattice alone (null: none)
    mcgb::SweepGraphs graphs;     // sweeps of the lattice alone
    mcgb::LaunchShape shape;      // autotuned launch shapes of the lattice alone
    const void* cone = nullptr;   // c(theta) table of the precision
    int slab_z0 = 0, slab_nz = 0, slab_lz = 0;  // a slab (mc_slab_create): its planes and the
                                                // lattice's Lz (slab_nz = 0: not a slab)
    long long slab_n = 0, slab_n_mov = 0;       // the whole lattice's sites and movable sites
    std::vector<uint8_t> film_bonds;   // kept for checkpoints
    std::vector<int32_t> film_grain;
    std::vector<double> film_axes;
    mc_lattice() = default;
    mc_lattice(const mc_lattice&) = delete;
    mc_lattice& operator=(const mc_lattice&) = delete;
    ~mc_lattice() { delete res; }
};

namespace mcgb {

int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
// A z slab of a larger lattice: global planes [z0, z0 + nz) of Lz.
struct SlabSpec {
    int z0, nz, Lz;
};
int create_lattice(const mc_desc* d, mc_handle* out, const SlabSpec* slab = nullptr);
int validate_desc(const mc_desc* d);
int row_fast(const LatParams& p, bool film);
int sublattices(int lattice);
int colour_kernel(const LatParams& p, bool film, int path);
size_t lattice_bytes(const mc_desc* d, bool slab = false);
int upload_params(mc_lattice* h);
size_t aos_bytes(const mc_desc* d);
int ensure_aos(mc_lattice* h);
void constraint_frame(double theta_deg, double phi_deg, double R[9]);
const KernelSet& kernel_set(int precision);
int read_state(mc_lattice* h, LatState* st);
int observables_from(const mc_lattice* h, const LatState& st, mc_observables* out);
// n sweeps of a launch set on stream s: whole graphs of kGraphSweeps
// sweeps, then the remainder launched directly.
int run_sweeps(SweepGraphs& gr, int precision, const LaunchSet& ls, const void* cone, int n, int measure,
               bool constrained, cudaStream_t s);
void destroy_graphs(SweepGraphs& gr);
LaunchSet single_launch_set(mc_lattice* h);
int autotune(int precision, LaunchSet& ls, const std::vector<mc_lattice*>& lats, const void* cone, int sweeps,
             int what, cudaStream_t s, mc_tune_report* out);
// Work units of wavefront lattices for a launch of `blocks` blocks (block b
// runs units [off[b], off[b+1]) of wu; nwu per lattice; span = the longest
// block's cost in row-steps).
struct WavePlan {
    std::vector<WaveWU> wu;
    std::vector<uint32_t> off, nwu;
    long long span = 0;
};
bool wave_desc(const mc_desc* d);
bool resident_desc(const mc_desc* d, bool slab);
WavePlan plan_wave(const std::vector<const LatParams*>& lats, uint32_t blocks);
int upload_wave_plan(const WavePlan& pl, const std::vector<LatDev*>& dev_lats, cudaStream_t s, void** d_mem,
                     WaveArgs* out);
// A launch bracketed by CUDA events (mc_group_time_passes / _kernels):
// kind kTimedWave = a wavefront sweep, kTimedPass = a colour pass (row or
// general kernels), kTimedPair = a constrained pair pass, kTimedResident =
// a resident launch (up to kResMaxSweeps sweeps).
enum { kTimedWave = 0, kTimedPass = 1, kTimedPair = 2, kTimedResident = 3, kTimedKinds = 4 };
struct TimedLaunch {
    cudaEvent_t a, b;
    int kind;
};
int enqueue_sweeps(const KernelSet& k, const LaunchSet& ls, const void* cone, int n, int measure, bool constrained,
                   cudaStream_t s, std::vector<TimedLaunch>* events);

}  // namespace mcgb
