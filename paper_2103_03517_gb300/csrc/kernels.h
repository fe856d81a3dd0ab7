// kernels.h -- host-side launchers of the libmc kernels, one set per
// precision (kernels_f64.cu, kernels_f32.cu).
#pragma once
#include <cuda_runtime.h>

#include "mc_internal.h"

namespace mcgb {

// Launch shapes the autotuner chooses among: an index into each kernel's
// candidate list (0 = the default, measured best on the batched workloads).
//   row:   FP32 row kernel, minimum resident blocks per SM (registers per
//          thread): all-periodic {3, 2}, boundaries and films {2, 3}; for a
//          resident lattice, threads per block {512, 640};
//   pair:  pair pass, consecutive tiles per grid-stride step {4, 8, 2}, and
//          4 with one more resident block per SM;
//   field: neighbour-field kernel, the same {4, 8, 2}.
constexpr int kRowShapes = 2, kPairShapes = 4, kFieldShapes = 3;
struct LaunchShape {
    int row = 0, pair = 0, field = 0;
};

// A resident lattice's launch: its arguments and two TMA descriptors
// (CUtensorMap, 128 bytes each) of its spins seen as a 64 x Ly x Lz x 6
// array (x, y, z, colour and component), with the boxes of a y face (64 x 1
// x bz x 3) and of a z face (64 x by x 1 x 3) of a brick.
struct alignas(128) ResidentPlan {
    unsigned char map_y[128];
    unsigned char map_z[128];
    ResidentArgs args;
};

struct KernelSet {
    // Table A1 colour pass over the lattices of g (ntiles = warp tiles of the
    // launch; the launcher sizes a persistent grid from the occupancy).
    // measure: 0 none, 1 magnetisation and energies, 2 also torques.
    void (*colour_pass)(const GroupArgs& g, uint32_t ntiles, const void* cone, int colour, int measure,
                        cudaStream_t s);
    // FP32 colour pass over lattices in the row layout (adjacent site pairs
    // per lane); gen = 0: all axes periodic, no film tables; gen = 1: any
    // boundaries and film tables.  Null in the FP64 set.  After an
    // unmeasured black pass (colour 1) it also launches the close of the
    // lattices' sweeps (row_close_kernel).  Returns the status of the
    // launches (made with programmatic serialisation).
    cudaError_t (*row_pass)(const GroupArgs& g, uint32_t ntiles, const void* cone, int colour, int measure,
                            int gen, int shape, cudaStream_t s);
    // Table A2 pair pass over sub-set (sub, colour) (sub = 0 for simple cubic
    // lattices); leader != 0 takes the pairs in site order
    // (LatParams::pair_leader).
    void (*pair_pass)(const GroupArgs& g, uint32_t ntiles, const void* cone, int colour, int leader, int shape,
                      int sub, cudaStream_t s);
    // End of an unmeasured constrained sweep of every lattice of g.
    void (*sweep_end)(const GroupArgs& g, cudaStream_t s);
    // Neighbour field of every site of the given colour into LatParams::pfield
    // (site tiles), before that colour's pair pass.
    void (*pair_field)(const GroupArgs& g, uint32_t ntiles, int colour, int shape, cudaStream_t s);
    // Zero M_L and its carried change of every lattice of g (before mlong).
    void (*ml_reset)(const GroupArgs& g, cudaStream_t s);
    // Exact M_L of every lattice of g (site tiles).
    void (*mlong)(const GroupArgs& g, uint32_t ntiles, cudaStream_t s);
    // Standalone sample + end of sweep (site tiles).
    void (*measure)(const GroupArgs& g, uint32_t ntiles, cudaStream_t s);
    // The same over lattices in the row layout (gen as in row_pass); with gen
    // = 0 it also stores the red sites' field for the next constrained sweep
    // (LatParams::pfield).  Null in the FP64 set.
    void (*row_sample)(const GroupArgs& g, uint32_t ntiles, int gen, cudaStream_t s);
    // bcc / fcc / hcp lattice L alone: a pass over sub-set (sub, colour) of
    // ntiles 32-site tiles (finalize != 0 closes the sweep), and the sample
    // over the 2 nsub sub-sets (ntiles = 2 nsub tiles_per_subset), which
    // closes it (level 2: with the torques); nb = the most neighbour entries
    // of a sub-lattice.
    void (*xtal_pass)(LatDev* L, uint32_t ntiles, const void* cone, int sub, int colour, int finalize, int nb,
                      cudaStream_t s);
    void (*xtal_sample)(LatDev* L, uint32_t ntiles, uint32_t tiles_per_subset, int nb, int level, cudaStream_t s);
    // Constrained sweeps of a crystal L: the neighbour field of sub-set (sub,
    // colour) into LatParams::pfield (ntiles 32-site tiles).
    void (*xtal_field)(LatDev* L, uint32_t ntiles, int sub, int colour, int nb, cudaStream_t s);
    // One grain sample of a film lattice (ntiles site tiles, n_grains grains).
    void (*grain_sample)(LatDev* L, uint32_t ntiles, int n_grains, cudaStream_t s);
    // Slice sums for the profile of one lattice.
    void (*profile)(LatDev* d, uint32_t Lh, uint32_t rows, cudaStream_t s);
    const char* name;
    // FP32 wavefront sweep (red and black pass in one launch) of the
    // lattices of a, nblocks blocks; dir = 0 reads spins and writes
    // spins_alt, dir = 1 the reverse; measure as for colour_pass.  Null in
    // the FP64 set.  Returns the status of the launch.
    cudaError_t (*wave_sweep)(const WaveArgs& a, uint32_t nblocks, const void* cone, int dir, int measure,
                              cudaStream_t s);
    // Blocks of the wavefront kernel resident on the current device at once
    // (the work-unit plan is made for this many).  Null in the FP64 set.
    uint32_t (*wave_blocks)();
    // Slabs of a lattice split along z (FP32 row layout; null in the FP64
    // set): export slab L's counts to LatParams::slab_counts, close L's
    // sweep from its (summed) counts.
    void (*slab_export)(LatDev* L, cudaStream_t s);
    void (*slab_close)(LatDev* L, int measure, cudaStream_t s);
    // Slabs on one device: the halo planes of one colour of n slabs, each
    // from its neighbours (dst / src: [slab][lower, upper] plane bases,
    // strides per slab), and export, sum and close of n slabs in one launch.
    cudaError_t (*slab_halo)(float* const (*dst)[2], const float* const (*src)[2], const uint32_t* stride,
                             const uint32_t (*src_stride)[2], uint32_t plane, int n, cudaStream_t s);
    cudaError_t (*slab_close_all)(LatDev* const* lats, int n, int measure, cudaStream_t s);
    // Resident sweeps (resident_pass.cuh) of the lattice of a plan: n sweeps
    // in cooperative launches of at most kResMaxSweeps, measure as for
    // colour_pass, shape 0 or 1 (blocks of 512 or 640 threads).  Null in the
    // FP64 set.  Returns the status of the launches.
    cudaError_t (*resident_sweeps)(const ResidentPlan& r, const void* cone, int n, int measure, int shape,
                                   cudaStream_t s);
    // The brick split of FP32 lattice p (host copy: dims, stride, spins) on
    // the current device and the tensor maps of its halo faces: fills
    // everything but args.lat and args.ctl; false when its rows do not fit
    // the SMs' shared memory.  Null in the FP64 set.
    bool (*resident_plan)(const LatParams& p, ResidentPlan* out);
};

// Launch tables of a set of lattices: site tiles and pair tiles of every
// lattice (lattice l owns tiles [start[l], start[l+1])), and for the colour
// passes the split by colour-pass kernel (LatParams::colour_kernel).
struct LaunchSet {
    GroupArgs all, pairs, pairs_lead;
    uint32_t nt_all = 0, nt_pairs = 0, nt_pairs_lead = 0;  // pair tiles: pair order, site order
    // colour passes: row kernel, row kernel with boundaries and films, the
    // general kernel (tiles)
    GroupArgs row, rowx, rest;
    uint32_t nt_row = 0, nt_rowx = 0, nt_rest = 0;
    // wavefront lattices (LatParams::wave): their work-unit plan (nb_wave
    // blocks; 0 = none), and the row-kernel list without them, which runs
    // beside a wavefront launch (row above keeps them, for sweeps that run
    // as two row passes)
    WaveArgs wave = {};
    uint32_t nb_wave = 0;
    GroupArgs row_rest;
    uint32_t nt_row_rest = 0;
    // resident lattices (LatParams::rctl) whose unconstrained sweeps run as
    // resident launches, one lattice after another: a lattice alone, or every
    // lattice of a group made only of large resident lattices; n_res launch
    // plans, owned by the lattices (none: n_res = 0)
    ResidentPlan* const* res = nullptr;
    int n_res = 0;
    int sample_level = 2;  // sample of a measured colour pass: 1 or 2 (torques)
    // a bcc / fcc lattice alone: its descriptor and sub-lattice count, else null
    LatDev* xtal = nullptr;
    int nsub = 1;
    int xnb_max = 0;  // most neighbour entries of its sub-lattices
    LaunchShape shape;  // autotuned launch shapes
};

const KernelSet& kernels_f64();
const KernelSet& kernels_f32();

}  // namespace mcgb
