// kernels.h -- host-side launchers of the libmc kernels, one set per
// precision (kernels_f64.cu, kernels_f32.cu).
#pragma once
#include <cuda_runtime.h>

#include "mc_internal.h"

namespace mcgb {

struct KernelSet {
    // Table A1 colour pass over the lattices of g (nblocks = grid size).
    void (*colour_pass)(const GroupArgs& g, uint32_t nblocks, const void* cone, int colour, int measure,
                        cudaStream_t s);
    // Table A2 pair pass; finalize != 0 closes the sweep in the last block.
    void (*pair_pass)(const GroupArgs& g, uint32_t nblocks, const void* cone, int colour, int finalize,
                      int measure, cudaStream_t s);
    // Exact M_L of every lattice of g (site-pass grid).
    void (*mlong)(const GroupArgs& g, uint32_t nblocks, cudaStream_t s);
    // Standalone sample + end of sweep (site-pass grid).
    void (*measure)(const GroupArgs& g, uint32_t nblocks, cudaStream_t s);
    // Slice sums for the profile of one lattice.
    void (*profile)(LatDev* d, uint32_t Lh, uint32_t rows, cudaStream_t s);
    const char* name;
};

const KernelSet& kernels_f64();
const KernelSet& kernels_f32();

}  // namespace mcgb
