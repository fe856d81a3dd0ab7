// kernels_f64.cu -- double instances of the libmc kernels and their launchers.
// Built with -fmad=false: no multiply-add contraction, so every FP64
// expression is evaluated as one IEEE operation at a time, left to right.
#include "kernels.h"
#include "pass_impl.cuh"
#include "xtal_pass.cuh"

namespace mcgb {
namespace {

using R = double;
constexpr int MINB = 1;  // minimum resident blocks per SM of the colour pass
constexpr int V = kSitesPerThreadF64;
constexpr int kPairChunk = 4;   // consecutive pair tiles per grid-stride step of the pair pass
constexpr int kFieldChunk = 4;  // the same for the neighbour-field kernel

#include "launchers_common.cuh"

template <int C>
void pair_pass_t(const GroupArgs& g, uint32_t ntiles, const void* cone, int colour, int sub, cudaStream_t s) {
    static const uint32_t cap = resident_blocks(pair_pass_kernel<R, 1, C, false>);
    pair_pass_kernel<R, 1, C, false><<<grid_for(ntiles, cap), kBlock, 0, s>>>(g, ntiles, static_cast<const R*>(cone),
                                                                           colour, sub);
}

// launch shapes: tiles per grid-stride step {default, 8, 2}; FP64 lattices
// always take pair order (LatParams::pair_leader)
void pair_pass(const GroupArgs& g, uint32_t ntiles, const void* cone, int colour, int leader, int shape, int sub,
               cudaStream_t s) {
    (void)leader;
    if (shape == 1) pair_pass_t<8>(g, ntiles, cone, colour, sub, s);
    else if (shape == 2) pair_pass_t<2>(g, ntiles, cone, colour, sub, s);
    else pair_pass_t<kPairChunk>(g, ntiles, cone, colour, sub, s);
}

}  // namespace

const KernelSet& kernels_f64() {
    static const KernelSet k{colour_pass, nullptr,     pair_pass,   sweep_end,         pair_field,
                             ml_reset,    mlong,       measure,     nullptr,           xtal_pass,
                             xtal_sample, xtal_field_launch, grain_sample, profile, "f64",
                             nullptr,     nullptr,     nullptr,           nullptr,      nullptr,
                             nullptr,     nullptr,     nullptr};
    return k;
}

}  // namespace mcgb
