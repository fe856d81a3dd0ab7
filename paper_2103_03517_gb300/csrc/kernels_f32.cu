// kernels_f32.cu -- float instances of the libmc kernels and their launchers.
// FP32 spins and energies (fast intrinsics: rsqrtf, __expf, __fdividef);
// FP64 for the sample, torque and M_L bookkeeping.
#include "kernels.h"
#include "pass_impl.cuh"

namespace mcgb {
namespace {

using R = float;

void colour_pass(const GroupArgs& g, uint32_t nblocks, const void* cone, int colour, int measure,
                 cudaStream_t s) {
    colour_pass_kernel<R><<<nblocks, kBlock, 0, s>>>(g, static_cast<const R*>(cone), colour, measure);
}

void pair_pass(const GroupArgs& g, uint32_t nblocks, const void* cone, int colour, int finalize, int measure,
               cudaStream_t s) {
    pair_pass_kernel<R><<<nblocks, kBlock, 0, s>>>(g, static_cast<const R*>(cone), colour, finalize, measure);
}

void mlong(const GroupArgs& g, uint32_t nblocks, cudaStream_t s) {
    mlong_kernel<R><<<nblocks, kBlock, 0, s>>>(g);
}

void measure(const GroupArgs& g, uint32_t nblocks, cudaStream_t s) {
    measure_kernel<R><<<nblocks, kBlock, 0, s>>>(g);
}

void profile(LatDev* d, uint32_t Lh, uint32_t rows, cudaStream_t s) {
    const uint32_t threads = Lh * ((rows + 31) / 32);
    profile_kernel<R><<<(threads + kBlock - 1) / kBlock, kBlock, 0, s>>>(d);
}

}  // namespace

const KernelSet& kernels_f32() {
    static const KernelSet k{colour_pass, pair_pass, mlong, measure, profile, "f32"};
    return k;
}

}  // namespace mcgb
