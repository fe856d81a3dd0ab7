// launchers_common.cuh -- host launchers shared by both precisions.  It is
// included inside `namespace mcgb { namespace { ... } }` of kernels_f32.cu
// and kernels_f64.cu, after each has defined R (the spin precision), V
// (sites per thread of a site tile), MINB (resident blocks per SM of the
// general colour pass) and kFieldChunk (tiles per grid-stride step of the
// neighbour-field kernel).
#pragma once

// Blocks of a persistent launch: resident blocks per SM x SMs (device 0 of
// the process is assumed representative; computed once per kernel).
template <typename K>
uint32_t resident_blocks(K kernel, int threads = kBlock) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
    if (per_sm < 1) per_sm = 1;
    return uint32_t(sms) * uint32_t(per_sm);
}

// blocks for ntiles warp tiles: one warp per tile at most, capped at residency
uint32_t grid_for(uint32_t ntiles, uint32_t cap, int threads = kBlock) {
    const uint32_t wpb = uint32_t(threads / 32);
    const uint32_t want = (ntiles + wpb - 1) / wpb;
    return want < cap ? (want > 0 ? want : 1) : cap;
}

template <int MEASURE>
void colour_pass_t(const GroupArgs& g, uint32_t ntiles, const R* cone, int colour, cudaStream_t s) {
    static const uint32_t cap = resident_blocks(colour_pass_kernel<R, V, MINB, MEASURE>);
    colour_pass_kernel<R, V, MINB, MEASURE><<<grid_for(ntiles, cap), kBlock, 0, s>>>(g, ntiles, cone, colour);
}

// measure: 0 none, 1 magnetisation and energies, 2 also torques
void colour_pass(const GroupArgs& g, uint32_t ntiles, const void* cone, int colour, int measure, cudaStream_t s) {
    const R* c = static_cast<const R*>(cone);
    if (measure >= 2) colour_pass_t<2>(g, ntiles, c, colour, s);
    else if (measure == 1) colour_pass_t<1>(g, ntiles, c, colour, s);
    else colour_pass_t<0>(g, ntiles, c, colour, s);
}

void sweep_end(const GroupArgs& g, cudaStream_t s) {
    sweep_end_kernel<R><<<(g.n + kBlock - 1) / kBlock, kBlock, 0, s>>>(g);
}

template <int C>
void pair_field_t(const GroupArgs& g, uint32_t ntiles, int colour, cudaStream_t s) {
    static const uint32_t cap = resident_blocks(pair_field_kernel<R, V, C>);
    pair_field_kernel<R, V, C><<<grid_for(ntiles, cap), kBlock, 0, s>>>(g, ntiles, colour);
}

// launch shapes: tiles per grid-stride step {default, 8, 2}
void pair_field(const GroupArgs& g, uint32_t ntiles, int colour, int shape, cudaStream_t s) {
    if (shape == 1) pair_field_t<8>(g, ntiles, colour, s);
    else if (shape == 2) pair_field_t<2>(g, ntiles, colour, s);
    else pair_field_t<kFieldChunk>(g, ntiles, colour, s);
}

void ml_reset(const GroupArgs& g, cudaStream_t s) {
    ml_reset_kernel<R><<<(g.n + kBlock - 1) / kBlock, kBlock, 0, s>>>(g);
}

void mlong(const GroupArgs& g, uint32_t ntiles, cudaStream_t s) {
    static const uint32_t cap = resident_blocks(mlong_kernel<R, V>);
    mlong_kernel<R, V><<<grid_for(ntiles, cap), kBlock, 0, s>>>(g, ntiles);
}

void measure(const GroupArgs& g, uint32_t ntiles, cudaStream_t s) {
    static const uint32_t cap = resident_blocks(measure_kernel<R, V>);
    measure_kernel<R, V><<<grid_for(ntiles, cap), kBlock, 0, s>>>(g, ntiles);
}

// Entry bound of the crystal kernels: the smallest instance that holds nb.
template <template <int> class F, typename... A>
void by_entries(int nb, A... a) {
    if (nb <= 8) F<8>::run(a...);
    else if (nb <= 12) F<12>::run(a...);
    else if (nb <= 14) F<14>::run(a...);
    else if (nb <= 18) F<18>::run(a...);
    else F<kXtalMaxNb>::run(a...);
}

template <int NB>
struct XtalPass {
    static void run(LatDev* L, uint32_t ntiles, const void* cone, int sub, int colour, int finalize, cudaStream_t s) {
        static const uint32_t cap = resident_blocks(xtal_pass_kernel<R, NB>);
        xtal_pass_kernel<R, NB><<<grid_for(ntiles, cap), kBlock, 0, s>>>(L, ntiles, static_cast<const R*>(cone), sub,
                                                                         colour, finalize);
    }
};

template <int NB>
struct XtalSample {
    template <int LEVEL>
    static void go(LatDev* L, uint32_t ntiles, uint32_t tiles_per_subset, cudaStream_t s) {
        static const uint32_t cap = resident_blocks(xtal_sample_kernel<R, NB, LEVEL>);
        xtal_sample_kernel<R, NB, LEVEL><<<grid_for(ntiles, cap), kBlock, 0, s>>>(L, ntiles, tiles_per_subset);
    }
    // level 2: with the torque sums
    static void run(LatDev* L, uint32_t ntiles, uint32_t tiles_per_subset, int level, cudaStream_t s) {
        if (level >= 2) go<2>(L, ntiles, tiles_per_subset, s);
        else go<1>(L, ntiles, tiles_per_subset, s);
    }
};

template <int NB>
struct XtalField {
    static void run(LatDev* L, uint32_t ntiles, int sub, int colour, cudaStream_t s) {
        static const uint32_t cap = resident_blocks(xtal_field_kernel<R, NB>);
        xtal_field_kernel<R, NB><<<grid_for(ntiles, cap), kBlock, 0, s>>>(L, ntiles, sub, colour);
    }
};

void xtal_field_launch(LatDev* L, uint32_t ntiles, int sub, int colour, int nb, cudaStream_t s) {
    by_entries<XtalField>(nb, L, ntiles, sub, colour, s);
}

void xtal_pass(LatDev* L, uint32_t ntiles, const void* cone, int sub, int colour, int finalize, int nb,
               cudaStream_t s) {
    by_entries<XtalPass>(nb, L, ntiles, cone, sub, colour, finalize, s);
}

void xtal_sample(LatDev* L, uint32_t ntiles, uint32_t tiles_per_subset, int nb, int level, cudaStream_t s) {
    by_entries<XtalSample>(nb, L, ntiles, tiles_per_subset, level, s);
}

void grain_sample(LatDev* L, uint32_t ntiles, int n_grains, cudaStream_t s) {
    static const uint32_t cap = resident_blocks(grain_sum_kernel<R, V>);
    grain_sum_kernel<R, V><<<grid_for(ntiles, cap), kBlock, 0, s>>>(L, ntiles);
    grain_finish_kernel<R><<<(n_grains + kBlock) / kBlock, kBlock, 0, s>>>(L);
}

void profile(LatDev* d, uint32_t Lh, uint32_t rows, cudaStream_t s) {
    const uint32_t threads = Lh * ((rows + 31) / 32);
    profile_kernel<R><<<(threads + kBlock - 1) / kBlock, kBlock, 0, s>>>(d);
}
