// kernels_f32.cu -- float instances of the libmc kernels and their launchers.
// FP32 spins and energies (fast intrinsics: rsqrtf, __expf, __fdividef);
// FP64 for the sample, torque and M_L bookkeeping.
#ifndef MC_MINB_F32
#define MC_MINB_F32 3
#endif
#ifndef MC_MINB_GEN_F32
#define MC_MINB_GEN_F32 2
#endif
#ifndef MC_MINB_PAIR_F32
#define MC_MINB_PAIR_F32 3
#endif
#ifndef MC_PAIR_CHUNK
#define MC_PAIR_CHUNK 4
#endif
#ifndef MC_PAIR_CHUNK_LEAD
#define MC_PAIR_CHUNK_LEAD 4
#endif
#include <algorithm>

#include "kernels.h"
#include "pass_impl.cuh"
#include "xtal_pass.cuh"
#include "row_pass.cuh"
#include "wave_pass.cuh"
#include "resident_pass.cuh"

namespace mcgb {
namespace {

using R = float;
constexpr int MINB = MC_MINB_F32;  // minimum resident blocks per SM of the colour pass
constexpr int MINB_GEN = MC_MINB_GEN_F32;  // the same for the row kernel with boundaries and films
constexpr int MINB_PAIR = MC_MINB_PAIR_F32;  // the same for the pair pass
constexpr int MINB_PAIR_LEAD = 2;            // the same for the pair pass in site order
constexpr int kPairChunk = MC_PAIR_CHUNK;    // consecutive pair tiles per grid-stride step
constexpr int kPairChunkLead = MC_PAIR_CHUNK_LEAD;  // the same in site order
constexpr int kFieldChunk = 4;               // the same for the neighbour-field kernel
constexpr int V = kSitesPerThreadF32;

#include "launchers_common.cuh"

template <int B, int MEASURE, int GEN>
cudaError_t row_pass_t(const GroupArgs& g, uint32_t ntiles, const R* cone, int colour, cudaStream_t s) {
    static const uint32_t cap = resident_blocks(row_pass_kernel<B, MEASURE, GEN>);
    // programmatic serialisation: the pass starts its blocks while the
    // previous launch drains and waits inside the kernel (griddepcontrol)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid_for(ntiles, cap));
    cfg.blockDim = dim3(kBlock);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, row_pass_kernel<B, MEASURE, GEN>, g, ntiles, cone, colour);
    if (e != cudaSuccess || colour != 1 || MEASURE > 0) return e;  // the unmeasured sweep's end
    cudaLaunchConfig_t cc = cfg;
    cc.gridDim = dim3(uint32_t(g.n));
    cc.blockDim = dim3(32);
    return cudaLaunchKernelEx(&cc, row_close_kernel, g, 0);
}

// launch shape 0: the default blocks per SM of the instance; 1: the other candidate
template <int GEN, int B0, int B1>
cudaError_t row_pass_g(const GroupArgs& g, uint32_t ntiles, const R* c, int colour, int measure, int shape,
                       cudaStream_t s) {
    if (shape == 1) {
        if (measure >= 2) return row_pass_t<B1, 2, GEN>(g, ntiles, c, colour, s);
        if (measure == 1) return row_pass_t<B1, 1, GEN>(g, ntiles, c, colour, s);
        return row_pass_t<B1, 0, GEN>(g, ntiles, c, colour, s);
    }
    if (measure >= 2) return row_pass_t<B0, 2, GEN>(g, ntiles, c, colour, s);
    if (measure == 1) return row_pass_t<B0, 1, GEN>(g, ntiles, c, colour, s);
    return row_pass_t<B0, 0, GEN>(g, ntiles, c, colour, s);
}

cudaError_t row_pass(const GroupArgs& g, uint32_t ntiles, const void* cone, int colour, int measure, int gen,
                     int shape, cudaStream_t s) {
    const R* c = static_cast<const R*>(cone);
    if (gen) return row_pass_g<1, MINB_GEN, MINB_GEN + 1>(g, ntiles, c, colour, measure, shape, s);
    return row_pass_g<0, MINB, MINB - 1>(g, ntiles, c, colour, measure, shape, s);
}

// the all-periodic instance samples red sites first and stores their field
// (the next constrained sweep's red field); the other keeps black
template <int GEN>
void row_sample_g(const GroupArgs& g, uint32_t ntiles, cudaStream_t s) {
    constexpr int B = GEN ? MINB_GEN : MINB;
    static const uint32_t cap = resident_blocks(row_pass_kernel<B, 2, GEN, 0>);
    row_pass_kernel<B, 2, GEN, 0><<<grid_for(ntiles, cap), kBlock, 0, s>>>(g, ntiles, nullptr, GEN ? 1 : 0);
}

void row_sample(const GroupArgs& g, uint32_t ntiles, int gen, cudaStream_t s) {
    if (gen) row_sample_g<1>(g, ntiles, s);
    else row_sample_g<0>(g, ntiles, s);
}

template <bool LEADER, int C, int B = LEADER ? MINB_PAIR_LEAD : MINB_PAIR, int NT = kBlock>
void pair_pass_t(const GroupArgs& g, uint32_t ntiles, const void* cone, int colour, int sub, cudaStream_t s) {
    static const uint32_t cap = resident_blocks(pair_pass_kernel<R, B, C, LEADER, NT>, NT);
    pair_pass_kernel<R, B, C, LEADER, NT><<<grid_for(ntiles, cap, NT), NT, 0, s>>>(
        g, ntiles, static_cast<const R*>(cone), colour, sub);
}

// launch shapes: tiles per grid-stride step {default, 8, 2}, and the
// default step with more resident warps per SM: pair order one more block
// of 256 threads (fewer registers, some spilled), site order blocks of 128
// threads, five per SM (20 warps at up to 102 registers, against 16 warps
// in two blocks of 256)
template <bool LEADER>
void pair_pass_s(const GroupArgs& g, uint32_t ntiles, const void* cone, int colour, int shape, int sub,
                 cudaStream_t s) {
    constexpr int C0 = LEADER ? kPairChunkLead : kPairChunk;
    constexpr int B0 = LEADER ? MINB_PAIR_LEAD : MINB_PAIR;
    if (shape == 1) pair_pass_t<LEADER, 8>(g, ntiles, cone, colour, sub, s);
    else if (shape == 2) pair_pass_t<LEADER, 2>(g, ntiles, cone, colour, sub, s);
    else if (shape == 3) {
        if constexpr (LEADER) pair_pass_t<LEADER, C0, 5, 128>(g, ntiles, cone, colour, sub, s);
        else pair_pass_t<LEADER, C0, B0 + 1>(g, ntiles, cone, colour, sub, s);
    } else pair_pass_t<LEADER, C0>(g, ntiles, cone, colour, sub, s);
}

void pair_pass(const GroupArgs& g, uint32_t ntiles, const void* cone, int colour, int leader, int shape, int sub,
               cudaStream_t s) {
    if (leader) pair_pass_s<true>(g, ntiles, cone, colour, shape, sub, s);
    else pair_pass_s<false>(g, ntiles, cone, colour, shape, sub, s);
}

// The wavefront kernel takes more than the default 48 KB of dynamic shared
// memory: opt in once per instance.
template <int MEASURE>
bool wave_opt_in() {
    static const bool ok = cudaFuncSetAttribute(wave_sweep_kernel<MEASURE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                int(kWaveSmemBytes)) == cudaSuccess;
    return ok;
}

template <int MEASURE>
cudaError_t wave_sweep_t(const WaveArgs& a, uint32_t nblocks, const R* cone, int dir, cudaStream_t s) {
    if (!wave_opt_in<MEASURE>()) return cudaErrorInvalidConfiguration;
    // programmatic serialisation, as for the row passes
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nblocks);
    cfg.blockDim = dim3(kWaveThreads);
    cfg.dynamicSmemBytes = kWaveSmemBytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, wave_sweep_kernel<MEASURE>, a, cone, dir);
}

cudaError_t wave_sweep(const WaveArgs& a, uint32_t nblocks, const void* cone, int dir, int measure, cudaStream_t s) {
    const R* c = static_cast<const R*>(cone);
    if (measure >= 2) return wave_sweep_t<2>(a, nblocks, c, dir, s);
    if (measure == 1) return wave_sweep_t<1>(a, nblocks, c, dir, s);
    return wave_sweep_t<0>(a, nblocks, c, dir, s);
}

uint32_t wave_blocks() {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (wave_opt_in<0>())
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wave_sweep_kernel<0>, kWaveThreads, kWaveSmemBytes);
    if (per_sm < 1) per_sm = 1;
    return uint32_t(sms) * uint32_t(per_sm);
}

// Resident sweeps: shape 0 = blocks of 512 threads (16 warps, up to 128
// registers), 1 = 640 threads (20 warps, up to 96 registers; 768 threads
// would spill at 80); one block per SM, opted in to the shared memory of the
// largest brick.
template <int NT, int MEASURE>
bool resident_opt_in() {
    static const bool ok = [] {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        return cudaFuncSetAttribute(resident_sweep_kernel<NT, MEASURE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    optin - int(kResStaticSmem)) == cudaSuccess;
    }();
    return ok;
}

template <int NT, int MEASURE>
cudaError_t resident_t(const ResidentPlan& r, const ResidentArgs& a, const R* cone, cudaStream_t s) {
    if (!resident_opt_in<NT, MEASURE>()) return cudaErrorInvalidConfiguration;
    // cooperative: the launch fails rather than run with a block not resident,
    // since the blocks wait for one another at the grid barriers
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(uint32_t(a.nyc * a.nzc));
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = a.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, resident_sweep_kernel<NT, MEASURE>, a,
                              *reinterpret_cast<const CUtensorMap*>(r.map_y),
                              *reinterpret_cast<const CUtensorMap*>(r.map_z), cone);
}

template <int NT>
cudaError_t resident_m(const ResidentPlan& r, const ResidentArgs& a, const R* cone, int measure, cudaStream_t s) {
    if (measure >= 2) return resident_t<NT, 2>(r, a, cone, s);
    if (measure == 1) return resident_t<NT, 1>(r, a, cone, s);
    return resident_t<NT, 0>(r, a, cone, s);
}

// n sweeps in launches of at most kResMaxSweeps, each after its control
// words are zeroed
cudaError_t resident_sweeps(const ResidentPlan& r, const void* cone, int n, int measure, int shape, cudaStream_t s) {
    const R* c = static_cast<const R*>(cone);
    for (int done = 0; done < n;) {
        ResidentArgs a = r.args;
        a.n_sweeps = n - done < kResMaxSweeps ? n - done : kResMaxSweeps;
        cudaError_t e = cudaMemsetAsync(a.ctl, 0, sizeof(ResCtl), s);
        if (e == cudaSuccess)
            e = shape == 1 ? resident_m<640>(r, a, c, measure, s) : resident_m<512>(r, a, c, measure, s);
        if (e != cudaSuccess) return e;
        done += a.n_sweeps;
    }
    return cudaSuccess;
}

// cuTensorMapEncodeTiled, taken from the driver at run time (the library
// links the CUDA runtime only).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
    static const EncodeTiledFn fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<EncodeTiledFn>(f);
    }();
    return fn;
}

// The bricks of a resident lattice of Ly x Lz rows on the current device:
// the split (nyc, nzc) with the fewest rows in the largest brick, then the
// fewest halo rows, then the fewest blocks, among those with one block per
// SM at most whose brick fits a block's shared memory (both launch shapes
// must keep a block resident).  Then the tensor maps of the halo faces: the
// spins as a 64 x Ly x Lz x 6 array of floats (x, y, z, 3 colour + component;
// strides 256 B, 256 Ly B, 4 stride B).  False if no split fits or a map
// cannot be made.
bool resident_plan(const LatParams& p, ResidentPlan* r) {
    const int Ly = p.Ly, Lz = p.Lz;
    ResidentArgs* out = &r->args;
    int dev = 0, sms = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const long long cap = (long long)optin - (long long)kResStaticSmem;
    long long best[3] = {0, 0, 0};
    bool found = false;
    for (int nyc = 1; nyc <= Ly && nyc <= sms; ++nyc)
        for (int nzc = 1; nzc <= Lz && nyc * nzc <= sms && nyc * nzc <= kResMaxBlocks; ++nzc) {
            const int by = (Ly + nyc - 1) / nyc, bz = (Lz + nzc - 1) / nzc;
            if (by > 255 || bz > 255) continue;
            const uint32_t smem = resident_smem_bytes(by, bz, nyc, nzc);
            if ((long long)smem > cap) continue;
            const long long key[3] = {(long long)by * bz, (long long)resident_halo_rows(by, bz, nyc, nzc),
                                      (long long)nyc * nzc};
            if (!found || std::lexicographical_compare(key, key + 3, best, best + 3)) {
                found = true;
                std::copy(key, key + 3, best);
                *out = ResidentArgs{};
                out->nyc = nyc;
                out->nzc = nzc;
                out->by = by;
                out->bz = bz;
                out->smem = smem;
            }
        }
    if (!found) return false;
    int per_sm = 0;
    if (!resident_opt_in<512, 0>() || !resident_opt_in<640, 0>()) return false;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, resident_sweep_kernel<640, 0>, 640, out->smem);
    if (per_sm < 1) return false;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, resident_sweep_kernel<512, 0>, 512, out->smem);
    if (per_sm < 1) return false;
    const EncodeTiledFn enc = encode_tiled();
    if (!enc) return false;
    const cuuint64_t dim[4] = {cuuint64_t(kResLh), cuuint64_t(Ly), cuuint64_t(Lz), 6};
    const cuuint64_t strides[3] = {cuuint64_t(kResLh) * 4, cuuint64_t(kResLh) * 4 * cuuint64_t(Ly),
                                   cuuint64_t(p.stride) * 4};
    const cuuint32_t box_y[4] = {cuuint32_t(kResLh), 1, cuuint32_t(out->bz), 3};
    const cuuint32_t box_z[4] = {cuuint32_t(kResLh), cuuint32_t(out->by), 1, 3};
    const cuuint32_t unit[4] = {1, 1, 1, 1};
    for (int k = 0; k < 2; ++k) {
        const CUresult e = enc(reinterpret_cast<CUtensorMap*>(k == 0 ? r->map_y : r->map_z),
                               CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, p.spins, dim, strides, k == 0 ? box_y : box_z,
                               unit, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (e != CUDA_SUCCESS) return false;
    }
    return true;
}

void slab_export(LatDev* L, cudaStream_t s) { slab_export_kernel<<<1, 32, 0, s>>>(L); }

void slab_close(LatDev* L, int measure, cudaStream_t s) { slab_close_kernel<<<1, 32, 0, s>>>(L, measure); }

cudaError_t slab_halo(float* const (*dst)[2], const float* const (*src)[2], const uint32_t* stride,
                      const uint32_t (*src_stride)[2], uint32_t plane, int n, cudaStream_t s) {
    if (n < 1 || n > kMaxSlabs) return cudaErrorInvalidValue;
    SlabHaloArgs a{};
    for (int i = 0; i < n; ++i) {
        for (int k = 0; k < 2; ++k) {
            a.dst[i][k] = dst[i][k];
            a.src[i][k] = src[i][k];
            a.src_stride[i][k] = src_stride[i][k];
        }
        a.stride[i] = stride[i];
    }
    a.plane = plane;
    a.n = n;
    const uint32_t bx = (plane + 255) / 256;
    slab_halo_kernel<<<dim3(bx < 64 ? bx : 64, 2, uint32_t(n)), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t slab_close_all(LatDev* const* lats, int n, int measure, cudaStream_t s) {
    if (n < 1 || n > kMaxSlabs) return cudaErrorInvalidValue;
    SlabDevs d{};
    for (int i = 0; i < n; ++i) d.lat[i] = lats[i];
    d.n = n;
    slab_close_all_kernel<<<1, 32 * (n < 32 ? n : 32), 0, s>>>(d, measure);
    return cudaGetLastError();
}

}  // namespace

const KernelSet& kernels_f32() {
    static const KernelSet k{colour_pass, row_pass,    pair_pass,   sweep_end,         pair_field,
                             ml_reset,    mlong,       measure,     row_sample,        xtal_pass,
                             xtal_sample, xtal_field_launch, grain_sample, profile, "f32",
                             wave_sweep,  wave_blocks, slab_export,       slab_close,   slab_halo,
                             slab_close_all, resident_sweeps, resident_plan};
    return k;
}

}  // namespace mcgb
