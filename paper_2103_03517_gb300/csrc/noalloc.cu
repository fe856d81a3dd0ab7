// noalloc.cu -- mc_sweep_noalloc: FP32 sweeps of a caller-owned lattice with
// no device allocation.  The scratch the sweep kernels need (the lattice
// descriptor with its counters and fixed-point sums, the launch tables, the
// cone table and the per-sweep sample ring) lives in one file-scope device
// array of fixed size instead of memory obtained from cudaMalloc.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "runtime.h"

namespace mcgb {
namespace {

constexpr int kMaxSamples = 256;                     // samples one call can return
constexpr size_t kScratchBytes = 32 * 1024;          // the whole scratch array

// Layout of the scratch array (byte offsets, 256-aligned pieces).
constexpr size_t kOffLat = 0;
constexpr size_t kOffLats = 1024;                    // LatDev* [1]
constexpr size_t kOffStartSite = kOffLats + 256;     // uint32_t [2]
constexpr size_t kOffStartPair = kOffStartSite + 256;
constexpr size_t kOffCone = kOffStartPair + 256;     // float [181]
constexpr size_t kOffRing = kOffCone + 1024;         // double [kMaxSamples][kRingWords]
constexpr size_t kUsed = kOffRing + size_t(kMaxSamples) * kRingWords * sizeof(double);
static_assert(sizeof(LatDev) <= kOffLats, "lattice descriptor does not fit its scratch slot");
static_assert(kUsed <= kScratchBytes, "scratch layout exceeds the array");

// Shared by every call on a device; contents persist from call to call.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch in the current device's context (in host code
// the name is only a stand-in).  Looked up on every call: the lookup
// allocates nothing and is cheap once the module is loaded, and an address
// kept from an earlier context would dangle after cudaDeviceReset.  The
// first call on a device loads the module, so it belongs before any stream
// capture.
int scratch_address(char** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
    *out = static_cast<char*>(p);
    return MC_OK;
}

}  // namespace
}  // namespace mcgb

using namespace mcgb;

extern "C" MC_API int mc_sweep_noalloc(float* spins, const int dims[3], double J, double K_u, const double axis[3],
                                       double K_c, const double H[3], double T, uint64_t seed, int64_t first_sweep,
                                       int n_sweeps, int* theta_deg, double* samples, void* stream) {
    if (!spins || !dims || !axis || !H || !theta_deg) return fail(MC_ERR_ARG, "null argument");
    if (n_sweeps < 0) return fail(MC_ERR_ARG, "n_sweeps < 0");
    if (samples && n_sweeps > kMaxSamples)
        return fail(MC_ERR_ARG, "n_sweeps %d exceeds the %d samples the no-allocation scratch holds per call",
                    n_sweeps, kMaxSamples);
    if (first_sweep < 0 || first_sweep + n_sweeps > int64_t(UINT32_MAX))
        return fail(MC_ERR_ARG, "sweep counter out of range");
    if (*theta_deg < 1 || *theta_deg > 180) return fail(MC_ERR_ARG, "theta must be in 1..180");
    mc_desc d;
    mc_desc_default(&d);
    for (int a = 0; a < 3; ++a) { d.dims[a] = dims[a]; d.axis[a] = axis[a]; d.H[a] = H[a]; }
    d.J = J; d.K_u = K_u; d.K_c = K_c; d.T = T; d.seed = seed;
    d.theta0_deg = *theta_deg;
    int rc = validate_desc(&d);
    if (rc) return rc;
    if (n_sweeps == 0) return MC_OK;

    char* base = nullptr;
    rc = scratch_address(&base);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // the lattice descriptor, parameters as in mc_create, state cleared
    LatDev host;
    std::memset(&host, 0, sizeof host);
    LatParams& p = host.p;
    p.Lx = dims[0]; p.Ly = dims[1]; p.Lz = dims[2]; p.Lh = p.Lx / 2;
    p.precision = MC_FP32;
    p.N = (long long)p.Lx * p.Ly * p.Lz;
    p.Nc = uint32_t(p.N / 2);
    p.stride = (p.Nc + 63) / 64 * 64;
    p.n_pairs = p.Nc / 2;
    p.n_mov = p.N;
    p.adapt_in_measure = 1;
    p.key0 = uint32_t(seed);
    p.key1 = uint32_t(seed >> 32);
    p.div_lh = make_fastdiv(uint32_t(p.Lh));
    p.div_ly = make_fastdiv(uint32_t(p.Ly));
    const uint32_t site_tile = uint32_t(32 * sites_per_thread(MC_FP32));
    p.nblocks_site = (p.Nc + site_tile - 1) / site_tile;
    p.nblocks_pair = (p.n_pairs + 31) / 32 > 0 ? (p.n_pairs + 31) / 32 : 1;
    p.sample_torque = 1;
    p.row_fast = row_fast(p, false);
    p.colour_kernel = colour_kernel(p, false, MC_PATH_AUTO);
    p.row_lanes = p.Lh / 2 < 32 ? (p.Lh / 2 > 0 ? p.Lh / 2 : 1) : 32;
    p.spins = spins;
    p.ring = reinterpret_cast<double*>(base + kOffRing);
    p.ring_cap = kMaxSamples;
    p.J = J; p.Ku = K_u; p.Kc = K_c; p.T = T;
    const double an = std::sqrt(axis[0] * axis[0] + axis[1] * axis[1] + axis[2] * axis[2]);
    for (int a = 0; a < 3; ++a) { p.e[a] = axis[a] / an; p.H[a] = H[a]; }
    p.fJ = (float)p.J; p.fKu = (float)p.Ku; p.fKc = (float)p.Kc; p.fT = (float)p.T;
    p.fBeta2 = (float)(-1.4426950408889634 / p.T);  // log2(e) = 1 / ln 2
    for (int a = 0; a < 3; ++a) { p.fe[a] = (float)p.e[a]; p.fH[a] = (float)p.H[a]; }
    host.st.theta = *theta_deg;
    host.st.sweep = uint32_t(first_sweep);

    LatDev* d_lat = reinterpret_cast<LatDev*>(base + kOffLat);
    const uint32_t starts[4] = {0, p.nblocks_site, 0, p.nblocks_pair};
    float cone[181];
    for (int deg = 0; deg <= 180; ++deg) {
        const double h = std::sin((double)deg * (M_PI / 360.0));
        cone[deg] = (float)(2.0 * (h * h));
    }
    cudaError_t e = cudaMemcpyAsync(d_lat, &host, sizeof host, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + kOffLats, &d_lat, sizeof d_lat, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + kOffStartSite, starts, 2 * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + kOffStartPair, starts + 2, 2 * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + kOffCone, cone, sizeof cone, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "no-allocation scratch set-up");

    LaunchSet ls;
    ls.all = GroupArgs{reinterpret_cast<LatDev* const*>(base + kOffLats),
                       reinterpret_cast<const uint32_t*>(base + kOffStartSite), 1};
    ls.pairs = GroupArgs{ls.all.lats, reinterpret_cast<const uint32_t*>(base + kOffStartPair), 1};
    ls.nt_all = p.nblocks_site;
    ls.nt_pairs = p.nblocks_pair;
    ls.sample_level = 2;
    if (p.colour_kernel == kColourRow) {  // every axis periodic: the row kernel or the general one
        ls.row = ls.all;
        ls.nt_row = ls.nt_all;
    } else {
        ls.rest = ls.all;
        ls.nt_rest = ls.nt_all;
    }
    rc = enqueue_sweeps(kernels_f32(), ls, base + kOffCone, n_sweeps, samples ? 1 : 0, false, s, nullptr);
    if (rc) return rc;
    if (samples) {
        e = cudaMemcpyAsync(samples, base + kOffRing, size_t(n_sweeps) * kRingWords * sizeof(double),
                            cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "copy of the samples");
    }
    int theta = 0;
    e = cudaMemcpyAsync(&theta, &d_lat->st.theta, sizeof theta, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "no-allocation sweep");
    *theta_deg = theta;
    return MC_OK;
}
