// mc_internal.h -- device-resident lattice descriptor shared by the host
// runtime and the kernels of libmc.
//
// Spin layout in HBM (both precisions): colour-split structure of arrays.
// Colour c = (x + y + z) mod 2 (0 = red, Sec. 2 checkerboard).  A site
// (x, y, z) of colour c has the colour index q = (x >> 1) + Lh (y + Ly z),
// Lh = Lx / 2, and component a of its spin lives at
//     spins[(3 c + a) * stride + q],   stride = Nc rounded up to 64.
// In row (y, z) the colour-c sites sit at x = ((y + z + c) & 1) + 2k, so the
// other colour's -x / +x neighbours of (k, y, z) are colour indices
// k + xoff - 1 and k + xoff in the same row, and the -y/+y/-z/+z neighbours
// share k in the adjacent rows.
#pragma once
#include <stdint.h>

namespace mcgb {

constexpr int kBlock = 256;          // threads per block of every pass kernel
// Sites per thread per tile of the site kernels (a site tile is kBlock * V
// colour indices of one lattice; a pair tile is kBlock pairs).
#ifndef MC_V_F32
#define MC_V_F32 2
#endif
constexpr int kSitesPerThreadF32 = MC_V_F32;   // a warp tile is 32 * V colour indices
constexpr int kSitesPerThreadF64 = 1;
constexpr int sites_per_thread(int precision) { return precision == 1 ? kSitesPerThreadF64 : kSitesPerThreadF32; }
constexpr int kNumSums = 12;         // per-sample lattice sums, see kSum*
constexpr int kRingWords = 14;       // doubles per ring sample
constexpr int kSlabWords = 16;       // slab count words: accepted, n_mov, N, the kNumSums sums
constexpr int kMomentWords = 26;     // running sums of per-sample observables
constexpr double kFixScale = 268435456.0;   // 2^28: fixed point of the FP64 sums
constexpr double kFixScaleF32 = 4194304.0;  // 2^22: fixed point of the FP32 sums

// Per-sample lattice sums (dimensionless, each bounded by 3 N):
enum {
    kSumMx = 0, kSumMy, kSumMz,      // sum S
    kSumEx,                          // sum over bonds S_i.S_j
    kSumU,                           // sum (S.e)^2
    kSumC,                           // sum Sx^2Sy^2 + Sx^2Sz^2 + Sy^2Sz^2
    kSumTux, kSumTuy, kSumTuz,       // sum (S.e)(S x e)
    kSumTcx, kSumTcy, kSumTcz        // sum S x c(S)
};

// Moment words (running sums over samples), same order as the oracle.
enum {
    kMomN = 0, kMomM = 1, kMomM2 = 4, kMomMabs = 7, kMomMl = 10, kMomMl2 = 11,
    kMomMl4 = 12, kMomE = 13, kMomE2 = 14, kMomParts = 15, kMomTq = 19, kMomTq2 = 22
};

// Unsigned 32-bit division by a runtime constant with a multiply
// (Granlund & Montgomery, PLDI 1994; round-up variant with the 33-bit
// correction of Hacker's Delight ch. 10): exact for every n < 2^32.
struct FastDiv {
    uint32_t d, mul, s1, s2;
};

inline FastDiv make_fastdiv(uint32_t d) {
    uint32_t l = 0;
    while ((uint64_t(1) << l) < d) ++l;
    FastDiv f;
    f.d = d;
    f.mul = uint32_t(((uint64_t(1) << 32) * ((uint64_t(1) << l) - d)) / d + 1);
    f.s1 = l > 0 ? 1 : 0;
    f.s2 = l > 0 ? l - 1 : 0;
    return f;
}

enum { kColourGeneral = 0, kColourRow = 1, kColourRowGen = 2 };

// One neighbour entry of a bcc / fcc / hcp sub-lattice: the neighbour's
// sub-lattice, its cell offset and its coupling (J1 or J2), with what the
// kernels need precomputed for the lattice's size: the offset taken modulo
// (Lx, Ly, Lz), the parity of dx + dy + dz (bit 0 of par; bit 1 marks a
// forward entry, one of each entry and its reverse), and for a site of
// colour c the element offset of the neighbour's x-component array.
constexpr int kXtalMaxSub = 4, kXtalMaxNb = 24;
struct XtalNb {
    int8_t sub, dx, dy, dz;
    float fJ;
    double J;
    uint32_t dxw, dyw, dzw, par;
    uint64_t off[2];
};

struct LatParams {
    int Lx, Ly, Lz, Lh;
    int bc[3];
    int precision;
    uint32_t Nc;            // sites per colour (and sub-lattice) = cells / 2
    uint32_t stride;        // Nc rounded up to 64
    uint32_t n_pairs;       // Nc / 2
    int perm_bits;          // Feistel word width b (domain 2^b >= Nc, b >= 1)
    long long N, n_mov;
    int adapt_in_measure;
    uint32_t key0, key1;
    FastDiv div_lh, div_ly;
    uint32_t nblocks_site;  // site tiles of this lattice
    uint32_t nblocks_pair;  // pair tiles of this lattice
    int sample_torque;      // measured sweeps also sum the torques
    int row_fast;           // all axes periodic and no film tables, and (FP64)
                            // Lh % 32 == 0, or (FP32) Lh a power of two <= 64 or a
                            // multiple of 64, Nc % 64 == 0: the row paths apply
    int row_lanes;          // FP32 row path: lanes per row group, min(Lh/2, 32)
    int nsub;               // sub-lattices: 1 simple cubic, 2 bcc, 4 fcc
    int pair_leader;        // constrained pass in site order (FP32, automatic kernel path)
    int xnb_n[kXtalMaxSub]; // bcc / fcc: neighbour entries per sub-lattice
    const void* xnb;        // bcc / fcc: [kXtalMaxSub][kXtalMaxNb] XtalNb, or null
    int colour_kernel;      // colour-pass kernel: kColourGeneral, kColourRow (FP32 row
                            // layout, all axes periodic, no film tables) or
                            // kColourRowGen (FP32 row layout, any boundaries and films)
    void* spins;
    void* spins_alt;        // wavefront lattices (wave != 0): the second spin buffer
                            // a fused sweep writes (same layout), else null
    int wave;               // FP32 all-periodic lattice of rows of Lh = 64 sites per
                            // colour and Ly a multiple of 16: its sweeps may run as
                            // one wavefront launch (wave_sweep_kernel)
    void* rctl;             // resident lattices: their ResCtl, else null
    const uint8_t* bonds;   // [2][stride] or null
    const int32_t* grain;   // [2][stride] or null
    const void* gaxis;      // [n_grains][4] in the lattice precision, or null
    double* ring;           // [ring_cap][kRingWords]
    int ring_cap;
    long long* profile;     // [3][Lx] fixed-point sums
    int n_grains;           // films: grains of the grain table (0 without one)
    long long* gsum;        // films: [n_grains][3] fixed-point spin sums of one grain sample
    const int32_t* gsize;   // films: [n_grains] spins per grain
    double* gacc;           // films: [n_grains + 1] sums over grain samples of |m_g|, then the count
    void* aos;              // constrained sweeps: [2 nsub][stride] (x, y, z, 0) copy of the
                            // spins (Spin4), written by mlong_kernel at the start of a run
                            // of constrained sweeps and kept in step by the pair passes;
                            // null until the lattice's first constrained sweep
    void* pfield;           // constrained sweeps: [stride] (h_x, h_y, h_z, 0) neighbour
                            // field of every site of the colour being updated, written by
                            // pair_field_kernel before each pair pass
    int slab;               // a z slab of a larger lattice (mc_slab_create): planes 0 and
                            // Lz - 1 are halo copies of the neighbouring slabs' planes,
                            // pinned and left out of the sample; passes never close
                            // the sweep (mc_slab_close does, from counts summed over slabs)
    int cflip;              // slab: global colour = local colour ^ cflip (the parity of
                            // the global plane under local plane 0)
    uint32_t site_off;      // slab: global site index - local site index (mod 2^32)
    long long* slab_counts; // slab: [kSlabWords] accepted, n_mov, N and the sums of the
                            // slab's own planes, exported by a pass for the sum over slabs
    double J, Ku, e[3], Kc, H[3], T;
    float fJ, fKu, fe[3], fKc, fH[3], fT;
    float fBeta2;           // FP32 Metropolis test: -log2(e) / T, so exp(-dE/T) = 2^(dE fBeta2)
    double R[9];            // constraint frame rows e1 = e_C, e2, e3
    float fR[9];
};

struct LatState {
    unsigned long long acc;         // accepted moves in the current sweep
    unsigned int done[4];           // finished blocks: red, black, M_L, measure
    int theta;                      // cone half-angle, degrees
    uint32_t sweep;                 // sweeps completed
    int error;                      // sticky mc_status
    int pad;
    long long last_acc;
    long long sums[kNumSums];       // fixed-point lattice sums of this sample
    long long ml_hi, ml_lo;         // exact M_L of this constrained sweep
    long long dml_hi, dml_lo;       // its change by this sweep's accepted pairs, carried
                                    // into ml_hi / ml_lo when the sweep ends
    long long ring_count;
    long long prof_samples;
    double moments[kMomentWords];
};

struct LatDev {
    LatParams p;
    LatState st;
};

// Arguments of a batched launch: lattice l owns tiles [start[l], start[l+1]).
struct GroupArgs {
    LatDev* const* lats;
    const uint32_t* start;
    int n;
};

// Wavefront sweep (wave_pass.cuh): lattices with rows of kWaveLh colour
// indices (Lx = 128) and Ly >= kWaveMinLy, cut into bands of at most
// kWaveTyMax rows and slabs of planes (work units).
constexpr int kWaveLh = 64;
constexpr int kWaveTyMax = 15;
constexpr int kWaveMinLy = 16;

// A work unit: band [y0, y0 + ty) x slab [z0, z0 + tz) of lattice `lat` (an
// index into WaveArgs::lats), full rows in x.
struct WaveWU {
    uint32_t lat, y0, z0, tz, ty, pad;
};

// Arguments of a wavefront launch: block b runs work units [off[b],
// off[b + 1]); lattice l has nwu[l] units in all, and the block finishing
// its last one closes its sweep.  inject: extra bytes expected by the
// first staged copy of block 0 (0 in normal runs; a host-set fault that
// makes that wait run out).
struct WaveArgs {
    LatDev* const* lats;
    const WaveWU* wu;
    const uint32_t* off;
    const uint32_t* nwu;
    int n;
    int inject;
};

// Resident sweeps (resident_pass.cuh): a lattice with rows of kResLh colour
// indices (Lx = 128) held in the shared memory of one block per brick of
// rows for a whole run of sweeps.
constexpr int kResLh = 64;
constexpr int kResMaxSweeps = 2048;  // sweeps per launch; longer runs take several

// Control words of one lattice's resident launch, in device memory, zeroed
// before every launch: the abort flag a block sets when one of its waits
// runs out; for sweep s, in slot s mod 3 (one slot fills, one is read, one
// is cleared), the blocks that have completed their black pass (high 32
// bits) and their accepted moves (low 32 bits) in one word, and the
// fixed-point sample sums; per block, the passes whose face rows it has
// written.
constexpr int kResMaxBlocks = 256;
constexpr int kResSlots = 3;
struct ResCtl {
    int abort;
    int pad;
    unsigned long long arrive_acc[kResSlots];
    long long sums[kResSlots][kNumSums];
    unsigned int done[kResMaxBlocks];
};

// A resident launch: nyc x nzc blocks, block b holding the rows [y0, y1) x
// [z0, z1) of its brick (y split into nyc near-equal parts, z into nzc);
// by, bz = the largest brick extents, which size the shared memory (smem
// bytes per block); n_sweeps sweeps; inject: an extra arrival the wait for a
// sweep's counts expects (0 in normal runs; a host-set fault that makes
// that wait run out).
struct ResidentArgs {
    LatDev* lat;
    ResCtl* ctl;
    int nyc, nzc, by, bz;
    uint32_t smem;
    int n_sweeps;
    int inject;
    uint32_t key0, key1;  // the lattice's Philox key, a launch constant
};

}  // namespace mcgb
