// runtime.cpp -- lattices, groups, observables and checkpoints of libmc
// (the C ABI of include/mc.h, except the server).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <queue>
#include <string>
#include <vector>

#include "kernels.h"
#include "mc.h"
#include "mc_internal.h"
#include "runtime.h"

namespace mcgb {

// ----------------------------------------------------------------- errors
static thread_local std::string g_error;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_error = buf;
    return code;
}

// MC_TRACE=1 in the environment prints the stages of lattice creation.
static void trace(const char* what) {
    static const int on = [] {
        const char* v = std::getenv("MC_TRACE");
        return v && v[0] == '1';
    }();
    if (on) {
        std::fprintf(stderr, "[libmc] %s\n", what);
        std::fflush(stderr);
    }
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? MC_ERR_NOMEM : MC_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
    } while (0)

// ------------------------------------------------------ per-device tables
// c(theta) = 1 - cos(theta) = 2 sin^2(theta / 2) for integer degrees (cone
// half-angle of Table A1), in both precisions, computed on the host.
struct DeviceTables {
    double* cone64 = nullptr;
    float* cone32 = nullptr;
};

static std::mutex g_tables_mu;
static std::vector<DeviceTables> g_tables;

int device_tables(int device, const double** c64, const float** c32) {
    std::lock_guard<std::mutex> lk(g_tables_mu);
    if ((int)g_tables.size() <= device) g_tables.resize(device + 1);
    DeviceTables& t = g_tables[device];
    if (!t.cone64) {
        double h64[181];
        float h32[181];
        for (int d = 0; d <= 180; ++d) {
            const double s = std::sin((double)d * (M_PI / 360.0));
            h64[d] = 2.0 * (s * s);
            h32[d] = (float)h64[d];
        }
        CK(cudaMalloc(&t.cone64, sizeof h64));
        CK(cudaMalloc(&t.cone32, sizeof h32));
        CK(cudaMemcpy(t.cone64, h64, sizeof h64, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(t.cone32, h32, sizeof h32, cudaMemcpyHostToDevice));
    }
    *c64 = t.cone64;
    *c32 = t.cone32;
    return MC_OK;
}

// Constraint frame of Table A2 (x-axis along e_C): rows e1 = e_C,
// e2 = (-sin phi, cos phi, 0), e3 = e1 x e2.
void constraint_frame(double theta_deg, double phi_deg, double R[9]) {
    const double th = theta_deg * (M_PI / 180.0), ph = phi_deg * (M_PI / 180.0);
    const double st = std::sin(th), ct = std::cos(th), sp = std::sin(ph), cp = std::cos(ph);
    R[0] = st * cp;  R[1] = st * sp;  R[2] = ct;
    R[3] = -sp;      R[4] = cp;       R[5] = 0.0;
    R[6] = -ct * cp; R[7] = -ct * sp; R[8] = st;
}

static int feistel_bits(uint32_t n) {
    int b = 1;
    while ((uint64_t(1) << b) < uint64_t(n)) ++b;
    return b;
}

static size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// FP32 row layout: rows of Lh sites per colour split evenly over the lanes
// of a 64-site tile (Lh a power of two <= 64, or a multiple of 64) and
// whole tiles (Nc % 64 == 0).
static bool row_layout(const LatParams& p) {
    const bool pow2_small = p.Lh >= 2 && p.Lh <= 64 && (p.Lh & (p.Lh - 1)) == 0;
    const bool long_rows = p.Lh % 64 == 0;
    return (pow2_small || long_rows) && p.Nc % 64 == 0;
}

// Whether a lattice takes the periodic row paths (see LatParams).
int row_fast(const LatParams& p, bool film) {
    if (film || p.bc[0] != MC_PERIODIC || p.bc[1] != MC_PERIODIC || p.bc[2] != MC_PERIODIC) return 0;
    if (p.precision == MC_FP64) return p.Lh % 32 == 0 ? 1 : 0;
    return row_layout(p) ? 1 : 0;
}

// Colour-pass kernel of a lattice (LatParams::colour_kernel).
int colour_kernel(const LatParams& p, bool film, int path) {
    if (p.precision != MC_FP32 || path == MC_PATH_GENERAL || !row_layout(p)) return kColourGeneral;
    return row_fast(p, film) ? kColourRow : kColourRowGen;
}

// ------------------------------------------------------------- lattices
static void set_float_params(LatParams& p) {
    p.fJ = (float)p.J; p.fKu = (float)p.Ku; p.fKc = (float)p.Kc; p.fT = (float)p.T;
    p.fBeta2 = (float)(-1.4426950408889634 / p.T);  // log2(e) = 1 / ln 2
    for (int a = 0; a < 3; ++a) { p.fe[a] = (float)p.e[a]; p.fH[a] = (float)p.H[a]; }
    for (int a = 0; a < 9; ++a) p.fR[a] = (float)p.R[a];
}

int sublattices(int lattice) { return lattice == MC_BCC ? 2 : (lattice == MC_FCC || lattice == MC_HCP ? 4 : 1); }

// Neighbour table of a bcc, fcc or hcp lattice from its basis (fractions of
// the cell; cell lengths ell, a = 1): entry (t, d) of sub-lattice s, d a
// cell offset in {-1, 0, 1}^3, is a neighbour when |(b_t + d - b_s) ell|^2
// equals the nearest-neighbour distance^2 (bcc 3/4, fcc 1/2, hcp 1;
// coupling J) or, for bcc and fcc with J2 != 0, 1 (the same sub-lattice one
// cell away; coupling J2).  Entries are ordered by t, then d_z, d_y, d_x
// from -1 to 1: the order in which the field is summed.  hcp: the
// orthohexagonal cell (1, sqrt 3, sqrt(8/3)) with sub-lattices (0,0,0),
// (1/2,1/2,0), (1/2,1/6,1/2), (0,2/3,1/2).
static void xtal_table(int lattice, double J, double J2, const LatParams& p, XtalNb out[kXtalMaxSub][kXtalMaxNb],
                       int n[kXtalMaxSub]) {
    const double bcc[2][3] = {{0, 0, 0}, {0.5, 0.5, 0.5}};
    const double fcc[4][3] = {{0, 0, 0}, {0.5, 0.5, 0}, {0.5, 0, 0.5}, {0, 0.5, 0.5}};
    const double hcp[4][3] = {{0, 0, 0}, {0.5, 0.5, 0}, {0.5, 1.0 / 6.0, 0.5}, {0, 2.0 / 3.0, 0.5}};
    const int ns = sublattices(lattice);
    const double(*b)[3] = lattice == MC_BCC ? bcc : (lattice == MC_FCC ? fcc : hcp);
    const double ell[3] = {1.0, lattice == MC_HCP ? std::sqrt(3.0) : 1.0, lattice == MC_HCP ? std::sqrt(8.0 / 3.0) : 1.0};
    const double nn2 = lattice == MC_BCC ? 0.75 : (lattice == MC_FCC ? 0.5 : 1.0);
    const bool with_j2 = lattice != MC_HCP && J2 != 0.0;
    for (int s = 0; s < ns; ++s) {
        n[s] = 0;
        for (int t = 0; t < ns; ++t)
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const double r[3] = {(b[t][0] + dx - b[s][0]) * ell[0], (b[t][1] + dy - b[s][1]) * ell[1],
                                             (b[t][2] + dz - b[s][2]) * ell[2]};
                        const double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
                        const bool nn = std::fabs(r2 - nn2) < 1e-9, nnn = with_j2 && std::fabs(r2 - 1.0) < 1e-9;
                        if (!nn && !nnn) continue;
                        XtalNb& e = out[s][n[s]++];
                        e.sub = int8_t(t);
                        e.dx = int8_t(dx);
                        e.dy = int8_t(dy);
                        e.dz = int8_t(dz);
                        e.J = nn ? J : J2;
                        e.fJ = float(e.J);
                        e.dxw = uint32_t((dx + p.Lx) % p.Lx);
                        e.dyw = uint32_t((dy + p.Ly) % p.Ly);
                        e.dzw = uint32_t((dz + p.Lz) % p.Lz);
                        e.par = uint32_t(dx + dy + dz + 4) & 1u;  // + 4 keeps the sum non-negative, parity unchanged
                        for (int c = 0; c < 2; ++c)
                            e.off[c] = (uint64_t(t) * 2 + ((uint32_t(c) + e.par) & 1u)) * 3 * uint64_t(p.stride);
                        // forward entries (bit 1): one of each entry and its reverse
                        // (sub-lattice t -> s, offset -d), so that summing S_i.S_j over
                        // them sees every bond once
                        const bool fwd = t > s || (t == s && (dz > 0 || (dz == 0 && (dy > 0 || (dy == 0 && dx > 0)))));
                        e.par |= fwd ? 2u : 0u;
                    }
    }
}

// Lattices whose sweeps may run as wavefront launches (wave_pass.cuh):
// FP32 simple cubic, every axis periodic, no film tables, rows of 64 sites
// per colour (Lx = 128), Ly >= 16, the wavefront kernel path asked for.
bool wave_desc(const mc_desc* d) {
    if (d->precision != MC_FP32 || d->lattice != MC_SC || d->kernel_path != MC_PATH_WAVE) return false;
    if (d->bond_mask || d->grain_id) return false;
    for (int a = 0; a < 3; ++a)
        if (d->boundary[a] != MC_PERIODIC) return false;
    return d->dims[0] == 2 * kWaveLh && d->dims[1] >= kWaveMinLy;
}

// Lattices whose sweeps may run held in shared memory (resident_pass.cuh):
// FP32 simple cubic, every axis periodic, no film tables, rows of 64 sites
// per colour (Lx = 128), not a slab, the automatic or resident kernel path;
// whether its rows fit is decided on the device (KernelSet::resident_plan).
bool resident_desc(const mc_desc* d, bool slab) {
    if (slab || d->precision != MC_FP32 || d->lattice != MC_SC) return false;
    if (d->kernel_path != MC_PATH_AUTO && d->kernel_path != MC_PATH_RESIDENT) return false;
    if (d->bond_mask || d->grain_id) return false;
    for (int a = 0; a < 3; ++a)
        if (d->boundary[a] != MC_PERIODIC) return false;
    return d->dims[0] == 2 * kResLh;
}

size_t lattice_bytes(const mc_desc* d, bool slab) {
    const uint64_t cells = uint64_t(d->dims[0]) * d->dims[1] * d->dims[2];
    const uint64_t Nc = cells / 2;
    const uint64_t stride = (Nc + 63) / 64 * 64;
    const size_t rs = d->precision == MC_FP64 ? 8 : 4;
    const int nsub = sublattices(d->lattice);
    size_t b = align256(sizeof(LatDev));
    b += align256(size_t(nsub) * 6 * stride * rs);
    if (wave_desc(d)) b += align256(6 * stride * rs);  // the second spin buffer
    if (nsub > 1) b += align256(sizeof(XtalNb) * kXtalMaxSub * kXtalMaxNb);
    if (d->bond_mask) b += align256(2 * stride);
    if (d->grain_id) {
        const size_t ng = size_t(std::max(d->n_grains, 1));
        b += align256(2 * stride * 4) + align256(4 * ng * rs);
        b += align256(3 * ng * 8) + align256(ng * 4) + align256((ng + 1) * 8);  // grain samples
    }
    const int cap = d->ring_capacity > 0 ? d->ring_capacity : 4096;
    b += align256(size_t(cap) * kRingWords * 8);
    b += align256(3 * size_t(d->dims[0]) * 8);
    // launch tables of the lattice alone: lattice pointer, site and pair starts
    b += align256(sizeof(void*)) + 2 * align256(2 * sizeof(uint32_t));
    if (slab) b += align256(kSlabWords * 8);
    if (resident_desc(d, slab)) b += align256(sizeof(ResCtl));
    return b;
}

int validate_desc(const mc_desc* d) {
    for (int a = 0; a < 3; ++a) {
        if (d->dims[a] < 1) return fail(MC_ERR_ARG, "dims[%d] = %d < 1", a, d->dims[a]);
        if (d->boundary[a] < 0 || d->boundary[a] > 3) return fail(MC_ERR_ARG, "boundary[%d] invalid", a);
        if ((d->boundary[a] == MC_PERIODIC || d->boundary[a] == MC_ANTIPERIODIC) && (d->dims[a] % 2))
            return fail(MC_ERR_ARG, "periodic axis %d has odd size %d (breaks the two-colouring)", a, d->dims[a]);
    }
    if (d->dims[0] % 2) return fail(MC_ERR_ARG, "Lx = %d must be even", d->dims[0]);
    const uint64_t N = uint64_t(d->dims[0]) * d->dims[1] * d->dims[2];
    if (N >= (uint64_t(1) << 32)) return fail(MC_ERR_ARG, "N = %llu spins exceeds 2^32 - 1", (unsigned long long)N);
    if (!(d->T > 0.0) || !std::isfinite(d->T)) return fail(MC_ERR_ARG, "T must be > 0");
    const double an = std::sqrt(d->axis[0] * d->axis[0] + d->axis[1] * d->axis[1] + d->axis[2] * d->axis[2]);
    if (!(an > 0.0)) return fail(MC_ERR_ARG, "|axis| = 0");
    if (d->precision != MC_FP32 && d->precision != MC_FP64) return fail(MC_ERR_ARG, "precision invalid");
    if (d->lattice < MC_SC || d->lattice > MC_HCP) return fail(MC_ERR_ARG, "lattice invalid");
    if (d->lattice == MC_HCP && d->J2 != 0.0) return fail(MC_ERR_ARG, "hcp lattices take J2 = 0");
    if (d->lattice != MC_SC) {
        for (int a = 0; a < 3; ++a)
            if (d->boundary[a] != MC_PERIODIC) return fail(MC_ERR_ARG, "bcc / fcc / hcp lattices need periodic cells");
        if (d->bond_mask || d->grain_id) return fail(MC_ERR_ARG, "bcc / fcc / hcp lattices take no film tables");
        if (!std::isfinite(d->J2)) return fail(MC_ERR_ARG, "J2 not finite");
    }
    if (d->kernel_path < MC_PATH_AUTO || d->kernel_path > MC_PATH_RESIDENT)
        return fail(MC_ERR_ARG, "kernel_path invalid");
    if (d->theta0_deg < 1 || d->theta0_deg > 180) return fail(MC_ERR_ARG, "theta0 must be in 1..180");
    if (d->init != MC_INIT_UNIFORM && d->init != MC_INIT_WALL) return fail(MC_ERR_ARG, "init invalid");
    if (d->init == MC_INIT_UNIFORM) {
        const double n = std::sqrt(d->init_dir[0] * d->init_dir[0] + d->init_dir[1] * d->init_dir[1] +
                                   d->init_dir[2] * d->init_dir[2]);
        if (!(n > 0.0)) return fail(MC_ERR_ARG, "|init_dir| = 0");
    }
    if (d->grain_id && (!d->grain_axis || d->n_grains < 1)) return fail(MC_ERR_ARG, "grain tables incomplete");
    if (d->grain_id)
        for (uint64_t i = 0; i < N; ++i)
            if (d->grain_id[i] < 0 || d->grain_id[i] >= d->n_grains) return fail(MC_ERR_ARG, "grain id out of range");
    if (d->bond_mask) {
        // every bond must be present from both ends
        const int L[3] = {d->dims[0], d->dims[1], d->dims[2]};
        for (int z = 0; z < L[2]; ++z)
            for (int y = 0; y < L[1]; ++y)
                for (int x = 0; x < L[0]; ++x) {
                    const uint64_t i = x + uint64_t(L[0]) * (y + uint64_t(L[1]) * z);
                    const int c[3] = {x, y, z};
                    for (int ax = 0; ax < 3; ++ax) {
                        int cc[3] = {c[0], c[1], c[2]};
                        if (cc[ax] + 1 >= L[ax] && d->boundary[ax] != MC_PERIODIC &&
                            d->boundary[ax] != MC_ANTIPERIODIC)
                            continue;
                        cc[ax] = (cc[ax] + 1) % L[ax];
                        const uint64_t j = cc[0] + uint64_t(L[0]) * (cc[1] + uint64_t(L[1]) * cc[2]);
                        const int fwd = (d->bond_mask[i] >> (2 * ax + 1)) & 1;
                        const int bwd = (d->bond_mask[j] >> (2 * ax)) & 1;
                        if (fwd != bwd) return fail(MC_ERR_ARG, "bond mask not symmetric at site %llu", (unsigned long long)i);
                    }
                }
    }
    return MC_OK;
}

// Site i = s + nsub (x + Lx (y + Ly z)) <-> component a of sub-lattice s,
// colour c = (x + y + z) & 1, index q = (x >> 1) + Lh (y + Ly z) at
// ((2 s + c) 3 + a) stride + q (nsub = 1: the simple cubic layout).
template <typename R, typename F>
static void for_each_site(const LatParams& p, F&& f) {
    for (int z = 0; z < p.Lz; ++z)
        for (int y = 0; y < p.Ly; ++y)
            for (int x = 0; x < p.Lx; ++x)
                for (int s = 0; s < p.nsub; ++s) {
                    const size_t i = size_t(s) + size_t(p.nsub) * (x + size_t(p.Lx) * (y + size_t(p.Ly) * z));
                    const int c = (x + y + z) & 1;
                    const size_t q = size_t(x >> 1) + size_t(p.Lh) * (y + size_t(p.Ly) * z);
                    f(i, (size_t(s) * 2 + c) * 3 * size_t(p.stride) + q);
                }
}

template <typename R>
static void to_device_layout(const LatParams& p, const double* xyz, R* out) {
    for_each_site<R>(p, [&](size_t i, size_t o) {
        for (int a = 0; a < 3; ++a) out[o + a * size_t(p.stride)] = (R)xyz[3 * i + a];
    });
}

template <typename R>
static void from_device_layout(const LatParams& p, const R* in, double* xyz) {
    for_each_site<R>(p, [&](size_t i, size_t o) {
        for (int a = 0; a < 3; ++a) xyz[3 * i + a] = (double)in[o + a * size_t(p.stride)];
    });
}

static void per_site_colour_split(const LatParams& p, const void* src, size_t elem, void* dst) {
    for (int z = 0; z < p.Lz; ++z)
        for (int y = 0; y < p.Ly; ++y)
            for (int x = 0; x < p.Lx; ++x) {
                const size_t i = x + size_t(p.Lx) * (y + size_t(p.Ly) * z);
                const int c = (x + y + z) & 1;
                const size_t q = size_t(x >> 1) + size_t(p.Lh) * (y + size_t(p.Ly) * z);
                std::memcpy(static_cast<char*>(dst) + (c * size_t(p.stride) + q) * elem,
                            static_cast<const char*>(src) + i * elem, elem);
            }
}

const KernelSet& kernel_set(int precision) { return precision == MC_FP64 ? kernels_f64() : kernels_f32(); }

// Bytes of what constrained sweeps gather from: the packed (x, y, z, 0)
// spin copy (a 4-vector per site of each sub-set: sub-lattice x colour) and
// the neighbour field of the sub-set being updated (a 4-vector per site).
size_t aos_bytes(const mc_desc* d) {
    const uint64_t Nc = uint64_t(d->dims[0]) * d->dims[1] * d->dims[2] / 2;
    const uint64_t stride = (Nc + 63) / 64 * 64;
    const uint64_t sets = 2 * uint64_t(sublattices(d->lattice));
    return size_t((sets + 1) * stride * 4) * (d->precision == MC_FP64 ? 8 : 4);
}

// Allocate the packed copy on the lattice's first constrained sweep (the
// parameters that point to it are uploaded by the caller).
int ensure_aos(mc_lattice* h) {
    if (h->d_aos) return MC_OK;
    const cudaError_t e = cudaMalloc(&h->d_aos, aos_bytes(&h->desc));
    if (e != cudaSuccess) {
        h->d_aos = nullptr;
        return cuda_fail(e, "cudaMalloc(packed spin copy)");
    }
    h->hp.aos = h->d_aos;
    const size_t rs = h->hp.precision == MC_FP64 ? 8 : 4;
    h->hp.pfield = static_cast<char*>(h->d_aos) + size_t(2 * h->hp.nsub) * h->hp.stride * 4 * rs;
    return MC_OK;
}

int upload_params(mc_lattice* h) {
    set_float_params(h->hp);
    CK(cudaMemcpyAsync(&h->d_lat->p, &h->hp, sizeof(LatParams), cudaMemcpyHostToDevice, h->stream));
    return MC_OK;
}

int create_lattice(const mc_desc* din, mc_handle* out, const SlabSpec* slab) {
    if (!din || !out) return fail(MC_ERR_ARG, "null argument");
    int rc = validate_desc(din);
    if (rc) return rc;
    trace("create: validated");
    mc_lattice* h = new mc_lattice();
    h->desc = *din;
    h->desc.bond_mask = nullptr;
    h->desc.grain_id = nullptr;
    h->desc.grain_axis = nullptr;
    const mc_desc* d = din;
    h->device = d->device;
    if (cudaSetDevice(d->device) != cudaSuccess) { delete h; return fail(MC_ERR_CUDA, "cudaSetDevice(%d) failed", d->device); }
    trace("create: device set");
    if (d->stream) {
        h->stream = static_cast<cudaStream_t>(d->stream);
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete h;
            return fail(MC_ERR_CUDA, "cudaStreamCreate failed");
        }
        h->owned_stream = h->stream;
    }
    LatParams& p = h->hp;
    std::memset(&p, 0, sizeof p);
    p.Lx = d->dims[0]; p.Ly = d->dims[1]; p.Lz = d->dims[2]; p.Lh = p.Lx / 2;
    for (int a = 0; a < 3; ++a) p.bc[a] = d->boundary[a];
    p.precision = d->precision;
    p.nsub = sublattices(d->lattice);
    p.N = (long long)p.nsub * p.Lx * p.Ly * p.Lz;
    p.Nc = uint32_t((long long)p.Lx * p.Ly * p.Lz / 2);
    p.stride = (p.Nc + 63) / 64 * 64;
    p.n_pairs = p.Nc / 2;
    p.perm_bits = feistel_bits(p.Nc);
    p.row_fast = row_fast(p, d->bond_mask != nullptr || d->grain_id != nullptr);
    p.colour_kernel = colour_kernel(p, d->bond_mask != nullptr || d->grain_id != nullptr, d->kernel_path);
    p.row_lanes = p.Lh / 2 < 32 ? (p.Lh / 2 > 0 ? p.Lh / 2 : 1) : 32;
    long long pinned = 0;
    for (int z = 0; z < p.Lz; ++z)
        for (int y = 0; y < p.Ly; ++y)
            for (int x = 0; x < p.Lx; ++x) {
                const int c[3] = {x, y, z};
                const int L[3] = {p.Lx, p.Ly, p.Lz};
                bool pin = false;
                for (int a = 0; a < 3; ++a) pin |= p.bc[a] == MC_PINNED && (c[a] == 0 || c[a] == L[a] - 1);
                pinned += pin;
            }
    p.n_mov = p.N - pinned;
    p.adapt_in_measure = d->adapt_in_measure;
    p.sample_torque = d->sample_torque ? 1 : 0;
    p.key0 = uint32_t(d->seed);
    p.key1 = uint32_t(d->seed >> 32);
    p.div_lh = make_fastdiv(uint32_t(p.Lh));
    p.div_ly = make_fastdiv(uint32_t(p.Ly));
    const uint32_t site_tile = p.nsub > 1 ? 32u : uint32_t(32 * sites_per_thread(p.precision));  // warp tiles
    p.nblocks_site = (p.Nc + site_tile - 1) / site_tile;
    p.nblocks_pair = (p.Nc + 63) / 64;  // pair tiles: 32 pairs, or 64 sites in site order
    if (p.nblocks_pair == 0) p.nblocks_pair = 1;
    // FP32 constrained passes take the pairs in site order: the leader side
    // is then read in index order and only the partner side is a random
    // gather (MC_PATH_GENERAL keeps pair order; both give the same pairs)
    p.pair_leader = d->kernel_path != MC_PATH_GENERAL && p.precision == MC_FP32 ? 1 : 0;
    p.J = p.nsub > 1 ? 1.0 : d->J;  // bcc / fcc: the couplings sit in the neighbour table
    p.Ku = d->K_u; p.Kc = d->K_c; p.T = d->T;
    const double an = std::sqrt(d->axis[0] * d->axis[0] + d->axis[1] * d->axis[1] + d->axis[2] * d->axis[2]);
    for (int a = 0; a < 3; ++a) { p.e[a] = d->axis[a] / an; p.H[a] = d->H[a]; }
    constraint_frame(0.0, 0.0, p.R);
    p.ring_cap = d->ring_capacity > 0 ? d->ring_capacity : 4096;
    h->desc.ring_capacity = p.ring_cap;
    if (slab) {
        // local plane 0 is global plane z0 - 1: colours and draw keys are the
        // global ones (global site = local site + Lx Ly (z0 - 1), mod 2^32;
        // the own planes, local z >= 1, land on global z >= z0 >= 0)
        p.slab = 1;
        p.cflip = (slab->z0 + 1) & 1;
        p.site_off = uint32_t(int64_t(p.Lx) * p.Ly * (slab->z0 - 1));
        h->slab_z0 = slab->z0;
        h->slab_nz = slab->nz;
        h->slab_lz = slab->Lz;
        h->slab_n = (long long)p.Lx * p.Ly * slab->Lz;
        h->slab_n_mov = p.n_mov / slab->nz * slab->Lz;  // the same movable sites in every plane
    }
    const size_t rs = d->precision == MC_FP64 ? 8 : 4;

    // one allocation, carved into 256-byte aligned pieces
    trace("create: parameters computed");
    h->bytes = lattice_bytes(d, slab != nullptr);
    cudaError_t e = cudaMalloc(&h->d_base, h->bytes);
    if (e != cudaSuccess) {
        if (h->owned_stream) cudaStreamDestroy(h->owned_stream);
        delete h;
        return cuda_fail(e, "cudaMalloc(lattice)");
    }
    char* cur = static_cast<char*>(h->d_base);
    auto take = [&](size_t b) { char* r = cur; cur += align256(b); return r; };
    h->d_lat = reinterpret_cast<LatDev*>(take(sizeof(LatDev)));
    p.spins = take(size_t(p.nsub) * 6 * size_t(p.stride) * rs);
    p.wave = wave_desc(d) ? 1 : 0;
    if (p.wave) p.spins_alt = take(6 * size_t(p.stride) * rs);
    XtalNb xt[kXtalMaxSub][kXtalMaxNb] = {};
    if (p.nsub > 1) {
        xtal_table(d->lattice, d->J, d->J2, p, xt, p.xnb_n);
        p.xnb = take(sizeof xt);
    }
    std::vector<uint8_t> hb;
    if (din->bond_mask) {
        hb.assign(2 * size_t(p.stride), 0);
        per_site_colour_split(p, din->bond_mask, 1, hb.data());
        p.bonds = reinterpret_cast<const uint8_t*>(take(2 * size_t(p.stride)));
        h->film_bonds.assign(din->bond_mask, din->bond_mask + p.N);
    }
    std::vector<int32_t> hg, hgs;
    std::vector<char> hax;
    if (din->grain_id) {
        hg.assign(2 * size_t(p.stride), 0);
        per_site_colour_split(p, din->grain_id, 4, hg.data());
        p.grain = reinterpret_cast<const int32_t*>(take(2 * size_t(p.stride) * 4));
        hax.assign(4 * size_t(d->n_grains) * rs, 0);
        for (int g = 0; g < d->n_grains; ++g) {
            const double* v = &din->grain_axis[3 * g];
            const double n = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            for (int a = 0; a < 3; ++a) {
                if (rs == 8) reinterpret_cast<double*>(hax.data())[4 * g + a] = v[a] / n;
                else reinterpret_cast<float*>(hax.data())[4 * g + a] = (float)(v[a] / n);
            }
        }
        p.gaxis = take(4 * size_t(d->n_grains) * rs);
        p.n_grains = d->n_grains;
        hgs.assign(size_t(d->n_grains), 0);
        for (long long i = 0; i < p.N; ++i) ++hgs[size_t(din->grain_id[i])];
        p.gsum = reinterpret_cast<long long*>(take(3 * size_t(d->n_grains) * 8));
        p.gsize = reinterpret_cast<const int32_t*>(take(size_t(d->n_grains) * 4));
        p.gacc = reinterpret_cast<double*>(take((size_t(d->n_grains) + 1) * 8));
        h->film_grain.assign(din->grain_id, din->grain_id + p.N);
        h->film_axes.assign(din->grain_axis, din->grain_axis + 3 * size_t(d->n_grains));
    }
    p.ring = reinterpret_cast<double*>(take(size_t(p.ring_cap) * kRingWords * 8));
    p.profile = reinterpret_cast<long long*>(take(3 * size_t(p.Lx) * 8));
    h->d_group_lats = reinterpret_cast<LatDev**>(take(sizeof(void*)));
    h->d_group_start = reinterpret_cast<uint32_t*>(take(2 * sizeof(uint32_t)));
    h->d_group_start_pair = reinterpret_cast<uint32_t*>(take(2 * sizeof(uint32_t)));
    if (slab) p.slab_counts = reinterpret_cast<long long*>(take(kSlabWords * 8));
    if (resident_desc(d, slab != nullptr)) {  // its control words, if its rows fit the SMs
        void* ctl = take(sizeof(ResCtl));
        ResidentPlan* rp = new ResidentPlan();
        if (kernels_f32().resident_plan(p, rp)) {
            p.rctl = ctl;
            rp->args.lat = h->d_lat;
            rp->args.ctl = static_cast<ResCtl*>(ctl);
            rp->args.key0 = p.key0;
            rp->args.key1 = p.key1;
            // fault injection for the tests of the bounded waits: the wait for
            // every block's count of a sweep expects one arrival too many
            const char* inj = std::getenv("MC_RESIDENT_INJECT_TIMEOUT");
            rp->args.inject = inj && inj[0] == '1' ? 1 : 0;
            h->res = rp;
        } else {
            delete rp;
        }
    }
    if (size_t(cur - static_cast<char*>(h->d_base)) > h->bytes) {
        cudaFree(h->d_base);
        if (h->owned_stream) cudaStreamDestroy(h->owned_stream);
        delete h;
        return fail(MC_ERR_STATE, "internal: lattice layout exceeds its allocation");
    }

    trace("create: allocated");
    // initial state
    std::vector<double> xyz(size_t(p.N) * 3);
    for (long long i = 0; i < p.N; ++i) {
        if (d->init == MC_INIT_WALL) {
            const int x = int((i / p.nsub) % p.Lx);
            xyz[3 * i] = 0; xyz[3 * i + 1] = 0; xyz[3 * i + 2] = x < p.Lx / 2 ? 1.0 : -1.0;
        } else {
            const double n = std::sqrt(d->init_dir[0] * d->init_dir[0] + d->init_dir[1] * d->init_dir[1] +
                                       d->init_dir[2] * d->init_dir[2]);
            for (int a = 0; a < 3; ++a) xyz[3 * i + a] = d->init_dir[a] / n;
        }
    }
    std::vector<char> hs(size_t(p.nsub) * 6 * size_t(p.stride) * rs, 0);
    if (rs == 8) to_device_layout(p, xyz.data(), reinterpret_cast<double*>(hs.data()));
    else to_device_layout(p, xyz.data(), reinterpret_cast<float*>(hs.data()));

    trace("create: host layout built");
    LatDev init;
    std::memset(&init, 0, sizeof init);
    init.st.theta = d->theta0_deg;
    rc = MC_OK;
    auto up = [&](void* dst, const void* src, size_t b) {
        if (rc == MC_OK) {
            cudaError_t ee = cudaMemcpyAsync(dst, src, b, cudaMemcpyHostToDevice, h->stream);
            if (ee != cudaSuccess) rc = cuda_fail(ee, "cudaMemcpyAsync(init)");
        }
    };
    set_float_params(p);
    init.p = p;
    up(h->d_lat, &init, sizeof init);
    up(p.spins, hs.data(), hs.size());
    if (!hb.empty()) up(const_cast<uint8_t*>(p.bonds), hb.data(), hb.size());
    if (p.nsub > 1) up(const_cast<void*>(p.xnb), xt, sizeof xt);
    if (!hg.empty()) {
        up(const_cast<int32_t*>(p.grain), hg.data(), hg.size() * 4);
        up(const_cast<void*>(p.gaxis), hax.data(), hax.size());
        up(const_cast<int32_t*>(p.gsize), hgs.data(), hgs.size() * 4);
        if (rc == MC_OK && (cudaMemsetAsync(p.gsum, 0, 3 * size_t(p.n_grains) * 8, h->stream) != cudaSuccess ||
                            cudaMemsetAsync(p.gacc, 0, (size_t(p.n_grains) + 1) * 8, h->stream) != cudaSuccess))
            rc = fail(MC_ERR_CUDA, "memset grain samples");
    }
    if (rc == MC_OK && cudaMemsetAsync(p.ring, 0, size_t(p.ring_cap) * kRingWords * 8, h->stream) != cudaSuccess)
        rc = fail(MC_ERR_CUDA, "memset ring");
    if (rc == MC_OK && cudaMemsetAsync(p.profile, 0, 3 * size_t(p.Lx) * 8, h->stream) != cudaSuccess)
        rc = fail(MC_ERR_CUDA, "memset profile");
    if (rc == MC_OK && p.slab_counts && cudaMemsetAsync(p.slab_counts, 0, kSlabWords * 8, h->stream) != cudaSuccess)
        rc = fail(MC_ERR_CUDA, "memset slab counts");
    LatDev* one = h->d_lat;
    const uint32_t st_site[2] = {0, p.nblocks_site};
    const uint32_t st_pair[2] = {0, p.nblocks_pair};
    up(h->d_group_lats, &one, sizeof one);
    up(h->d_group_start, st_site, sizeof st_site);
    up(h->d_group_start_pair, st_pair, sizeof st_pair);
    trace("create: uploads queued");
    if (rc == MC_OK) {
        const double* c64;
        const float* c32;
        rc = device_tables(h->device, &c64, &c32);
        h->cone = d->precision == MC_FP64 ? (const void*)c64 : (const void*)c32;
    }
    trace("create: tables ready");
    if (rc == MC_OK && cudaStreamSynchronize(h->stream) != cudaSuccess) rc = fail(MC_ERR_CUDA, "init sync");
    if (rc == MC_OK && p.wave) {  // the wavefront plan of the lattice alone
        const uint32_t blocks = kernels_f32().wave_blocks();
        const WavePlan pl = plan_wave({&p}, blocks);
        rc = upload_wave_plan(pl, {h->d_lat}, h->stream, &h->d_wave, &h->wave_args);
        h->wave_nblocks = uint32_t(pl.off.size() - 1);
    }
    trace("create: done");
    if (rc != MC_OK) {
        if (h->d_wave) cudaFree(h->d_wave);
        cudaFree(h->d_base);
        if (h->owned_stream) cudaStreamDestroy(h->owned_stream);
        delete h;
        return rc;
    }
    *out = h;
    return MC_OK;
}

// Launch tables of the lattice alone (one colour-pass kernel).
LaunchSet single_launch_set(mc_lattice* h) {
    LaunchSet ls;
    ls.all = GroupArgs{h->d_group_lats, h->d_group_start, 1};
    ls.nt_all = h->hp.nblocks_site;
    if (h->hp.pair_leader) {
        ls.pairs_lead = GroupArgs{h->d_group_lats, h->d_group_start_pair, 1};
        ls.nt_pairs_lead = h->hp.nblocks_pair;
    } else {
        ls.pairs = GroupArgs{h->d_group_lats, h->d_group_start_pair, 1};
        ls.nt_pairs = h->hp.nblocks_pair;
    }
    ls.sample_level = h->hp.sample_torque ? 2 : 1;
    ls.shape = h->shape;
    if (h->hp.nsub > 1) {
        ls.xtal = h->d_lat;
        ls.nsub = h->hp.nsub;
        for (int i = 0; i < h->hp.nsub; ++i) ls.xnb_max = std::max(ls.xnb_max, h->hp.xnb_n[i]);
    } else if (h->hp.colour_kernel == kColourRow) {
        ls.row = ls.all;
        ls.nt_row = ls.nt_all;
        if (h->res) {
            ls.res = &h->res;
            ls.n_res = 1;
        }
        if (h->hp.wave) {
            ls.wave = h->wave_args;
            ls.nb_wave = h->wave_nblocks;
        } else {
            ls.row_rest = ls.all;
            ls.nt_row_rest = ls.nt_all;
        }
    } else if (h->hp.colour_kernel == kColourRowGen) {
        ls.rowx = ls.all;
        ls.nt_rowx = ls.nt_all;
    } else {
        ls.rest = ls.all;
        ls.nt_rest = ls.nt_all;
    }
    return ls;
}

// ------------------------------------------------------------ wavefront plan
// Work units of the wavefront lattices for `blocks` resident blocks: every
// lattice is cut into bands of at most kWaveTyMax rows, each band into slabs
// of planes.
// A unit of tz planes takes about 2 tz + 5 row-steps of a block (tz + 3
// phases, the first three and the last only half full).  Two plans are
// tried and the one with the shorter longest block kept: (a) every band cut
// into slabs of at most T planes (each T from 1 to the tallest lattice),
// units handed out longest first to the least loaded block; (b) the bands'
// planes laid end to end and cut into `blocks` equal runs (a run that
// crosses a band boundary becomes two units).
static long long wave_cost(uint32_t tz) { return 2ll * tz + 5; }

WavePlan plan_wave(const std::vector<const LatParams*>& lats, uint32_t blocks) {
    struct Band { uint32_t lat, y0, lz, ty; };
    std::vector<Band> bands;
    uint32_t lz_max = 1;
    long long planes = 0;
    for (size_t l = 0; l < lats.size(); ++l) {
        // the fewest bands of at most kWaveTyMax rows, heights as equal as possible
        const int Ly = lats[l]->Ly, nb = (Ly + kWaveTyMax - 1) / kWaveTyMax;
        for (int b = 0, y0 = 0; b < nb; ++b) {
            const int ty = Ly / nb + (b < Ly % nb ? 1 : 0);
            bands.push_back({uint32_t(l), uint32_t(y0), uint32_t(lats[l]->Lz), uint32_t(ty)});
            y0 += ty;
        }
        lz_max = std::max(lz_max, uint32_t(lats[l]->Lz));
        planes += (long long)nb * lats[l]->Lz;
    }
    if (blocks < 1) blocks = 1;
    std::vector<std::vector<WaveWU>> best;
    long long best_span = -1;
    auto consider = [&](std::vector<std::vector<WaveWU>>& bins) {
        long long span = 0;
        for (auto& b : bins) {
            long long c = 0;
            for (auto& u : b) c += wave_cost(u.tz);
            span = std::max(span, c);
        }
        if (best_span < 0 || span < best_span) {
            best_span = span;
            best.swap(bins);
        }
    };
    // (a) slabs of at most T planes, longest first onto the least loaded block
    for (uint32_t T = 1; T <= lz_max; ++T) {
        std::vector<WaveWU> units;
        for (const Band& b : bands) {
            const uint32_t ns = (b.lz + T - 1) / T;
            for (uint32_t k = 0, z = 0; k < ns; ++k) {
                const uint32_t tz = b.lz / ns + (k < b.lz % ns ? 1u : 0u);
                units.push_back({b.lat, b.y0, z, tz, b.ty, 0});
                z += tz;
            }
        }
        std::stable_sort(units.begin(), units.end(), [](const WaveWU& x, const WaveWU& y) { return x.tz > y.tz; });
        std::vector<std::vector<WaveWU>> bins(blocks);
        std::priority_queue<std::pair<long long, uint32_t>, std::vector<std::pair<long long, uint32_t>>,
                            std::greater<>> heap;
        for (uint32_t i = 0; i < blocks; ++i) heap.push({0, i});
        for (const WaveWU& u : units) {
            auto [load, i] = heap.top();
            heap.pop();
            bins[i].push_back(u);
            heap.push({load + wave_cost(u.tz), i});
        }
        consider(bins);
    }
    // (b) equal runs of the planes laid end to end
    {
        std::vector<std::vector<WaveWU>> bins(blocks);
        long long pos = 0;  // first plane of the current band in the end-to-end order
        for (const Band& b : bands) {
            for (uint32_t i = 0; i < blocks; ++i) {
                const long long r0 = planes * i / blocks, r1 = planes * (i + 1) / blocks;
                const long long a = std::max(r0, pos), e = std::min(r1, pos + (long long)b.lz);
                if (a < e) bins[i].push_back({b.lat, b.y0, uint32_t(a - pos), uint32_t(e - a), b.ty, 0});
            }
            pos += b.lz;
        }
        consider(bins);
    }
    WavePlan pl;
    pl.nwu.assign(lats.size(), 0);
    pl.off.push_back(0);
    for (auto& b : best) {
        std::sort(b.begin(), b.end(), [](const WaveWU& x, const WaveWU& y) {
            return x.lat != y.lat ? x.lat < y.lat : (x.y0 != y.y0 ? x.y0 < y.y0 : x.z0 < y.z0);
        });
        for (auto& u : b) {
            pl.wu.push_back(u);
            ++pl.nwu[u.lat];
        }
        pl.off.push_back(uint32_t(pl.wu.size()));
    }
    pl.span = best_span;
    return pl;
}

// Upload a plan (with the lattices' device descriptors, in plan order) into
// one device allocation; *d_mem is freed by the owner with cudaFree.
int upload_wave_plan(const WavePlan& pl, const std::vector<LatDev*>& dev_lats, cudaStream_t s, void** d_mem,
                     WaveArgs* out) {
    const size_t b_lats = align256(sizeof(LatDev*) * dev_lats.size());
    const size_t b_nwu = align256(sizeof(uint32_t) * pl.nwu.size());
    const size_t b_off = align256(sizeof(uint32_t) * pl.off.size());
    const size_t b_wu = align256(sizeof(WaveWU) * std::max<size_t>(pl.wu.size(), 1));
    const size_t total = b_lats + b_nwu + b_off + b_wu;
    std::vector<char> host(total, 0);
    std::copy(dev_lats.begin(), dev_lats.end(), reinterpret_cast<LatDev**>(host.data()));
    std::copy(pl.nwu.begin(), pl.nwu.end(), reinterpret_cast<uint32_t*>(host.data() + b_lats));
    std::copy(pl.off.begin(), pl.off.end(), reinterpret_cast<uint32_t*>(host.data() + b_lats + b_nwu));
    std::copy(pl.wu.begin(), pl.wu.end(), reinterpret_cast<WaveWU*>(host.data() + b_lats + b_nwu + b_off));
    void* d = nullptr;
    cudaError_t e = cudaMalloc(&d, total);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(wavefront plan)");
    e = cudaMemcpyAsync(d, host.data(), total, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_fail(e, "wavefront plan upload");
    }
    char* db = static_cast<char*>(d);
    out->lats = reinterpret_cast<LatDev* const*>(db);
    out->nwu = reinterpret_cast<const uint32_t*>(db + b_lats);
    out->off = reinterpret_cast<const uint32_t*>(db + b_lats + b_nwu);
    out->wu = reinterpret_cast<const WaveWU*>(db + b_lats + b_nwu + b_off);
    out->n = int(dev_lats.size());
    // fault injection for the tests of the bounded waits: block 0's first
    // staged copy expects 16 bytes that never arrive, so its wait runs out
    const char* inj = std::getenv("MC_WAVE_INJECT_TIMEOUT");
    out->inject = inj && inj[0] == '1' ? 16 : 0;
    *d_mem = d;
    return MC_OK;
}

// Enqueue n sweeps of the lattices of a launch set; with events != nullptr
// every colour pass or pair pass is bracketed by a pair of events.
int enqueue_sweeps(const KernelSet& k, const LaunchSet& ls, const void* cone, int n, int measure, bool constrained,
                   cudaStream_t s, std::vector<TimedLaunch>* events) {
    auto timed_kind = [&](int kind, auto&& launch) {
        if (events) {
            cudaEvent_t a, b;
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            cudaEventRecord(a, s);
            launch();
            cudaEventRecord(b, s);
            events->push_back(TimedLaunch{a, b, kind});
        } else {
            launch();
        }
    };
    auto timed = [&](auto&& launch) { timed_kind(constrained ? kTimedPair : kTimedPass, launch); };
    // all n sweeps held in shared memory, lattice after lattice (see kResMinSweeps)
    if (!constrained && ls.n_res && k.resident_sweeps && n >= kResMinSweeps) {
        cudaError_t e = cudaSuccess;
        for (int i = 0; i < ls.n_res && e == cudaSuccess; ++i)
            for (int done = 0; done < n && e == cudaSuccess; done += kResMaxSweeps) {
                const int m = std::min(n - done, kResMaxSweeps);
                timed_kind(kTimedResident, [&] {
                    e = k.resident_sweeps(*ls.res[i], cone, m, measure ? ls.sample_level : 0, ls.shape.row, s);
                });
            }
        if (e != cudaSuccess) return cuda_fail(e, "resident sweep launch");
        return MC_OK;
    }
    cudaError_t launch_err = cudaSuccess;  // first failed launch of the row kernels
    auto colour_pass = [&](int colour, int meas) {
        if (ls.nt_row) {
            const cudaError_t e = k.row_pass(ls.row, ls.nt_row, cone, colour, meas, 0, ls.shape.row, s);
            if (launch_err == cudaSuccess) launch_err = e;
        }
        if (ls.nt_rowx) {
            const cudaError_t e = k.row_pass(ls.rowx, ls.nt_rowx, cone, colour, meas, 1, ls.shape.row, s);
            if (launch_err == cudaSuccess) launch_err = e;
        }
        if (ls.nt_rest) k.colour_pass(ls.rest, ls.nt_rest, cone, colour, meas, s);
    };
    if (ls.xtal) {  // bcc / fcc / hcp: the 2 nsub sub-sets in turn, then the sample
        for (int i = 0; i < n; ++i) {
            if (!constrained) {
                for (int sub = 0; sub < ls.nsub; ++sub)
                    for (int colour = 0; colour < 2; ++colour) {
                        const bool last = sub == ls.nsub - 1 && colour == 1;
                        timed([&] {
                            k.xtal_pass(ls.xtal, ls.nt_all, cone, sub, colour, last && !measure ? 1 : 0, ls.xnb_max,
                                        s);
                        });
                    }
            } else {  // Table A2 per sub-set, as for the two colours of a simple cubic lattice
                if (i == 0) {
                    k.ml_reset(ls.all, s);
                    k.mlong(ls.all, ls.nt_all, s);
                }
                for (int sub = 0; sub < ls.nsub; ++sub)
                    for (int colour = 0; colour < 2; ++colour) {
                        k.xtal_field(ls.xtal, ls.nt_all, sub, colour, ls.xnb_max, s);
                        timed([&] {
                            if (ls.nt_pairs) k.pair_pass(ls.pairs, ls.nt_pairs, cone, colour, 0, ls.shape.pair, sub, s);
                            if (ls.nt_pairs_lead)
                                k.pair_pass(ls.pairs_lead, ls.nt_pairs_lead, cone, colour, 1, ls.shape.pair, sub, s);
                        });
                    }
                if (!measure) k.sweep_end(ls.all, s);
            }
            if (measure)
                k.xtal_sample(ls.xtal, uint32_t(2 * ls.nsub) * ls.nt_all, ls.nt_all, ls.xnb_max, ls.sample_level, s);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
        return MC_OK;
    }
    // the lattices beside a wavefront launch: the row list without the
    // wavefront lattices, the boundary and general lists
    auto rest_pass = [&](int colour, int meas) {
        if (ls.nt_row_rest) {
            const cudaError_t e = k.row_pass(ls.row_rest, ls.nt_row_rest, cone, colour, meas, 0, ls.shape.row, s);
            if (launch_err == cudaSuccess) launch_err = e;
        }
        if (ls.nt_rowx) {
            const cudaError_t e = k.row_pass(ls.rowx, ls.nt_rowx, cone, colour, meas, 1, ls.shape.row, s);
            if (launch_err == cudaSuccess) launch_err = e;
        }
        if (ls.nt_rest) k.colour_pass(ls.rest, ls.nt_rest, cone, colour, meas, s);
    };
    const bool rest_any = ls.nt_row_rest || ls.nt_rowx || ls.nt_rest;
    bool red_field_ready = false;  // the next constrained sweep's red field is stored
    for (int i = 0; i < n; ++i) {
        // wavefront lattices sweep two at a time, spins -> spins_alt -> spins,
        // so that every call leaves their state in spins; an odd last sweep
        // of the call runs as two row passes
        const bool wave = !constrained && ls.nb_wave && k.wave_sweep && (i % 2 == 1 || i + 1 < n);
        if (wave) {
            timed_kind(kTimedWave, [&] {
                const cudaError_t e =
                    k.wave_sweep(ls.wave, ls.nb_wave, cone, i % 2, measure ? ls.sample_level : 0, s);
                if (launch_err == cudaSuccess) launch_err = e;
            });
            if (rest_any) {
                timed([&] { rest_pass(0, 0); });
                timed([&] { rest_pass(1, measure ? ls.sample_level : 0); });
            }
        } else if (!constrained) {
            timed([&] { colour_pass(0, 0); });
            timed([&] { colour_pass(1, measure ? ls.sample_level : 0); });
        } else {
            if (i == 0) {  // M_L and the packed copy afresh; later sweeps carry both
                k.ml_reset(ls.all, s);
                k.mlong(ls.all, ls.nt_all, s);
            }
            for (int colour = 0; colour < 2; ++colour) {
                // a measured sweep of all-periodic row lattices leaves the red field
                // behind in its sample (row_sample); otherwise sum it here
                if (!(colour == 0 && red_field_ready)) k.pair_field(ls.all, ls.nt_all, colour, ls.shape.field, s);
                timed([&] {
                    if (ls.nt_pairs) k.pair_pass(ls.pairs, ls.nt_pairs, cone, colour, 0, ls.shape.pair, 0, s);
                    if (ls.nt_pairs_lead)
                        k.pair_pass(ls.pairs_lead, ls.nt_pairs_lead, cone, colour, 1, ls.shape.pair, 0, s);
                });
            }
            if (!measure) k.sweep_end(ls.all, s);  // a measured sweep ends in its sample
            red_field_ready = false;
            if (measure) {
                if (k.row_sample) {  // row-layout lattices sample in the row kernels
                    if (ls.nt_row) k.row_sample(ls.row, ls.nt_row, 0, s);
                    if (ls.nt_rowx) k.row_sample(ls.rowx, ls.nt_rowx, 1, s);
                    if (ls.nt_rest) k.measure(ls.rest, ls.nt_rest, s);
                    red_field_ready = ls.nt_row && !ls.nt_rowx && !ls.nt_rest;
                } else {
                    k.measure(ls.all, ls.nt_all, s);
                }
            }
        }
    }
    if (launch_err != cudaSuccess) return cuda_fail(launch_err, "row kernel launch");
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return MC_OK;
}

int run_sweeps(SweepGraphs& gr, int precision, const LaunchSet& ls, const void* cone, int n, int measure,
               bool constrained, cudaStream_t s) {
    const KernelSet& k = kernel_set(precision);
    // resident sweeps run many to a launch: nothing to capture
    if (!constrained && ls.n_res && n >= kResMinSweeps)
        return enqueue_sweeps(k, ls, cone, n, measure, constrained, s, nullptr);
    const int reps = n / kGraphSweeps;
    if (reps > 0) {
        cudaGraphExec_t& ex = gr.exec[constrained ? 1 : 0][measure ? 1 : 0];
        if (!ex) {
            cudaGraph_t graph;
            cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
            const int rc = enqueue_sweeps(k, ls, cone, kGraphSweeps, measure, constrained, s, nullptr);
            e = cudaStreamEndCapture(s, &graph);
            if (rc) return rc;
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&ex, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                ex = nullptr;
                return cuda_fail(e, "cudaGraphInstantiate");
            }
        }
        for (int r = 0; r < reps; ++r) {
            const cudaError_t e = cudaGraphLaunch(ex, s);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
        }
    }
    return enqueue_sweeps(k, ls, cone, n - reps * kGraphSweeps, measure, constrained, s, nullptr);
}

void destroy_graphs(SweepGraphs& gr) {
    for (auto& row : gr.exec)
        for (auto& ex : row)
            if (ex) {
                cudaGraphExecDestroy(ex);
                ex = nullptr;
            }
}

int read_state(mc_lattice* h, LatState* st) {
    CK(cudaMemcpyAsync(st, &h->d_lat->st, sizeof(LatState), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return MC_OK;
}

// Ensemble averages of Sec. 3 (Eq. 6 in reduced units) from a copy of the
// lattice's device state; returns the sticky device error, if any.
int observables_from(const mc_lattice* h, const LatState& st, mc_observables* out) {
    std::memset(out, 0, sizeof *out);
    const double* mo = st.moments;
    const double n = mo[kMomN];
    out->n_samples = (int64_t)n;
    out->sweeps_done = st.sweep;
    out->theta_deg = st.theta;
    out->error = st.error;
    // a slab's count and sample are the whole lattice's
    const long long n_mov = h->slab_nz ? h->slab_n_mov : h->hp.n_mov;
    out->accept_last = double(st.last_acc) / double(n_mov > 0 ? n_mov : 1);
    if (n > 0) {
        for (int a = 0; a < 3; ++a) {
            out->m[a] = mo[kMomM + a] / n;
            out->m2[a] = mo[kMomM2 + a] / n;
            out->m_abs[a] = mo[kMomMabs + a] / n;
            out->torque[a] = mo[kMomTq + a] / n;
            out->torque2[a] = mo[kMomTq2 + a] / n;
        }
        out->ml = mo[kMomMl] / n;
        out->ml2 = mo[kMomMl2] / n;
        out->ml4 = mo[kMomMl4] / n;
        out->e = mo[kMomE] / n;
        out->e2 = mo[kMomE2] / n;
        for (int a = 0; a < 4; ++a) out->e_parts[a] = mo[kMomParts + a] / n;
        const double NT = double(h->slab_nz ? h->slab_n : h->hp.N) / h->hp.T;
        out->chi[0] = NT * (out->ml2 - out->ml * out->ml);
        for (int a = 0; a < 3; ++a) out->chi[1 + a] = NT * (out->m2[a] - out->m[a] * out->m[a]);
        out->binder = out->ml2 > 0 ? 1.0 - out->ml4 / (3.0 * out->ml2 * out->ml2) : 0.0;
    }
    if (st.error) return fail(st.error, "device reported error %d", st.error);
    return MC_OK;
}

}  // namespace mcgb

using namespace mcgb;

// ===================================================================== ABI
extern "C" {

MC_API const char* mc_last_error(void) { return g_error.c_str(); }
MC_API const char* mc_version(void) { return "libmc 1.0 (sm_103a)"; }

MC_API void mc_desc_default(mc_desc* d) {
    if (!d) return;
    std::memset(d, 0, sizeof *d);
    d->dims[0] = d->dims[1] = d->dims[2] = 16;
    d->precision = MC_FP32;
    d->J = 1.0;
    d->axis[2] = 1.0;
    d->T = 1.0;
    d->theta0_deg = 30;
    d->adapt_in_measure = 1;
    d->init = MC_INIT_UNIFORM;
    d->init_dir[2] = 1.0;
    d->ring_capacity = 4096;
    d->sample_torque = 1;
}

MC_API int mc_create(const int dims[3], double J, double K_u, const double axis[3], double K_c, const double H[3],
                     double T, uint64_t seed, mc_handle* out) {
    if (!dims || !axis || !H) return fail(MC_ERR_ARG, "null argument");
    mc_desc d;
    mc_desc_default(&d);
    for (int a = 0; a < 3; ++a) { d.dims[a] = dims[a]; d.axis[a] = axis[a]; d.H[a] = H[a]; }
    d.J = J; d.K_u = K_u; d.K_c = K_c; d.T = T; d.seed = seed;
    return create_lattice(&d, out);
}

MC_API int mc_create_ex(const mc_desc* d, mc_handle* out) { return create_lattice(d, out); }

MC_API int mc_destroy(mc_handle h) {
    if (!h) return MC_OK;
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    destroy_graphs(h->graphs);
    cudaFree(h->d_base);
    if (h->d_aos) cudaFree(h->d_aos);
    if (h->d_wave) cudaFree(h->d_wave);
    if (h->owned_stream) cudaStreamDestroy(h->owned_stream);
    delete h;
    return MC_OK;
}

MC_API int mc_set_temperature(mc_handle h, double T) {
    if (!h) return fail(MC_ERR_ARG, "null handle");
    if (!(T > 0.0) || !std::isfinite(T)) return fail(MC_ERR_ARG, "T must be > 0");
    h->hp.T = T;
    h->desc.T = T;
    return upload_params(h);
}

MC_API int mc_set_field(mc_handle h, const double H[3]) {
    if (!h || !H) return fail(MC_ERR_ARG, "null argument");
    for (int a = 0; a < 3; ++a) { h->hp.H[a] = H[a]; h->desc.H[a] = H[a]; }
    return upload_params(h);
}

MC_API int mc_sweep(mc_handle h, int n_sweeps, int measure) {
    if (!h || n_sweeps < 0) return fail(MC_ERR_ARG, "invalid argument");
    if (h->slab_nz) return fail(MC_ERR_STATE, "a slab sweeps through mc_slab_pass / mc_slab_close or mc_slab_sweep");
    NvtxRange range("mc_sweep");
    cudaSetDevice(h->device);
    return run_sweeps(h->graphs, h->hp.precision, single_launch_set(h), h->cone, n_sweeps, measure ? 1 : 0, false,
                      h->stream);
}

MC_API int mc_constrained_sweep(mc_handle h, double theta_c_deg, double phi_c_deg, int n_sweeps, int measure) {
    if (!h || n_sweeps < 0) return fail(MC_ERR_ARG, "invalid argument");
    NvtxRange range("mc_constrained_sweep");
    if (!(theta_c_deg >= 0.0 && theta_c_deg <= 180.0)) return fail(MC_ERR_ARG, "theta_c outside [0, 180]");
    if (!std::isfinite(phi_c_deg)) return fail(MC_ERR_ARG, "phi_c not finite");
    for (int a = 0; a < 3; ++a)
        if (h->hp.bc[a] == MC_PINNED) return fail(MC_ERR_ARG, "constrained sweeps need no pinned boundary");
    cudaSetDevice(h->device);
    int rc = ensure_aos(h);
    if (rc) return rc;
    constraint_frame(theta_c_deg, phi_c_deg, h->hp.R);
    rc = upload_params(h);
    if (rc) return rc;
    return run_sweeps(h->graphs, h->hp.precision, single_launch_set(h), h->cone, n_sweeps, measure ? 1 : 0, true,
                      h->stream);
}

MC_API int mc_sync(mc_handle h) {
    if (!h) return fail(MC_ERR_ARG, "null handle");
    cudaSetDevice(h->device);
    LatState st;
    int rc = read_state(h, &st);
    if (rc) return rc;
    if (st.error) return fail(st.error, "device reported error %d", st.error);
    return MC_OK;
}

MC_API int mc_anisotropy_scaling(mc_handle h, double out[2]) {
    if (!h || !out) return fail(MC_ERR_ARG, "null argument");
    mc_observables o;
    const int rc = mc_measure(h, &o);
    if (rc) return rc;
    if (o.n_samples == 0) return fail(MC_ERR_STATE, "no samples since the last reset");
    const double Ku = h->hp.Ku, Kc = h->hp.Kc;
    out[0] = Ku != 0.0 ? 1.0 - 3.0 * (o.e_parts[1] + Ku) / (2.0 * Ku) : std::nan("");
    out[1] = Kc != 0.0 ? 1.0 - 5.0 * o.e_parts[2] / (3.0 * (Kc / 3.0)) : std::nan("");
    return MC_OK;
}

MC_API int mc_measure(mc_handle h, mc_observables* out) {
    if (!h || !out) return fail(MC_ERR_ARG, "null argument");
    cudaSetDevice(h->device);
    LatState st;
    int rc = read_state(h, &st);
    if (rc) return rc;
    return observables_from(h, st, out);
}

MC_API int mc_profile_sample(mc_handle h) {
    if (h && h->hp.nsub > 1) return fail(MC_ERR_ARG, "profiles need a simple cubic lattice");
    if (h && h->slab_nz) return fail(MC_ERR_ARG, "a slab's planes include halo copies: profile the whole lattice");
    if (!h) return fail(MC_ERR_ARG, "null handle");
    cudaSetDevice(h->device);
    kernel_set(h->hp.precision).profile(h->d_lat, uint32_t(h->hp.Lh), uint32_t(h->hp.Ly) * h->hp.Lz, h->stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "profile launch");
    return MC_OK;
}

MC_API int mc_profile(mc_handle h, int component, double* out, int len) {
    if (h && h->hp.nsub > 1) return fail(MC_ERR_ARG, "profiles need a simple cubic lattice");
    if (!h || !out || component < 0 || component > 2 || len < h->hp.Lx) return fail(MC_ERR_ARG, "invalid argument");
    cudaSetDevice(h->device);
    std::vector<long long> sums(size_t(h->hp.Lx));
    CK(cudaMemcpyAsync(sums.data(), h->hp.profile + size_t(component) * h->hp.Lx, sums.size() * 8,
                       cudaMemcpyDeviceToHost, h->stream));
    LatState st;
    int rc = read_state(h, &st);
    if (rc) return rc;
    const double denom = double(st.prof_samples) * h->hp.Ly * h->hp.Lz;
    for (int x = 0; x < h->hp.Lx; ++x) out[x] = denom > 0 ? double(sums[x]) / kFixScale / denom : 0.0;
    return MC_OK;
}

MC_API int mc_grain_sample(mc_handle h) {
    if (!h) return fail(MC_ERR_ARG, "null handle");
    if (!h->hp.n_grains) return fail(MC_ERR_ARG, "the lattice has no grain table");
    cudaSetDevice(h->device);
    kernel_set(h->hp.precision).grain_sample(h->d_lat, h->hp.nblocks_site, h->hp.n_grains, h->stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "grain sample launch");
    return MC_OK;
}

MC_API int mc_grain_magnetization(mc_handle h, double* out, int len, int64_t* n_samples) {
    if (!h || !out) return fail(MC_ERR_ARG, "null argument");
    if (!h->hp.n_grains) return fail(MC_ERR_ARG, "the lattice has no grain table");
    if (len < h->hp.n_grains) return fail(MC_ERR_ARG, "out holds %d < %d grains", len, h->hp.n_grains);
    cudaSetDevice(h->device);
    std::vector<double> acc(size_t(h->hp.n_grains) + 1);
    CK(cudaMemcpyAsync(acc.data(), h->hp.gacc, acc.size() * 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    const double n = acc.back();
    for (int g = 0; g < h->hp.n_grains; ++g) out[g] = n > 0 ? acc[size_t(g)] / n : 0.0;
    if (n_samples) *n_samples = int64_t(n);
    return MC_OK;
}

MC_API int mc_samples(mc_handle h, mc_sample* out, int max, int* n) {
    if (!h || !n || (max > 0 && !out)) return fail(MC_ERR_ARG, "invalid argument");
    cudaSetDevice(h->device);
    LatState st;
    int rc = read_state(h, &st);
    if (rc) return rc;
    const int cap = h->hp.ring_cap;
    const long long have = std::min<long long>(st.ring_count, cap);
    const long long cnt = std::min<long long>(have, max);
    std::vector<double> ring(size_t(cap) * kRingWords);
    CK(cudaMemcpy(ring.data(), h->hp.ring, ring.size() * 8, cudaMemcpyDeviceToHost));
    const long long first = st.ring_count - cnt;
    for (long long s = 0; s < cnt; ++s) {
        const double* r = &ring[size_t((first + s) % cap) * kRingWords];
        mc_sample& o = out[s];
        o.sweep = (int64_t)r[0];
        o.theta_deg = (int32_t)r[1];
        o.pad = 0;
        o.accepted = (int64_t)r[2];
        for (int a = 0; a < 3; ++a) o.m[a] = r[3 + a];
        for (int a = 0; a < 4; ++a) o.e_parts[a] = r[6 + a];
        for (int a = 0; a < 3; ++a) o.torque[a] = r[10 + a];
    }
    *n = (int)cnt;
    return MC_OK;
}

MC_API int mc_reset_stats(mc_handle h) {
    if (!h) return fail(MC_ERR_ARG, "null handle");
    cudaSetDevice(h->device);
    LatDev* d = h->d_lat;
    CK(cudaMemsetAsync(d->st.moments, 0, sizeof(d->st.moments), h->stream));
    CK(cudaMemsetAsync(&d->st.ring_count, 0, sizeof(long long), h->stream));
    CK(cudaMemsetAsync(&d->st.prof_samples, 0, sizeof(long long), h->stream));
    CK(cudaMemsetAsync(h->hp.profile, 0, 3 * size_t(h->hp.Lx) * 8, h->stream));
    if (h->hp.n_grains) CK(cudaMemsetAsync(h->hp.gacc, 0, (size_t(h->hp.n_grains) + 1) * 8, h->stream));
    return MC_OK;
}

MC_API size_t mc_state_bytes(mc_handle h) {
    if (!h) return 0;
    return size_t(h->hp.nsub) * 6 * size_t(h->hp.stride) * (h->hp.precision == MC_FP64 ? 8 : 4);
}

MC_API int mc_export_state(mc_handle h, void* host_buf, size_t bytes) {
    if (!h || !host_buf || bytes != mc_state_bytes(h)) return fail(MC_ERR_ARG, "invalid argument");
    cudaSetDevice(h->device);
    CK(cudaMemcpyAsync(host_buf, h->hp.spins, bytes, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return MC_OK;
}

MC_API int mc_import_state(mc_handle h, const void* host_buf, size_t bytes) {
    if (!h || !host_buf || bytes != mc_state_bytes(h)) return fail(MC_ERR_ARG, "invalid argument");
    cudaSetDevice(h->device);
    CK(cudaMemcpyAsync(h->hp.spins, host_buf, bytes, cudaMemcpyHostToDevice, h->stream));
    return MC_OK;
}

MC_API int mc_get_spins(mc_handle h, double* host_xyz, size_t n) {
    if (!h || !host_xyz || n != size_t(h->hp.N)) return fail(MC_ERR_ARG, "invalid argument");
    std::vector<char> buf(mc_state_bytes(h));
    int rc = mc_export_state(h, buf.data(), buf.size());
    if (rc) return rc;
    if (h->hp.precision == MC_FP64) from_device_layout(h->hp, reinterpret_cast<const double*>(buf.data()), host_xyz);
    else from_device_layout(h->hp, reinterpret_cast<const float*>(buf.data()), host_xyz);
    return MC_OK;
}

MC_API int mc_set_spins(mc_handle h, const double* host_xyz, size_t n) {
    if (!h || !host_xyz || n != size_t(h->hp.N)) return fail(MC_ERR_ARG, "invalid argument");
    std::vector<char> buf(mc_state_bytes(h), 0);
    if (h->hp.precision == MC_FP64) to_device_layout(h->hp, host_xyz, reinterpret_cast<double*>(buf.data()));
    else to_device_layout(h->hp, host_xyz, reinterpret_cast<float*>(buf.data()));
    int rc = mc_import_state(h, buf.data(), buf.size());
    if (rc) return rc;
    CK(cudaStreamSynchronize(h->stream));
    return MC_OK;
}

MC_API int mc_get_theta(mc_handle h, int* theta_deg, int64_t* sweeps_done) {
    if (!h) return fail(MC_ERR_ARG, "null handle");
    cudaSetDevice(h->device);
    LatState st;
    int rc = read_state(h, &st);
    if (rc) return rc;
    if (theta_deg) *theta_deg = st.theta;
    if (sweeps_done) *sweeps_done = st.sweep;
    return MC_OK;
}

// ------------------------------------------------------------- checkpoint
static const char kMagic[8] = {'M', 'C', 'G', 'B', 'C', 'K', '0', '4'};

MC_API int mc_save(mc_handle h, const char* path) {
    if (!h || !path) return fail(MC_ERR_ARG, "null argument");
    if (h->slab_nz) return fail(MC_ERR_STATE, "a slab is checkpointed through its lattice (mc_get_spins of every slab)");
    cudaSetDevice(h->device);
    LatState st;
    int rc = read_state(h, &st);
    if (rc) return rc;
    std::vector<char> spins(mc_state_bytes(h));
    rc = mc_export_state(h, spins.data(), spins.size());
    if (rc) return rc;
    std::vector<double> ring(size_t(h->hp.ring_cap) * kRingWords);
    std::vector<long long> prof(3 * size_t(h->hp.Lx));
    std::vector<double> gacc(h->hp.n_grains ? size_t(h->hp.n_grains) + 1 : 0);
    CK(cudaMemcpy(ring.data(), h->hp.ring, ring.size() * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(prof.data(), h->hp.profile, prof.size() * 8, cudaMemcpyDeviceToHost));
    if (!gacc.empty()) CK(cudaMemcpy(gacc.data(), h->hp.gacc, gacc.size() * 8, cudaMemcpyDeviceToHost));
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(MC_ERR_IO, "cannot open %s for writing", path);
    mc_desc d = h->desc;
    d.stream = nullptr;
    d.bond_mask = nullptr;
    d.grain_id = nullptr;
    d.grain_axis = nullptr;
    const uint64_t nb = h->film_bonds.size(), ng = h->film_grain.size(), na = h->film_axes.size();
    bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(&d, sizeof d, 1, f) == 1 &&
              std::fwrite(&h->hp.R, sizeof h->hp.R, 1, f) == 1 && std::fwrite(&st, sizeof st, 1, f) == 1 &&
              std::fwrite(&nb, 8, 1, f) == 1 && std::fwrite(&ng, 8, 1, f) == 1 && std::fwrite(&na, 8, 1, f) == 1;
    if (ok && nb) ok = std::fwrite(h->film_bonds.data(), 1, nb, f) == nb;
    if (ok && ng) ok = std::fwrite(h->film_grain.data(), 4, ng, f) == ng;
    if (ok && na) ok = std::fwrite(h->film_axes.data(), 8, na, f) == na;
    ok = ok && std::fwrite(ring.data(), 8, ring.size(), f) == ring.size() &&
         std::fwrite(prof.data(), 8, prof.size(), f) == prof.size() &&
         std::fwrite(gacc.data(), 8, gacc.size(), f) == gacc.size() &&
         std::fwrite(spins.data(), 1, spins.size(), f) == spins.size();
    ok = (std::fclose(f) == 0) && ok;
    return ok ? MC_OK : fail(MC_ERR_IO, "write to %s failed", path);
}

MC_API int mc_load(const char* path, mc_handle* out) {
    if (!path || !out) return fail(MC_ERR_ARG, "null argument");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(MC_ERR_IO, "cannot open %s", path);
    char magic[8];
    mc_desc d;
    double R[9];
    LatState st;
    uint64_t nb = 0, ng = 0, na = 0;
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMagic, 8) == 0 &&
              std::fread(&d, sizeof d, 1, f) == 1 && std::fread(R, sizeof R, 1, f) == 1 &&
              std::fread(&st, sizeof st, 1, f) == 1 && std::fread(&nb, 8, 1, f) == 1 &&
              std::fread(&ng, 8, 1, f) == 1 && std::fread(&na, 8, 1, f) == 1;
    const uint64_t N = ok ? uint64_t(d.dims[0]) * d.dims[1] * d.dims[2] : 0;
    ok = ok && (nb == 0 || nb == N) && (ng == 0 || ng == N) && na == 3 * uint64_t(ng ? d.n_grains : 0);
    std::vector<uint8_t> bonds(ok ? nb : 0);
    std::vector<int32_t> grain(ok ? ng : 0);
    std::vector<double> axes(ok ? na : 0);
    if (ok && nb) ok = std::fread(bonds.data(), 1, nb, f) == nb;
    if (ok && ng) ok = std::fread(grain.data(), 4, ng, f) == ng;
    if (ok && na) ok = std::fread(axes.data(), 8, na, f) == na;
    if (!ok) { std::fclose(f); return fail(MC_ERR_IO, "%s is not a valid checkpoint", path); }
    d.stream = nullptr;
    d.bond_mask = nb ? bonds.data() : nullptr;
    d.grain_id = ng ? grain.data() : nullptr;
    d.grain_axis = ng ? axes.data() : nullptr;
    if (!ng) d.n_grains = 0;
    mc_handle h = nullptr;
    int rc = create_lattice(&d, &h);
    if (rc) { std::fclose(f); return rc; }
    std::vector<double> ring(size_t(h->hp.ring_cap) * kRingWords);
    std::vector<long long> prof(3 * size_t(h->hp.Lx));
    std::vector<double> gacc(h->hp.n_grains ? size_t(h->hp.n_grains) + 1 : 0);
    std::vector<char> spins(mc_state_bytes(h));
    ok = std::fread(ring.data(), 8, ring.size(), f) == ring.size() &&
         std::fread(prof.data(), 8, prof.size(), f) == prof.size() &&
         std::fread(gacc.data(), 8, gacc.size(), f) == gacc.size() &&
         std::fread(spins.data(), 1, spins.size(), f) == spins.size();
    std::fclose(f);
    if (!ok) { mc_destroy(h); return fail(MC_ERR_IO, "%s is truncated", path); }
    std::memcpy(h->hp.R, R, sizeof R);
    rc = upload_params(h);
    if (!rc && cudaMemcpy(&h->d_lat->st, &st, sizeof st, cudaMemcpyHostToDevice) != cudaSuccess) rc = MC_ERR_CUDA;
    if (!rc && cudaMemcpy(h->hp.ring, ring.data(), ring.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess) rc = MC_ERR_CUDA;
    if (!rc && cudaMemcpy(h->hp.profile, prof.data(), prof.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess) rc = MC_ERR_CUDA;
    if (!rc && !gacc.empty() &&
        cudaMemcpy(h->hp.gacc, gacc.data(), gacc.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess)
        rc = MC_ERR_CUDA;
    if (!rc) rc = mc_import_state(h, spins.data(), spins.size());
    if (!rc && cudaStreamSynchronize(h->stream) != cudaSuccess) rc = MC_ERR_CUDA;
    if (rc) { mc_destroy(h); return rc == MC_ERR_CUDA ? fail(rc, "restoring %s failed", path) : rc; }
    *out = h;
    return MC_OK;
}

}  // extern "C"
