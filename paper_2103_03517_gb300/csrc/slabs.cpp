// slabs.cpp -- one lattice split into z slabs (the domain decomposition of
// the paper's multi-GPU projection, Sec. 2): each slab holds its own planes
// plus one halo plane on each side, copied from the neighbouring slabs
// after every colour pass; the accepted moves and sample sums of a sweep
// are summed over the slabs before the sweep is closed, so that every slab
// keeps the cone angle, sweep counter and samples of the unsplit lattice.
// Draws are keyed by global site index and colour, so the split chain is
// the unsplit chain.  The exchanges and the sum are left to the caller
// between devices (mc_slab_plane, mc_slab_export); mc_slab_sweep does both
// for slabs on one device.
#include <cstring>

#include "runtime.h"

using namespace mcgb;

namespace {

int check_slab(mc_handle h) {
    if (!h) return fail(MC_ERR_ARG, "null handle");
    if (!h->slab_nz) return fail(MC_ERR_ARG, "not a slab (mc_slab_create)");
    return MC_OK;
}

// Component pointers and site count of local plane zl of local colour c.
void plane_ptrs(const mc_lattice* h, int c, int zl, void* ptrs[3], size_t* count) {
    const LatParams& p = h->hp;
    const size_t plane = size_t(p.Lh) * size_t(p.Ly);
    float* s = static_cast<float*>(p.spins);
    for (int a = 0; a < 3; ++a) ptrs[a] = s + size_t(3 * c + a) * p.stride + plane * size_t(zl);
    if (count) *count = plane;
}

// Local plane of `which`: 0 first own, 1 last own, 2 lower halo, 3 upper halo.
int plane_of(const mc_lattice* h, int which) {
    switch (which) {
        case 0: return 1;
        case 1: return h->slab_nz;
        case 2: return 0;
        default: return h->slab_nz + 1;
    }
}

}  // namespace

extern "C" {

MC_API int mc_slab_create(const mc_desc* d, int z0, int nz, mc_handle* out) {
    if (!d || !out) return fail(MC_ERR_ARG, "null argument");
    int rc = validate_desc(d);
    if (rc) return rc;
    const int Lz = d->dims[2];
    if (d->precision != MC_FP32 || d->lattice != MC_SC) return fail(MC_ERR_ARG, "slabs are FP32 simple cubic lattices");
    if (d->boundary[2] != MC_PERIODIC) return fail(MC_ERR_ARG, "slabs split a lattice periodic in z");
    if (d->bond_mask || d->grain_id) return fail(MC_ERR_ARG, "slabs take no film tables");
    if (d->kernel_path == MC_PATH_GENERAL) return fail(MC_ERR_ARG, "slabs run on the row kernel");
    if (nz < 1 || z0 < 0 || z0 + nz > Lz) return fail(MC_ERR_ARG, "planes [%d, %d) outside 0..%d", z0, z0 + nz, Lz);
    mc_desc ld = *d;
    ld.dims[2] = nz + 2;
    ld.boundary[2] = MC_PINNED;  // the halo planes do not move
    ld.kernel_path = MC_PATH_AUTO;
    const SlabSpec spec{z0, nz, Lz};
    rc = create_lattice(&ld, out, &spec);
    if (rc) return rc;
    if ((*out)->hp.colour_kernel != kColourRowGen) {
        mc_destroy(*out);
        *out = nullptr;
        return fail(MC_ERR_ARG, "a slab needs the FP32 row layout (Lx/2 a power of two <= 64 or a multiple of 64, "
                                "Lx Ly (nz + 2) / 2 a multiple of 64)");
    }
    return MC_OK;
}

MC_API int mc_slab_info(mc_handle h, int* z0, int* nz, int* Lz) {
    int rc = check_slab(h);
    if (rc) return rc;
    if (z0) *z0 = h->slab_z0;
    if (nz) *nz = h->slab_nz;
    if (Lz) *Lz = h->slab_lz;
    return MC_OK;
}

MC_API int mc_slab_pass(mc_handle h, int colour, int measure) {
    int rc = check_slab(h);
    if (rc) return rc;
    if (colour != 0 && colour != 1) return fail(MC_ERR_ARG, "colour must be 0 (red) or 1 (black)");
    if (measure && colour != 1) return fail(MC_ERR_ARG, "the sample is taken in the black pass");
    cudaSetDevice(h->device);
    const LaunchSet ls = single_launch_set(h);
    const int level = measure ? (h->hp.sample_torque ? 2 : 1) : 0;
    const cudaError_t e = kernels_f32().row_pass(ls.rowx, ls.nt_rowx, h->cone, colour ^ h->hp.cflip, level, 1,
                                                 ls.shape.row, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "slab pass");
    return MC_OK;
}

MC_API int mc_slab_plane(mc_handle h, int colour, int which, void* ptrs[3], size_t* count) {
    int rc = check_slab(h);
    if (rc) return rc;
    if (!ptrs || colour < 0 || colour > 1 || which < 0 || which > 3) return fail(MC_ERR_ARG, "invalid argument");
    plane_ptrs(h, colour ^ h->hp.cflip, plane_of(h, which), ptrs, count);
    return MC_OK;
}

MC_API int mc_slab_export(mc_handle h, int64_t** counts) {
    int rc = check_slab(h);
    if (rc) return rc;
    cudaSetDevice(h->device);
    kernels_f32().slab_export(h->d_lat, h->stream);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "slab export");
    if (counts) *counts = reinterpret_cast<int64_t*>(h->hp.slab_counts);
    return MC_OK;
}

MC_API int mc_slab_close(mc_handle h, int measure) {
    int rc = check_slab(h);
    if (rc) return rc;
    cudaSetDevice(h->device);
    kernels_f32().slab_close(h->d_lat, measure ? 1 : 0, h->stream);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "slab close");
    return MC_OK;
}

MC_API int mc_slab_sweep(const mc_handle* slabs, int n, int n_sweeps, int measure) {
    if (!slabs || n < 1 || n > 64 || n_sweeps < 0) return fail(MC_ERR_ARG, "invalid argument");
    for (int i = 0; i < n; ++i) {
        int rc = check_slab(slabs[i]);
        if (rc) return rc;
        const mc_lattice* a = slabs[i];
        const mc_lattice* b = slabs[(i + 1) % n];
        if (a->device != slabs[0]->device || a->stream != slabs[0]->stream)
            return fail(MC_ERR_ARG, "the slabs of mc_slab_sweep share one device and one stream");
        if (a->slab_lz != slabs[0]->slab_lz || a->hp.Lx != slabs[0]->hp.Lx || a->hp.Ly != slabs[0]->hp.Ly)
            return fail(MC_ERR_ARG, "the slabs belong to different lattices");
        if ((a->slab_z0 + a->slab_nz) % a->slab_lz != b->slab_z0)
            return fail(MC_ERR_ARG, "slab %d does not end where slab %d begins", i, (i + 1) % n);
    }
    if (slabs[0]->slab_z0 != 0) return fail(MC_ERR_ARG, "the first slab starts at plane 0");
    cudaSetDevice(slabs[0]->device);
    const cudaStream_t s = slabs[0]->stream;
    const KernelSet& k = kernels_f32();
    // halo copies of each colour: slab i's lower halo from slab i-1's last
    // own plane, its upper halo from slab i+1's first own plane
    float* dst[2][64][2];
    const float* src[2][64][2];
    uint32_t stride[64], src_stride[64][2];
    std::vector<LatDev*> lats(n);
    size_t plane = 0;
    for (int colour = 0; colour < 2; ++colour)
        for (int i = 0; i < n; ++i) {
            const mc_lattice* up = slabs[(i + 1) % n];
            const mc_lattice* dn = slabs[(i + n - 1) % n];
            void* p[3];
            plane_ptrs(slabs[i], colour ^ slabs[i]->hp.cflip, plane_of(slabs[i], 2), p, &plane);
            dst[colour][i][0] = static_cast<float*>(p[0]);
            plane_ptrs(slabs[i], colour ^ slabs[i]->hp.cflip, plane_of(slabs[i], 3), p, nullptr);
            dst[colour][i][1] = static_cast<float*>(p[0]);
            plane_ptrs(dn, colour ^ dn->hp.cflip, plane_of(dn, 1), p, nullptr);
            src[colour][i][0] = static_cast<const float*>(p[0]);
            plane_ptrs(up, colour ^ up->hp.cflip, plane_of(up, 0), p, nullptr);
            src[colour][i][1] = static_cast<const float*>(p[0]);
            stride[i] = slabs[i]->hp.stride;
            src_stride[i][0] = dn->hp.stride;
            src_stride[i][1] = up->hp.stride;
            lats[i] = slabs[i]->d_lat;
        }
    for (int it = 0; it < n_sweeps; ++it) {
        for (int colour = 0; colour < 2; ++colour) {
            const int meas = measure && colour == 1;
            for (int i = 0; i < n; ++i) {
                int rc = mc_slab_pass(slabs[i], colour, meas);
                if (rc) return rc;
            }
            const cudaError_t e = k.slab_halo(dst[colour], src[colour], stride, src_stride, uint32_t(plane), n, s);
            if (e != cudaSuccess) return cuda_fail(e, "slab halo copy");
        }
        const cudaError_t e = k.slab_close_all(lats.data(), n, measure ? 1 : 0, s);
        if (e != cudaSuccess) return cuda_fail(e, "slab close");
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "slab sweep");
    return MC_OK;
}

}  // extern "C"
