// xtal_pass.cuh -- colour passes and sample of the bcc and fcc lattices
// (Sec. 2: bcc as 2 interleaved simple cubic sub-lattices, fcc as 4, each
// split red/black by cell parity and visited in turn).  Spins of sub-lattice
// s and colour c are the simple cubic colour arrays of that sub-lattice:
// component a at spins[((2 s + c) 3 + a) stride + q], q = (x >> 1) + Lh (y +
// Ly z) for cell (x, y, z).  Every neighbour comes from the lattice's table
// (XtalNb: sub-lattice, cell offset, coupling J1 or J2) in its order, with
// the coupling inside the field h, so the exchange term of Eq. 2 is -(d.h).
// One lattice per launch, one lane per site, persistent warps; the table
// entries sit in shared memory for the launch.
#pragma once
#include "pass_impl.cuh"

namespace mcgb {

// Cell of colour index q of colour c (periodic cells, Lx even).
struct XCell {
    uint32_t x, y, z;
};

__device__ __forceinline__ XCell xtal_cell(const LatParams& p, int colour, uint32_t q) {
    const uint32_t row = fast_div(q, p.div_lh);
    const uint32_t k = q - row * uint32_t(p.Lh);
    const uint32_t z = fast_div(row, p.div_ly);
    const uint32_t y = row - z * uint32_t(p.Ly);
    const uint32_t xoff = (y + z + uint32_t(colour)) & 1u;
    return XCell{2u * k + xoff, y, z};
}

// Stage the neighbour entries of sub-lattices [sub0, sub0 + nsub) in shared
// memory (block-wide; every thread must reach it).
template <int NMAX>
__device__ __forceinline__ void xtal_stage(const LatParams& p, int sub0, int nsub, XtalNb* tab) {
    const XtalNb* src = static_cast<const XtalNb*>(p.xnb);
    for (int i = threadIdx.x; i < nsub * NMAX; i += blockDim.x) {
        const int s = i / NMAX, e = i - s * NMAX;
        if (e < p.xnb_n[sub0 + s]) tab[i] = src[(sub0 + s) * kXtalMaxNb + e];
    }
    __syncthreads();
}

// h = sum over the n <= NMAX entries tab[0 .. n) of J S_j, in table order;
// the site is cell c of the given colour.  Each entry's cell offset is taken
// modulo the lattice size in advance, so a neighbour's cell wraps by one
// compare per axis; its colour array follows from the entry's parity.
// HALF: the forward entries only (every bond once over the lattice).
template <typename R, int NMAX, bool HALF = false>
__device__ __forceinline__ V3<R> xtal_field(const LatParams& p, const R* s, const XtalNb* tab, int n, XCell c,
                                            int colour) {
    const uint32_t Lx = uint32_t(p.Lx), Ly = uint32_t(p.Ly), Lz = uint32_t(p.Lz), Lh = uint32_t(p.Lh);
    const size_t stride = p.stride;
    V3<R> h{R(0), R(0), R(0)};
#pragma unroll
    for (int e = 0; e < NMAX; ++e) {
        if (e < n && (!HALF || (tab[e].par & 2u))) {
            const XtalNb& t = tab[e];
            uint32_t xx = c.x + t.dxw, yy = c.y + t.dyw, zz = c.z + t.dzw;
            xx = xx >= Lx ? xx - Lx : xx;
            yy = yy >= Ly ? yy - Ly : yy;
            zz = zz >= Lz ? zz - Lz : zz;
            const uint32_t q = (xx >> 1) + Lh * (yy + Ly * zz);
            const R* b = s + t.off[colour];
            R J;
            if constexpr (kIsF64<R>) J = t.J;
            else J = t.fJ;
            h.x = h.x + J * b[q];
            h.y = h.y + J * b[stride + q];
            h.z = h.z + J * b[2 * stride + q];
        }
    }
    return h;
}

// Pass over sub-set (sub, colour); finalize != 0 closes the sweep (the last
// sub-set of an unmeasured sweep).  NMAX bounds the sub-lattice's entries.
template <typename R, int NMAX>
__global__ void __launch_bounds__(kBlock) xtal_pass_kernel(LatDev* L, uint32_t ntiles, const R* __restrict__ cone,
                                                           int sub, int colour, int finalize) {
    __shared__ XtalNb tab[NMAX];
    const LatParams& p = L->p;
    xtal_stage<NMAX>(p, sub, 1, tab);
    const int n = p.xnb_n[sub];
    const WarpChunk wc = warp_chunk(ntiles);
    if (wc.begin >= wc.end) return;
    const int lane = wc.lane;
    const Par<R> par = load_par<R>(p);
    const R c = cone[L->st.theta];
    const uint32_t sweep = L->st.sweep;
    const uint32_t tag = tag_of(colour, kPurposeMove);
    R* __restrict__ s = static_cast<R*>(p.spins);
    const V3<R> e_ax{par.e[0], par.e[1], par.e[2]};
    unsigned nacc = 0;
    for (uint32_t tile = wc.begin; tile < wc.end; ++tile) {
        const uint32_t q = tile * 32u + uint32_t(lane);
        if (q >= p.Nc) continue;
        const XCell cell = xtal_cell(p, colour, q);
        const uint32_t site =
            uint32_t(sub) + uint32_t(p.nsub) * (cell.x + uint32_t(p.Lx) * (cell.y + uint32_t(p.Ly) * cell.z));
        R* own = s + (size_t(sub) * 2 + colour) * 3 * p.stride;
        const V3<R> S{own[q], own[p.stride + q], own[2 * size_t(p.stride) + q]};
        V3<R> Sn;
        R P;
        if (!cone_trial(S, c, site, sweep, tag, p.key0, p.key1, Sn, P)) continue;
        const V3<R> h = xtal_field<R, NMAX>(p, s, tab, n, cell, colour);
        if (metropolis(delta_e(par, S, Sn, h, e_ax), par, P)) {
            own[q] = Sn.x;
            own[p.stride + q] = Sn.y;
            own[2 * size_t(p.stride) + q] = Sn.z;
            ++nacc;
        }
    }
    publish(L->st, lane, nacc, false, 0, colour, wc.end - wc.begin, ntiles, finalize != 0,
            [&] { finalize_sweep(p, L->st, 0, false, lane); });
}

// Constrained sweeps (Table A2) of a crystal: the neighbour field of every
// site of sub-set (sub, colour) into LatParams::pfield as (h_x, h_y, h_z, 0),
// summed in table order from the spins (which the pair passes keep in step;
// the sub-set's own spins are not among its neighbours).
template <typename R, int NMAX>
__global__ void __launch_bounds__(kBlock) xtal_field_kernel(LatDev* L, uint32_t ntiles, int sub, int colour) {
    __shared__ XtalNb tab[NMAX];
    const LatParams& p = L->p;
    xtal_stage<NMAX>(p, sub, 1, tab);
    const int n = p.xnb_n[sub];
    const WarpChunk wc = warp_chunk(ntiles);
    if (wc.begin >= wc.end) return;
    const R* s = static_cast<const R*>(p.spins);
    Spin4<R>* fld = static_cast<Spin4<R>*>(p.pfield);
    for (uint32_t tile = wc.begin; tile < wc.end; ++tile) {
        const uint32_t q = tile * 32u + uint32_t(wc.lane);
        if (q >= p.Nc) continue;
        const V3<R> h = xtal_field<R, NMAX>(p, s, tab, n, xtal_cell(p, colour, q), colour);
        fld[q] = Spin4<R>{h.x, h.y, h.z, R(0)};
    }
}

// Sample of the current state: M, the exchange sum over every bond once
// (sum_i S_i . h_i over the forward entries), the uniaxial, cubic and torque
// sums; tiles of 32 sites
// over the 2 nsub sub-sets; closes the sweep.  The warp sums are reduced in
// the working precision in a fixed butterfly order and rounded to fixed
// point on lane i (int64 in both precisions, so that large couplings cannot
// overflow).
template <typename R, int NMAX, int LEVEL>
__global__ void __launch_bounds__(kBlock) xtal_sample_kernel(LatDev* L, uint32_t ntiles, uint32_t tiles_per_subset) {
    constexpr int NS = LEVEL >= 2 ? kNumSums : kSumTux;  // sums sampled (LEVEL 2: with the torques)
    __shared__ XtalNb tab[kXtalMaxSub * NMAX];
    const LatParams& p = L->p;
    xtal_stage<NMAX>(p, 0, p.nsub, tab);
    const WarpChunk wc = warp_chunk(ntiles);
    if (wc.begin >= wc.end) return;
    const int lane = wc.lane;
    const Par<R> par = load_par<R>(p);
    const R* s = static_cast<const R*>(p.spins);
    const V3<R> e_ax{par.e[0], par.e[1], par.e[2]};
    long long fix = 0;
    for (uint32_t tile = wc.begin; tile < wc.end; ++tile) {
        const uint32_t set = tile / tiles_per_subset;  // 2 sub + colour
        const int sub = int(set >> 1), colour = int(set & 1u);
        const uint32_t q = (tile - set * tiles_per_subset) * 32u + uint32_t(lane);
        Sums<R> sums;
        for (int i = 0; i < kNumSums; ++i) sums.v[i] = R(0);
        if (q < p.Nc) {
            const XCell cell = xtal_cell(p, colour, q);
            const R* own = s + (size_t(sub) * 2 + colour) * 3 * p.stride;
            const V3<R> S{own[q], own[p.stride + q], own[2 * size_t(p.stride) + q]};
            const V3<R> h = xtal_field<R, NMAX, true>(p, s, tab + sub * NMAX, p.xnb_n[sub], cell, colour);
            add_site<R, LEVEL>(sums, S, e_ax);
            sums.v[kSumEx] = S.x * h.x + S.y * h.y + S.z * h.z;
        }
        if constexpr (kIsF64<R>) {
            R mine = R(0);
#pragma unroll
            for (int i = 0; i < NS; ++i) {
                R v = sums.v[i];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == i) mine = v;
            }
            fix += __double2ll_rn(mine * kFixScale);
        } else {
            fix += warp_tile_fix<R, NS>(sums, lane);  // per-lane fixed point, integer warp sums
        }
    }
    publish(L->st, lane, 0, true, fix, 3, wc.end - wc.begin, ntiles, true,
            [&] { finalize_sweep(p, L->st, 1, LEVEL >= 2, lane); });
}

}  // namespace mcgb
