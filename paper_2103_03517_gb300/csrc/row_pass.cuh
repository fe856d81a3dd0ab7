// row_pass.cuh -- FP32 colour pass (Table A1) over lattices in the row layout:
// Lx even, rows of Lh = Lx/2 sites per colour a power of two <= 64 or a
// multiple of 64, and Nc a multiple of 64, so that every warp tile is full
// and its rows split evenly over the lanes.  Two instances: GEN = 0 for
// lattices with every axis periodic and no film tables (the batched m(T)
// workload), GEN = 1 for any boundary modes (open, pinned, anti-periodic),
// bond masks and per-grain easy axes (walls, granular films).  Neither holds
// the general-geometry code of the general colour pass, so that they run in
// fewer registers.
//
// Lane L of a tile of 64 colour indices q0 .. q0 + 63 takes the adjacent pair
// q = q0 + 2L, q + 1 of one row, so that every spin is read as a float2 (one
// load per component for both sites) and one Philox call keys the draws of
// both sites to the first.  Rows of Lh <= 64 sites per colour are covered by
// groups of G = Lh/2 lanes (row_lanes), rows of Lh > 64 by segments of 64.
// The other colour's spins at k and k+1 give three of the four x neighbours
// of the pair; the fourth, at k-1 or k+2, is the neighbouring lane's pair,
// taken by a warp shuffle inside the row group (wrapping the row) or, at the
// ends of a 64-site segment of a longer row, loaded on its own.  The
// neighbour sum keeps the order -x, +x, -y, +y, -z, +z.  In the GEN instance
// every neighbour enters with a factor 1, -1 (across an anti-periodic face)
// or 0 (absent: open face or missing bond), an exact product.
#pragma once
#include "pair_math.cuh"

namespace mcgb {

constexpr int kRowSlots = 18;  // float2 loads per lane per tile

__device__ __forceinline__ float2 ld2(const float* a, size_t i) { return *reinterpret_cast<const float2*>(a + i); }

// Factor of a neighbour across a face of an axis with boundary mode bc.
__device__ __forceinline__ float face_factor(int bc) { return bc == 0 ? 1.0f : (bc == 3 ? -1.0f : 0.0f); }

// Spins and neighbour sums of lane L's pair in the tile starting at q0,
// packed (site 0 in .x, site 1 in .y, as loaded); returns the lattice index
// of the pair's first site (its parity is the row's x offset).  GEN:
// mov[v] = site v is not on a pinned plane.
template <int GEN>
__device__ __forceinline__ uint32_t row_pair_sums(const LatParams& p, const float* s, int colour, uint32_t q0,
                                                  int lane, P3& S, P3& h, P3& O, bool mov[2]) {
    const uint32_t stride = p.stride;
    const float* own = s + size_t(3 * colour) * stride;
    const float* oth = s + size_t(3 * (colour ^ 1)) * stride;
    const uint32_t Lh = uint32_t(p.Lh), Ly = uint32_t(p.Ly), Lz = uint32_t(p.Lz), plane = Lh * Ly;
    const uint32_t q = q0 + 2u * uint32_t(lane);
    const uint32_t row = fast_div(q, p.div_lh);
    const uint32_t k = q - row * Lh;
    const uint32_t z = fast_div(row, p.div_ly);
    const uint32_t y = row - z * Ly;
    const uint32_t xoff = (y + z + uint32_t(colour)) & 1u;
    const uint32_t qn[6] = {q, q, y > 0 ? q - Lh : q + Lh * (Ly - 1), y + 1 < Ly ? q + Lh : q - Lh * (Ly - 1),
                            z > 0 ? q - plane : q + plane * (Lz - 1), z + 1 < Lz ? q + plane : q - plane * (Lz - 1)};
    float2 v[kRowSlots];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        const float* base = j == 0 ? own : oth;
#pragma unroll
        for (int a = 0; a < 3; ++a) v[3 * j + a] = ld2(base + size_t(a) * stride, qn[j]);
    }
    const int G = p.row_lanes;
    const int gbase = lane & ~(G - 1);
    const int left = gbase | ((lane - 1) & (G - 1));
    const int right = gbase | ((lane + 1) & (G - 1));
    // other colour at k - 1 (left lane's second) and k + 2 (right lane's first)
    V3<float> lft{__shfl_sync(0xffffffffu, v[3].y, left), __shfl_sync(0xffffffffu, v[4].y, left),
                  __shfl_sync(0xffffffffu, v[5].y, left)};
    V3<float> rgt{__shfl_sync(0xffffffffu, v[3].x, right), __shfl_sync(0xffffffffu, v[4].x, right),
                  __shfl_sync(0xffffffffu, v[5].x, right)};
    if (Lh > 64u) {  // ends of a 64-site segment of a longer row
        if (lane == 0) {
            const uint32_t qe = k == 0 ? q + Lh - 1 : q - 1;
            lft = V3<float>{oth[qe], oth[stride + qe], oth[2 * size_t(stride) + qe]};
        }
        if (lane == 31) {
            const uint32_t qe = k + 2 == Lh ? q + 2 - Lh : q + 2;
            rgt = V3<float>{oth[qe], oth[stride + qe], oth[2 * size_t(stride) + qe]};
        }
    }
    // the other colour at the pair's own indices: one x neighbour of each
    // site (and the site of the other colour the sample pairs with it)
    O = P3{v[3], v[4], v[5]};
    if constexpr (GEN == 0) {
        // the other x neighbour: site 0 has (xoff ? o1 : lft), site 1 has
        // (xoff ? rgt : o0); the -x + +x sum is the same either way round
        const P3 a{make_float2(xoff ? v[3].y : lft.x, xoff ? rgt.x : v[3].x),
                   make_float2(xoff ? v[4].y : lft.y, xoff ? rgt.y : v[4].x),
                   make_float2(xoff ? v[5].y : lft.z, xoff ? rgt.z : v[5].x)};
        h.x = p2add(p2add(p2add(p2add(p2add(O.x, a.x), v[6]), v[9]), v[12]), v[15]);
        h.y = p2add(p2add(p2add(p2add(p2add(O.y, a.y), v[7]), v[10]), v[13]), v[16]);
        h.z = p2add(p2add(p2add(p2add(p2add(O.z, a.z), v[8]), v[11]), v[14]), v[17]);
        mov[0] = mov[1] = true;
    } else {
        const int bx = p.bc[0], by = p.bc[1], bz = p.bc[2];
        const uint32_t x0 = xoff + 2u * k;  // x of site 0; site 1 is at x0 + 2
        // face factors: -x of site 0, +x of site 1, -y, +y, -z, +z of both
        const float fxm = x0 == 0 ? face_factor(bx) : 1.0f;
        const float fxp = x0 + 3 == uint32_t(p.Lx) ? face_factor(bx) : 1.0f;
        const float fym = y > 0 ? 1.0f : face_factor(by), fyp = y + 1 < Ly ? 1.0f : face_factor(by);
        const float fzm = z > 0 ? 1.0f : face_factor(bz), fzp = z + 1 < Lz ? 1.0f : face_factor(bz);
        // bond bits of the two sites (adjacent bytes), all present without a mask
        const uint32_t mm = p.bonds ? uint32_t(__ldg(reinterpret_cast<const unsigned short*>(
                                          p.bonds + size_t(colour) * stride + q)))
                                    : 0x3F3Fu;
        auto fac = [mm](int bit, float base) { return ((mm >> bit) & 1u) ? base : 0.0f; };
        // -x and +x neighbours of the two sites, and each term's factor (an
        // exact 1, -1 or 0), packed (site 0, site 1)
        const P3 xm{make_float2(xoff ? v[3].x : lft.x, xoff ? v[3].y : v[3].x),
                    make_float2(xoff ? v[4].x : lft.y, xoff ? v[4].y : v[4].x),
                    make_float2(xoff ? v[5].x : lft.z, xoff ? v[5].y : v[5].x)};
        const P3 xp{make_float2(xoff ? v[3].y : v[3].x, xoff ? rgt.x : v[3].y),
                    make_float2(xoff ? v[4].y : v[4].x, xoff ? rgt.y : v[4].y),
                    make_float2(xoff ? v[5].y : v[5].x, xoff ? rgt.z : v[5].y)};
        const float2 Fxm = make_float2(fac(0, fxm), fac(8, 1.0f)), Fxp = make_float2(fac(1, 1.0f), fac(9, fxp));
        const float2 Fym = make_float2(fac(2, fym), fac(10, fym)), Fyp = make_float2(fac(3, fyp), fac(11, fyp));
        const float2 Fzm = make_float2(fac(4, fzm), fac(12, fzm)), Fzp = make_float2(fac(5, fzp), fac(13, fzp));
        h.x = p2fma(Fzp, v[15], p2fma(Fzm, v[12], p2fma(Fyp, v[9], p2fma(Fym, v[6], p2fma(Fxp, xp.x, p2mul(Fxm, xm.x))))));
        h.y = p2fma(Fzp, v[16], p2fma(Fzm, v[13], p2fma(Fyp, v[10], p2fma(Fym, v[7], p2fma(Fxp, xp.y, p2mul(Fxm, xm.y))))));
        h.z = p2fma(Fzp, v[17], p2fma(Fzm, v[14], p2fma(Fyp, v[11], p2fma(Fym, v[8], p2fma(Fxp, xp.z, p2mul(Fxm, xm.z))))));
        const bool row_pinned = (by == 2 && (y == 0 || y + 1 == Ly)) || (bz == 2 && (z == 0 || z + 1 == Lz));
        mov[0] = !row_pinned && !(bx == 2 && x0 == 0);
        mov[1] = !row_pinned && !(bx == 2 && x0 + 3 == uint32_t(p.Lx));
    }
    S = P3{v[0], v[1], v[2]};
    return xoff + 2u * k + uint32_t(p.Lx) * row;
}

// Easy axis of grain table entry g (float4 rows).
__device__ __forceinline__ V3<float> grain_axis(const LatParams& p, int colour, uint32_t q) {
    const int32_t g = __ldg(&p.grain[uint32_t(colour) * p.stride + q]);
    const float4 a = __ldg(static_cast<const float4*>(p.gaxis) + g);
    return V3<float>{a.x, a.y, a.z};
}

// MOVE = 0: no moves; the sample of the current state, closing the lattice's
// sweep as the standalone sample does after a constrained sweep: with colour
// c, each site of colour c, the site of the other colour with its index, and
// the six bonds of the first (every bond has one end of each colour).  With
// colour 0 and a constrained lattice (LatParams::pfield set) it also stores
// the red sites' neighbour sums as the field of the next sweep's red pair
// pass: the same terms in the same order as pair_field_kernel's (the -x, +x
// pair commutes), so the same bits.
template <int MINB, int MEASURE, int GEN, int MOVE = 1>
__global__ void __launch_bounds__(kBlock, MINB) row_pass_kernel(GroupArgs g, uint32_t ntiles,
                                                                const float* __restrict__ cone, int colour) {
    constexpr int NS = MEASURE >= 2 ? kNumSums : kSumTux;  // sums sampled
    // Programmatic dependent launch (a colour pass launched after another):
    // the next launch's blocks may take the SM slots this launch frees, and
    // this launch waits for the previous one to complete (its spins, cone
    // angle and counters) before it reads any of them.  Launched without
    // the attribute, both instructions do nothing.
    asm volatile("griddepcontrol.launch_dependents;");
    const WarpChunk wc = warp_chunk(ntiles);
    const int lane = wc.lane;
    const uint32_t tag = tag_of(colour, kPurposeMove);
    uint32_t tile = wc.begin;
    int l = tile < wc.end ? lattice_of_tile(g, tile) : 0;
    asm volatile("griddepcontrol.wait;" ::: "memory");
    while (tile < wc.end) {
        LatDev* L = g.lats[l];
        const LatParams& p = L->p;
        const uint32_t t0 = __ldg(&g.start[l]);
        const uint32_t t1 = min(__ldg(&g.start[l + 1]), wc.end);
        const uint32_t run = t1 - tile;
        const Par<float> par = load_par<float>(p);
        const float c = MOVE ? cone[L->st.theta] : 0.0f;
        const uint32_t sweep = L->st.sweep;
        float* __restrict__ s = static_cast<float*>(p.spins);
        const V3<float> e_ax{par.e[0], par.e[1], par.e[2]};
        // unmeasured passes: the lattice's Philox round keys, once per run, in
        // the warp's slots (ten shared loads per draw instead of twenty adds;
        // the measured pass keeps the adds, which need no registers there)
        __shared__ uint2 round_keys[kBlock / 32][10];
        uint2* rk = round_keys[threadIdx.x >> 5];
        if constexpr (MEASURE == 0) {
            __syncwarp();  // the previous run's keys are no longer read
            if (lane < 10)
                rk[lane] = make_uint2(p.key0 + uint32_t(lane) * 0x9E3779B9u, p.key1 + uint32_t(lane) * 0xBB67AE85u);
            __syncwarp();
        }
        unsigned nacc = 0;
        long long fix = 0;
        int lf[NS];  // this lane's fixed-point parts of the sample, kPartTiles tiles at a time
#pragma unroll
        for (int i = 0; i < NS; ++i) lf[i] = 0;
        uint32_t nparts = 0;
        for (; tile < t1; ++tile) {
            const uint32_t q0 = (tile - t0) * 64u;
            P3 S, h, O;
            bool mov[2];
            const uint32_t site0 = row_pair_sums<GEN>(p, s, colour, q0, lane, S, h, O, mov);
            P3 e, eo;  // per-site easy axes (films with grain axes)
            const bool grains = GEN != 0 && p.grain;
            if constexpr (GEN != 0) {
                if (grains) {
                    V3<float> a[2], b[2];
#pragma unroll
                    for (int v = 0; v < 2; ++v) {
                        a[v] = grain_axis(p, colour, q0 + 2u * uint32_t(lane) + v);
                        b[v] = grain_axis(p, colour ^ 1, q0 + 2u * uint32_t(lane) + v);
                    }
                    e = pack(a);
                    eo = pack(b);
                }
            }
            if (!grains) e = eo = P3{p2(e_ax.x), p2(e_ax.y), p2(e_ax.z)};
            P3 Sf = S;
            bool any = false;
            // a slab draws with its sites' global indices and colours, and
            // leaves its halo planes out of the sample
            uint32_t key_site = site0, key_tag = tag;
            bool sampled = true;
            if constexpr (GEN != 0) {
                if (p.slab) {
                    key_site = site0 + p.site_off;
                    key_tag = tag_of(colour ^ p.cflip, kPurposeMove);
                    const uint32_t plane = uint32_t(p.Lx) * uint32_t(p.Ly);
                    sampled = site0 >= plane && site0 < plane * uint32_t(p.Lz - 1);
                }
            }
            if constexpr (MOVE != 0) {
                const uint4 w = MEASURE == 0 ? philox_smem(make_uint4(key_site, sweep, key_tag, 0u), rk)
                                             : philox(make_uint4(key_site, sweep, key_tag, 0u), p.key0, p.key1);
                const unsigned n = pair_move(par, c, w, S, h, mov, grains ? &e : nullptr, Sf);
                nacc += n;
                any = n != 0;
            }
            if constexpr (MOVE == 0 && GEN == 0) {
                if (colour == 0 && p.pfield) {
                    Spin4<float>* fld = static_cast<Spin4<float>*>(p.pfield) + q0 + 2u * uint32_t(lane);
                    fld[0] = Spin4<float>{h.x.x, h.y.x, h.z.x, 0.0f};
                    fld[1] = Spin4<float>{h.x.y, h.y.y, h.z.y, 0.0f};
                }
            }
            if (any) {  // both sites of the pair in one 8-byte store per component
                float* own = s + size_t(3 * colour) * p.stride + q0 + 2u * uint32_t(lane);
                *reinterpret_cast<float2*>(own) = Sf.x;
                *reinterpret_cast<float2*>(own + p.stride) = Sf.y;
                *reinterpret_cast<float2*>(own + 2 * size_t(p.stride)) = Sf.z;
            }
            if constexpr (MEASURE > 0) {
                if (sampled) pair_tile_parts<MEASURE, NS>(par, Sf, h, e, O, eo, lf);
                if (++nparts == uint32_t(kPartTiles)) {
                    fix += pair_parts_flush<NS>(lf, lane);
                    nparts = 0;
                }
            }
        }
        if constexpr (MEASURE > 0) {
            if (nparts) fix += pair_parts_flush<NS>(lf, lane);
        }
        if constexpr (MOVE != 0) {
            // a measured black pass closes the sweep itself; after an unmeasured
            // one row_close_kernel does (its warps then need no fence), and
            // slabs close in mc_slab_close
            const bool closes = MEASURE > 0 && colour == 1 && !(GEN != 0 && p.slab);
            publish(L->st, lane, nacc, MEASURE > 0, fix, colour, run, p.nblocks_site, closes, [&] {
                finalize_sweep(p, L->st, MEASURE > 0 ? 1 : 0, p.sample_torque != 0, lane);
            });
        } else {
            publish(L->st, lane, 0, true, fix, 3, run, p.nblocks_site, true,
                    [&] { finalize_sweep(p, L->st, 1, true, lane); });
        }
        ++l;
    }
}

// End of an unmeasured sweep of every lattice of g after its black pass, one
// warp per lattice (slabs are closed by mc_slab_close instead).  Launched
// after the pass with programmatic serialisation: it waits for the pass to
// complete, so the pass's warps publish their counts with no fence.
__global__ void row_close_kernel(GroupArgs g, int measure) {
    asm volatile("griddepcontrol.launch_dependents;");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int l = int(blockIdx.x);
    if (l >= g.n) return;
    LatDev* L = g.lats[l];
    if (L->p.slab) return;
    finalize_sweep(L->p, L->st, measure, L->p.sample_torque != 0, int(threadIdx.x & 31));
}

// ------------------------------------------------------------------------
// Slabs of one lattice split along z (the decomposition of Sec. 2's
// multi-GPU projection).  A slab's passes publish their accepted moves and
// sample sums but never close the sweep.  After the black pass each slab
// exports its counts (slab_export_kernel), the counts are summed over all
// slabs (an all-reduce between devices), and every slab closes the sweep
// from the totals (slab_close_kernel; slab_close_all_kernel does all three
// for slabs on one device): the cone rule of Table A1 with the total accepted
// count and movable sites, the sample with the total sums and sites, so
// that every slab keeps the same cone angle, sweep counter and samples as
// the unsplit lattice.
// ------------------------------------------------------------------------
constexpr int kMaxSlabs = 64;
// Halo planes of one colour of n slabs on one device: slab i's lower halo
// from slab i-1's last own plane and its upper halo from slab i+1's first
// own plane (periodic), component a at offset a * stride[i] of each base.
struct SlabHaloArgs {
    float* dst[kMaxSlabs][2];       // lower, upper halo plane (component 0)
    const float* src[kMaxSlabs][2]; // the neighbours' boundary planes
    uint32_t stride[kMaxSlabs];     // component stride of slab i (floats)
    uint32_t src_stride[kMaxSlabs][2];
    uint32_t plane;                 // sites of the colour per plane
    int n;
};

// Grid: (chunks of the plane, 2 sides, n slabs); a thread copies one site
// of the plane in all three components per step.
__global__ void slab_halo_kernel(SlabHaloArgs a) {
    const int i = int(blockIdx.z), side = int(blockIdx.y);
    float* dst = a.dst[i][side];
    const float* src = a.src[i][side];
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < a.plane; v += gridDim.x * blockDim.x)
#pragma unroll
        for (int c = 0; c < 3; ++c) dst[size_t(c) * a.stride[i] + v] = src[size_t(c) * a.src_stride[i][side] + v];
}

// Export, sum over the n slabs and close, fused for slabs on one device:
// warp w takes slabs w, w + 32, ...; the counts meet in shared memory.
struct SlabDevs {
    LatDev* lat[kMaxSlabs];
    int n;
};

__global__ void slab_close_all_kernel(SlabDevs d, int measure) {
    __shared__ long long words[kMaxSlabs][kSlabWords];
    __shared__ long long total[kSlabWords];
    const int lane = int(threadIdx.x & 31), warp = int(threadIdx.x >> 5), nw = int(blockDim.x >> 5);
    for (int i = warp; i < d.n; i += nw) {
        LatState& st = d.lat[i]->st;
        const LatParams& p = d.lat[i]->p;
        if (lane == 0) {
            words[i][0] = (long long)atomicExch(&st.acc, 0ull);
            words[i][1] = p.n_mov;
            words[i][2] = p.N - 2ll * p.Lx * p.Ly;
        }
        if (lane < kNumSums)
            words[i][3 + lane] = (long long)atomicExch(reinterpret_cast<unsigned long long*>(&st.sums[lane]), 0ull);
        if (lane >= 3 + kNumSums && lane < kSlabWords) words[i][lane] = 0;
    }
    __syncthreads();
    if (warp == 0 && lane < kSlabWords) {
        long long t = 0;
        for (int j = 0; j < d.n; ++j) t += words[j][lane];
        total[lane] = t;
    }
    __syncthreads();
    for (int i = warp; i < d.n; i += nw) {
        LatState& st = d.lat[i]->st;
        const LatParams& p = d.lat[i]->p;
        if (lane < kSlabWords) p.slab_counts[lane] = total[lane];
        if (lane == 0) st.acc = (unsigned long long)total[0];
        if (lane < kNumSums) st.sums[lane] = total[3 + lane];
        __syncwarp();
        finalize_sweep(p, st, measure, p.sample_torque != 0, lane, total[1], total[2]);
    }
}

// One warp: accepted moves, movable sites, own sites and the sums, moved
// out of the lattice's accumulators (which are cleared).
__global__ void slab_export_kernel(LatDev* L) {
    const int lane = int(threadIdx.x & 31);
    LatState& st = L->st;
    const LatParams& p = L->p;
    long long* c = p.slab_counts;
    if (lane == 0) {
        c[0] = (long long)atomicExch(&st.acc, 0ull);
        c[1] = p.n_mov;
        c[2] = p.N - 2ll * p.Lx * p.Ly;  // the halo planes are not the slab's
    }
    if (lane < kNumSums)
        c[3 + lane] = (long long)atomicExch(reinterpret_cast<unsigned long long*>(&st.sums[lane]), 0ull);
    if (lane >= 3 + kNumSums && lane < kSlabWords) c[lane] = 0;
}

// One warp: the sweep's end from the summed counts.
__global__ void slab_close_kernel(LatDev* L, int measure) {
    const int lane = int(threadIdx.x & 31);
    LatState& st = L->st;
    const LatParams& p = L->p;
    const long long* c = p.slab_counts;
    if (lane == 0) st.acc = (unsigned long long)c[0];
    if (lane < kNumSums) st.sums[lane] = c[3 + lane];
    __syncwarp();
    finalize_sweep(p, st, measure, p.sample_torque != 0, lane, c[1], c[2]);
}

}  // namespace mcgb
