// row_pass.cuh -- FP32 colour pass (Table A1) over row_fast lattices:
// periodic lattices whose rows of one colour split evenly over the lanes of a
// warp tile.  The kernel holds no general-geometry code, so that it runs in
// fewer registers than the general colour pass.
//
// Lane L of a tile of 64 colour indices q0 .. q0 + 63 takes the adjacent pair
// q = q0 + 2L, q + 1 of one row, so that every spin is read as a float2 (one
// copy per component for both sites) and one Philox call keys the draws of
// both sites to the first.  Rows of Lh <= 64 sites per colour are covered by
// groups of G = Lh/2 lanes (row_lanes), rows of Lh > 64 by segments of 64.
// The other colour's spins at k and k+1 give three of the four x neighbours
// of the pair; the fourth, at k-1 or k+2, is the neighbouring lane's pair,
// taken by a warp shuffle inside the row group (wrapping the row) or, at the
// ends of a 64-site segment of a longer row, loaded on its own.  The
// neighbour sum keeps the order -x, +x, -y, +y, -z, +z.
#pragma once
#include "pass_impl.cuh"

namespace mcgb {

constexpr int kRowSlots = 18;  // float2 loads per lane per tile

__device__ __forceinline__ float2 ld2(const float* a, size_t i) { return *reinterpret_cast<const float2*>(a + i); }

// Spins and neighbour sums of lane L's pair in the tile starting at q0;
// returns the lattice index of the pair's first site (its parity is the
// row's x offset).
__device__ __forceinline__ uint32_t row_pair_sums(const LatParams& p, const float* s, int colour, uint32_t q0,
                                                  int lane, V3<float> S[2], V3<float> h[2], V3<float> O[2]) {
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
    const V3<float> o0{v[3].x, v[4].x, v[5].x}, o1{v[3].y, v[4].y, v[5].y};
    // x neighbours: site 0 has o0 and (xoff ? o1 : lft), site 1 has o1 and
    // (xoff ? rgt : o0); the -x + +x sum is the same either way round
    const V3<float> a0 = xoff ? o1 : lft, a1 = xoff ? rgt : o0;
    h[0].x = ((((o0.x + a0.x) + v[6].x) + v[9].x) + v[12].x) + v[15].x;
    h[0].y = ((((o0.y + a0.y) + v[7].x) + v[10].x) + v[13].x) + v[16].x;
    h[0].z = ((((o0.z + a0.z) + v[8].x) + v[11].x) + v[14].x) + v[17].x;
    h[1].x = ((((o1.x + a1.x) + v[6].y) + v[9].y) + v[12].y) + v[15].y;
    h[1].y = ((((o1.y + a1.y) + v[7].y) + v[10].y) + v[13].y) + v[16].y;
    h[1].z = ((((o1.z + a1.z) + v[8].y) + v[11].y) + v[14].y) + v[17].y;
    S[0] = V3<float>{v[0].x, v[1].x, v[2].x};
    S[1] = V3<float>{v[0].y, v[1].y, v[2].y};
    O[0] = o0;
    O[1] = o1;
    return xoff + 2u * k + uint32_t(p.Lx) * row;
}

template <int MINB, int MEASURE>
__global__ void __launch_bounds__(kBlock, MINB) row_pass_kernel(GroupArgs g, uint32_t ntiles,
                                                                const float* __restrict__ cone, int colour) {
    constexpr int NS = MEASURE >= 2 ? kNumSums : kSumTux;  // sums sampled
    const WarpChunk wc = warp_chunk(ntiles);
    const int lane = wc.lane;
    const uint32_t tag = tag_of(colour, kPurposeMove);
    uint32_t tile = wc.begin;
    int l = tile < wc.end ? lattice_of_tile(g, tile) : 0;
    while (tile < wc.end) {
        LatDev* L = g.lats[l];
        const LatParams& p = L->p;
        const uint32_t t0 = __ldg(&g.start[l]);
        const uint32_t t1 = min(__ldg(&g.start[l + 1]), wc.end);
        const uint32_t run = t1 - tile;
        const Par<float> par = load_par<float>(p);
        const float c = cone[L->st.theta];
        const uint32_t sweep = L->st.sweep;
        float* __restrict__ s = static_cast<float*>(p.spins);
        const V3<float> e_ax{par.e[0], par.e[1], par.e[2]};
        unsigned nacc = 0;
        long long fix = 0;
        for (; tile < t1; ++tile) {
            V3<float> S[2], h[2], O[2];
            const uint32_t site0 = row_pair_sums(p, s, colour, (tile - t0) * 64u, lane, S, h, O);
            const uint4 w = philox(make_uint4(site0, sweep, tag, 0u), p.key0, p.key1);
            float P[2], sd[2], cp[2], sp[2];
            direct_draw_two(w, P, sd, cp, sp);
            V3<float> Sf[2];
            bool any = false;
#pragma unroll
            for (int v = 0; v < 2; ++v) {
                const V3<float> Sn = cap_point_direct(S[v], c, sd[v], cp[v], sp[v]);
                const bool acc = metropolis(delta_e(par, S[v], Sn, h[v], e_ax), par.T, P[v]);
                Sf[v] = acc ? Sn : S[v];
                nacc += acc ? 1u : 0u;
                any = any || acc;
            }
            if (any) {  // both sites of the pair in one 8-byte store per component
                float* own = s + size_t(3 * colour) * p.stride + (tile - t0) * 64u + 2u * uint32_t(lane);
                *reinterpret_cast<float2*>(own) = make_float2(Sf[0].x, Sf[1].x);
                *reinterpret_cast<float2*>(own + p.stride) = make_float2(Sf[0].y, Sf[1].y);
                *reinterpret_cast<float2*>(own + 2 * size_t(p.stride)) = make_float2(Sf[0].z, Sf[1].z);
            }
            if constexpr (MEASURE > 0) {
                Sums<float> sums;
#pragma unroll
                for (int i = 0; i < kNumSums; ++i) sums.v[i] = 0.0f;
                const bool nu = par.Ku != 0.0f, nc = par.Kc != 0.0f;
#pragma unroll
                for (int v = 0; v < 2; ++v) {
                    add_site<float, MEASURE>(sums, Sf[v], e_ax, nu, nc);
                    sums.v[kSumEx] += Sf[v].x * h[v].x + Sf[v].y * h[v].y + Sf[v].z * h[v].z;
                    add_site<float, MEASURE>(sums, O[v], e_ax, nu, nc);
                }
                fix += warp_tile_fix<float, NS>(sums, lane);
            }
        }
        publish(L->st, lane, nacc, MEASURE > 0, fix, colour, run, p.nblocks_site, [&] {
            if (colour == 1) finalize_sweep(p, L->st, MEASURE > 0 ? 1 : 0, p.sample_torque != 0);
        });
        ++l;
    }
}

}  // namespace mcgb
