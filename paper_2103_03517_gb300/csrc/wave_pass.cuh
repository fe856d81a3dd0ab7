// wave_pass.cuh -- one FP32 sweep of Table A1 (red pass, then black pass)
// in a single launch, for all-periodic lattices whose rows hold Lh = 64
// sites per colour (Lx = 128) and Ly >= 16: the 128^3 lattices of the
// batched m(T) workload.
//
// The sweep reads the spins from one buffer and writes every spin, moved or
// not, to a second one (LatParams::spins_alt), so that the old state stays
// readable for the whole launch.  A block owns a work unit: a band of ty <=
// 15 rows (y) times a slab of tz planes (z), full rows in x.  It marches up
// the slab: in phase j it updates red plane z0 - 1 + j and black plane
// z0 + j - 3, so that every black site sees its six red neighbours already
// moved, as the black pass of Table A1 does.  The red sites one row outside
// the band and one plane outside the slab are moved as well, from the old
// state, with the same draws as their owner block uses (the Philox counter
// is the site and the sweep): they are bit-identical to what the owner
// writes, and only the owner writes them or counts them.
//
// Work split: 16 warps, 4 per scheduler; in a phase warp w moves red row w
// and black row w of the band (row indices counted from the halo row below
// it), and warp 0 also red row 16 of a 15-row band: 32 rows of 64 sites
// per phase, two per warp, so that no warp or scheduler carries more of a
// phase than another.
//
// Staging (per block, dynamic shared memory): the old black planes of the
// band +- 2 rows (a ring of 6 planes, two phases ahead), the old red planes
// of the band +- 1 row (a ring of 3) and the new red planes (a ring of 4).
// The old planes arrive by bulk asynchronous copies (cp.async.bulk), issued
// by the lanes of warp 0 two phases before they are needed and tracked by
// one mbarrier per ring slot; every wait is bounded and, when it runs out,
// the lattice's error is set to MC_ERR_TIMEOUT and the block stops.
//
// Each spin is read once from HBM and written once per sweep (24 B per
// update, plus the halo rows and planes, which mostly hit L2).  The Philox
// counters, the trial points, the energy change and the sample sums are
// those of the two-pass row kernel (row_pass.cuh, pair_math.cuh), term for
// term and in the same order, so a wavefront sweep gives the spins of a red
// and a black row pass.
#pragma once
#include "pair_math.cuh"

namespace mcgb {

constexpr int kWaveWarps = 16;
constexpr int kWaveThreads = 32 * kWaveWarps;
constexpr int kWaveBRows = kWaveTyMax + 4;        // staged old black rows: band +- 2
constexpr int kWaveRRows = kWaveTyMax + 2;        // red rows: band +- 1
constexpr int kWaveBSlots = 6, kWaveROSlots = 3, kWaveRNSlots = 4;
constexpr int kWaveBComp = kWaveBRows * kWaveLh;  // floats of one component of a black slot
constexpr int kWaveRComp = kWaveRRows * kWaveLh;
constexpr size_t kWaveSmemFloats =
    size_t(kWaveBSlots) * 3 * kWaveBComp + size_t(kWaveROSlots + kWaveRNSlots) * 3 * kWaveRComp;
constexpr size_t kWaveSmemBytes = kWaveSmemFloats * 4 + 16 * 8;  // + the mbarriers
constexpr long long kWaveWaitCycles = 1ll << 31;  // about one second at 2 GHz
static_assert(kWaveTyMax + 2 <= 2 * kWaveWarps + 1, "the red rows of a band must fit the warps' tasks");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of the given parity to complete; false if it does not
// within kWaveWaitCycles.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaveWaitCycles) return false;
    return true;
}

// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned)
// from global to this block's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// One staged plane: rows y_first .. y_first + nrows - 1 (wrapped in Ly) of
// plane z of one colour, into a ring slot laid out [3][cap][64] (cap rows
// per component), completing on bar.
struct StagePlane {
    float* slot;
    const float* colour_base;
    int cap, y_first, nrows, z;
    uint64_t* bar;
};

// Piece `piece` (0, 1, 2) of component a of a staged plane: the rows of the
// plane split where they wrap in Ly (y_first >= -2, nrows <= Ly + 4, so at
// most three pieces).
__device__ __forceinline__ void stage_piece(const StagePlane& s, uint32_t stride, int Ly, int a, int piece,
                                            uint64_t* bar) {
    int y = s.y_first < 0 ? s.y_first + Ly : s.y_first, done = 0, n = min(s.nrows, Ly - y);
    for (int k = 0; k < piece; ++k) {  // skip to the piece
        done += n;
        y = 0;
        n = min(s.nrows - done, Ly);
    }
    if (n <= 0) return;
    const float* src = s.colour_base + size_t(a) * stride + (size_t(s.z) * size_t(Ly) + size_t(y)) * kWaveLh;
    bulk_g2s(s.slot + (a * s.cap + done) * kWaveLh, src, uint32_t(n * kWaveLh * 4), bar);
}

__device__ __forceinline__ float2 lds2(const float* row, int lane) {
    return *reinterpret_cast<const float2*>(row + 2 * lane);
}

// Spins and neighbour sums of lane L's two sites (colour indices 2L, 2L + 1)
// of one row, all rows in shared memory, packed (site 0 in .x): own (the
// site's colour), and of the other colour the same row xr and the rows -y,
// +y, -z and +z, each row with its own component stride (cs_*, floats).
// The x neighbours and the sums are those of the row kernel: -x + +x, then
// -y, +y, -z, +z.
__device__ __forceinline__ void wave_pair_sums(const float* own, int cs_own, const float* xr, int cs_xr,
                                               const float* ym, int cs_ym, const float* yp, int cs_yp,
                                               const float* zm, int cs_zm, const float* zp, int cs_zp, int lane,
                                               uint32_t xoff, P3& S, P3& h, P3& O) {
    float2 v[18];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        v[a] = lds2(own + a * cs_own, lane);
        v[3 + a] = lds2(xr + a * cs_xr, lane);
        v[6 + a] = lds2(ym + a * cs_ym, lane);
        v[9 + a] = lds2(yp + a * cs_yp, lane);
        v[12 + a] = lds2(zm + a * cs_zm, lane);
        v[15 + a] = lds2(zp + a * cs_zp, lane);
    }
    const int left = (lane - 1) & 31, right = (lane + 1) & 31;  // a row is the whole warp, wrapped
    const V3<float> lft{__shfl_sync(0xffffffffu, v[3].y, left), __shfl_sync(0xffffffffu, v[4].y, left),
                        __shfl_sync(0xffffffffu, v[5].y, left)};
    const V3<float> rgt{__shfl_sync(0xffffffffu, v[3].x, right), __shfl_sync(0xffffffffu, v[4].x, right),
                        __shfl_sync(0xffffffffu, v[5].x, right)};
    O = P3{v[3], v[4], v[5]};
    const P3 a{make_float2(xoff ? v[3].y : lft.x, xoff ? rgt.x : v[3].x),
               make_float2(xoff ? v[4].y : lft.y, xoff ? rgt.y : v[4].x),
               make_float2(xoff ? v[5].y : lft.z, xoff ? rgt.z : v[5].x)};
    h.x = p2add(p2add(p2add(p2add(p2add(O.x, a.x), v[6]), v[9]), v[12]), v[15]);
    h.y = p2add(p2add(p2add(p2add(p2add(O.y, a.y), v[7]), v[10]), v[13]), v[16]);
    h.z = p2add(p2add(p2add(p2add(p2add(O.z, a.z), v[8]), v[11]), v[14]), v[17]);
    S = P3{v[0], v[1], v[2]};
}

__device__ __forceinline__ void sts_p3(float* row, int cs, int lane, const P3& v) {
    *reinterpret_cast<float2*>(row + 2 * lane) = v.x;
    *reinterpret_cast<float2*>(row + cs + 2 * lane) = v.y;
    *reinterpret_cast<float2*>(row + 2 * cs + 2 * lane) = v.z;
}

__device__ __forceinline__ void stg_pair(float* colour_base, uint32_t stride, uint32_t q, const P3& Sf) {
    float* d = colour_base + q;
    *reinterpret_cast<float2*>(d) = Sf.x;
    *reinterpret_cast<float2*>(d + stride) = Sf.y;
    *reinterpret_cast<float2*>(d + 2 * size_t(stride)) = Sf.z;
}

// dir = 0: read spins, write spins_alt; dir = 1: the reverse.  MEASURE as
// in the row kernel (1: magnetisation and energies, 2: also torques); the
// block that finishes a lattice's last work unit closes its sweep.
template <int MEASURE>
__global__ void __launch_bounds__(kWaveThreads, 1) wave_sweep_kernel(WaveArgs a, const float* __restrict__ cone,
                                                                     int dir) {
    constexpr int NS = MEASURE >= 2 ? kNumSums : kSumTux;
    extern __shared__ __align__(128) float wsm[];
    float* bslot = wsm;                                               // [6][3][19][64] old black
    float* roslot = bslot + kWaveBSlots * 3 * kWaveBComp;             // [3][3][17][64] old red
    float* rnslot = roslot + kWaveROSlots * 3 * kWaveRComp;           // [4][3][17][64] new red
    uint64_t* bar = reinterpret_cast<uint64_t*>(rnslot + kWaveRNSlots * 3 * kWaveRComp);  // 6 + 3
    __shared__ int abort_flag;
    asm volatile("griddepcontrol.launch_dependents;");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        for (int i = 0; i < kWaveBSlots + kWaveROSlots; ++i) mbar_init(&bar[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    __syncthreads();
    asm volatile("griddepcontrol.wait;" ::: "memory");
    uint32_t nb = 0, nr = 0;  // staged copies planned so far (old black, old red): ring slot and parity
    uint32_t ib = 0, ir = 0;  // planes issued so far (warp 0)
    const uint32_t w_end = a.off[blockIdx.x + 1];
    bool aborted = false;
    uint32_t extra = blockIdx.x == 0 ? uint32_t(a.inject) : 0u;  // warp 0 only
    for (uint32_t wi = a.off[blockIdx.x]; wi < w_end && !aborted; ++wi) {
        const WaveWU u = a.wu[wi];
        LatDev* L = a.lats[u.lat];
        const LatParams& p = L->p;
        const Par<float> par = load_par<float>(p);
        const int Ly = p.Ly, Lz = p.Lz, tz = int(u.tz), ty = int(u.ty), y0 = int(u.y0), z0 = int(u.z0);
        const uint32_t stride = p.stride, Lx = uint32_t(p.Lx);
        const uint32_t sweep = L->st.sweep;
        const PhiloxKeys K = philox_keys(p.key0, p.key1);
        const float c = cone[L->st.theta];
        const float* src = static_cast<const float*>(dir ? p.spins_alt : p.spins);
        float* dst = static_cast<float*>(dir ? p.spins : p.spins_alt);
        float* dst_red = dst;
        float* dst_blk = dst + 3 * size_t(stride);
        const uint32_t nb0 = nb, nr0 = nr;
        // old black plane index i = plane z0 - 2 + i (i = 0 .. tz + 3), rows
        // y0 - 2 .. y0 + ty + 1; old red index i = plane z0 - 1 + i (i = 0 ..
        // tz + 1), rows y0 - 1 .. y0 + ty
        auto b_plane = [&](int i) {
            const uint32_t g = nb0 + uint32_t(i);
            const int z = z0 - 2 + i;  // in [-2, Lz + 1], Lz >= 2
            return StagePlane{bslot + (g % kWaveBSlots) * 3 * kWaveBComp, src + 3 * size_t(stride), kWaveBRows,
                              y0 - 2, ty + 4, z < 0 ? z + Lz : (z >= Lz ? z - Lz : z), &bar[g % kWaveBSlots]};
        };
        auto r_plane = [&](int i) {
            const uint32_t g = nr0 + uint32_t(i);
            const int z = z0 - 1 + i;  // in [-1, Lz]
            return StagePlane{roslot + (g % kWaveROSlots) * 3 * kWaveRComp, src, kWaveRRows, y0 - 1, ty + 2,
                              z < 0 ? z + Lz : (z >= Lz ? z - Lz : z), &bar[kWaveBSlots + g % kWaveROSlots]};
        };
        // warp 0 stages old black planes b_lo .. b_hi - 1 and old red planes
        // r_lo .. r_hi - 1: lane 0 arms each plane's barrier with its bytes,
        // then the lanes issue the pieces (plane, piece, component) between them
        auto stage = [&](int b_lo, int b_hi, int r_lo, int r_hi) {
            const int nbp = max(b_hi - b_lo, 0), nrp = max(r_hi - r_lo, 0);
            if (lane == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                for (int i = 0; i < nbp + nrp; ++i) {
                    const StagePlane sp = i < nbp ? b_plane(b_lo + i) : r_plane(r_lo + i - nbp);
                    mbar_expect_tx(sp.bar, uint32_t(3 * sp.nrows * kWaveLh * 4) + extra);
                    extra = 0;
                }
                if (nbp) ib = nb0 + uint32_t(b_hi);
                if (nrp) ir = nr0 + uint32_t(r_hi);
            }
            __syncwarp();
            for (int k = lane; k < 9 * (nbp + nrp); k += 32) {
                const int i = k / 9, piece = (k % 9) / 3, comp = k % 3;
                const StagePlane sp = i < nbp ? b_plane(b_lo + i) : r_plane(r_lo + i - nbp);
                stage_piece(sp, stride, Ly, comp, piece, sp.bar);
            }
        };
        if (warp == 0) stage(0, 5, 0, 3);
        nb += uint32_t(tz + 4);
        nr += uint32_t(tz + 2);
        unsigned nacc = 0;
        long long fix = 0;
        for (int j = 0; j <= tz + 2; ++j) {
            if (j > 0 && warp == 0) stage(j + 4, min(j + 5, tz + 4), j + 2, min(j + 3, tz + 2));
            const bool red = j <= tz + 1, black = j >= 3;
            if (red) {  // old black planes j .. j + 2 and old red plane j
                bool ok = true;
                for (int i = (j == 0 ? 0 : j + 2); i <= j + 2; ++i) {
                    const uint32_t g = nb0 + uint32_t(i);
                    ok = ok && mbar_wait(&bar[g % kWaveBSlots], (g / kWaveBSlots) & 1u);
                }
                const uint32_t g = nr0 + uint32_t(j);
                ok = ok && mbar_wait(&bar[kWaveBSlots + g % kWaveROSlots], (g / kWaveROSlots) & 1u);
                if (!ok) abort_flag = 1;
            }
            // ring slots of this phase (uniform over the block): red plane
            // zr = z0 - 1 + j reads old black j .. j + 2 and old red j, writes
            // new red j; black plane zb = z0 + j - 3 reads old black j - 1 and
            // new red j - 3 .. j - 1
            const float* b0 = bslot + ((nb0 + j) % kWaveBSlots) * 3 * kWaveBComp;      // plane zr - 1
            const float* b1 = bslot + ((nb0 + j + 1) % kWaveBSlots) * 3 * kWaveBComp;  // plane zr
            const float* b2 = bslot + ((nb0 + j + 2) % kWaveBSlots) * 3 * kWaveBComp;  // plane zr + 1
            const float* ro = roslot + ((nr0 + j) % kWaveROSlots) * 3 * kWaveRComp;
            float* rn = rnslot + (j % kWaveRNSlots) * 3 * kWaveRComp;
            const float* bo = bslot + ((nb0 + j + kWaveBSlots - 1) % kWaveBSlots) * 3 * kWaveBComp;
            const float* rm = rnslot + ((j + 1) % kWaveRNSlots) * 3 * kWaveRComp;  // j - 3: plane zb - 1
            const float* r0 = rnslot + ((j + 2) % kWaveRNSlots) * 3 * kWaveRComp;  // j - 2: plane zb
            const float* rp = rnslot + ((j + 3) % kWaveRNSlots) * 3 * kWaveRComp;  // j - 1: plane zb + 1
            int zr = z0 - 1 + j;  // in [-1, Lz]
            zr = zr < 0 ? zr + Lz : (zr >= Lz ? zr - Lz : zr);
            int zb = z0 + j - 3;
            zb = zb >= Lz ? zb - Lz : zb;
            // warp w: red row w, then black row w (rows counted from the halo
            // row below the band: red 0 .. ty + 1, black 1 .. ty); warp 0 takes
            // red row 16 of a 15-row band in place of a black row
            for (int k = 0; k < 2; ++k) {
                const bool is_red = k == 0 || warp == 0;
                const int r = k == 0 ? warp : (warp == 0 ? kWaveWarps : warp);
                if (is_red ? !(red && r <= ty + 1) : !(black && r <= ty)) continue;
                P3 S, h, O, Sf;
                const bool mov[2] = {true, true};
                if (is_red) {  // red row r of plane zr
                    int y = y0 - 1 + r;  // in [-1, Ly]
                    y = y < 0 ? y + Ly : (y >= Ly ? y - Ly : y);
                    const uint32_t xoff = uint32_t(y + zr) & 1u;
                    wave_pair_sums(ro + r * kWaveLh, kWaveRComp, b1 + (r + 1) * kWaveLh, kWaveBComp,
                                   b1 + r * kWaveLh, kWaveBComp, b1 + (r + 2) * kWaveLh, kWaveBComp,
                                   b0 + (r + 1) * kWaveLh, kWaveBComp, b2 + (r + 1) * kWaveLh, kWaveBComp, lane,
                                   xoff, S, h, O);
                    const uint32_t row = uint32_t(y) + uint32_t(Ly) * uint32_t(zr);
                    const uint32_t site0 = xoff + 4u * uint32_t(lane) + Lx * row;
                    const uint4 w = philox_rk(make_uint4(site0, sweep, tag_of(0, kPurposeMove), 0u), K);
                    const unsigned n = pair_move(par, c, w, S, h, mov, nullptr, Sf);
                    sts_p3(rn + r * kWaveLh, kWaveRComp, lane, Sf);
                    if (r >= 1 && r <= ty && j >= 1 && j <= tz) {  // owned: in the band and the slab
                        stg_pair(dst_red, stride, row * kWaveLh + 2u * uint32_t(lane), Sf);
                        nacc += n;
                    }
                } else {  // black row r of plane zb
                    const int y = y0 - 1 + r;
                    const uint32_t xoff = uint32_t(y + zb + 1) & 1u;
                    wave_pair_sums(bo + (r + 1) * kWaveLh, kWaveBComp, r0 + r * kWaveLh, kWaveRComp,
                                   r0 + (r - 1) * kWaveLh, kWaveRComp, r0 + (r + 1) * kWaveLh, kWaveRComp,
                                   rm + r * kWaveLh, kWaveRComp, rp + r * kWaveLh, kWaveRComp, lane, xoff, S, h, O);
                    const uint32_t row = uint32_t(y) + uint32_t(Ly) * uint32_t(zb);
                    const uint32_t site0 = xoff + 4u * uint32_t(lane) + Lx * row;
                    const uint4 w = philox_rk(make_uint4(site0, sweep, tag_of(1, kPurposeMove), 0u), K);
                    nacc += pair_move(par, c, w, S, h, mov, nullptr, Sf);
                    stg_pair(dst_blk, stride, row * kWaveLh + 2u * uint32_t(lane), Sf);
                    if constexpr (MEASURE > 0) {
                        const P3 e{p2(par.e[0]), p2(par.e[1]), p2(par.e[2])};
                        fix += pair_tile_sample<MEASURE, NS>(par, Sf, h, e, O, e, lane);
                    }
                }
            }
            __syncthreads();
            if (abort_flag) {
                aborted = true;
                break;
            }
        }
        // counts of the unit, then the lattice's unit count; the block that
        // completes the lattice closes its sweep
        nacc = __reduce_add_sync(0xffffffffu, nacc);
        if (lane == 0 && nacc) atomicAdd(&L->st.acc, (unsigned long long)nacc);
        if (MEASURE > 0 && lane < kNumSums && fix)
            atomicAdd(reinterpret_cast<unsigned long long*>(&L->st.sums[lane]), static_cast<unsigned long long>(fix));
        if (aborted) {
            if (tid == 0) atomicCAS(&L->st.error, 0, -4);  // MC_ERR_TIMEOUT
            break;
        }
        __threadfence();
        __syncthreads();
        if (MEASURE == 0 && tid == 0) {
            const unsigned prev = atomicAdd(&L->st.done[1], 1u);
            if (prev + 1 == a.nwu[u.lat]) {
                __threadfence();
                L->st.done[1] = 0;
                finalize_sweep_unmeasured(p, L->st);
            }
        }
        if (MEASURE > 0 && warp == 0) {  // the whole warp closes a measured sweep if this unit completes the lattice
            unsigned closing = 0;
            if (lane == 0) {
                const unsigned prev = atomicAdd(&L->st.done[1], 1u);
                if (prev + 1 == a.nwu[u.lat]) {
                    __threadfence();
                    L->st.done[1] = 0;
                    closing = 1;
                }
            }
            if (__shfl_sync(0xffffffffu, closing, 0)) {
                __threadfence();
                finalize_sweep(p, L->st, 1, p.sample_torque != 0, lane);
            }
            __syncwarp();
        }
    }
    // no copy may still be writing this block's shared memory when it exits:
    // wait (bounded) on the last plane issued to every slot
    if (aborted && tid == 0) {
        for (int s = 0; s < kWaveBSlots; ++s)
            if (ib > uint32_t(s)) {
                const uint32_t g = ib - 1 - uint32_t(s);
                mbar_wait(&bar[g % kWaveBSlots], (g / kWaveBSlots) & 1u);
            }
        for (int s = 0; s < kWaveROSlots; ++s)
            if (ir > uint32_t(s)) {
                const uint32_t g = ir - 1 - uint32_t(s);
                mbar_wait(&bar[kWaveBSlots + g % kWaveROSlots], (g / kWaveROSlots) & 1u);
            }
    }
}

}  // namespace mcgb
