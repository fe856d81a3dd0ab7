// wave_pass.cuh -- one FP32 sweep of Table A1 (red pass, then black pass)
// in a single launch, for all-periodic lattices whose rows hold Lh = 64
// sites per colour (Lx = 128) and Ly a multiple of 16: the 128^3 lattices of
// the batched m(T) workload.
//
// The sweep reads the spins from one buffer and writes every spin, moved or
// not, to a second one (LatParams::spins_alt), so that the old state stays
// readable for the whole launch.  A block owns a work unit: a band of 16
// rows (y) times a slab of tz planes (z), full rows in x.  It marches up the
// slab: in phase j it updates red plane z0 - 1 + j and black plane z0 + j - 3,
// so that every black site sees its six red neighbours already moved, as the
// black pass of Table A1 does.  The red sites one row outside the band and
// one plane outside the slab are moved as well, from the old state, with
// the same draws as their owner block uses (the Philox counter is the site
// and the sweep): they are bit-identical to what the owner writes, and only
// the owner writes them or counts them.
//
// Staging (per block, dynamic shared memory): the old black planes of the
// band +- 2 rows (a ring of 6 planes, two phases ahead), the old red planes
// of the band +- 1 row (a ring of 3) and the new red planes (a ring of 4).
// The old planes arrive by bulk asynchronous copies (cp.async.bulk), issued
// by one thread two phases before they are needed and tracked by one
// mbarrier per ring slot; every wait is bounded and, when it runs out, the
// lattice's error is set to MC_ERR_TIMEOUT and the block stops.
//
// Each spin is read once from HBM and written once per sweep (24 B per
// update, plus the halo rows and planes, which mostly hit L2).  The Philox
// counters, the trial points, the energy change and the sample sums are
// those of the two-pass row kernel (row_pass.cuh), term for term and in the
// same order, so a wavefront sweep gives the spins of a red and a black row
// pass.
#pragma once
#include "pass_impl.cuh"

namespace mcgb {

constexpr int kWaveWarps = 17;                    // 18 red + 16 black rows = 2 rows per warp a phase
constexpr int kWaveThreads = 32 * kWaveWarps;
constexpr int kWaveBRows = kWaveTy + 4;           // staged old black rows: band +- 2
constexpr int kWaveRRows = kWaveTy + 2;           // red rows: band +- 1
constexpr int kWaveBSlots = 6, kWaveROSlots = 3, kWaveRNSlots = 4;
constexpr int kWaveBComp = kWaveBRows * kWaveLh;  // floats of one component of a black slot
constexpr int kWaveRComp = kWaveRRows * kWaveLh;
constexpr size_t kWaveSmemFloats =
    size_t(kWaveBSlots) * 3 * kWaveBComp + size_t(kWaveROSlots + kWaveRNSlots) * 3 * kWaveRComp;
constexpr size_t kWaveSmemBytes = kWaveSmemFloats * 4 + 16 * 8;  // + the mbarriers
constexpr long long kWaveWaitCycles = 1ll << 31;  // about one second at 2 GHz

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

// Stage rows y_first .. y_first + nrows - 1 (wrapped in Ly) of plane z of
// one colour into a ring slot laid out [3][nrows][64]: one expect_tx for
// the whole plane, then up to three contiguous pieces per component.
__device__ __forceinline__ void wave_stage(float* slot, const float* colour_base, uint32_t stride, int Ly,
                                           int y_first, int nrows, int z, uint64_t* bar, uint32_t extra) {
    mbar_expect_tx(bar, uint32_t(3 * nrows * kWaveLh * 4) + extra);
    const float* plane = colour_base + size_t(z) * size_t(Ly) * kWaveLh;
    for (int a = 0; a < 3; ++a) {
        const float* comp = plane + size_t(a) * stride;
        float* d = slot + a * nrows * kWaveLh;
        int y = y_first < 0 ? y_first + Ly : y_first, left = nrows;  // y_first in [-2, Ly)
        while (left > 0) {
            const int n = min(left, Ly - y);
            bulk_g2s(d, comp + size_t(y) * kWaveLh, uint32_t(n * kWaveLh * 4), bar);
            d += n * kWaveLh;
            left -= n;
            y = 0;
        }
    }
}

__device__ __forceinline__ float2 lds2(const float* row, int lane) {
    return *reinterpret_cast<const float2*>(row + 2 * lane);
}

// Spins and neighbour sums of lane L's two sites (colour indices 2L, 2L + 1)
// of one row, all rows in shared memory: own (the site's colour, component
// stride cs_own), and of the other colour the same row xr and the rows -y,
// +y (component stride cs_xy), -z (cs_zm) and +z (cs_zp).  The x neighbours
// and the sums are those of the row kernel: -x + +x, then -y, +y, -z, +z.
__device__ __forceinline__ void wave_pair_sums(const float* own, int cs_own, const float* xr, const float* ym,
                                               const float* yp, int cs_xy, const float* zm, int cs_zm,
                                               const float* zp, int cs_zp, int lane, uint32_t xoff, V3<float> S[2],
                                               V3<float> h[2], V3<float> O[2]) {
    float2 v[18];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        v[a] = lds2(own + a * cs_own, lane);
        v[3 + a] = lds2(xr + a * cs_xy, lane);
        v[6 + a] = lds2(ym + a * cs_xy, lane);
        v[9 + a] = lds2(yp + a * cs_xy, lane);
        v[12 + a] = lds2(zm + a * cs_zm, lane);
        v[15 + a] = lds2(zp + a * cs_zp, lane);
    }
    const int left = (lane - 1) & 31, right = (lane + 1) & 31;  // a row is the whole warp, wrapped
    const V3<float> lft{__shfl_sync(0xffffffffu, v[3].y, left), __shfl_sync(0xffffffffu, v[4].y, left),
                        __shfl_sync(0xffffffffu, v[5].y, left)};
    const V3<float> rgt{__shfl_sync(0xffffffffu, v[3].x, right), __shfl_sync(0xffffffffu, v[4].x, right),
                        __shfl_sync(0xffffffffu, v[5].x, right)};
    const V3<float> o0{v[3].x, v[4].x, v[5].x}, o1{v[3].y, v[4].y, v[5].y};
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
}

// Trial moves and Metropolis tests of lane L's two sites (Table A1, Eq. 1-2),
// with the draws of the row kernel: one Philox call keyed by the first site.
__device__ __forceinline__ unsigned wave_move(const Par<float>& par, float c, uint32_t site0, uint32_t sweep,
                                              uint32_t tag, uint32_t k0, uint32_t k1, const V3<float> S[2],
                                              const V3<float> h[2], V3<float> Sf[2]) {
    const V3<float> e_ax{par.e[0], par.e[1], par.e[2]};
    const uint4 w = philox(make_uint4(site0, sweep, tag, 0u), k0, k1);
    float P[2], sd[2], cp[2], sp[2];
    direct_draw_two(w, P, sd, cp, sp);
    unsigned nacc = 0;
#pragma unroll
    for (int v = 0; v < 2; ++v) {
        const V3<float> Sn = cap_point_direct(S[v], c, sd[v], cp[v], sp[v]);
        const bool acc = metropolis(delta_e(par, S[v], Sn, h[v], e_ax), par, P[v]);
        Sf[v] = acc ? Sn : S[v];
        nacc += acc ? 1u : 0u;
    }
    return nacc;
}

__device__ __forceinline__ void sts2(float* row, int lane, float a, float b) {
    *reinterpret_cast<float2*>(row + 2 * lane) = make_float2(a, b);
}

__device__ __forceinline__ void stg_pair(float* colour_base, uint32_t stride, uint32_t q, const V3<float> Sf[2]) {
    float* d = colour_base + q;
    *reinterpret_cast<float2*>(d) = make_float2(Sf[0].x, Sf[1].x);
    *reinterpret_cast<float2*>(d + stride) = make_float2(Sf[0].y, Sf[1].y);
    *reinterpret_cast<float2*>(d + 2 * size_t(stride)) = make_float2(Sf[0].z, Sf[1].z);
}

// dir = 0: read spins, write spins_alt; dir = 1: the reverse.  MEASURE as
// in the row kernel (1: magnetisation and energies, 2: also torques); the
// block that finishes a lattice's last work unit closes its sweep.
template <int MEASURE>
__global__ void __launch_bounds__(kWaveThreads, 1) wave_sweep_kernel(WaveArgs a, const float* __restrict__ cone,
                                                                     int dir) {
    constexpr int NS = MEASURE >= 2 ? kNumSums : kSumTux;
    extern __shared__ __align__(128) float wsm[];
    float* bslot = wsm;                                               // [6][3][20][64] old black
    float* roslot = bslot + kWaveBSlots * 3 * kWaveBComp;             // [3][3][18][64] old red
    float* rnslot = roslot + kWaveROSlots * 3 * kWaveRComp;           // [4][3][18][64] new red
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
    uint32_t ib = 0, ir = 0;  // copies issued so far (thread 0)
    const uint32_t w_end = a.off[blockIdx.x + 1];
    bool aborted = false;
    int extra = blockIdx.x == 0 ? a.inject : 0;
    for (uint32_t wi = a.off[blockIdx.x]; wi < w_end && !aborted; ++wi) {
        const WaveWU u = a.wu[wi];
        LatDev* L = a.lats[u.lat];
        const LatParams& p = L->p;
        const Par<float> par = load_par<float>(p);
        const int Ly = p.Ly, Lz = p.Lz, tz = int(u.tz), y0 = int(u.y0), z0 = int(u.z0);
        const uint32_t stride = p.stride, Lx = uint32_t(p.Lx);
        const uint32_t sweep = L->st.sweep, k0 = p.key0, k1 = p.key1;
        const float c = cone[L->st.theta];
        const float* src = static_cast<const float*>(dir ? p.spins_alt : p.spins);
        float* dst = static_cast<float*>(dir ? p.spins : p.spins_alt);
        const float* src_red = src;
        const float* src_blk = src + 3 * size_t(stride);
        float* dst_red = dst;
        float* dst_blk = dst + 3 * size_t(stride);
        const uint32_t nb0 = nb, nr0 = nr;
        // old black plane index i = plane z0 - 2 + i (i = 0 .. tz + 3), old red
        // index i = plane z0 - 1 + i (i = 0 .. tz + 1)
        auto issue_b = [&](int i) {
            const uint32_t g = nb0 + uint32_t(i);
            const int z = z0 - 2 + i;  // in [-2, Lz + 1], Lz >= 2
            wave_stage(bslot + (g % kWaveBSlots) * 3 * kWaveBComp, src_blk, stride, Ly, y0 - 2, kWaveBRows,
                       z < 0 ? z + Lz : (z >= Lz ? z - Lz : z), &bar[g % kWaveBSlots], uint32_t(extra));
            extra = 0;
            ib = g + 1;
        };
        auto issue_r = [&](int i) {
            const uint32_t g = nr0 + uint32_t(i);
            const int z = z0 - 1 + i;  // in [-1, Lz]
            wave_stage(roslot + (g % kWaveROSlots) * 3 * kWaveRComp, src_red, stride, Ly, y0 - 1, kWaveRRows,
                       z < 0 ? z + Lz : (z >= Lz ? z - Lz : z), &bar[kWaveBSlots + g % kWaveROSlots], 0u);
            ir = g + 1;
        };
        if (tid == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            for (int i = 0; i < 5; ++i) issue_b(i);
            for (int i = 0; i < 3; ++i) issue_r(i);
        }
        nb += uint32_t(tz + 4);
        nr += uint32_t(tz + 2);
        unsigned nacc = 0;
        long long fix = 0;
        for (int j = 0; j <= tz + 2; ++j) {
            if (j > 0 && tid == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                if (j + 4 <= tz + 3) issue_b(j + 4);
                if (j + 2 <= tz + 1) issue_r(j + 2);
            }
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
            const int nred = red ? kWaveRRows : 0, ntask = nred + (black ? kWaveTy : 0);
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
            for (int t = warp; t < ntask; t += kWaveWarps) {
                V3<float> S[2], h[2], O[2], Sf[2];
                if (t < nred) {  // red row r of plane zr
                    const int r = t;
                    int y = y0 - 1 + r;  // in [-1, Ly]
                    y = y < 0 ? y + Ly : (y >= Ly ? y - Ly : y);
                    const uint32_t xoff = uint32_t(y + zr) & 1u;
                    wave_pair_sums(ro + r * kWaveLh, kWaveRComp, b1 + (r + 1) * kWaveLh, b1 + r * kWaveLh,
                                   b1 + (r + 2) * kWaveLh, kWaveBComp, b0 + (r + 1) * kWaveLh, kWaveBComp,
                                   b2 + (r + 1) * kWaveLh, kWaveBComp, lane, xoff, S, h, O);
                    const uint32_t row = uint32_t(y) + uint32_t(Ly) * uint32_t(zr);
                    const uint32_t site0 = xoff + 4u * uint32_t(lane) + Lx * row;
                    const unsigned n = wave_move(par, c, site0, sweep, tag_of(0, kPurposeMove), k0, k1, S, h, Sf);
                    float* rw = rn + r * kWaveLh;
                    sts2(rw, lane, Sf[0].x, Sf[1].x);
                    sts2(rw + kWaveRComp, lane, Sf[0].y, Sf[1].y);
                    sts2(rw + 2 * kWaveRComp, lane, Sf[0].z, Sf[1].z);
                    if (r >= 1 && r <= kWaveTy && j >= 1 && j <= tz) {  // owned: in the band and the slab
                        stg_pair(dst_red, stride, row * kWaveLh + 2u * uint32_t(lane), Sf);
                        nacc += n;
                    }
                } else {  // black row r of plane zb
                    const int r = t - nred + 1;
                    const int y = y0 - 1 + r;
                    const uint32_t xoff = uint32_t(y + zb + 1) & 1u;
                    wave_pair_sums(bo + (r + 1) * kWaveLh, kWaveBComp, r0 + r * kWaveLh, r0 + (r - 1) * kWaveLh,
                                   r0 + (r + 1) * kWaveLh, kWaveRComp, rm + r * kWaveLh, kWaveRComp,
                                   rp + r * kWaveLh, kWaveRComp, lane, xoff, S, h, O);
                    const uint32_t row = uint32_t(y) + uint32_t(Ly) * uint32_t(zb);
                    const uint32_t site0 = xoff + 4u * uint32_t(lane) + Lx * row;
                    nacc += wave_move(par, c, site0, sweep, tag_of(1, kPurposeMove), k0, k1, S, h, Sf);
                    stg_pair(dst_blk, stride, row * kWaveLh + 2u * uint32_t(lane), Sf);
                    if constexpr (MEASURE > 0) {
                        Sums<float> sums;
#pragma unroll
                        for (int i = 0; i < kNumSums; ++i) sums.v[i] = 0.0f;
                        const bool nu = par.Ku != 0.0f, nc = par.Kc != 0.0f;
                        const V3<float> e_ax{par.e[0], par.e[1], par.e[2]};
#pragma unroll
                        for (int v = 0; v < 2; ++v) {
                            add_site<float, MEASURE>(sums, Sf[v], e_ax, nu, nc);
                            sums.v[kSumEx] += Sf[v].x * h[v].x + Sf[v].y * h[v].y + Sf[v].z * h[v].z;
                            add_site<float, MEASURE>(sums, O[v], e_ax, nu, nc);
                        }
                        fix += warp_tile_fix<float, NS>(sums, lane);
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
        if (tid == 0) {
            const unsigned prev = atomicAdd(&L->st.done[1], 1u);
            if (prev + 1 == a.nwu[u.lat]) {
                __threadfence();
                L->st.done[1] = 0;
                finalize_sweep(p, L->st, MEASURE > 0 ? 1 : 0, p.sample_torque != 0);
            }
        }
    }
    // no copy may still be writing this block's shared memory when it exits:
    // wait (bounded) on the last copy issued to every slot
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
