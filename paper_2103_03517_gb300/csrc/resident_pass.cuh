// resident_pass.cuh -- FP32 sweeps of Table A1 over one lattice held in the
// SMs' shared memory for a whole run of sweeps: every axis periodic, rows of
// Lh = 64 sites per colour (Lx = 128), and few enough rows that they fit the
// blocks' shared memory (a 128^3 lattice, 25 MB of spins, on 152 SMs).
//
// The lattice's rows (y, z) are cut into nyc x nzc bricks of whole rows, one
// per block of a cooperative launch (every block resident at once).  A block
// loads its brick, both colours, into shared memory once, runs the launch's
// sweeps on it and writes it back at the end.  In a colour pass a warp takes
// one row of the brick at a time: 64 sites of the colour, two per lane, as in
// the row kernel, with the same neighbour sums in the same order, the same
// draws keyed by site and sweep, the same trial point and test.  The chain is
// therefore the row passes' chain, bit for bit.
//
// Neighbours in other bricks.  The rows on a brick's faces are also written
// to the lattice in global memory as they are moved; once all of them are,
// the block publishes the pass (ResCtl::done, a release), half-way through
// it.  At the start of the next pass warp 0 waits (acquire) for the blocks of
// the four neighbouring bricks to have published the previous pass, then
// fetches the other colour's rows just outside the brick (its halo) with four
// tensor copies (TMA), one per face, each a box of 64 x 1 x bz x 3 or 64 x by
// x 1 x 3 floats (x, y, z, component) of the lattice.  Rows are handed out
// to the warps one at a time from a shared counter: first one interior row
// per warp (its neighbours all in the brick) while the copies land, then the
// face rows, then the other interior rows.  A block's face rows of a colour
// are written again two passes later, after its neighbours have published
// the pass in between, whose face rows needed their copies to have landed.
//
// The cone angle changes between sweeps (Table A1): the red pass of sweep
// s + 1 needs the accepted count of all of sweep s.  After its black pass a
// block adds its sample sums (measured sweeps) into slot s mod 3 of the
// control words and then, in one atomic with release semantics, its accepted
// count and its arrival into the slot's count word.  At the start of the next
// red pass the block's last warp waits until every block has arrived (while
// warp 0 issues the halo copies) and applies the cone rule to the total.  Warp 0 of block
// 0 then closes sweep s in the lattice state (cone angle, sample, moments,
// ring, sweep counter) from the same totals, as the closing warp of a row
// pass does, and clears slot s + 2 mod 3 (read by every block before it
// arrived for sweep s; filled again only after block 0 has arrived for sweep
// s + 1).
//
// Every wait is bounded.  The waits on other blocks and on the halo copies
// give up after about one second (kResWaitCycles); the block then raises the
// abort flag, so that the other blocks leave at their next wait, sets the
// lattice's error to MC_ERR_TIMEOUT, waits (bounded) for its copies in
// flight and returns without writing its brick back.
#pragma once
#include <cuda.h>  // CUtensorMap

#include "wave_pass.cuh"  // mbarrier helpers, wave_pair_sums, sts_p3, stg_pair

namespace mcgb {

constexpr int kResRow = 3 * kResLh;  // floats of one row of one colour: [3][64]
constexpr long long kResWaitCycles = 1ll << 31;  // about one second at 2 GHz
constexpr uint32_t kResStaticSmem = 1024;        // bound on the kernel's static shared memory

// Halo rows of a brick of at most by x bz rows: the rows beside its y faces
// (2 bz, when y is split) and beside its z faces (2 by, when z is split).
__host__ __device__ inline uint32_t resident_halo_rows(int by, int bz, int nyc, int nzc) {
    return uint32_t((nyc > 1 ? 2 * bz : 0) + (nzc > 1 ? 2 * by : 0));
}

// Dynamic shared memory of a block (from its first 128-byte boundary): the
// brick [2][by bz][3][64] floats (row r of a colour = (z - z0) by_block +
// (y - y0)), the halo faces -y, +y [3][bz][64] and -z, +z [3][by][64] (the
// boxes of the tensor copies), then the order in which the rows are handed
// out (one 16-bit word per row).
__host__ __device__ inline uint32_t resident_smem_bytes(int by, int bz, int nyc, int nzc) {
    const uint32_t rows = 2u * uint32_t(by * bz) + resident_halo_rows(by, bz, nyc, nzc);
    return 128u + rows * uint32_t(kResRow) * 4u + ((2u * uint32_t(by * bz) + 15u) & ~15u);
}

// Tensor copy of the box at (c0, c1, c2, c3) of map into shared memory,
// completing on bar.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* a) {
    unsigned v;
    asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* a) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.u64 %0, [%1];" : "=l"(v) : "l"(a) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned* a, unsigned v) {
    asm volatile("st.release.gpu.u32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}

__device__ __forceinline__ void red_release_add_u64(unsigned long long* a, unsigned long long v) {
    asm volatile("red.release.gpu.add.u64 [%0], %1;" ::"l"(a), "l"(v) : "memory");
}

// Bounded wait (one thread) until *w >= want; false if the wait runs out (the
// abort flag is then raised) or another block has raised it.
__device__ __forceinline__ bool res_wait_u32(const unsigned* w, unsigned want, int* abort) {
    if (ld_acquire_u32(w) >= want) return true;
    const long long t0 = clock64();
    while (ld_acquire_u32(w) < want) {
        if (*reinterpret_cast<volatile int*>(abort)) return false;
        if (clock64() - t0 > kResWaitCycles) {
            atomicExch(abort, 1);
            return false;
        }
    }
    return true;
}

// The same for the arrivals (high 32 bits) of a count word: wait until they
// reach want, then return the word in *out.
__device__ __forceinline__ bool res_wait_arrivals(const unsigned long long* w, unsigned want, int* abort,
                                                  unsigned long long* out) {
    unsigned long long v = ld_acquire_u64(w);
    if (unsigned(v >> 32) < want) {
        const long long t0 = clock64();
        while (unsigned((v = ld_acquire_u64(w)) >> 32) < want) {
            if (*reinterpret_cast<volatile int*>(abort)) return false;
            if (clock64() - t0 > kResWaitCycles) {
                atomicExch(abort, 1);
                return false;
            }
        }
    }
    *out = v;
    return true;
}

// NT threads per block (one block per SM); MEASURE as in the row kernel.
template <int NT, int MEASURE>
__global__ void __launch_bounds__(NT, 1)
    resident_sweep_kernel(ResidentArgs a, const __grid_constant__ CUtensorMap map_y,
                          const __grid_constant__ CUtensorMap map_z, const float* __restrict__ cone) {
    constexpr int NS = MEASURE >= 2 ? kNumSums : kSumTux;  // sums sampled
    constexpr int NW = NT / 32;
    extern __shared__ __align__(128) float rsm_raw[];
    __shared__ uint64_t hbar;                  // the halo copies of the current pass
    __shared__ int claim[2];                   // next row of the pass, by pass parity
    __shared__ int fdone[2];                   // face rows moved in the pass, by pass parity
    __shared__ unsigned cta_acc;               // accepted moves of the block in the sweep
    __shared__ long long cta_sums[kNumSums];   // its fixed-point sample sums
    __shared__ int s_theta, s_fail;
    LatDev* const L = a.lat;
    const LatParams& p = L->p;
    ResCtl* const ctl = a.ctl;
    const int tid = int(threadIdx.x), lane = tid & 31, warp = tid >> 5;
    const int Ly = p.Ly, Lz = p.Lz, nyc = a.nyc, nzc = a.nzc;
    const int bi = int(blockIdx.x) % nyc, bj = int(blockIdx.x) / nyc;
    const int y0 = bi * Ly / nyc, by = (bi + 1) * Ly / nyc - y0;
    const int z0 = bj * Lz / nzc, bz = (bj + 1) * Lz / nzc - z0;
    const int nr = by * bz, NR = a.by * a.bz;
    // interior rows (all neighbours in the brick) and face rows; the order
    // hands out k0 interior rows, then the nf face rows, then the rest
    const int ni = (nyc > 1 ? max(by - 2, 0) : by) * (nzc > 1 ? max(bz - 2, 0) : bz);
    const int nf = nr - ni, k0 = min(ni, NW);
    const bool has_halo = nyc > 1 || nzc > 1;
    const uint32_t stride = p.stride;
    float* const s = static_cast<float*>(p.spins);
    float* const brick = rsm_raw + ((128u - (smem_u32(rsm_raw) & 127u)) & 127u) / 4u;  // 128-byte aligned
    float* const halo = brick + size_t(2) * NR * kResRow;
    // the halo faces and the component stride of a face row
    const int fy = nyc > 1 ? 3 * a.bz * kResLh : 0, cy = a.bz * kResLh, cz = a.by * kResLh;
    float* const face_ym = halo;
    float* const face_yp = halo + fy;
    float* const face_zm = halo + 2 * fy;
    float* const face_zp = face_zm + 3 * cz;
    uint16_t* const order = reinterpret_cast<uint16_t*>(halo + size_t(resident_halo_rows(a.by, a.bz, nyc, nzc)) * kResRow);
    // lanes 0-3 of warp 0 watch the blocks of the -y, +y, -z, +z bricks
    int nb = -1;
    if (lane < 2 && nyc > 1) nb = bj * nyc + (lane == 0 ? (bi + nyc - 1) % nyc : (bi + 1) % nyc);
    if (lane >= 2 && lane < 4 && nzc > 1) nb = (lane == 2 ? (bj + nzc - 1) % nzc : (bj + 1) % nzc) * nyc + bi;
    if (tid == 0) {
        mbar_init(&hbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        claim[0] = claim[1] = 0;
        fdone[0] = fdone[1] = 0;
        cta_acc = 0;
        s_fail = 0;
        // an entry is ly | lz << 8
        int k = 0, seen = 0;
        for (int phase = 0; phase < 3; ++phase)
            for (int lz = 0; lz < bz; ++lz)
                for (int ly = 0; ly < by; ++ly) {
                    const bool f = (nyc > 1 && (ly == 0 || ly == by - 1)) || (nzc > 1 && (lz == 0 || lz == bz - 1));
                    const bool take = phase == 1 ? f : (!f && (phase == 0 ? seen < k0 : seen >= k0 + ni));
                    if (!f && phase != 1) ++seen;
                    if (take) order[k++] = uint16_t(ly | (lz << 8));
                }
    }
    if (tid < kNumSums) cta_sums[tid] = 0;
    // the brick, both colours: row component (c, r, comp) as 16 float4
    const int n4 = 2 * nr * 3 * (kResLh / 4);
    for (int i = tid; i < n4; i += NT) {
        const int f = i & 15, rc = i >> 4, comp = rc % 3, cr = rc / 3, c = cr / nr, r = cr - c * nr;
        const int ly = r % by, lz = r / by;
        const size_t q = size_t(kResLh) * (size_t(y0 + ly) + size_t(Ly) * size_t(z0 + lz));
        const float4 v = __ldg(reinterpret_cast<const float4*>(s + size_t(3 * c + comp) * stride + q) + f);
        reinterpret_cast<float4*>(brick + (size_t(c) * NR + r) * kResRow + comp * kResLh)[f] = v;
    }
    int theta = L->st.theta;
    const uint32_t sweep0 = L->st.sweep;
    __syncthreads();
    const Par<float> par = load_par<float>(p);
    const unsigned G = gridDim.x + unsigned(a.inject);  // arrivals that complete a sweep
    uint32_t issued = 0;  // passes whose halo copies were issued (warp 0)
    bool alive = true;
    // block 0, warp 0: the close of sweep sw from slot sw mod 3, clearing slot sw + 2 mod 3
    auto close_sweep = [&](int sw) {
        const int k = sw % kResSlots, z = (sw + 2) % kResSlots;
        if (lane == 0) {
            L->st.acc = *reinterpret_cast<volatile unsigned long long*>(&ctl->arrive_acc[k]) & 0xFFFFFFFFull;
            ctl->arrive_acc[z] = 0;
        }
        if (MEASURE > 0 && lane < kNumSums) {
            L->st.sums[lane] = *reinterpret_cast<volatile long long*>(&ctl->sums[k][lane]);
            ctl->sums[z][lane] = 0;
        }
        __syncwarp();
        finalize_sweep(p, L->st, MEASURE > 0 ? 1 : 0, p.sample_torque != 0, lane);
    };
    for (int sw = 0; sw < a.n_sweeps && alive; ++sw) {
        const uint32_t sweep = sweep0 + uint32_t(sw);
        unsigned nacc = 0;
        for (int c = 0; c < 2; ++c) {
            const uint32_t t = 2u * uint32_t(sw) + uint32_t(c);  // pass of the launch
            const int oc = c ^ 1;
            if (tid == 0) {  // the next pass's counters (their last use ended at the last barrier)
                claim[(t + 1) & 1] = 0;
                fdone[(t + 1) & 1] = 0;
            }
            if (warp == 0) {
                bool ok = true;
                if (has_halo) {
                    // the neighbouring blocks' face rows of pass t - 1
                    const bool mine = nb < 0 || res_wait_u32(&ctl->done[nb], t, &ctl->abort);
                    ok = __all_sync(0xffffffffu, mine);
                    __syncwarp();
                    if (ok && lane == 0) {  // the other colour's rows beside the brick, a tensor copy per face
                        asm volatile("fence.proxy.async;" ::: "memory");
                        mbar_expect_tx(&hbar, uint32_t((2 * fy + (nzc > 1 ? 6 * cz : 0)) * 4));
                        if (nyc > 1) {
                            tma_load_4d(face_ym, &map_y, 0, y0 > 0 ? y0 - 1 : Ly - 1, z0, 3 * oc, &hbar);
                            tma_load_4d(face_yp, &map_y, 0, y0 + by < Ly ? y0 + by : 0, z0, 3 * oc, &hbar);
                        }
                        if (nzc > 1) {
                            tma_load_4d(face_zm, &map_z, 0, y0, z0 > 0 ? z0 - 1 : Lz - 1, 3 * oc, &hbar);
                            tma_load_4d(face_zp, &map_z, 0, y0, z0 + bz < Lz ? z0 + bz : 0, 3 * oc, &hbar);
                        }
                    }
                    if (ok) issued = t + 1;
                }
                if (lane == 0 && !ok) s_fail = 1;
            }
            // the last warp, at the same time: every block's count of the last sweep
            if (c == 0 && sw > 0 && warp == NW - 1 && lane == 0) {
                unsigned long long w = 0;
                if (res_wait_arrivals(&ctl->arrive_acc[(sw - 1) % kResSlots], G, &ctl->abort, &w))
                    s_theta = (MEASURE == 0 || p.adapt_in_measure)
                                  ? cone_rule(theta, (long long)(w & 0xFFFFFFFFull), p.n_mov)
                                  : theta;
                else
                    s_fail = 1;
            }
            if (c == 0 && sw > 0) {
                __syncthreads();  // the cone angle of this sweep
                if (s_fail) {
                    alive = false;
                    break;
                }
                theta = s_theta;
                if (blockIdx.x == 0 && warp == 0) close_sweep(sw - 1);
            }
            const float cval = cone[theta];
            bool halo_ready = !has_halo;
            int lf[NS];  // this lane's fixed-point parts of the sample, kPartTiles rows at a time
#pragma unroll
            for (int i = 0; i < NS; ++i) lf[i] = 0;
            uint32_t nparts = 0;
            long long fix = 0;
            for (;;) {
                int k = 0;
                if (lane == 0) k = atomicAdd(&claim[t & 1], 1);
                k = __shfl_sync(0xffffffffu, k, 0);
                if (k >= nr) break;
                const bool face = k >= k0 && k < k0 + nf;
                if (face && !halo_ready) {
                    if (*reinterpret_cast<volatile int*>(&s_fail) || !mbar_wait(&hbar, t & 1u)) {
                        if (lane == 0) s_fail = 1;
                        break;
                    }
                    halo_ready = true;
                }
                const int e = order[k], ly = e & 0xFF, lz = e >> 8, r = lz * by + ly;
                const int y = y0 + ly, z = z0 + lz;
                float* own = brick + (size_t(c) * NR + r) * kResRow;
                const float* oth = brick + (size_t(oc) * NR + r) * kResRow;
                // the four neighbour rows: in the brick (wrapping when it spans
                // the axis) or a row of a halo face
                const bool yi0 = ly > 0 || nyc == 1, yi1 = ly + 1 < by || nyc == 1;
                const bool zi0 = lz > 0 || nzc == 1, zi1 = lz + 1 < bz || nzc == 1;
                const float* ym = yi0 ? oth + (ly > 0 ? -kResRow : (by - 1) * kResRow) : face_ym + lz * kResLh;
                const float* yp = yi1 ? oth + (ly + 1 < by ? kResRow : -(by - 1) * kResRow) : face_yp + lz * kResLh;
                const float* zm = zi0 ? oth + (lz > 0 ? -by * kResRow : (bz - 1) * by * kResRow) : face_zm + ly * kResLh;
                const float* zp =
                    zi1 ? oth + (lz + 1 < bz ? by * kResRow : -(bz - 1) * by * kResRow) : face_zp + ly * kResLh;
                const uint32_t xoff = uint32_t(y + z + c) & 1u;
                P3 S, h, O, Sf;
                wave_pair_sums(own, kResLh, oth, kResLh, ym, yi0 ? kResLh : cy, yp, yi1 ? kResLh : cy, zm,
                               zi0 ? kResLh : cz, zp, zi1 ? kResLh : cz, lane, xoff, S, h, O);
                const uint32_t row = uint32_t(y) + uint32_t(Ly) * uint32_t(z);
                const uint32_t site0 = xoff + 4u * uint32_t(lane) + 2u * uint32_t(kResLh) * row;
                // the key is a kernel parameter, so its round keys are launch constants
                const uint4 w = philox(make_uint4(site0, sweep, tag_of(c, kPurposeMove), 0u), a.key0, a.key1);
                const bool mov[2] = {true, true};
                nacc += pair_move(par, cval, w, S, h, mov, nullptr, Sf);
                sts_p3(own, kResLh, lane, Sf);
                if (face) {  // into the lattice for the neighbouring blocks; the last one publishes the pass
                    stg_pair(s + size_t(3 * c) * stride, stride, row * uint32_t(kResLh) + 2u * uint32_t(lane), Sf);
                    __syncwarp();
                    if (lane == 0) {
                        __threadfence_block();
                        if (atomicAdd(&fdone[t & 1], 1) == nf - 1) {
                            __threadfence_block();
                            st_release_u32(&ctl->done[blockIdx.x], t + 1);
                        }
                    }
                }
                if constexpr (MEASURE > 0) {
                    if (c == 1) {
                        const P3 ea{p2(par.e[0]), p2(par.e[1]), p2(par.e[2])};
                        pair_tile_parts<MEASURE, NS>(par, Sf, h, ea, O, ea, lf);
                        if (++nparts == uint32_t(kPartTiles)) {
                            fix += pair_parts_flush<NS>(lf, lane);
                            nparts = 0;
                        }
                    }
                }
            }
            if (c == 1) {  // the warp's count (and sums) of the sweep into the block's
                if constexpr (MEASURE > 0) {
                    if (nparts) fix += pair_parts_flush<NS>(lf, lane);
                }
                const unsigned wacc = __reduce_add_sync(0xffffffffu, nacc);
                if (lane == 0 && wacc) atomicAdd(&cta_acc, wacc);
                if (MEASURE > 0 && lane < NS && fix)
                    atomicAdd(reinterpret_cast<unsigned long long*>(&cta_sums[lane]), static_cast<unsigned long long>(fix));
            }
            __syncthreads();  // the pass is complete in the block
            if (s_fail) {
                alive = false;
                break;
            }
            if (c == 1 && warp == 0) {  // the block's sums, then its count and arrival (a release)
                const int k = sw % kResSlots;
                if (MEASURE > 0 && lane < NS) {
                    const long long v = cta_sums[lane];
                    cta_sums[lane] = 0;
                    if (v) atomicAdd(reinterpret_cast<unsigned long long*>(&ctl->sums[k][lane]),
                                     static_cast<unsigned long long>(v));
                }
                __syncwarp();
                if (lane == 0) {
                    const unsigned v = cta_acc;
                    cta_acc = 0;
                    red_release_add_u64(&ctl->arrive_acc[k], (1ull << 32) | v);
                }
            }
        }
    }
    if (alive && blockIdx.x == 0) {  // the close of the launch's last sweep, after every block's count
        unsigned long long w = 0;
        if (tid == 0 && !res_wait_arrivals(&ctl->arrive_acc[(a.n_sweeps - 1) % kResSlots], G, &ctl->abort, &w))
            s_fail = 1;
        __syncthreads();
        if (s_fail) alive = false;
        else if (warp == 0) close_sweep(a.n_sweeps - 1);
    }
    if (!alive) {
        if (tid == 0) {
            atomicExch(&ctl->abort, 1);
            if (issued > 0) mbar_wait(&hbar, (issued - 1u) & 1u);  // no copy may land after the block exits
            atomicCAS(&L->st.error, 0, -4);                         // MC_ERR_TIMEOUT
        }
        return;
    }
    // the brick back into the lattice
    for (int i = tid; i < n4; i += NT) {
        const int f = i & 15, rc = i >> 4, comp = rc % 3, cr = rc / 3, c = cr / nr, r = cr - c * nr;
        const int ly = r % by, lz = r / by;
        const size_t q = size_t(kResLh) * (size_t(y0 + ly) + size_t(Ly) * size_t(z0 + lz));
        reinterpret_cast<float4*>(s + size_t(3 * c + comp) * stride + q)[f] =
            reinterpret_cast<const float4*>(brick + (size_t(c) * NR + r) * kResRow + comp * kResLh)[f];
    }
}

}  // namespace mcgb
