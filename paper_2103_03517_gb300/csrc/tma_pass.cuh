// tma_pass.cuh -- FP32 colour pass (Table A1) for periodic lattices whose
// rows hold 32..256 sites per colour (Lh a power of two), with the planes
// staged in shared memory by the Tensor Memory Accelerator.
//
// Work item: one brick of a colour -- every k of BY = 512 / Lh consecutive
// rows y0..y0+BY-1 -- over ZC consecutive z planes; a block walks a
// contiguous run of items, the chunks of a brick in z order, as one stream.
// Per plane the block updates the brick's 512 sites (256 threads x an adjacent pair (k,
// k+1) of a row, as on the row path: same pairing, same Philox keying, same
// neighbour-sum order).  Shared memory holds
//   own[3]   : the brick of the colour being updated at planes z .. z+2,
//              as [component][BY rows][Lh] (one 4D TMA box each),
//   oth[5]   : a rolling window of the other colour at planes z-1 .. z+3,
//              each as [component][BY + 2 rows][Lh] -- the brick's rows plus
//              one halo row on either side (wrapped in y), three TMA boxes
//              per component.
// Planes are loaded kTmaAhead = 2 steps before they are computed; the
// updated own plane goes back to HBM with a TMA store.  Every wait on an
// mbarrier is bounded: on expiry the block records MC_ERR_TIMEOUT in the
// lattice and stops.
#pragma once
#include <cuda.h>

#include "pass_impl.cuh"

namespace mcgb {

constexpr int kTmaThreads = 256;
constexpr int kTmaSitesPerPlane = 512;   // BY * Lh
constexpr int kTmaZChunk = 16;           // planes per work item
constexpr int kTmaAhead = 2;            // planes loaded ahead of the one computed
constexpr int kTmaOwnBufs = kTmaAhead + 1;
constexpr int kTmaOthSlots = kTmaAhead + 3;
constexpr uint32_t kTmaSpinLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait for the phase of the given parity; false on expiry.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (uint32_t i = 0; i < kTmaSpinLimit; ++i)
        if (mbar_test(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                         uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void tma_store(const CUtensorMap* map, int c0, int c1, int c2, int c3, const void* src) {
    asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%2, %3, %4, %5}], [%1];" ::"l"(map),
                 "r"(smem_addr(src)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Tensor maps of one lattice, per colour: [0] own box (Lh, BY, 1, 3),
// [1] brick rows of one component (Lh, BY, 1, 1), [2] one row (Lh, 1, 1, 1).
struct TmaMaps {
    CUtensorMap m[2][3];
};

template <int MEASURE>
__global__ void __launch_bounds__(kTmaThreads, 2) tma_pass_kernel(GroupArgs g, uint32_t nitems,
                                                                  const float* __restrict__ cone, int colour,
                                                                  uint32_t slot_floats) {
    constexpr int NSUM = MEASURE >= 2 ? kNumSums : kSumTux;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // 128-byte aligned base (the launch adds slack): every TMA destination
    // below is a multiple of 128 bytes from it
    unsigned char* smem =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);  // own buffers, then other slots
    float* own_buf = reinterpret_cast<float*>(smem + 128);
    float* oth_buf = own_buf + kTmaOwnBufs * 3 * kTmaSitesPerPlane;
    __shared__ unsigned s_acc;
    __shared__ long long s_sums[kNumSums];
    __shared__ int s_fail;
    const int tid = threadIdx.x, lane = tid & 31;
    const int other = colour ^ 1;
    if (tid == 0) {
        for (int i = 0; i < kTmaOwnBufs + kTmaOthSlots; ++i) mbar_init(&bar[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    __syncthreads();
    // bit i = parity of the number of loads issued into buffer i (own
    // buffers first, then the other slots); identical in every thread.  The
    // latest load into buffer i completes the phase of parity (bit i) ^ 1.
    uint32_t issued = 0;
    bool failed = false;
    // this block's contiguous run of work items; items are ordered so that
    // the z chunks of one brick are adjacent, and a run of them is walked as
    // one z segment with one pipeline fill
    const uint32_t per = (nitems + gridDim.x - 1) / gridDim.x;
    uint32_t item = min(blockIdx.x * per, nitems);
    const uint32_t item_end = min(item + per, nitems);
    while (item < item_end && !failed) {
        int l = 0;
        {
            int lo = 0, hi = g.n - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (__ldg(&g.start[mid]) <= item) lo = mid; else hi = mid - 1;
            }
            l = lo;
        }
        LatDev* L = g.lats[l];
        const LatParams& p = L->p;
        const int Lh = p.Lh, Ly = p.Ly, Lz = p.Lz;
        const int BY = kTmaSitesPerPlane / Lh;
        const int nzc = Lz / kTmaZChunk;
        const uint32_t lat0 = __ldg(&g.start[l]);
        const uint32_t local = item - lat0;
        const int brick = int(local / uint32_t(nzc));
        const uint32_t seg_end = min(item_end, lat0 + uint32_t(brick + 1) * uint32_t(nzc));
        const int zs = int(local % uint32_t(nzc)) * kTmaZChunk;
        const int ze = zs + int(seg_end - item) * kTmaZChunk;
        const int y0 = brick * BY;
        const TmaMaps* maps = static_cast<const TmaMaps*>(p.tmaps);
        const CUtensorMap* m_own = &maps->m[colour][0];
        const CUtensorMap* m_row = &maps->m[other][1];
        const CUtensorMap* m_one = &maps->m[other][2];
        const Par<float> par = load_par<float>(p);
        const float c = cone[L->st.theta];
        const uint32_t sweep = L->st.sweep;
        const uint32_t tag = tag_of(colour, kPurposeMove);
        const int slot_comp = (BY + 2) * Lh;  // floats per component in a slot
        const uint32_t oth_bytes = uint32_t(3 * slot_comp) * 4u;
        const uint32_t own_bytes = uint32_t(3 * kTmaSitesPerPlane) * 4u;
        const int ylo = (y0 - 1 + Ly) % Ly, yhi = (y0 + BY) % Ly;
        auto oslot = [](int zz) { return ((zz % kTmaOthSlots) + kTmaOthSlots) % kTmaOthSlots; };
        // issue the other colour's plane zz (unwrapped index) into its slot
        auto load_other = [&](int zz) {
            const int s = oslot(zz);
            if (tid == 0) {
                const int zw = ((zz % Lz) + Lz) % Lz;
                float* dst = oth_buf + size_t(s) * slot_floats;
                uint64_t* bb = &bar[kTmaOwnBufs + s];
                mbar_expect_tx(bb, oth_bytes);
                for (int a = 0; a < 3; ++a) {
                    float* d = dst + a * slot_comp;
                    tma_load(d, m_one, 0, ylo, zw, a, bb);
                    tma_load(d + Lh, m_row, 0, y0, zw, a, bb);
                    tma_load(d + (BY + 1) * Lh, m_one, 0, yhi, zw, a, bb);
                }
            }
            issued ^= 1u << (kTmaOwnBufs + s);
        };
        auto load_own = [&](int zz) {
            const int b = zz % kTmaOwnBufs;
            if (tid == 0) {
                bulk_wait_read();  // the store of the plane that used this buffer has read it
                mbar_expect_tx(&bar[b], own_bytes);
                tma_load(own_buf + size_t(b) * 3 * kTmaSitesPerPlane, m_own, 0, y0, zz, 0, &bar[b]);
            }
            issued ^= 1u << b;
        };
        if (tid == 0) {
            s_acc = 0;
            for (int i = 0; i < kNumSums; ++i) s_sums[i] = 0;
        }
        // pipeline fill: other planes zs-1 .. zs+1+kTmaAhead-1, own zs .. zs+kTmaAhead-1
        for (int zz = zs - 1; zz <= min(zs + kTmaAhead, ze); ++zz) load_other(zz);
        for (int zz = zs; zz < min(zs + kTmaAhead, ze); ++zz) load_own(zz);
        // thread -> row r of the brick and the pair (k, k + 1)
        const int half = Lh >> 1;
        const int r = tid / half;
        const int k = 2 * (tid - r * half);
        const int sidx = r * Lh + k;        // in an own plane
        const int oidx = (r + 1) * Lh + k;  // in an other slot (row 0 is the low halo)
        const int y = y0 + r;
        unsigned nacc = 0;
        long long fix = 0;
        for (int z = zs; z < ze; ++z) {
            if (z + 1 + kTmaAhead <= ze) load_other(z + 1 + kTmaAhead);
            if (z + kTmaAhead < ze) load_own(z + kTmaAhead);
            const int bo = z % kTmaOwnBufs;
            bool ok = mbar_wait(&bar[bo], ((issued >> bo) & 1u) ^ 1u);
            for (int dz = -1; dz <= 1 && ok; ++dz) {
                const int sl = kTmaOwnBufs + oslot(z + dz);
                ok = mbar_wait(&bar[sl], ((issued >> sl) & 1u) ^ 1u);
            }
            if (!ok) {
                s_fail = 1;
                atomicCAS(&L->st.error, 0, -4);
            }
            __syncthreads();
            if (s_fail) { failed = true; break; }
            float* own = own_buf + size_t(bo) * 3 * kTmaSitesPerPlane;
            const float* om = oth_buf + size_t(oslot(z - 1)) * slot_floats;
            const float* o0 = oth_buf + size_t(oslot(z)) * slot_floats;
            const float* op = oth_buf + size_t(oslot(z + 1)) * slot_floats;
            const bool xoff = ((y + z + colour) & 1) != 0;
            V3<float> S[2], h[2], O[2];
            {
                float2 sv[3], ov[3], ym[3], yp[3], zm[3], zp[3];
                float e[3];
                const int ke = xoff ? ((k + 2) & (Lh - 1)) : ((k - 1) & (Lh - 1));
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    sv[a] = *reinterpret_cast<const float2*>(own + a * kTmaSitesPerPlane + sidx);
                    ov[a] = *reinterpret_cast<const float2*>(o0 + a * slot_comp + oidx);
                    ym[a] = *reinterpret_cast<const float2*>(o0 + a * slot_comp + oidx - Lh);
                    yp[a] = *reinterpret_cast<const float2*>(o0 + a * slot_comp + oidx + Lh);
                    zm[a] = *reinterpret_cast<const float2*>(om + a * slot_comp + oidx);
                    zp[a] = *reinterpret_cast<const float2*>(op + a * slot_comp + oidx);
                    e[a] = o0[a * slot_comp + (r + 1) * Lh + ke];
                }
                const V3<float> o0v{ov[0].x, ov[1].x, ov[2].x}, o1v{ov[0].y, ov[1].y, ov[2].y};
                const V3<float> ev{e[0], e[1], e[2]};
                const V3<float> xm0 = xoff ? o0v : ev, xp0 = xoff ? o1v : o0v;
                const V3<float> xm1 = xoff ? o1v : o0v, xp1 = xoff ? ev : o1v;
                h[0].x = ((((xm0.x + xp0.x) + ym[0].x) + yp[0].x) + zm[0].x) + zp[0].x;
                h[0].y = ((((xm0.y + xp0.y) + ym[1].x) + yp[1].x) + zm[1].x) + zp[1].x;
                h[0].z = ((((xm0.z + xp0.z) + ym[2].x) + yp[2].x) + zm[2].x) + zp[2].x;
                h[1].x = ((((xm1.x + xp1.x) + ym[0].y) + yp[0].y) + zm[0].y) + zp[0].y;
                h[1].y = ((((xm1.y + xp1.y) + ym[1].y) + yp[1].y) + zm[1].y) + zp[1].y;
                h[1].z = ((((xm1.z + xp1.z) + ym[2].y) + yp[2].y) + zm[2].y) + zp[2].y;
                S[0] = V3<float>{sv[0].x, sv[1].x, sv[2].x};
                S[1] = V3<float>{sv[0].y, sv[1].y, sv[2].y};
                O[0] = o0v;
                O[1] = o1v;
            }
            const uint32_t site0 = uint32_t(xoff) + 2u * uint32_t(k) +
                                   uint32_t(p.Lx) * (uint32_t(y) + uint32_t(Ly) * uint32_t(z));
            const uint4 w = philox(make_uint4(site0, sweep, tag, 0u), p.key0, p.key1);
            float P[2], sd[2], cp[2], sp[2];
            direct_draw_two(w, P, sd, cp, sp);
            const V3<float> e_ax{par.e[0], par.e[1], par.e[2]};
            V3<float> Sf[2];
#pragma unroll
            for (int v = 0; v < 2; ++v) {
                const V3<float> Sn = cap_point_direct(S[v], c, sd[v], cp[v], sp[v]);
                const float dE = delta_e(par, S[v], Sn, h[v], e_ax);
                const bool acc = metropolis(dE, par.T, P[v]);
                Sf[v] = acc ? Sn : S[v];
                nacc += acc ? 1u : 0u;
            }
            *reinterpret_cast<float2*>(own + sidx) = make_float2(Sf[0].x, Sf[1].x);
            *reinterpret_cast<float2*>(own + kTmaSitesPerPlane + sidx) = make_float2(Sf[0].y, Sf[1].y);
            *reinterpret_cast<float2*>(own + 2 * kTmaSitesPerPlane + sidx) = make_float2(Sf[0].z, Sf[1].z);
            if constexpr (MEASURE > 0) {
                Sums<float> sums;
                for (int i = 0; i < kNumSums; ++i) sums.v[i] = 0.0f;
                const bool nu = par.Ku != 0.0f, nc = par.Kc != 0.0f;
#pragma unroll
                for (int v = 0; v < 2; ++v) {
                    add_site<float, MEASURE>(sums, Sf[v], e_ax, nu, nc);
                    sums.v[kSumEx] += Sf[v].x * h[v].x + Sf[v].y * h[v].y + Sf[v].z * h[v].z;
                    add_site<float, MEASURE>(sums, O[v], e_ax, nu, nc);
                }
                fix += warp_tile_fix<float, NSUM>(sums, lane);
            }
            fence_async_shared();
            __syncthreads();
            if (tid == 0) tma_store(m_own, 0, y0, z, 0, own);
        }
        if (failed) break;
        // publish the segment: accepted moves, sample sums, its item count
        nacc = __reduce_add_sync(0xffffffffu, nacc);
        if (lane == 0 && nacc) atomicAdd(&s_acc, nacc);
        if (MEASURE > 0 && lane < NSUM && fix)
            atomicAdd(reinterpret_cast<unsigned long long*>(&s_sums[lane]), static_cast<unsigned long long>(fix));
        __syncthreads();
        if (tid == 0) {
            if (s_acc) atomicAdd(&L->st.acc, (unsigned long long)s_acc);
            if (MEASURE > 0)
                for (int i = 0; i < NSUM; ++i)
                    if (s_sums[i])
                        atomicAdd(reinterpret_cast<unsigned long long*>(&L->st.sums[i]),
                                  static_cast<unsigned long long>(s_sums[i]));
            __threadfence();
            const unsigned items = seg_end - item;
            const unsigned prev = atomicAdd(&L->st.done[colour], items);
            if (prev + items == p.nblocks_tma) {
                __threadfence();
                L->st.done[colour] = 0;
                if (colour == 1) finalize_sweep(p, L->st, MEASURE > 0 ? 1 : 0, p.sample_torque != 0);
            }
        }
        __syncthreads();
        item = seg_end;
    }
    if (tid == 0) {
        // after a wait gave up, give the loads still in flight a bounded
        // chance to land before the block exits (a no-op otherwise)
        for (int i = 0; i < kTmaOwnBufs + kTmaOthSlots; ++i)
            if (!mbar_wait(&bar[i], ((issued >> i) & 1u) ^ 1u)) break;
        bulk_wait_all();
    }
}

}  // namespace mcgb
