// pass_impl.cuh -- colour-pass, pair-pass and reduction kernels of libmc,
// written once for both precisions.  Included by kernels_f64.cu (compiled
// with -fmad=false: every FP64 operation is one IEEE operation in source
// order, which makes the FP64 mode reproduce a serial FP64 reference bit for
// bit) and by kernels_f32.cu (FP32 spins, fast intrinsics).
#pragma once
#include <type_traits>

#include "device_common.cuh"

namespace mcgb {

template <typename R>
constexpr bool kIsF64 = std::is_same<R, double>::value;

template <typename R>
struct Par {
    R J, Ku, e[3], Kc, H[3], T;
    R Rm[9];
};

template <typename R>
__device__ __forceinline__ Par<R> load_par(const LatParams& p) {
    Par<R> q;
    if constexpr (kIsF64<R>) {
        q.J = p.J; q.Ku = p.Ku; q.Kc = p.Kc; q.T = p.T;
        for (int a = 0; a < 3; ++a) { q.e[a] = p.e[a]; q.H[a] = p.H[a]; }
        for (int a = 0; a < 9; ++a) q.Rm[a] = p.R[a];
    } else {
        q.J = p.fJ; q.Ku = p.fKu; q.Kc = p.fKc; q.T = p.fT;
        for (int a = 0; a < 3; ++a) { q.e[a] = p.fe[a]; q.H[a] = p.fH[a]; }
        for (int a = 0; a < 9; ++a) q.Rm[a] = p.fR[a];
    }
    return q;
}

// ------------------------------------------------------------------------
// Site geometry of colour index q of colour c.
// ------------------------------------------------------------------------
struct Geo {
    uint32_t q;
    int k, y, z, xoff, x;
    uint32_t site;
};

__device__ __forceinline__ Geo geometry(const LatParams& p, int colour, uint32_t q) {
    Geo g;
    g.q = q;
    const uint32_t row = fast_div(q, p.div_lh);
    g.k = int(q - row * uint32_t(p.Lh));
    g.z = int(fast_div(row, p.div_ly));
    g.y = int(row - uint32_t(g.z) * uint32_t(p.Ly));
    g.xoff = (g.y + g.z + colour) & 1;
    g.x = g.xoff + 2 * g.k;
    g.site = uint32_t(g.x) + uint32_t(p.Lx) * (uint32_t(g.y) + uint32_t(p.Ly) * uint32_t(g.z));
    return g;
}

__device__ __forceinline__ bool pinned(const LatParams& p, const Geo& g) {
    return (p.bc[0] == 2 && (g.x == 0 || g.x == p.Lx - 1)) ||
           (p.bc[1] == 2 && (g.y == 0 || g.y == p.Ly - 1)) ||
           (p.bc[2] == 2 && (g.z == 0 || g.z == p.Lz - 1));
}

// Other-colour indices of the six neighbours in the order -x,+x,-y,+y,-z,+z
// and a presence mask (boundaries and, for films, the bond mask).
__device__ __forceinline__ uint32_t neighbours(const LatParams& p, const Geo& g, int colour,
                                               uint32_t nq[6]) {
    uint32_t present = 0;
    const uint32_t q = g.q;
    const uint32_t Lh = uint32_t(p.Lh);
    const uint32_t plane = Lh * uint32_t(p.Ly);
    // -x
    if (g.k + g.xoff - 1 >= 0) { nq[0] = q + g.xoff - 1; present |= 1u; }
    else if (p.bc[0] == 0) { nq[0] = q - g.k + Lh - 1; present |= 1u; }
    // +x
    if (g.k + g.xoff < p.Lh) { nq[1] = q + g.xoff; present |= 2u; }
    else if (p.bc[0] == 0) { nq[1] = q - g.k; present |= 2u; }
    // -y
    if (g.y > 0) { nq[2] = q - Lh; present |= 4u; }
    else if (p.bc[1] == 0) { nq[2] = q + Lh * uint32_t(p.Ly - 1); present |= 4u; }
    // +y
    if (g.y < p.Ly - 1) { nq[3] = q + Lh; present |= 8u; }
    else if (p.bc[1] == 0) { nq[3] = q - Lh * uint32_t(p.Ly - 1); present |= 8u; }
    // -z
    if (g.z > 0) { nq[4] = q - plane; present |= 16u; }
    else if (p.bc[2] == 0) { nq[4] = q + plane * uint32_t(p.Lz - 1); present |= 16u; }
    // +z
    if (g.z < p.Lz - 1) { nq[5] = q + plane; present |= 32u; }
    else if (p.bc[2] == 0) { nq[5] = q - plane * uint32_t(p.Lz - 1); present |= 32u; }
    if (p.bonds) present &= uint32_t(__ldg(&p.bonds[uint32_t(colour) * p.stride + q]));
    return present;
}

template <typename R>
__device__ __forceinline__ V3<R> load_spin(const R* s, uint32_t stride, int colour, uint32_t q) {
    const R* b = s + size_t(3 * colour) * stride;
    return V3<R>{b[q], b[stride + q], b[2 * size_t(stride) + q]};
}

template <typename R>
__device__ __forceinline__ void store_spin(R* s, uint32_t stride, int colour, uint32_t q, V3<R> v) {
    R* b = s + size_t(3 * colour) * stride;
    b[q] = v.x;
    b[stride + q] = v.y;
    b[2 * size_t(stride) + q] = v.z;
}

// Sum of the present other-colour neighbours, accumulated -x,+x,-y,+y,-z,+z.
template <typename R>
__device__ __forceinline__ V3<R> neighbour_sum(const R* s, uint32_t stride, int other, const uint32_t nq[6],
                                               uint32_t present) {
    V3<R> h{R(0), R(0), R(0)};
    const R* b = s + size_t(3 * other) * stride;
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        if (present & (1u << d)) {
            h.x = h.x + b[nq[d]];
            h.y = h.y + b[stride + nq[d]];
            h.z = h.z + b[2 * size_t(stride) + nq[d]];
        }
    }
    return h;
}

template <typename R>
__device__ __forceinline__ V3<R> easy_axis(const LatParams& p, const Par<R>& par, int colour, uint32_t q) {
    if (p.grain) {
        const int32_t g = __ldg(&p.grain[uint32_t(colour) * p.stride + q]);
        const R* a = static_cast<const R*>(p.gaxis) + 4 * size_t(g);
        return V3<R>{a[0], a[1], a[2]};
    }
    return V3<R>{par.e[0], par.e[1], par.e[2]};
}

template <typename R>
__device__ __forceinline__ R cubic_q(V3<R> s) {
    const R x2 = s.x * s.x, y2 = s.y * s.y, z2 = s.z * s.z;
    return x2 * y2 + x2 * z2 + y2 * z2;
}

// Energy change of Eq. 2 for S -> Sn with the neighbour sum h fixed:
// dE = -J d.h - K_u((Sn.e)^2 - (S.e)^2) + K_c(q(Sn) - q(S)) - H.d, d = Sn - S.
template <typename R>
__device__ __forceinline__ R delta_e(const Par<R>& par, V3<R> S, V3<R> Sn, V3<R> h, V3<R> e) {
    const R d0 = Sn.x - S.x, d1 = Sn.y - S.y, d2 = Sn.z - S.z;
    const R e_ex = -(par.J * (d0 * h.x + d1 * h.y + d2 * h.z));
    const R pn = Sn.x * e.x + Sn.y * e.y + Sn.z * e.z;
    const R po = S.x * e.x + S.y * e.y + S.z * e.z;
    const R e_u = -(par.Ku * (pn * pn - po * po));
    const R e_c = par.Kc * (cubic_q(Sn) - cubic_q(S));
    const R e_z = -(par.H[0] * d0 + par.H[1] * d1 + par.H[2] * d2);
    return e_ex + e_u + e_c + e_z;
}

// Trial move UniformRandom_RotateSpin(S, theta) of Table A1: uniform by
// solid angle on the cap of half-angle theta about S (c = 1 - cos theta),
// by the disk method generalised to a cap and the orthonormal basis of
// Duff et al. (JCGT 2017); attempt a uses the words (w0, w1) of draw a, at
// most 16 attempts; P = w2 of draw 0.
template <typename R>
__device__ __forceinline__ bool cone_trial(V3<R> S, R c, uint32_t idx, uint32_t sweep, uint32_t tag,
                                           uint32_t k0, uint32_t k1, V3<R>& out, R& P) {
    uint4 w = philox(make_uint4(idx, sweep, tag, 0u), k0, k1);
    R u1, u2;
    if constexpr (kIsF64<R>) {
        P = (double)w.z * 0x1p-32;
        u1 = (double)w.x * 0x1p-31 - 1.0;
        u2 = (double)w.y * 0x1p-31 - 1.0;
    } else {
        P = (float)(w.z >> 8) * 0x1p-24f;
        u1 = (float)(w.x >> 8) * 0x1p-23f - 1.0f;
        u2 = (float)(w.y >> 8) * 0x1p-23f - 1.0f;
    }
    R s = u1 * u1 + u2 * u2;
    uint32_t draw = 0;
    while (!(s < R(1))) {
        if (++draw == 16u) return false;
        w = philox(make_uint4(idx, sweep, tag, draw), k0, k1);
        if constexpr (kIsF64<R>) {
            u1 = (double)w.x * 0x1p-31 - 1.0;
            u2 = (double)w.y * 0x1p-31 - 1.0;
        } else {
            u1 = (float)(w.x >> 8) * 0x1p-23f - 1.0f;
            u2 = (float)(w.y >> 8) * 0x1p-23f - 1.0f;
        }
        s = u1 * u1 + u2 * u2;
    }
    const R sc = s * c;
    const R zp = R(1) - sc;
    const R r = sqrt(c * (R(2) - sc));
    const R xp = u1 * r;
    const R yp = u2 * r;
    // basis {b1, b2, S} (Duff et al. 2017)
    const R sgn = copysign(R(1), S.z);
    const R a = R(-1) / (sgn + S.z);
    const R b = S.x * S.y * a;
    const R b1x = R(1) + sgn * S.x * S.x * a, b1y = sgn * b, b1z = -sgn * S.x;
    const R b2x = b, b2y = sgn + S.y * S.y * a, b2z = -S.y;
    const R nx = xp * b1x + yp * b2x + zp * S.x;
    const R ny = xp * b1y + yp * b2y + zp * S.y;
    const R nz = xp * b1z + yp * b2z + zp * S.z;
    if constexpr (kIsF64<R>) {
        const double norm = sqrt(nx * nx + ny * ny + nz * nz);
        out = V3<R>{nx / norm, ny / norm, nz / norm};
    } else {
        const float inv = rsqrtf(nx * nx + ny * ny + nz * nz);
        out = V3<R>{nx * inv, ny * inv, nz * inv};
    }
    return true;
}

// Metropolis acceptance, Eq. 1: accept iff P < exp(-dE/T).
template <typename R>
__device__ __forceinline__ bool metropolis(R dE, R T, R P) {
    if (dE <= R(0)) return true;
    if constexpr (kIsF64<R>) return P < exp_fp64(-(dE / T));
    else return P < __expf(-__fdividef(dE, T));
}

// ------------------------------------------------------------------------
// Block reduction of the per-thread measurement sums into the lattice's
// fixed-point accumulators (deterministic: integer adds commute).
// ------------------------------------------------------------------------
template <typename R>
struct Sums {
    R v[kNumSums];
};

template <typename R>
__device__ __forceinline__ void add_site(Sums<R>& s, V3<R> S, V3<R> e) {
    s.v[kSumMx] += S.x;
    s.v[kSumMy] += S.y;
    s.v[kSumMz] += S.z;
    const R pe = S.x * e.x + S.y * e.y + S.z * e.z;
    s.v[kSumU] += pe * pe;
    s.v[kSumC] += cubic_q(S);
    s.v[kSumTux] += pe * (S.y * e.z - S.z * e.y);
    s.v[kSumTuy] += pe * (S.z * e.x - S.x * e.z);
    s.v[kSumTuz] += pe * (S.x * e.y - S.y * e.x);
    const R x2 = S.x * S.x, y2 = S.y * S.y, z2 = S.z * S.z;
    const R c0 = S.x * (y2 + z2), c1 = S.y * (x2 + z2), c2 = S.z * (x2 + y2);
    s.v[kSumTcx] += S.y * c2 - S.z * c1;
    s.v[kSumTcy] += S.z * c0 - S.x * c2;
    s.v[kSumTcz] += S.x * c1 - S.y * c0;
}

template <typename R>
__device__ __forceinline__ void block_reduce_sums(Sums<R>& s, LatState& st) {
    __shared__ double red[kBlock / 32][kNumSums];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < kNumSums; ++i) {
        R v = s.v[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][i] = double(v);
    }
    __syncthreads();
    if (threadIdx.x < kNumSums) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < kBlock / 32; ++w) t += red[w][threadIdx.x];
        atomicAdd(reinterpret_cast<unsigned long long*>(&st.sums[threadIdx.x]),
                  static_cast<unsigned long long>(to_fix(t)));
    }
}

// ------------------------------------------------------------------------
// End of a sweep (Table A1 / A2, after the black pass): cone adaptation,
// the sample of Sec. 3 (if measuring), the sweep counter.  Runs on one
// thread of the last block to finish.
// ------------------------------------------------------------------------
__device__ inline void finalize_sweep(const LatParams& p, LatState& st, int measure) {
    const long long acc = (long long)atomicExch(&st.acc, 0ull);
    st.last_acc = acc;
    if (!measure || p.adapt_in_measure) {
        if (2 * acc > p.n_mov) { if (st.theta < 180) st.theta += 1; }
        else { if (st.theta > 1) st.theta -= 1; }
    }
    st.ml_hi = 0;
    st.ml_lo = 0;
    if (measure) {
        double v[kNumSums];
        for (int i = 0; i < kNumSums; ++i) {
            // two's complement fixed point: reinterpret the 64-bit word as signed
            const long long raw =
                (long long)atomicExch(reinterpret_cast<unsigned long long*>(&st.sums[i]), 0ull);
            v[i] = double(raw) / kFixScale;
        }
        const double N = double(p.N);
        const double m[3] = {v[kSumMx] / N, v[kSumMy] / N, v[kSumMz] / N};
        const double ml2 = m[0] * m[0] + m[1] * m[1] + m[2] * m[2];
        const double ml = sqrt(ml2);
        const double e_ex = -p.J * v[kSumEx] / N, e_u = -p.Ku * v[kSumU] / N, e_c = p.Kc * v[kSumC] / N;
        const double e_z = -(p.H[0] * v[kSumMx] + p.H[1] * v[kSumMy] + p.H[2] * v[kSumMz]) / N;
        const double e = e_ex + e_u + e_c + e_z;
        double tq[3];
        tq[0] = (2.0 * p.Ku * v[kSumTux] - 2.0 * p.Kc * v[kSumTcx] + (v[kSumMy] * p.H[2] - v[kSumMz] * p.H[1])) / N;
        tq[1] = (2.0 * p.Ku * v[kSumTuy] - 2.0 * p.Kc * v[kSumTcy] + (v[kSumMz] * p.H[0] - v[kSumMx] * p.H[2])) / N;
        tq[2] = (2.0 * p.Ku * v[kSumTuz] - 2.0 * p.Kc * v[kSumTcz] + (v[kSumMx] * p.H[1] - v[kSumMy] * p.H[0])) / N;
        double* mo = st.moments;
        mo[kMomN] += 1.0;
        for (int a = 0; a < 3; ++a) {
            mo[kMomM + a] += m[a];
            mo[kMomM2 + a] += m[a] * m[a];
            mo[kMomMabs + a] += fabs(m[a]);
            mo[kMomTq + a] += tq[a];
            mo[kMomTq2 + a] += tq[a] * tq[a];
        }
        mo[kMomMl] += ml;
        mo[kMomMl2] += ml2;
        mo[kMomMl4] += ml2 * ml2;
        mo[kMomE] += e;
        mo[kMomE2] += e * e;
        mo[kMomParts + 0] += e_ex;
        mo[kMomParts + 1] += e_u;
        mo[kMomParts + 2] += e_c;
        mo[kMomParts + 3] += e_z;
        if (p.ring) {
            double* r = p.ring + (st.ring_count % p.ring_cap) * kRingWords;
            r[0] = double(st.sweep); r[1] = double(st.theta); r[2] = double(acc);
            r[3] = m[0]; r[4] = m[1]; r[5] = m[2];
            r[6] = e_ex; r[7] = e_u; r[8] = e_c; r[9] = e_z;
            r[10] = tq[0]; r[11] = tq[1]; r[12] = tq[2]; r[13] = 0.0;
        }
        st.ring_count += 1;
    }
    st.sweep += 1;
}

// Count a finished block; the last block of the pass runs `last`.
template <typename F>
__device__ __forceinline__ void block_done(LatState& st, int slot, uint32_t nblocks, F&& last) {
    __threadfence();
    const unsigned prev = atomicAdd(&st.done[slot], 1u);
    if (prev == nblocks - 1) {
        __threadfence();
        st.done[slot] = 0;
        last();
    }
}

// ------------------------------------------------------------------------
// Colour pass of Table A1 (one thread per site of the colour), batched over
// the lattices of a group.  colour 1 with measure != 0 also takes the
// sample: each black thread adds its own site, the red site with the same
// colour index, and its bonds to the six red neighbours (every bond joins
// a red and a black site, so each bond is counted once).
// ------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kBlock) colour_pass_kernel(GroupArgs g, const R* __restrict__ cone, int colour,
                                                             int measure) {
    __shared__ int s_lat;
    __shared__ unsigned s_acc;
    if (threadIdx.x == 0) { s_lat = find_lattice(g); s_acc = 0; }
    __syncthreads();
    const int l = s_lat;
    LatDev* L = g.lats[l];
    const LatParams& p = L->p;
    LatState& st = L->st;
    const Par<R> par = load_par<R>(p);
    const int theta = st.theta;
    const uint32_t sweep = st.sweep;
    const R c = cone[theta];
    R* __restrict__ s = static_cast<R*>(p.spins);
    const uint32_t q = (blockIdx.x - g.start[l]) * kBlock + threadIdx.x;
    const bool active = q < p.Nc;
    const int other = colour ^ 1;
    bool accepted = false;
    Sums<R> sums;
    if (measure) for (int i = 0; i < kNumSums; ++i) sums.v[i] = R(0);
    if (active) {
        const Geo geo = geometry(p, colour, q);
        const V3<R> S = load_spin(s, p.stride, colour, q);
        uint32_t nq[6];
        const uint32_t present = neighbours(p, geo, colour, nq);
        const V3<R> e = easy_axis(p, par, colour, q);
        V3<R> Sf = S;
        const bool movable = !pinned(p, geo);
        V3<R> h{R(0), R(0), R(0)};
        if (movable || measure) h = neighbour_sum(s, p.stride, other, nq, present);
        if (movable) {
            V3<R> Sn;
            R P;
            if (cone_trial(S, c, geo.site, sweep, tag_of(colour, kPurposeMove), p.key0, p.key1, Sn, P)) {
                const R dE = delta_e(par, S, Sn, h, e);
                if (metropolis(dE, par.T, P)) {
                    store_spin(s, p.stride, colour, q, Sn);
                    Sf = Sn;
                    accepted = true;
                }
            }
        }
        if (measure) {
            add_site(sums, Sf, e);
            sums.v[kSumEx] += Sf.x * h.x + Sf.y * h.y + Sf.z * h.z;
            const V3<R> Sr = load_spin(s, p.stride, other, q);
            add_site(sums, Sr, easy_axis(p, par, other, q));
        }
    }
    const unsigned ballot = __ballot_sync(0xffffffffu, accepted);
    if ((threadIdx.x & 31) == 0 && ballot) atomicAdd(&s_acc, unsigned(__popc(ballot)));
    if (measure) block_reduce_sums(sums, st);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_acc) atomicAdd(&st.acc, (unsigned long long)s_acc);
        block_done(st, colour, p.nblocks_site, [&] {
            if (colour == 1) finalize_sweep(p, st, measure);
        });
    }
}

// ------------------------------------------------------------------------
// Exact M_L = sum_i S_i . e_C (Table A2) as fixed point: FP64 terms t give
// q = trunc(t 2^52) split as hi 2^26 + lo; FP32 terms give q = trunc(t 2^40)
// split as hi 2^14 + lo.  Integer sums, so the result is independent of
// the order of the reduction.
// ------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kBlock) mlong_kernel(GroupArgs g) {
    __shared__ int s_lat;
    __shared__ long long s_hi[kBlock / 32], s_lo[kBlock / 32];
    if (threadIdx.x == 0) s_lat = find_lattice(g);
    __syncthreads();
    const int l = s_lat;
    LatDev* L = g.lats[l];
    const LatParams& p = L->p;
    const R* s = static_cast<const R*>(p.spins);
    const uint32_t q = (blockIdx.x - g.start[l]) * kBlock + threadIdx.x;
    long long hi = 0, lo = 0;
    if (q < p.Nc) {
        R e1[3];
        if constexpr (kIsF64<R>) { e1[0] = p.R[0]; e1[1] = p.R[1]; e1[2] = p.R[2]; }
        else { e1[0] = p.fR[0]; e1[1] = p.fR[1]; e1[2] = p.fR[2]; }
        for (int colour = 0; colour < 2; ++colour) {
            const V3<R> S = load_spin(s, p.stride, colour, q);
            const R t = e1[0] * S.x + e1[1] * S.y + e1[2] * S.z;
            if constexpr (kIsF64<R>) {
                const long long v = (long long)(t * 0x1p52);
                const long long h = v >> 26;
                hi += h;
                lo += v - h * (1ll << 26);
            } else {
                const long long v = __float2ll_rz(t * 0x1p40f);
                const long long h = v >> 14;
                hi += h;
                lo += v - h * (1ll << 14);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        hi += __shfl_xor_sync(0xffffffffu, hi, o);
        lo += __shfl_xor_sync(0xffffffffu, lo, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { s_hi[warp] = hi; s_lo[warp] = lo; }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long th = 0, tl = 0;
        for (int w = 0; w < kBlock / 32; ++w) { th += s_hi[w]; tl += s_lo[w]; }
        atomicAdd(reinterpret_cast<unsigned long long*>(&L->st.ml_hi), static_cast<unsigned long long>(th));
        atomicAdd(reinterpret_cast<unsigned long long*>(&L->st.ml_lo), static_cast<unsigned long long>(tl));
    }
}

template <typename R>
__device__ __forceinline__ double mlong_value(long long hi, long long lo) {
    if constexpr (kIsF64<R>) return (double)hi * 0x1p-26 + (double)lo * 0x1p-52;
    else return (double)hi * 0x1p-26 + (double)lo * 0x1p-40;
}

// ShuffleRedBlackSpins (Sec. 2, Table A2) as a keyed bijection: 4-round
// balanced Feistel network on 2h-bit words with cycle-walking (Black and
// Rogaway 2002); round function = lowbias32 hash (C. Wellons, 2018) of the
// right half xor the round key; round keys = Philox(0, sweep, colour |
// purpose 2, 0).
__device__ __forceinline__ uint32_t hash32(uint32_t v) {
    v ^= v >> 16;
    v *= 0x7feb352du;
    v ^= v >> 15;
    v *= 0x846ca68bu;
    v ^= v >> 16;
    return v;
}

__device__ __forceinline__ uint32_t permute(uint32_t i, uint32_t n, int h, uint4 rk) {
    const uint32_t mask = (1u << h) - 1u;
    const uint32_t keys[4] = {rk.x, rk.y, rk.z, rk.w};
    uint32_t v = i;
    do {
        uint32_t l = v >> h, r = v & mask;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t f = hash32(r ^ keys[k]) & mask;
            const uint32_t nl = r;
            r = l ^ f;
            l = nl;
        }
        v = (l << h) | r;
    } while (v >= n);
    return v;
}

template <typename R>
__device__ __forceinline__ V3<R> rotate(const R* Rm, V3<R> s) {
    return V3<R>{Rm[0] * s.x + Rm[1] * s.y + Rm[2] * s.z, Rm[3] * s.x + Rm[4] * s.y + Rm[5] * s.z,
                 Rm[6] * s.x + Rm[7] * s.y + Rm[8] * s.z};
}
template <typename R>
__device__ __forceinline__ V3<R> rotate_back(const R* Rm, V3<R> h) {
    return V3<R>{h.x * Rm[0] + h.y * Rm[3] + h.z * Rm[6], h.x * Rm[1] + h.y * Rm[4] + h.z * Rm[7],
                 h.x * Rm[2] + h.y * Rm[5] + h.z * Rm[8]};
}

// ------------------------------------------------------------------------
// Constrained pair pass of Table A2 (one thread per pair), batched.  Pairs
// are (pi(2p), pi(2p+1)) of the colour's shuffled indices; the cone move is
// made on i in the frame whose x-axis is e_C, j compensates the transverse
// components, x'_j = sign(x_j) sqrt(|S_j|^2 - y'_j^2 - z'_j^2).  The pair is
// accepted iff P < (M'_L/M_L)^2 |x_j / x'_j| exp(-(dE_i + dE_j)/T); M_L is
// the exact value from mlong_kernel, fixed for the whole iteration.
// Rejected without a test: 16 failed disk draws, t <= 0, M'_L <= 0.
// ------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kBlock) pair_pass_kernel(GroupArgs g, const R* __restrict__ cone, int colour,
                                                           int finalize, int measure) {
    __shared__ int s_lat;
    __shared__ unsigned s_acc;
    __shared__ double s_ml;
    if (threadIdx.x == 0) {
        s_lat = find_lattice(g);
        s_acc = 0;
        const LatDev* L0 = g.lats[s_lat];
        s_ml = mlong_value<R>(L0->st.ml_hi, L0->st.ml_lo);
    }
    __syncthreads();
    const int l = s_lat;
    LatDev* L = g.lats[l];
    const LatParams& p = L->p;
    LatState& st = L->st;
    const double ML = s_ml;
    const Par<R> par = load_par<R>(p);
    const int theta = st.theta;
    const uint32_t sweep = st.sweep;
    const R c = cone[theta];
    R* __restrict__ s = static_cast<R*>(p.spins);
    const uint32_t pr = (blockIdx.x - g.start[l]) * kBlock + threadIdx.x;
    const int other = colour ^ 1;
    bool accepted = false;
    if (!(ML > 0.0)) {
        if (threadIdx.x == 0) atomicCAS(&st.error, 0, -5);
    } else if (pr < p.n_pairs) {
        const uint4 rk = philox(make_uint4(0u, sweep, tag_of(colour, kPurposePerm), 0u), p.key0, p.key1);
        const uint32_t qi = permute(2 * pr, p.Nc, p.perm_h, rk);
        const uint32_t qj = permute(2 * pr + 1, p.Nc, p.perm_h, rk);
        const V3<R> Si = load_spin(s, p.stride, colour, qi);
        const V3<R> Sj = load_spin(s, p.stride, colour, qj);
        const V3<R> hi = rotate(par.Rm, Si);
        const V3<R> hj = rotate(par.Rm, Sj);
        V3<R> hni;
        R P;
        if (cone_trial(hi, c, pr, sweep, tag_of(colour, kPurposePair), p.key0, p.key1, hni, P)) {
            const R ynj = (hj.y + hi.y) - hni.y;
            const R znj = (hj.z + hi.z) - hni.z;
            const R t = (hj.x * hj.x + hj.y * hj.y + hj.z * hj.z) - ynj * ynj - znj * znj;
            if (t > R(0)) {
                R xnj = sqrt(t);
                if (hj.x < R(0)) xnj = -xnj;
                bool ok;
                R rM;
                if constexpr (kIsF64<R>) {
                    const double MLn = ML + hni.x + xnj - hi.x - hj.x;
                    ok = MLn > 0.0;
                    const double ratio = MLn / ML;
                    rM = ratio * ratio;
                } else {
                    // FP32 spins: the change of M_L is evaluated in FP32 and
                    // applied to the FP64 M_L as (1 + delta / M_L)^2.
                    const float delta = ((hni.x + xnj) - hi.x) - hj.x;
                    const float fml = float(ML);
                    ok = fml + delta > 0.0f;
                    const float ratio = 1.0f + delta / fml;
                    rM = ratio * ratio;
                }
                if (ok) {
                    const V3<R> hnj{xnj, ynj, znj};
                    const V3<R> Sni = rotate_back(par.Rm, hni);
                    const V3<R> Snj = rotate_back(par.Rm, hnj);
                    const Geo gi = geometry(p, colour, qi);
                    const Geo gj = geometry(p, colour, qj);
                    uint32_t nqi[6], nqj[6];
                    const uint32_t pi_ = neighbours(p, gi, colour, nqi);
                    const uint32_t pj_ = neighbours(p, gj, colour, nqj);
                    const V3<R> h_i = neighbour_sum(s, p.stride, other, nqi, pi_);
                    const V3<R> h_j = neighbour_sum(s, p.stride, other, nqj, pj_);
                    const R dEi = delta_e(par, Si, Sni, h_i, easy_axis(p, par, colour, qi));
                    const R dEj = delta_e(par, Sj, Snj, h_j, easy_axis(p, par, colour, qj));
                    const R dE = dEi + dEj;
                    R r = rM;
                    r = r * (fabs(hj.x) / fabs(xnj));
                    if constexpr (kIsF64<R>) r = r * exp_fp64(-(dE / par.T));
                    else r = r * __expf(-__fdividef(dE, par.T));
                    if (P < r) {
                        store_spin(s, p.stride, colour, qi, Sni);
                        store_spin(s, p.stride, colour, qj, Snj);
                        accepted = true;
                    }
                }
            }
        }
    }
    const unsigned ballot = __ballot_sync(0xffffffffu, accepted);
    if ((threadIdx.x & 31) == 0 && ballot) atomicAdd(&s_acc, 2u * unsigned(__popc(ballot)));
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_acc) atomicAdd(&st.acc, (unsigned long long)s_acc);
        block_done(st, colour, p.nblocks_pair, [&] {
            if (finalize) finalize_sweep(p, st, measure);
        });
    }
}

// ------------------------------------------------------------------------
// Standalone sample of the current state (after a constrained sweep): same
// sums as the fused black-pass measurement; the last block closes the sweep.
// ------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kBlock) measure_kernel(GroupArgs g) {
    __shared__ int s_lat;
    if (threadIdx.x == 0) s_lat = find_lattice(g);
    __syncthreads();
    const int l = s_lat;
    LatDev* L = g.lats[l];
    const LatParams& p = L->p;
    LatState& st = L->st;
    const Par<R> par = load_par<R>(p);
    const R* s = static_cast<const R*>(p.spins);
    const uint32_t q = (blockIdx.x - g.start[l]) * kBlock + threadIdx.x;
    Sums<R> sums;
    for (int i = 0; i < kNumSums; ++i) sums.v[i] = R(0);
    if (q < p.Nc) {
        const Geo geo = geometry(p, 1, q);
        uint32_t nq[6];
        const uint32_t present = neighbours(p, geo, 1, nq);
        const V3<R> h = neighbour_sum(s, p.stride, 0, nq, present);
        const V3<R> Sb = load_spin(s, p.stride, 1, q);
        add_site(sums, Sb, easy_axis(p, par, 1, q));
        sums.v[kSumEx] += Sb.x * h.x + Sb.y * h.y + Sb.z * h.z;
        add_site(sums, load_spin(s, p.stride, 0, q), easy_axis(p, par, 0, q));
    }
    block_reduce_sums(sums, st);
    __syncthreads();
    if (threadIdx.x == 0) block_done(st, 3, p.nblocks_site, [&] { finalize_sweep(p, st, 1); });
}

// ------------------------------------------------------------------------
// Slice sums of every spin component over the (y, z) planes of each x
// (domain-wall profile, Sec. 3), fixed point.  One thread per (k, 32-row
// chunk): red sites of row parity r sit at x = r + 2k, black at 1 - r + 2k.
// ------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kBlock) profile_kernel(LatDev* L) {
    const LatParams& p = L->p;
    const R* s = static_cast<const R*>(p.spins);
    const uint32_t rows = uint32_t(p.Ly) * uint32_t(p.Lz);
    const uint32_t chunks = (rows + 31) / 32;
    const uint32_t t = blockIdx.x * kBlock + threadIdx.x;
    if (t == 0) atomicAdd(reinterpret_cast<unsigned long long*>(&L->st.prof_samples), 1ull);
    if (t >= uint32_t(p.Lh) * chunks) return;
    const uint32_t k = t % uint32_t(p.Lh);
    const uint32_t chunk = t / uint32_t(p.Lh);
    double acc[2][3] = {{0, 0, 0}, {0, 0, 0}};  // [x parity][component]
    for (uint32_t row = chunk * 32; row < min(rows, chunk * 32 + 32); ++row) {
        const uint32_t y = row % uint32_t(p.Ly), z = row / uint32_t(p.Ly);
        const int par = int((y + z) & 1u);
        const uint32_t q = k + uint32_t(p.Lh) * row;
        const V3<R> Sr = load_spin(s, p.stride, 0, q);
        const V3<R> Sb = load_spin(s, p.stride, 1, q);
        acc[par][0] += Sr.x; acc[par][1] += Sr.y; acc[par][2] += Sr.z;
        acc[par ^ 1][0] += Sb.x; acc[par ^ 1][1] += Sb.y; acc[par ^ 1][2] += Sb.z;
    }
    for (int xp = 0; xp < 2; ++xp)
        for (int a = 0; a < 3; ++a)
            atomicAdd(reinterpret_cast<unsigned long long*>(&p.profile[a * p.Lx + 2 * k + xp]),
                      static_cast<unsigned long long>(to_fix(acc[xp][a])));
}

}  // namespace mcgb
