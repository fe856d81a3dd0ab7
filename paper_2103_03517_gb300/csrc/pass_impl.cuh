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
    R beta2;  // FP32: -log2(e) / T (unused in FP64)
    R Rm[9];
};

template <typename R>
__device__ __forceinline__ Par<R> load_par(const LatParams& p) {
    Par<R> q;
    if constexpr (kIsF64<R>) {
        q.J = p.J; q.Ku = p.Ku; q.Kc = p.Kc; q.T = p.T;
        q.beta2 = 0.0;
        for (int a = 0; a < 3; ++a) { q.e[a] = p.e[a]; q.H[a] = p.H[a]; }
        for (int a = 0; a < 9; ++a) q.Rm[a] = p.R[a];
    } else {
        q.J = p.fJ; q.Ku = p.fKu; q.Kc = p.fKc; q.T = p.fT;
        q.beta2 = p.fBeta2;
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
// and a mask: bit d = neighbour d present (boundaries and, for films, the
// bond mask), bit 8 + d = the bond to it crosses an anti-periodic face and
// couples to -S (kFlipShift).
constexpr int kFlipShift = 8;

__device__ __forceinline__ bool wraps(int bc) { return bc == 0 || bc == 3; }

__device__ __forceinline__ uint32_t neighbours(const LatParams& p, const Geo& g, int colour,
                                               uint32_t nq[6]) {
    uint32_t present = 0;
    const uint32_t q = g.q;
    const uint32_t Lh = uint32_t(p.Lh);
    const uint32_t plane = Lh * uint32_t(p.Ly);
    const uint32_t fx = p.bc[0] == 3 ? 1u : 0u, fy = p.bc[1] == 3 ? 1u : 0u, fz = p.bc[2] == 3 ? 1u : 0u;
    // -x
    if (g.k + g.xoff - 1 >= 0) { nq[0] = q + g.xoff - 1; present |= 1u; }
    else if (wraps(p.bc[0])) { nq[0] = q - g.k + Lh - 1; present |= 1u | (fx << kFlipShift); }
    // +x
    if (g.k + g.xoff < p.Lh) { nq[1] = q + g.xoff; present |= 2u; }
    else if (wraps(p.bc[0])) { nq[1] = q - g.k; present |= 2u | (fx << (kFlipShift + 1)); }
    // -y
    if (g.y > 0) { nq[2] = q - Lh; present |= 4u; }
    else if (wraps(p.bc[1])) { nq[2] = q + Lh * uint32_t(p.Ly - 1); present |= 4u | (fy << (kFlipShift + 2)); }
    // +y
    if (g.y < p.Ly - 1) { nq[3] = q + Lh; present |= 8u; }
    else if (wraps(p.bc[1])) { nq[3] = q - Lh * uint32_t(p.Ly - 1); present |= 8u | (fy << (kFlipShift + 3)); }
    // -z
    if (g.z > 0) { nq[4] = q - plane; present |= 16u; }
    else if (wraps(p.bc[2])) { nq[4] = q + plane * uint32_t(p.Lz - 1); present |= 16u | (fz << (kFlipShift + 4)); }
    // +z
    if (g.z < p.Lz - 1) { nq[5] = q + plane; present |= 32u; }
    else if (wraps(p.bc[2])) { nq[5] = q - plane * uint32_t(p.Lz - 1); present |= 32u | (fz << (kFlipShift + 5)); }
    if (p.bonds) present &= uint32_t(__ldg(&p.bonds[uint32_t(colour) * p.stride + q])) | ~0x3Fu;
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

// (x, y, z, 0) of one site: the packed spin copy of constrained sweeps, one
// 16-byte (FP32) or 32-byte (FP64) load per site.
template <typename R>
struct alignas(4 * sizeof(R)) Spin4 {
    R x, y, z, w;
};

// Sum of the present other-colour neighbours, accumulated -x,+x,-y,+y,-z,+z;
// a neighbour across an anti-periodic face enters as -S.
template <typename R>
__device__ __forceinline__ V3<R> neighbour_sum(const R* s, uint32_t stride, int other, const uint32_t nq[6],
                                               uint32_t present) {
    V3<R> h{R(0), R(0), R(0)};
    const R* b = s + size_t(3 * other) * stride;
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        if (present & (1u << d)) {
            const R vx = b[nq[d]], vy = b[stride + nq[d]], vz = b[2 * size_t(stride) + nq[d]];
            if (present & (1u << (kFlipShift + d))) {
                h.x = h.x - vx;
                h.y = h.y - vy;
                h.z = h.z - vz;
            } else {
                h.x = h.x + vx;
                h.y = h.y + vy;
                h.z = h.z + vz;
            }
        }
    }
    return h;
}

// The same sum from the packed copy of the other colour.
template <typename R>
__device__ __forceinline__ V3<R> neighbour_sum4(const Spin4<R>* a, const uint32_t nq[6], uint32_t present) {
    V3<R> h{R(0), R(0), R(0)};
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        if (present & (1u << d)) {
            const Spin4<R> v = a[nq[d]];
            if (present & (1u << (kFlipShift + d))) {
                h.x = h.x - v.x;
                h.y = h.y - v.y;
                h.z = h.z - v.z;
            } else {
                h.x = h.x + v.x;
                h.y = h.y + v.y;
                h.z = h.z + v.z;
            }
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
    if constexpr (!kIsF64<R>) {
        // FP32: zero couplings cost nothing (their terms are exactly zero)
        R dE = e_ex + e_u;
        if (par.Kc != R(0)) dE += par.Kc * (cubic_q(Sn) - cubic_q(S));
        if (par.H[0] != R(0) || par.H[1] != R(0) || par.H[2] != R(0))
            dE += -(par.H[0] * d0 + par.H[1] * d1 + par.H[2] * d2);
        return dE;
    } else {
        const R e_c = par.Kc * (cubic_q(Sn) - cubic_q(S));
        const R e_z = -(par.H[0] * d0 + par.H[1] * d1 + par.H[2] * d2);
        return e_ex + e_u + e_c + e_z;
    }
}

// Trial move UniformRandom_RotateSpin(S, theta) of Table A1: uniform by
// solid angle on the cap of half-angle theta about S (c = 1 - cos theta),
// by the disk method generalised to a cap and the orthonormal basis of
// Duff et al. (JCGT 2017); attempt a uses the words (w0, w1) of draw a, at
// most 16 attempts; P = w2 of draw 0.  Split in three steps so that a warp
// can draw the words of several sites before any data-dependent branch.
template <typename R>
__device__ __forceinline__ void disk_point(uint4 w, R& u1, R& u2) {
    if constexpr (kIsF64<R>) {
        u1 = (double)w.x * 0x1p-31 - 1.0;
        u2 = (double)w.y * 0x1p-31 - 1.0;
    } else {
        u1 = (float)(w.x >> 8) * 0x1p-23f - 1.0f;
        u2 = (float)(w.y >> 8) * 0x1p-23f - 1.0f;
    }
}

template <typename R>
__device__ __forceinline__ R uniform_p(uint4 w) {
    if constexpr (kIsF64<R>) return (double)w.z * 0x1p-32;
    else return (float)(w.z >> 8) * 0x1p-24f;
}

// Redraw rejected disk points (s >= 1) with draws 1..15; false if all fail.
template <typename R>
__device__ __forceinline__ bool disk_retry(R& u1, R& u2, R& s, uint32_t idx, uint32_t sweep, uint32_t tag,
                                           uint32_t k0, uint32_t k1) {
    uint32_t draw = 0;
    while (!(s < R(1))) {
        if (++draw == 16u) return false;
        const uint4 w = philox(make_uint4(idx, sweep, tag, draw), k0, k1);
        disk_point<R>(w, u1, u2);
        s = u1 * u1 + u2 * u2;
    }
    return true;
}

// Map the disk point to the cap about S and renormalise.
template <typename R>
__device__ __forceinline__ V3<R> cap_point(V3<R> S, R c, R u1, R u2, R s) {
    const R sc = s * c;
    const R zp = R(1) - sc;
    const R r = sqrt(c * (R(2) - sc));
    const R xp = u1 * r;
    const R yp = u2 * r;
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
        return V3<R>{nx / norm, ny / norm, nz / norm};
    } else {
        const float inv = rsqrtf(nx * nx + ny * ny + nz * nz);
        return V3<R>{nx * inv, ny * inv, nz * inv};
    }
}

// FP32 mode samples the cap directly, without rejection: s = w0 / 2^32 is
// uniform on [0, 1), so z' = 1 - s c is uniform on [cos theta, 1], and the
// azimuth phi = 2 pi (w1 / 2^32 - 1/2) is uniform; (x', y') = r (cos phi,
// sin phi) with r = sqrt(s c (2 - s c)) = sqrt(1 - z'^2).  Same law as the
// disk method of the FP64 mode, no divergent retry loop in a warp.
__device__ __forceinline__ void direct_draw(uint4 w, float& s, float& cp, float& sp) {
    s = (float)(w.x >> 8) * 0x1p-24f;
    const float phi = ((float)(w.y >> 8) * 0x1p-24f - 0.5f) * 6.28318530717958647692f;
    __sincosf(phi, &sp, &cp);
}

// FP32 trial point: the cap point at z' = 1 - s c and azimuth phi is built
// about -sigma z and carried onto S by the Householder reflection of
// v = S + sigma z, which maps -sigma z to S (sigma = sign(S_z) keeps
// v.v = 2 (1 + sigma S_z) >= 2).  A reflection maps the uniform cap about
// -sigma z to the uniform cap about S, so the law is that of the frame of
// Duff et al. used by the FP64 mode, in fewer operations.
__device__ __forceinline__ V3<float> cap_point_direct(V3<float> S, float c, float s, float cp, float sp) {
    const float sc = s * c;
    const float r = sqrtf(sc * (2.0f - sc));
    const float sgn = copysignf(1.0f, S.z);
    const float px = r * cp, py = r * sp, pz = -sgn * (1.0f - sc);
    const float vz = S.z + sgn;
    const float d = S.x * px + S.y * py + vz * pz;
    const float k = __fdividef(d, 1.0f + sgn * S.z);
    const float nx = px - k * S.x, ny = py - k * S.y, nz = pz - k * vz;
    const float inv = rsqrtf(nx * nx + ny * ny + nz * nz);
    return V3<float>{nx * inv, ny * inv, nz * inv};
}

// FP32, two sites per lane: one Philox call, keyed by the first site's
// index, supplies the draws of both sites, 64 bits each: P (22 bits),
// s (21 bits), phi (21 bits).
__device__ __forceinline__ void direct_draw_two(uint4 w, float P[2], float s[2], float cp[2], float sp[2]) {
    P[0] = (float)(w.x >> 10) * 0x1p-22f;
    P[1] = (float)(w.y >> 10) * 0x1p-22f;
    s[0] = (float)(((w.x & 0x3FFu) << 11) | (w.z & 0x7FFu)) * 0x1p-21f;
    s[1] = (float)(((w.y & 0x3FFu) << 11) | (w.w & 0x7FFu)) * 0x1p-21f;
    const float f0 = ((float)(w.z >> 11) * 0x1p-21f - 0.5f) * 6.28318530717958647692f;
    const float f1 = ((float)(w.w >> 11) * 0x1p-21f - 0.5f) * 6.28318530717958647692f;
    __sincosf(f0, &sp[0], &cp[0]);
    __sincosf(f1, &sp[1], &cp[1]);
}

template <typename R>
__device__ __forceinline__ bool cone_trial(V3<R> S, R c, uint32_t idx, uint32_t sweep, uint32_t tag,
                                           uint32_t k0, uint32_t k1, V3<R>& out, R& P) {
    const uint4 w = philox(make_uint4(idx, sweep, tag, 0u), k0, k1);
    P = uniform_p<R>(w);
    if constexpr (!kIsF64<R>) {
        float s, cp, sp;
        direct_draw(w, s, cp, sp);
        out = cap_point_direct(S, c, s, cp, sp);
        return true;
    } else {
        R u1, u2;
        disk_point<R>(w, u1, u2);
        R s = u1 * u1 + u2 * u2;
        if (!disk_retry(u1, u2, s, idx, sweep, tag, k0, k1)) return false;
        out = cap_point(S, c, u1, u2, s);
        return true;
    }
}

// Metropolis acceptance, Eq. 1: accept iff P < exp(-dE/T).  FP32 evaluates
// exp(-dE/T) as 2^(dE beta2) with beta2 = -log2(e)/T fixed per lattice: one
// multiply and one hardware exp2.
template <typename R>
__device__ __forceinline__ R boltzmann(R dE, const Par<R>& par) {
    if constexpr (kIsF64<R>) return exp_fp64(-(dE / par.T));
    else return exp2f(dE * par.beta2);
}

template <typename R>
__device__ __forceinline__ bool metropolis(R dE, const Par<R>& par, R P) {
    if (dE <= R(0)) return true;
    return P < boltzmann(dE, par);
}

// ------------------------------------------------------------------------
// Block reduction of the per-thread measurement sums into the lattice's
// fixed-point accumulators (deterministic: integer adds commute).
// ------------------------------------------------------------------------
template <typename R>
struct Sums {
    R v[kNumSums];
};

// Sample sums of one site: LEVEL 1 = magnetisation and the single-site
// energy sums, LEVEL 2 = also the torque sums.  FP32 skips the uniaxial or
// cubic sum when its constant is zero (its energy is zero whatever the sum).
template <typename R, int LEVEL = 2>
__device__ __forceinline__ void add_site(Sums<R>& s, V3<R> S, V3<R> e, bool need_u = true, bool need_c = true) {
    s.v[kSumMx] += S.x;
    s.v[kSumMy] += S.y;
    s.v[kSumMz] += S.z;
    const R pe = S.x * e.x + S.y * e.y + S.z * e.z;
    if (kIsF64<R> || need_u) s.v[kSumU] += pe * pe;
    if (kIsF64<R> || need_c) s.v[kSumC] += cubic_q(S);
    if constexpr (LEVEL >= 2) {
        s.v[kSumTux] += pe * (S.y * e.z - S.z * e.y);
        s.v[kSumTuy] += pe * (S.z * e.x - S.x * e.z);
        s.v[kSumTuz] += pe * (S.x * e.y - S.y * e.x);
        const R x2 = S.x * S.x, y2 = S.y * S.y, z2 = S.z * S.z;
        const R c0 = S.x * (y2 + z2), c1 = S.y * (x2 + z2), c2 = S.z * (x2 + y2);
        s.v[kSumTcx] += S.y * c2 - S.z * c1;
        s.v[kSumTcy] += S.z * c0 - S.x * c2;
        s.v[kSumTcz] += S.x * c1 - S.y * c0;
    }
}

// ------------------------------------------------------------------------
// Measurement sums of one warp tile as fixed point on lane i for sum i.
// FP64: reduced across the warp in a fixed butterfly order, then rounded at
// 2^28 (int64).  FP32: each lane rounds its own part at 2^22 and the warp
// adds the integers (one redux per sum), so that no FP64 instruction runs on
// the FP32 path.  A lane's part covers at most two sites of each colour, so
// it is below 16 in magnitude (the bond sum S.h is at most 6 a site) and the
// warp total fits an int32.  Tiles are aligned to the lattice and integer
// sums commute, so the totals do not depend on the batch a lattice runs in.
// ------------------------------------------------------------------------
template <typename R, int NS = kNumSums>
__device__ __forceinline__ long long warp_tile_fix(const Sums<R>& s, int lane) {
    if constexpr (kIsF64<R>) {
        R mine = R(0);
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            R v = s.v[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == i) mine = v;
        }
        return __double2ll_rn(mine * kFixScale);
    } else {
        static_assert(kSitesPerThreadF32 <= 2, "a lane's FP32 sample part must stay below 16");
        int mine = 0;
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            const int t = __reduce_add_sync(0xffffffffu, __float2int_rn(s.v[i] * float(kFixScaleF32)));
            if (lane == i) mine = t;
        }
        return (long long)mine;
    }
}

// ------------------------------------------------------------------------
// End of a sweep (Table A1 / A2, after the black pass): the cone adaptation
// and the carried M_L on one thread; returns the sweep's accepted count.
// ------------------------------------------------------------------------
// The cone rule of Table A1: theta one degree up when more than half of the
// movable sites accepted, else one degree down, within [1, 180].
__device__ __forceinline__ int cone_rule(int theta, long long acc, long long n_mov) {
    if (2 * acc > n_mov) return theta < 180 ? theta + 1 : theta;
    return theta > 1 ? theta - 1 : theta;
}

__device__ inline long long close_counts(const LatParams& p, LatState& st, int measure, long long n_mov) {
    const long long acc = (long long)atomicExch(&st.acc, 0ull);
    st.last_acc = acc;
    if (!measure || p.adapt_in_measure) st.theta = cone_rule(st.theta, acc, n_mov);
    st.ml_hi += st.dml_hi;  // M_L of the next sweep (exact: integer sums)
    st.ml_lo += st.dml_lo;
    st.dml_hi = 0;
    st.dml_lo = 0;
    return acc;
}

// End of an unmeasured sweep, on one thread.
__device__ inline void finalize_sweep_unmeasured(const LatParams& p, LatState& st) {
    close_counts(p, st, 0, p.n_mov);
    st.sweep += 1;
}

// End of a sweep on all 32 lanes of the warp that completed the lattice's
// pass: lane 0 closes the counts; if measuring, the sample of Sec. 3 is
// spread over the lanes.  Lane i takes fixed-point sum i; lanes 0-9 divide
// one numerator each by N (m, the four energy parts, the torque); lane k
// adds moment word k and writes ring word k.  Every quantity is the same
// expression of the same sums as in a serial evaluation.  The sample then costs one
// FP64 division and one memory round trip per lane instead of a serial
// chain on one thread, which sat at the end of every measured pass.
// n_mov and N (the movable sites of the cone rule and the sites of the
// sample) default to the lattice's own; a slab closes with the totals over
// all slabs of its lattice.
__device__ inline void finalize_sweep(const LatParams& p, LatState& st, int measure, bool torque, int lane,
                                      long long n_mov = -1, long long N = -1) {
    constexpr unsigned kAll = 0xffffffffu;
    long long acc = 0;
    int theta = 0;
    uint32_t sweep = 0;
    long long slot = 0;
    if (lane == 0) {
        acc = close_counts(p, st, measure, n_mov < 0 ? p.n_mov : n_mov);
        theta = st.theta;
        sweep = st.sweep;
        slot = p.ring_cap > 0 ? st.ring_count % p.ring_cap : 0;
    }
    if (measure) {
        acc = __shfl_sync(kAll, acc, 0);
        theta = __shfl_sync(kAll, theta, 0);
        sweep = __shfl_sync(kAll, sweep, 0);
        slot = __shfl_sync(kAll, slot, 0);
        // the scales are powers of two, so the products are the quotients
        const double inv_scale = p.precision == 1 ? 1.0 / kFixScale : 1.0 / kFixScaleF32;
        double mine = 0.0;
        if (lane < kNumSums)
            mine = double((long long)atomicExch(reinterpret_cast<unsigned long long*>(&st.sums[lane]), 0ull)) *
                   inv_scale;
        // the sums each numerator needs, fetched by per-lane shuffles: lanes
        // 0-2 m_a; 3-5 the exchange, uniaxial and cubic sums; 6 the three m
        // components (Zeeman); 7 + a the torque sums of axis a and the two
        // other m components (their field cross product)
        const int a = lane - 7;  // torque axis of lanes 7-9
        const int a1 = a == 0 ? 1 : (a == 1 ? 2 : 0), a2 = a == 0 ? 2 : (a == 1 ? 0 : 1);
        const int i1 = lane < 3 ? kSumMx + lane
                       : lane == 3 ? kSumEx
                       : lane == 4 ? kSumU
                       : lane == 5 ? kSumC
                       : lane == 6 ? kSumMx
                       : lane < 10 ? kSumTux + a
                                   : 0;
        const int i2 = lane == 6 ? kSumMy : (lane >= 7 && lane < 10 ? kSumTcx + a : 0);
        const int i3 = lane == 6 ? kSumMz : (lane >= 7 && lane < 10 ? kSumMx + a1 : 0);
        const int i4 = lane >= 7 && lane < 10 ? kSumMx + a2 : 0;
        const double s1 = __shfl_sync(kAll, mine, i1), s2 = __shfl_sync(kAll, mine, i2);
        const double s3 = __shfl_sync(kAll, mine, i3), s4 = __shfl_sync(kAll, mine, i4);
        double num = 0.0;
        if (lane < 3) num = s1;
        else if (lane == 3) num = -p.J * s1;
        else if (lane == 4) num = -p.Ku * s1;
        else if (lane == 5) num = p.Kc * s1;
        else if (lane == 6) num = -(p.H[0] * s1 + p.H[1] * s2 + p.H[2] * s3);
        else if (lane < 10 && torque) num = 2.0 * p.Ku * s1 - 2.0 * p.Kc * s2 + (s3 * p.H[a2] - s4 * p.H[a1]);
        const double quo = num / double(N < 0 ? p.N : N);
        // lanes 0-2: m; 3-6: the energy parts E_ex, E_u, E_c, E_Z; 7-9: tau
        const double m0 = __shfl_sync(kAll, quo, 0), m1 = __shfl_sync(kAll, quo, 1), m2 = __shfl_sync(kAll, quo, 2);
        const double e_ex = __shfl_sync(kAll, quo, 3), e_u = __shfl_sync(kAll, quo, 4);
        const double e_c = __shfl_sync(kAll, quo, 5), e_z = __shfl_sync(kAll, quo, 6);
        const double ml2 = m0 * m0 + m1 * m1 + m2 * m2;
        const double ml = sqrt(ml2);
        const double e = e_ex + e_u + e_c + e_z;
        // moment word `lane`, in the order of the enum: N, m_a, m_a^2, |m_a|,
        // |m|, |m|^2, |m|^4, E, E^2, the four parts, tau_a, tau_a^2; x is the
        // quotient the word is built from (m_a, a part or tau_a)
        const int src = lane < kMomM2     ? lane - kMomM
                        : lane < kMomMabs ? lane - kMomM2
                        : lane < kMomMl   ? lane - kMomMabs
                        : lane < kMomParts ? 0
                        : lane < kMomTq   ? 3 + lane - kMomParts
                        : lane < kMomTq2  ? 7 + lane - kMomTq
                        : lane < kMomTq2 + 3 ? 7 + lane - kMomTq2
                                          : 0;
        const double x = __shfl_sync(kAll, quo, src < 0 ? 0 : src);
        const double inc = lane == kMomN      ? 1.0
                           : lane < kMomM2    ? x
                           : lane < kMomMabs  ? x * x
                           : lane < kMomMl    ? fabs(x)
                           : lane == kMomMl   ? ml
                           : lane == kMomMl2  ? ml2
                           : lane == kMomMl4  ? ml2 * ml2
                           : lane == kMomE    ? e
                           : lane == kMomE2   ? e * e
                           : lane < kMomTq    ? x
                           : lane < kMomTq2   ? x
                                              : x * x;
        if (lane < kMomTq2 + 3) st.moments[lane] += inc;
        // ring word `lane`: sweep, theta, accepted, m, the four parts, tau, 0
        const double y = __shfl_sync(kAll, quo, lane >= 3 && lane < 13 ? lane - 3 : 0);
        if (p.ring && lane < kRingWords) {
            const double w = lane == 0 ? double(sweep) : lane == 1 ? double(theta) : lane == 2 ? double(acc)
                             : lane < 13 ? y : 0.0;
            p.ring[slot * kRingWords + lane] = w;
        }
        if (lane == 0) st.ring_count += 1;
    }
    if (lane == 0) st.sweep += 1;
}

// ------------------------------------------------------------------------
// Work split of every batched kernel: the launch holds as many blocks as are
// resident on the GPU at once, and each warp owns one contiguous chunk of
// warp tiles (a warp tile = 32 * V colour indices, or 32 pairs, of one
// lattice; lattice l owns tiles [g.start[l], g.start[l+1])).  A warp walks
// its chunk lattice by lattice and publishes each lattice's counts once per
// run of tiles; no block-wide barrier is involved.
// ------------------------------------------------------------------------
struct WarpChunk {
    uint32_t begin, end;
    int lane;
};

__device__ __forceinline__ WarpChunk warp_chunk(uint32_t ntiles) {
    // even split: warp w takes [w T / W, (w + 1) T / W), so chunks differ by
    // at most one tile and no warp of the launch idles while T >= W
    const uint32_t nwarps = gridDim.x * uint32_t(kBlock / 32);
    const uint32_t w = blockIdx.x * uint32_t(kBlock / 32) + (threadIdx.x >> 5);
    WarpChunk c;
    c.begin = uint32_t(uint64_t(w) * ntiles / nwarps);
    c.end = uint32_t(uint64_t(w + 1) * ntiles / nwarps);
    c.lane = int(threadIdx.x & 31);
    return c;
}

__device__ __forceinline__ int lattice_of_tile(const GroupArgs& g, uint32_t tile) {
    int lo = 0, hi = g.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&g.start[mid]) <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Publish one warp's run of `tiles` tiles of lattice L: accepted moves and
// fixed-point sums (lane i holds sum i).  In a pass that closes the sweep
// (closes != 0) the warp then counts its tiles, and the warp that completes
// the lattice's pass runs `last` on all its lanes after a fence that orders
// every warp's counts before it.  Any other pass stops after the counts: they are
// read by a later launch, which the kernel boundary orders, so its warps
// neither fence nor count.
template <typename F>
__device__ __forceinline__ void publish(LatState& st, int lane, unsigned nacc, bool with_sums, long long fix, int slot,
                                        uint32_t tiles, uint32_t ntiles_lattice, bool closes, F&& last) {
    nacc = __reduce_add_sync(0xffffffffu, nacc);
    if (lane == 0 && nacc) atomicAdd(&st.acc, (unsigned long long)nacc);
    if (with_sums && lane < kNumSums && fix)
        atomicAdd(reinterpret_cast<unsigned long long*>(&st.sums[lane]), static_cast<unsigned long long>(fix));
    if (!closes) return;
    __threadfence();
    __syncwarp();
    unsigned closing = 0;
    if (lane == 0) {
        const unsigned prev = atomicAdd(&st.done[slot], tiles);
        if (prev + tiles == ntiles_lattice) {
            __threadfence();
            st.done[slot] = 0;
            closing = 1;
        }
    }
    if (__shfl_sync(0xffffffffu, closing, 0)) {
        __threadfence();  // every lane reads what the other warps published
        last();
    }
    __syncwarp();
}

template <typename R>
__device__ __forceinline__ double mlong_value(long long hi, long long lo) {
    if constexpr (kIsF64<R>) return (double)hi * 0x1p-26 + (double)lo * 0x1p-52;
    else return (double)hi * 0x1p-30;
}

// ------------------------------------------------------------------------
// Loads of one warp tile of a uniform periodic lattice whose rows hold a
// multiple of 32 sites per colour (row_fast): the tile is V segments of 32
// consecutive colour indices, each inside one row (y, z) of the colour.  Per
// segment the row, its x parity and the -y/+y/-z/+z row offsets are uniform;
// every lane loads its own spin and the other colour's spin at the same k,
// which is one of its two x neighbours and, by a warp shuffle, the other x
// neighbour of the adjacent lane (an edge lane loads one value across the
// segment boundary, wrapping the row).  The other-colour spin at the same k
// is also the red site a black site samples.  The neighbour sum keeps the
// order -x, +x, -y, +y, -z, +z of the general path.
// ------------------------------------------------------------------------
template <typename R, int V>
__device__ __forceinline__ void row_segments(const LatParams& p, const Par<R>& par, const R* s, int colour,
                                             uint32_t tile_q0, int lane, V3<R> S[V], V3<R> h[V], V3<R> e[V],
                                             V3<R> O[V], uint32_t site[V]) {
    const int other = colour ^ 1;
    const uint32_t stride = p.stride;
    const R* own = s + size_t(3 * colour) * stride;
    const R* oth = s + size_t(3 * other) * stride;
    const uint32_t Lh = uint32_t(p.Lh), plane = Lh * uint32_t(p.Ly);
    V3<R> E[V], Ym[V], Yp[V], Zm[V], Zp[V];
    int xoff[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const uint32_t qs = tile_q0 + uint32_t(32 * v);  // segment start (uniform)
        const uint32_t row = fast_div(qs, p.div_lh);
        const uint32_t k0 = qs - row * Lh;
        const uint32_t z = fast_div(row, p.div_ly);
        const uint32_t y = row - z * uint32_t(p.Ly);
        xoff[v] = int((y + z + uint32_t(colour)) & 1u);
        const uint32_t q = qs + uint32_t(lane);
        site[v] = uint32_t(xoff[v]) + 2u * (k0 + uint32_t(lane)) + uint32_t(p.Lx) * row;
        S[v] = V3<R>{own[q], own[stride + q], own[2 * size_t(stride) + q]};
        O[v] = V3<R>{oth[q], oth[stride + q], oth[2 * size_t(stride) + q]};
        // the x neighbour across the segment edge: k0 - 1 for lane 0 when
        // xoff = 0, k0 + 32 for lane 31 when xoff = 1 (wrapped in the row)
        const bool edge = xoff[v] ? lane == 31 : lane == 0;
        if (edge) {
            const uint32_t qe = xoff[v] ? (k0 + 32 == Lh ? qs - k0 : qs + 32) : (k0 == 0 ? qs + Lh - 1 : qs - 1);
            E[v] = V3<R>{oth[qe], oth[stride + qe], oth[2 * size_t(stride) + qe]};
        } else {
            E[v] = V3<R>{R(0), R(0), R(0)};
        }
        const uint32_t qym = y > 0 ? q - Lh : q + Lh * uint32_t(p.Ly - 1);
        const uint32_t qyp = y + 1 < uint32_t(p.Ly) ? q + Lh : q - Lh * uint32_t(p.Ly - 1);
        const uint32_t qzm = z > 0 ? q - plane : q + plane * uint32_t(p.Lz - 1);
        const uint32_t qzp = z + 1 < uint32_t(p.Lz) ? q + plane : q - plane * uint32_t(p.Lz - 1);
        Ym[v] = V3<R>{oth[qym], oth[stride + qym], oth[2 * size_t(stride) + qym]};
        Yp[v] = V3<R>{oth[qyp], oth[stride + qyp], oth[2 * size_t(stride) + qyp]};
        Zm[v] = V3<R>{oth[qzm], oth[stride + qzm], oth[2 * size_t(stride) + qzm]};
        Zp[v] = V3<R>{oth[qzp], oth[stride + qzp], oth[2 * size_t(stride) + qzp]};
        e[v] = V3<R>{par.e[0], par.e[1], par.e[2]};
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
        // other-colour spin at k - 1 (xoff = 0) or k + 1 (xoff = 1)
        V3<R> N;
        if (xoff[v]) {
            N.x = __shfl_down_sync(0xffffffffu, O[v].x, 1);
            N.y = __shfl_down_sync(0xffffffffu, O[v].y, 1);
            N.z = __shfl_down_sync(0xffffffffu, O[v].z, 1);
            if (lane == 31) N = E[v];
        } else {
            N.x = __shfl_up_sync(0xffffffffu, O[v].x, 1);
            N.y = __shfl_up_sync(0xffffffffu, O[v].y, 1);
            N.z = __shfl_up_sync(0xffffffffu, O[v].z, 1);
            if (lane == 0) N = E[v];
        }
        const V3<R> Xm = xoff[v] ? O[v] : N;
        const V3<R> Xp = xoff[v] ? N : O[v];
        V3<R> a{R(0), R(0), R(0)};
        a.x = a.x + Xm.x; a.y = a.y + Xm.y; a.z = a.z + Xm.z;
        a.x = a.x + Xp.x; a.y = a.y + Xp.y; a.z = a.z + Xp.z;
        a.x = a.x + Ym[v].x; a.y = a.y + Ym[v].y; a.z = a.z + Ym[v].z;
        a.x = a.x + Yp[v].x; a.y = a.y + Yp[v].y; a.z = a.z + Yp[v].z;
        a.x = a.x + Zm[v].x; a.y = a.y + Zm[v].y; a.z = a.z + Zm[v].z;
        a.x = a.x + Zp[v].x; a.y = a.y + Zp[v].y; a.z = a.z + Zp[v].z;
        h[v] = a;
    }
}

// ------------------------------------------------------------------------
// Colour pass of Table A1, batched over the lattices of a group (MEASURE:
// black pass of a measurement sweep: 1 = magnetisation and energies, 2 = also
// torques).  FP64 row_fast lattices take the row path of 32-site segments,
// the others the general path; FP32 row_fast lattices are launched on
// row_pass_kernel instead.  Every lane updates V
// adjacent sites per warp tile; the loads of all V sites are issued before
// any of them is computed.  colour 1 with measure != 0 also takes the sample:
// each black site adds itself, the red site with the same colour index, and
// its bonds to the six red neighbours (every bond joins a red and a black
// site, so each bond is counted once).
// ------------------------------------------------------------------------
template <typename R, int V, int MINB, int MEASURE>
__global__ void __launch_bounds__(kBlock, MINB) colour_pass_kernel(GroupArgs g, uint32_t ntiles, const R* __restrict__ cone,
                                                                   int colour) {
    constexpr int measure = MEASURE > 0 ? 1 : 0;
    constexpr int NS = MEASURE >= 2 ? kNumSums : kSumTux;  // sums sampled
    const WarpChunk wc = warp_chunk(ntiles);
    const int lane = wc.lane;
    const int other = colour ^ 1;
    uint32_t tile = wc.begin;
    int l = tile < wc.end ? lattice_of_tile(g, tile) : 0;
    while (tile < wc.end) {
        LatDev* L = g.lats[l];
        const LatParams& p = L->p;
        const uint32_t t0 = __ldg(&g.start[l]);
        const uint32_t t1 = min(__ldg(&g.start[l + 1]), wc.end);
        const uint32_t run = t1 - tile;
        const Par<R> par = load_par<R>(p);
        const R c = cone[L->st.theta];
        const uint32_t sweep = L->st.sweep;
        R* __restrict__ s = static_cast<R*>(p.spins);
        unsigned nacc = 0;
        long long fix = 0;
        for (; tile < t1; ++tile) {
            const uint32_t base = (tile - t0) * uint32_t(32 * V) + uint32_t(lane);
            V3<R> S[V], h[V], e[V], Sr[V];
            uint32_t site[V], qv[V];
            bool act[V], mov[V];
            if (kIsF64<R> && p.row_fast) {  // FP32 row_fast lattices take row_pass_kernel
                row_segments<R, V>(p, par, s, colour, base - uint32_t(lane), lane, S, h, e, Sr, site);
#pragma unroll
                for (int v = 0; v < V; ++v) qv[v] = base + uint32_t(32 * v);
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    act[v] = true;
                    mov[v] = true;
                    e[v] = V3<R>{par.e[0], par.e[1], par.e[2]};
                }
            } else {
                // a lane's V sites are adjacent colour indices, as on the row
                // paths, so both paths key the same draws to the same sites
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const uint32_t q = (base - uint32_t(lane)) + uint32_t(V * lane + v);
                    qv[v] = q;
                    act[v] = q < p.Nc;
                    mov[v] = false;
                    site[v] = 0;
                    h[v] = V3<R>{R(0), R(0), R(0)};
                    if (act[v]) {
                        const Geo geo = geometry(p, colour, q);
                        site[v] = geo.site;
                        S[v] = load_spin(s, p.stride, colour, q);
                        uint32_t nq[6];
                        const uint32_t present = neighbours(p, geo, colour, nq);
                        mov[v] = !pinned(p, geo);
                        if (mov[v] || measure) h[v] = neighbour_sum(s, p.stride, other, nq, present);
                        e[v] = easy_axis(p, par, colour, q);
                        if (measure) Sr[v] = load_spin(s, p.stride, other, q);
                    }
                }
            }
            // draw 0 of every site first: V independent Philox chains
            const uint32_t tag = tag_of(colour, kPurposeMove);
            // FP64: disk point (u1, u2), s = |u|^2; FP32: s, cos phi, sin phi
            R u1[V], u2[V], sd[V], P[V];
            if constexpr (!kIsF64<R> && V == 2) {
                const uint4 w = philox(make_uint4(site[0], sweep, tag, 0u), p.key0, p.key1);
                direct_draw_two(w, P, sd, u1, u2);
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const uint4 w = philox(make_uint4(site[v], sweep, tag, 0u), p.key0, p.key1);
                    P[v] = uniform_p<R>(w);
                    if constexpr (kIsF64<R>) {
                        disk_point<R>(w, u1[v], u2[v]);
                        sd[v] = u1[v] * u1[v] + u2[v] * u2[v];
                    } else {
                        direct_draw(w, sd[v], u1[v], u2[v]);
                    }
                }
            }
            Sums<R> sums;
            if (measure)
                for (int i = 0; i < kNumSums; ++i) sums.v[i] = R(0);  // unused tail stays 0
#pragma unroll
            for (int v = 0; v < V; ++v) {
                if (!act[v]) continue;
                V3<R> Sf = S[v];
                bool drawn;
                V3<R> Sn;
                if constexpr (kIsF64<R>) {
                    drawn = mov[v] && disk_retry(u1[v], u2[v], sd[v], site[v], sweep, tag, p.key0, p.key1);
                    if (drawn) Sn = cap_point(S[v], c, u1[v], u2[v], sd[v]);
                } else {
                    drawn = mov[v];
                    if (drawn) Sn = cap_point_direct(S[v], c, sd[v], u1[v], u2[v]);
                }
                if (drawn) {
                    const R dE = delta_e(par, S[v], Sn, h[v], e[v]);
                    if (metropolis(dE, par, P[v])) {
                        store_spin(s, p.stride, colour, qv[v], Sn);
                        Sf = Sn;
                        ++nacc;
                    }
                }
                if (measure) {
                    const bool nu = par.Ku != R(0), nc = par.Kc != R(0);
                    add_site<R, MEASURE>(sums, Sf, e[v], nu, nc);
                    sums.v[kSumEx] += Sf.x * h[v].x + Sf.y * h[v].y + Sf.z * h[v].z;
                    add_site<R, MEASURE>(sums, Sr[v], easy_axis(p, par, other, qv[v]), nu, nc);
                }
            }
            if (measure) fix += warp_tile_fix<R, NS>(sums, lane);
        }
        publish(L->st, lane, nacc, measure != 0, fix, colour, run, p.nblocks_site, colour == 1, [&] {
            finalize_sweep(p, L->st, measure, p.sample_torque != 0, lane);
        });
        ++l;
    }
}

// ------------------------------------------------------------------------
// Exact M_L = sum_i S_i . e_C (Table A2) as fixed point, order independent:
// FP64 terms t give q = trunc(t 2^52) split as hi 2^26 + lo; FP32 terms give
// q = trunc(t 2^30) (an int32).  ml_add adds the term of one spin with sign
// +1 or -1, so that the pair passes can carry M_L from sweep to sweep as
// the exact sum over the new state; t is one IEEE operation at a time in
// both precisions (no contraction), the same wherever it is taken.
// ------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R ml_term(const R* e1, V3<R> S) {
    if constexpr (kIsF64<R>) {
        return __dadd_rn(__dadd_rn(__dmul_rn(e1[0], S.x), __dmul_rn(e1[1], S.y)), __dmul_rn(e1[2], S.z));
    } else {
        return __fadd_rn(__fadd_rn(__fmul_rn(e1[0], S.x), __fmul_rn(e1[1], S.y)), __fmul_rn(e1[2], S.z));
    }
}

template <typename R>
__device__ __forceinline__ void ml_add(long long& hi, long long& lo, R t, int sign) {
    if constexpr (kIsF64<R>) {
        const long long w = (long long)(t * 0x1p52);
        const long long hh = w >> 26;
        hi += sign * hh;
        lo += sign * (w - hh * (1ll << 26));
    } else {
        hi += sign * (long long)__float2int_rz(t * 0x1p30f);
    }
}

// M_L of every lattice of g into the zeroed ml_hi / ml_lo, site tiles as in
// the colour pass; it also writes the packed (x, y, z, 0) copy of every
// sub-set (sub-lattice x colour; the two colours of a simple cubic lattice)
// that the pair passes gather from and keep in step.
// ------------------------------------------------------------------------
template <typename R, int V>
__global__ void __launch_bounds__(kBlock) mlong_kernel(GroupArgs g, uint32_t ntiles) {
    const WarpChunk wc = warp_chunk(ntiles);
    const int lane = wc.lane;
    uint32_t tile = wc.begin;
    int l = tile < wc.end ? lattice_of_tile(g, tile) : 0;
    while (tile < wc.end) {
        LatDev* L = g.lats[l];
        const LatParams& p = L->p;
        const uint32_t t0 = __ldg(&g.start[l]);
        const uint32_t t1 = min(__ldg(&g.start[l + 1]), wc.end);
        const R* s = static_cast<const R*>(p.spins);
        Spin4<R>* a4 = static_cast<Spin4<R>*>(p.aos);
        R e1[3];
        if constexpr (kIsF64<R>) { e1[0] = p.R[0]; e1[1] = p.R[1]; e1[2] = p.R[2]; }
        else { e1[0] = p.fR[0]; e1[1] = p.fR[1]; e1[2] = p.fR[2]; }
        long long hi = 0, lo = 0;
        for (; tile < t1; ++tile) {
            const uint32_t base = (tile - t0) * uint32_t(32 * V) + uint32_t(lane);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const uint32_t q = base + uint32_t(32 * v);
                if (q >= p.Nc) continue;
                for (int k = 0; k < 2 * p.nsub; ++k) {  // sub-set k = 2 sub + colour
                    const V3<R> S = load_spin(s, p.stride, k, q);
                    if (a4) a4[size_t(k) * p.stride + q] = Spin4<R>{S.x, S.y, S.z, R(0)};
                    ml_add<R>(hi, lo, ml_term<R>(e1, S), 1);
                }
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            hi += __shfl_xor_sync(0xffffffffu, hi, o);
            lo += __shfl_xor_sync(0xffffffffu, lo, o);
        }
        if (lane == 0) {
            atomicAdd(reinterpret_cast<unsigned long long*>(&L->st.ml_hi), static_cast<unsigned long long>(hi));
            if (lo) atomicAdd(reinterpret_cast<unsigned long long*>(&L->st.ml_lo), static_cast<unsigned long long>(lo));
        }
        ++l;
    }
}

// End of an unmeasured constrained sweep, after its last pair pass (one
// thread per lattice): cone adaptation, M_L carried, the sweep counter.
template <typename R>
__global__ void sweep_end_kernel(GroupArgs g) {
    const int l = int(blockIdx.x * blockDim.x + threadIdx.x);
    if (l >= g.n) return;
    LatDev* L = g.lats[l];
    finalize_sweep_unmeasured(L->p, L->st);
}

// Zero M_L and its carried change before mlong_kernel sums M_L afresh (one
// thread per lattice).
template <typename R>
__global__ void ml_reset_kernel(GroupArgs g) {
    const int l = int(blockIdx.x * blockDim.x + threadIdx.x);
    if (l >= g.n) return;
    LatState& st = g.lats[l]->st;
    st.ml_hi = 0;
    st.ml_lo = 0;
    st.dml_hi = 0;
    st.dml_lo = 0;
}

// ShuffleRedBlackSpins (Sec. 2, Table A2) as a keyed bijection of [0, n):
// a 4-round alternating Feistel network on b-bit words, b the least width
// with 2^b >= n, with cycle-walking (Black and Rogaway 2002).  Round k takes
// the low w bits R and the high b - w bits L to (R, L ^ F_k(R)), R now on
// top, w = ceil(b/2) in rounds 0 and 2 and floor(b/2) in rounds 1 and 3
// (the alternating splits of the FFX mode, Bellare, Rogaway and Spies 2010;
// for even b every round is balanced).  F_k = lowbias32 hash (C. Wellons,
// 2018) of R xor round key k, cut to b - w bits; round keys = Philox(0,
// sweep, colour | purpose 2, 0).  With 2^b < 2n a walk takes under two
// steps on average, and none at all when n is a power of two.
__device__ __forceinline__ uint32_t hash32(uint32_t v) {
    v ^= v >> 16;
    v *= 0x7feb352du;
    v ^= v >> 15;
    v *= 0x846ca68bu;
    v ^= v >> 16;
    return v;
}

__device__ __forceinline__ uint32_t feistel_round(uint32_t v, int b, int w, uint32_t key) {
    const uint32_t r = v & ((1u << w) - 1u);
    const uint32_t l = v >> w;
    return (r << (b - w)) | (l ^ (hash32(r ^ key) & ((1u << (b - w)) - 1u)));
}

// Inverse of feistel_round: R is the top w bits, L = low bits ^ F(R).
__device__ __forceinline__ uint32_t feistel_round_inv(uint32_t v, int b, int w, uint32_t key) {
    const uint32_t r = v >> (b - w);
    const uint32_t l = (v ^ hash32(r ^ key)) & ((1u << (b - w)) - 1u);
    return (l << w) | r;
}

__device__ __forceinline__ uint32_t permute(uint32_t i, uint32_t n, int b, uint4 rk) {
    const int wa = (b + 1) >> 1, wb = b >> 1;
    uint32_t v = i;
    do {
        v = feistel_round(v, b, wa, rk.x);
        v = feistel_round(v, b, wb, rk.y);
        v = feistel_round(v, b, wa, rk.z);
        v = feistel_round(v, b, wb, rk.w);
    } while (v >= n);
    return v;
}

// Inverse of permute: the rounds undone in reverse order, with the same
// cycle-walking: from y = permute(i) the backward walk passes only values
// >= n until it reaches i.
__device__ __forceinline__ uint32_t permute_inv(uint32_t y, uint32_t n, int b, uint4 rk) {
    const int wa = (b + 1) >> 1, wb = b >> 1;
    uint32_t v = y;
    do {
        v = feistel_round_inv(v, b, wb, rk.w);
        v = feistel_round_inv(v, b, wa, rk.z);
        v = feistel_round_inv(v, b, wb, rk.y);
        v = feistel_round_inv(v, b, wa, rk.x);
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
// Constrained pair pass of Table A2 (one lane per pair), batched
// (pair_move below, pair_pass_kernel after it).  Pairs are (pi(2p),
// pi(2p+1)) of the colour's shuffled indices, taken 32 per warp tile in pair
// order or led by the sites of 64-site tiles in site order; the cone move is
// made on i in the frame whose x-axis is e_C, j compensates the transverse
// components, x'_j = sign(x_j) sqrt(|S_j|^2 - y'_j^2 - z'_j^2).  The pair is
// accepted iff
// P < (M'_L/M_L)^2 |x_j / x'_j| exp(-(dE_i + dE_j)/T); M_L is the exact sum
// over the state at the start of the sweep, fixed for the whole iteration
// (mlong_kernel sums it at the start of a run of sweeps; after that every
// accepted pair adds the exact change of its two terms, carried into M_L
// when the sweep ends).  Rejected without a
// test: 16 failed disk draws, t <= 0, M'_L <= 0.  Spins are gathered from the
// packed copy (one sector per site instead of one per component); accepted
// moves are written to the spins and to the copy of the pass's colour.
// ------------------------------------------------------------------------
// One pair of the pass (pair index pr of the lattice, sites qi and qj);
// returns the accepted spin count (0 or 2).  Each member needs its spin and
// its neighbour field, both gathered from packed 4-vectors (the field was
// summed for every site of the colour by pair_field_kernel, in the order of
// neighbour_sum4), and issued together before the move is drawn.
// pair_move_with takes the four gathered items (spins and fields of i
// and j) from the caller, which may have staged them ahead of the move.
template <typename R>
__device__ __forceinline__ unsigned pair_move_with(const LatParams& p, const Par<R>& par, R* __restrict__ s,
                                                   Spin4<R>* own4, const Spin4<R>& si4, const Spin4<R>& sj4,
                                                   const Spin4<R>& fi4, const Spin4<R>& fj4, uint32_t pr, uint32_t qi,
                                                   uint32_t qj, R c, uint32_t sweep, int colour, int set, uint32_t tag,
                                                   double ML, long long& dhi, long long& dlo) {
    const V3<R> h_i{fi4.x, fi4.y, fi4.z};
    const V3<R> h_j{fj4.x, fj4.y, fj4.z};
    const V3<R> Si{si4.x, si4.y, si4.z};
    const V3<R> Sj{sj4.x, sj4.y, sj4.z};
    const V3<R> hi = rotate(par.Rm, Si);
    const V3<R> hj = rotate(par.Rm, Sj);
    V3<R> hni;
    R P;
    if (!cone_trial(hi, c, pr, sweep, tag, p.key0, p.key1, hni, P)) return 0;
    const R ynj = (hj.y + hi.y) - hni.y;
    const R znj = (hj.z + hi.z) - hni.z;
    const R t = (hj.x * hj.x + hj.y * hj.y + hj.z * hj.z) - ynj * ynj - znj * znj;
    if (!(t > R(0))) return 0;
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
        // FP32 spins: the change of M_L is evaluated in FP32 and applied to
        // the FP64 M_L as (1 + delta / M_L)^2.
        const float fml = float(ML);
        const float delta = ((hni.x + xnj) - hi.x) - hj.x;
        ok = fml + delta > 0.0f;
        const float ratio = 1.0f + delta / fml;
        rM = ratio * ratio;
    }
    if (!ok) return 0;
    const V3<R> hnj{xnj, ynj, znj};
    const V3<R> Sni = rotate_back(par.Rm, hni);
    const V3<R> Snj = rotate_back(par.Rm, hnj);
    const R dEi = delta_e(par, Si, Sni, h_i, easy_axis(p, par, colour, qi));
    const R dEj = delta_e(par, Sj, Snj, h_j, easy_axis(p, par, colour, qj));
    const R dE = dEi + dEj;
    R r = rM;
    r = r * (fabs(hj.x) / fabs(xnj));
    r = r * boltzmann(dE, par);
    if (!(P < r)) return 0;
    store_spin(s, p.stride, set, qi, Sni);
    store_spin(s, p.stride, set, qj, Snj);
    own4[qi] = Spin4<R>{Sni.x, Sni.y, Sni.z, R(0)};
    own4[qj] = Spin4<R>{Snj.x, Snj.y, Snj.z, R(0)};
    ml_add<R>(dhi, dlo, ml_term<R>(par.Rm, Sni), 1);  // M_L of the next sweep
    ml_add<R>(dhi, dlo, ml_term<R>(par.Rm, Snj), 1);
    ml_add<R>(dhi, dlo, ml_term<R>(par.Rm, Si), -1);
    ml_add<R>(dhi, dlo, ml_term<R>(par.Rm, Sj), -1);
    return 2;
}

template <typename R>
__device__ __forceinline__ unsigned pair_move(const LatParams& p, const Par<R>& par, R* __restrict__ s,
                                              Spin4<R>* own4, const Spin4<R>* fld, uint32_t pr, uint32_t qi,
                                              uint32_t qj, R c, uint32_t sweep, int colour, int set, uint32_t tag,
                                              double ML, long long& dhi, long long& dlo) {
    const Spin4<R> si4 = own4[qi], sj4 = own4[qj];
    const Spin4<R> fi4 = fld[qi], fj4 = fld[qj];
    return pair_move_with<R>(p, par, s, own4, si4, sj4, fi4, fj4, pr, qi, qj, c, sweep, colour, set, tag, ML, dhi,
                             dlo);
}

// 16-byte asynchronous copy global -> shared (L2 only), and its groups
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const uint32_t sa = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Slots of a warp's ring of waiting leaders in the site-order pair pass:
// at most 31 wait between tiles, and a tile adds at most 64.
constexpr uint32_t kLeaderRing = 128;

// Tiles are taken in grid-stride order, CHUNK consecutive tiles per step: at
// any moment the warps hold a window of about CHUNK tiles each, a few
// lattices of the batch, so that the random gathers of partners and their
// neighbours stay in L2.  A warp adds its accepted moves and M_L change
// once per lattice in a chunk.
template <typename R, int MINB, int CHUNK, bool LEADER, int NT = kBlock>
__global__ void __launch_bounds__(NT, MINB) pair_pass_kernel(GroupArgs g, uint32_t ntiles,
                                                             const R* __restrict__ cone, int colour, int sub) {
    const int lane = int(threadIdx.x & 31);
    const uint32_t nwarps = gridDim.x * uint32_t(NT / 32);
    const uint32_t w = blockIdx.x * uint32_t(NT / 32) + (threadIdx.x >> 5);
    int l = 0;
    for (uint32_t c0 = w * CHUNK; c0 < ntiles; c0 += nwarps * CHUNK) {
        const uint32_t c1 = min(c0 + uint32_t(CHUNK), ntiles);
        for (uint32_t tile = c0; tile < c1;) {
            while (__ldg(&g.start[l + 1]) <= tile) ++l;
            const uint32_t t0 = __ldg(&g.start[l]);
            const uint32_t t1 = min(__ldg(&g.start[l + 1]), c1);
            LatDev* L = g.lats[l];
            const LatParams& p = L->p;
            const double ML = mlong_value<R>(L->st.ml_hi, L->st.ml_lo);
            Spin4<R>* a4 = static_cast<Spin4<R>*>(p.aos);
            unsigned nacc = 0;
            long long dhi = 0, dlo = 0;
            if (!(ML > 0.0)) {
                if (lane == 0) atomicCAS(&L->st.error, 0, -5);
            } else if (!a4) {
                if (lane == 0) atomicCAS(&L->st.error, 0, -6);
            } else {
                const Par<R> par = load_par<R>(p);
                const R c = cone[L->st.theta];
                const uint32_t sweep = L->st.sweep;
                R* __restrict__ s = static_cast<R*>(p.spins);
                // sub-set set = 2 sub + colour (a simple cubic lattice: sub = 0); a
                // crystal sub-set's draws carry the sub-lattice in bits 4.. of the tag
                const int set = 2 * sub + colour;
                const uint32_t tsub = uint32_t(sub) << 4;
                const uint4 rk =
                    philox(make_uint4(0u, sweep, tag_of(colour, kPurposePerm) | tsub, 0u), p.key0, p.key1);
                const uint32_t tag = tag_of(colour, kPurposePair) | tsub;
                Spin4<R>* own4 = a4 + size_t(set) * p.stride;
                const Spin4<R>* fld = static_cast<const Spin4<R>*>(p.pfield);
                if constexpr (LEADER) {
                    // The 64 sites of each tile in index order; each site whose
                    // position r = pi^-1(q) is even leads the pair (pi(r),
                    // pi(r+1)).  A tile has about 32 leaders, rarely exactly, so
                    // leaders wait in a per-warp ring in shared memory (a leader
                    // writes its (q, r) at its rank among the tile's leaders)
                    // until a full warp of them is ready; the ring is emptied at
                    // the end of the run.  The ring holds at most 31 waiting
                    // leaders plus one tile's 64.  A batch of 32 leaders first
                    // finds its partners and starts the four 16-byte gathers of
                    // each pair (spins and fields of i and j) into one of two
                    // shared-memory stages; its moves are made one batch later,
                    // while the next batch's gathers are in flight.  The pairs
                    // of a pass are disjoint and their draws are keyed by pair,
                    // so neither the grouping nor the order changes a result.
                    static_assert(sizeof(Spin4<R>) == 16, "the staged gathers copy 16-byte items");
                    __shared__ uint2 ring[NT / 32][kLeaderRing];
                    __shared__ Spin4<R> stage[NT / 32][2][4][32];  // [warp][stage][item][lane]
                    const int wid = int(threadIdx.x >> 5);
                    uint2* lq = ring[wid];
                    const uint32_t below = (1u << lane) - 1u;
                    uint32_t head = 0, tail = 0;  // leaders queued and taken (warp-uniform)
                    uint32_t pend_pr = 0, pend_qi = 0, pend_qj = 0;
                    bool pend = false, pend_lane = false;  // a batch in flight; this lane has a pair of it
                    int sl = 0;                            // the stage of the next batch
                    // take the n <= 32 oldest leaders and start their gathers into stage sl
                    auto issue = [&](uint32_t n, uint32_t& pr, uint32_t& qi, uint32_t& qj) {
                        const bool mine = uint32_t(lane) < n;
                        if (mine) {
                            const uint2 e = lq[(tail + uint32_t(lane)) % kLeaderRing];
                            qi = e.x;
                            pr = e.y >> 1;
                            qj = permute(e.y + 1u, p.Nc, p.perm_bits, rk);
                            cp_async16(&stage[wid][sl][0][lane], own4 + qi);
                            cp_async16(&stage[wid][sl][1][lane], own4 + qj);
                            cp_async16(&stage[wid][sl][2][lane], fld + qi);
                            cp_async16(&stage[wid][sl][3][lane], fld + qj);
                        }
                        cp_async_commit();
                        tail += n;
                        return mine;
                    };
                    // the moves of the batch in flight, from the other stage
                    auto finish = [&]() {
                        const int st = sl ^ 1;
                        if (pend_lane)
                            nacc += pair_move_with<R>(p, par, s, own4, stage[wid][st][0][lane], stage[wid][st][1][lane],
                                                      stage[wid][st][2][lane], stage[wid][st][3][lane], pend_pr,
                                                      pend_qi, pend_qj, c, sweep, colour, set, tag, ML, dhi, dlo);
                    };
                    auto take = [&](uint32_t n) {
                        uint32_t pr = 0, qi = 0, qj = 0;
                        const bool mine = issue(n, pr, qi, qj);
                        if (pend) {
                            cp_async_wait<1>();  // all but the batch just started
                            finish();
                        }
                        pend = true;
                        pend_lane = mine;
                        pend_pr = pr;
                        pend_qi = qi;
                        pend_qj = qj;
                        sl ^= 1;
                    };
                    for (uint32_t t = tile; t < t1; ++t) {
                        const uint32_t qa = (t - t0) * 64u + uint32_t(lane), qb = qa + 32u;
                        const uint32_t ra = qa < p.Nc ? permute_inv(qa, p.Nc, p.perm_bits, rk) : 1u;
                        const uint32_t rb = qb < p.Nc ? permute_inv(qb, p.Nc, p.perm_bits, rk) : 1u;
                        const bool la = !(ra & 1u) && ra + 1u < p.Nc, lb = !(rb & 1u) && rb + 1u < p.Nc;
                        const uint32_t ma = __ballot_sync(0xffffffffu, la), mb = __ballot_sync(0xffffffffu, lb);
                        const uint32_t ca = uint32_t(__popc(ma));
                        __syncwarp();  // the ring slots taken by the last batch are free again
                        if (la) lq[(head + uint32_t(__popc(ma & below))) % kLeaderRing] = make_uint2(qa, ra);
                        if (lb) lq[(head + ca + uint32_t(__popc(mb & below))) % kLeaderRing] = make_uint2(qb, rb);
                        head += ca + uint32_t(__popc(mb));
                        __syncwarp();
                        while (head - tail >= 32u) take(32u);  // full batches, oldest leaders first
                    }
                    if (head != tail) take(head - tail);
                    if (pend) {
                        cp_async_wait<0>();
                        finish();
                    }
                    __syncwarp();
                } else {
                    for (uint32_t t = tile; t < t1; ++t) {
                        const uint32_t pr = (t - t0) * 32u + uint32_t(lane);
                        if (pr < p.n_pairs) {
                            const uint32_t qi = permute(2 * pr, p.Nc, p.perm_bits, rk);
                            const uint32_t qj = permute(2 * pr + 1, p.Nc, p.perm_bits, rk);
                            nacc += pair_move<R>(p, par, s, own4, fld, pr, qi, qj, c, sweep, colour, set, tag, ML, dhi,
                                                 dlo);
                        }
                    }
                }
            }
            // accepted moves and the change of M_L of this run of tiles; the
            // sweep is closed by a later launch (sweep_end_kernel or the
            // sample), so no warp waits on a fence for its scattered stores
            nacc = __reduce_add_sync(0xffffffffu, nacc);
            for (int o = 16; o > 0; o >>= 1) {
                dhi += __shfl_xor_sync(0xffffffffu, dhi, o);
                dlo += __shfl_xor_sync(0xffffffffu, dlo, o);
            }
            if (lane == 0) {
                if (nacc) atomicAdd(&L->st.acc, (unsigned long long)nacc);
                if (dhi) atomicAdd(reinterpret_cast<unsigned long long*>(&L->st.dml_hi), (unsigned long long)dhi);
                if (dlo) atomicAdd(reinterpret_cast<unsigned long long*>(&L->st.dml_lo), (unsigned long long)dlo);
            }
            tile = t1;
        }
    }
}

// ------------------------------------------------------------------------
// Neighbour field h of every site of one colour (the pair pass of that
// colour reads it for both members of each pair): the other colour's packed
// spins summed in the order -x, +x, -y, +y, -z, +z, as neighbour_sum4 does,
// written as (h_x, h_y, h_z, 0).  The other colour does not change during
// the pass, so the field holds for all of it.  Tiles go to the warps
// CHUNK at a time in grid-stride order, so that the warps in flight cover
// one compact window of the batch and the +-z planes a tile reads are still
// in L2 when the tiles two planes on read them again (with one contiguous
// run per warp those reads were a large part of the launch apart, and every
// plane came from DRAM 3 times).  Lattices with every axis periodic and no
// bond mask take the neighbours without the general path's boundary and
// bond tests (the same indices and order).
// ------------------------------------------------------------------------
template <typename R, int V>
__device__ __forceinline__ void field_tile_periodic(const LatParams& p, const Spin4<R>* __restrict__ oth4,
                                                    Spin4<R>* __restrict__ fld, int colour, uint32_t base) {
    const uint32_t Lh = uint32_t(p.Lh), Ly = uint32_t(p.Ly), Lz = uint32_t(p.Lz), plane = Lh * Ly;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const uint32_t q = base + uint32_t(32 * v);
        if (q >= p.Nc) continue;
        const uint32_t row = fast_div(q, p.div_lh);
        const uint32_t k = q - row * Lh;
        const uint32_t z = fast_div(row, p.div_ly);
        const uint32_t y = row - z * Ly;
        const uint32_t kx = k + ((y + z + uint32_t(colour)) & 1u);  // +x neighbour's k before the wrap
        const uint32_t qrow = q - k;
        const uint32_t nq[6] = {qrow + (kx == 0 ? Lh - 1 : kx - 1), qrow + (kx == Lh ? 0 : kx),
                                y > 0 ? q - Lh : q + Lh * (Ly - 1), y + 1 < Ly ? q + Lh : q - Lh * (Ly - 1),
                                z > 0 ? q - plane : q + plane * (Lz - 1), z + 1 < Lz ? q + plane : q - plane * (Lz - 1)};
        Spin4<R> a[6];
#pragma unroll
        for (int d = 0; d < 6; ++d) a[d] = oth4[nq[d]];
        V3<R> h{R(0), R(0), R(0)};
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            h.x = h.x + a[d].x;
            h.y = h.y + a[d].y;
            h.z = h.z + a[d].z;
        }
        fld[q] = Spin4<R>{h.x, h.y, h.z, R(0)};
    }
}

template <typename R, int V, int CHUNK>
__global__ void __launch_bounds__(kBlock) pair_field_kernel(GroupArgs g, uint32_t ntiles, int colour) {
    const uint32_t nwarps = gridDim.x * uint32_t(kBlock / 32);
    const uint32_t w = blockIdx.x * uint32_t(kBlock / 32) + (threadIdx.x >> 5);
    const uint32_t lane = threadIdx.x & 31u;
    const int other = colour ^ 1;
    int l = 0;
    for (uint32_t c0 = w * CHUNK; c0 < ntiles; c0 += nwarps * CHUNK) {
        const uint32_t c1 = min(c0 + uint32_t(CHUNK), ntiles);
        for (uint32_t tile = c0; tile < c1;) {
            while (__ldg(&g.start[l + 1]) <= tile) ++l;  // tiles only move forward
            const uint32_t t0 = __ldg(&g.start[l]);
            const uint32_t t1 = min(__ldg(&g.start[l + 1]), c1);
            const LatParams& p = g.lats[l]->p;
            const Spin4<R>* oth4 = static_cast<const Spin4<R>*>(p.aos) + size_t(other) * p.stride;
            Spin4<R>* fld = static_cast<Spin4<R>*>(p.pfield);
            if (p.aos && fld) {
                if ((p.bc[0] | p.bc[1] | p.bc[2]) == 0 && !p.bonds) {  // every axis periodic
                    for (uint32_t t = tile; t < t1; ++t)
                        field_tile_periodic<R, V>(p, oth4, fld, colour, (t - t0) * uint32_t(32 * V) + lane);
                } else {
                    for (uint32_t t = tile; t < t1; ++t) {
                        const uint32_t base = (t - t0) * uint32_t(32 * V) + lane;
#pragma unroll
                        for (int v = 0; v < V; ++v) {
                            const uint32_t q = base + uint32_t(32 * v);
                            if (q >= p.Nc) continue;
                            const Geo geo = geometry(p, colour, q);
                            uint32_t nq[6];
                            const uint32_t present = neighbours(p, geo, colour, nq);
                            const V3<R> h = neighbour_sum4(oth4, nq, present);
                            fld[q] = Spin4<R>{h.x, h.y, h.z, R(0)};
                        }
                    }
                }
            }
            tile = t1;
        }
    }
}

// ------------------------------------------------------------------------
// Standalone sample of the current state (after a constrained sweep): same
// sums as the fused black-pass measurement, site tiles; the warp that
// completes a lattice closes its sweep.
// ------------------------------------------------------------------------
template <typename R, int V>
__global__ void __launch_bounds__(kBlock) measure_kernel(GroupArgs g, uint32_t ntiles) {
    const WarpChunk wc = warp_chunk(ntiles);
    const int lane = wc.lane;
    uint32_t tile = wc.begin;
    int l = tile < wc.end ? lattice_of_tile(g, tile) : 0;
    while (tile < wc.end) {
        LatDev* L = g.lats[l];
        const LatParams& p = L->p;
        const uint32_t t0 = __ldg(&g.start[l]);
        const uint32_t t1 = min(__ldg(&g.start[l + 1]), wc.end);
        const uint32_t run = t1 - tile;
        const Par<R> par = load_par<R>(p);
        const R* s = static_cast<const R*>(p.spins);
        long long fix = 0;
        for (; tile < t1; ++tile) {
            const uint32_t base = (tile - t0) * uint32_t(32 * V) + uint32_t(lane);
            Sums<R> sums;
            for (int i = 0; i < kNumSums; ++i) sums.v[i] = R(0);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const uint32_t q = base + uint32_t(32 * v);
                if (q >= p.Nc) continue;
                const Geo geo = geometry(p, 1, q);
                uint32_t nq[6];
                const uint32_t present = neighbours(p, geo, 1, nq);
                const V3<R> h = neighbour_sum(s, p.stride, 0, nq, present);
                const V3<R> Sb = load_spin(s, p.stride, 1, q);
                add_site(sums, Sb, easy_axis(p, par, 1, q));
                sums.v[kSumEx] += Sb.x * h.x + Sb.y * h.y + Sb.z * h.z;
                add_site(sums, load_spin(s, p.stride, 0, q), easy_axis(p, par, 0, q));
            }
            fix += warp_tile_fix(sums, lane);
        }
        publish(L->st, lane, 0, true, fix, 3, run, p.nblocks_site, true, [&] { finalize_sweep(p, L->st, 1, true, lane); });
        ++l;
    }
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

// ------------------------------------------------------------------------
// One grain sample of a film (Sec. 4: every grain contributes its own Bloch
// term to Eq. 8): the spins of each grain summed as fixed point, then
// m_g = |sum S| / N_g added to the grain's accumulator.  Site tiles over
// both colours; the lanes of a warp that hold the same grain pool their
// values (one atomic per grain present in the warp).
// ------------------------------------------------------------------------
template <typename R, int V>
__global__ void __launch_bounds__(kBlock) grain_sum_kernel(LatDev* L, uint32_t ntiles) {
    const LatParams& p = L->p;
    const WarpChunk wc = warp_chunk(ntiles);
    const int lane = wc.lane;
    const R* s = static_cast<const R*>(p.spins);
    for (uint32_t tile = wc.begin; tile < wc.end; ++tile) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const uint32_t q = tile * uint32_t(32 * V) + uint32_t(32 * v + lane);
            for (int colour = 0; colour < 2; ++colour) {
                const bool ok = q < p.Nc;
                const int32_t g = ok ? __ldg(&p.grain[uint32_t(colour) * p.stride + q]) : -1;
                const V3<R> S = ok ? load_spin(s, p.stride, colour, q) : V3<R>{R(0), R(0), R(0)};
                const long long f[3] = {to_fix(double(S.x)), to_fix(double(S.y)), to_fix(double(S.z))};
                const unsigned peers = __match_any_sync(0xffffffffu, g);
                long long sum[3] = {0, 0, 0};
                for (unsigned m = peers; m; m &= m - 1u) {
                    const int src = __ffs(m) - 1;
#pragma unroll
                    for (int a = 0; a < 3; ++a) sum[a] += __shfl_sync(peers, f[a], src);
                }
                if (g >= 0 && lane == __ffs(peers) - 1)
#pragma unroll
                    for (int a = 0; a < 3; ++a)
                        atomicAdd(reinterpret_cast<unsigned long long*>(&p.gsum[3 * size_t(g) + a]),
                                  static_cast<unsigned long long>(sum[a]));
            }
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(kBlock) grain_finish_kernel(LatDev* L) {
    const LatParams& p = L->p;
    const int g = int(blockIdx.x * blockDim.x + threadIdx.x);
    if (g == 0) p.gacc[p.n_grains] += 1.0;
    if (g >= p.n_grains) return;
    double M[3];
    for (int a = 0; a < 3; ++a) {
        M[a] = double(p.gsum[3 * size_t(g) + a]) / kFixScale;
        p.gsum[3 * size_t(g) + a] = 0;
    }
    p.gacc[g] += sqrt(M[0] * M[0] + M[1] * M[1] + M[2] * M[2]) / double(p.gsize[g]);
}

}  // namespace mcgb
