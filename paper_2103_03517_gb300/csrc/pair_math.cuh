// pair_math.cuh -- the FP32 trial move, energy change (Eq. 2), Metropolis
// test (Eq. 1) and sample sums of a lane's two sites, evaluated two sites at
// a time with the packed FP32 instructions of sm_100 and later
// (add / mul / fma .f32x2): one instruction does the same IEEE operation on
// both sites.  Shared by the row kernel (row_pass.cuh) and the wavefront
// kernel (wave_pass.cuh), so that both run the same operations in the same
// order and give the same bits.  The law of the trial point and the
// acceptance test are those of the scalar FP32 path (cap_point_direct,
// delta_e, metropolis in pass_impl.cuh).
#pragma once
#include "pass_impl.cuh"

namespace mcgb {

// ---------------------------------------------------------------- packed ops
__device__ __forceinline__ float2 p2add(float2 a, float2 b) {
    float2 r;
    asm("{\n\t.reg .b64 a, b, r;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
        "add.rn.ftz.f32x2 r, a, b;\n\tmov.b64 {%0, %1}, r;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

__device__ __forceinline__ float2 p2sub(float2 a, float2 b) {
    float2 r;
    asm("{\n\t.reg .b64 a, b, r;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
        "sub.rn.ftz.f32x2 r, a, b;\n\tmov.b64 {%0, %1}, r;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

__device__ __forceinline__ float2 p2mul(float2 a, float2 b) {
    float2 r;
    asm("{\n\t.reg .b64 a, b, r;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
        "mul.rn.ftz.f32x2 r, a, b;\n\tmov.b64 {%0, %1}, r;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

// a * b + c, one rounding per lane
__device__ __forceinline__ float2 p2fma(float2 a, float2 b, float2 c) {
    float2 r;
    asm("{\n\t.reg .b64 a, b, c, r;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\tmov.b64 c, {%6, %7};\n\t"
        "fma.rn.ftz.f32x2 r, a, b, c;\n\tmov.b64 {%0, %1}, r;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return r;
}

__device__ __forceinline__ float2 p2(float v) { return make_float2(v, v); }

// 1 / x to the hardware's approximation (the reciprocal that fast-math
// division by x uses)
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Three packed components: component a of site 0 in .x, of site 1 in .y.
struct P3 {
    float2 x, y, z;
};

__device__ __forceinline__ P3 pack(const V3<float> s[2]) {
    return P3{make_float2(s[0].x, s[1].x), make_float2(s[0].y, s[1].y), make_float2(s[0].z, s[1].z)};
}

__device__ __forceinline__ void unpack(const P3& p, V3<float> s[2]) {
    s[0] = V3<float>{p.x.x, p.y.x, p.z.x};
    s[1] = V3<float>{p.x.y, p.y.y, p.z.y};
}

// a.b of two packed vectors
__device__ __forceinline__ float2 pdot(const P3& a, const P3& b) {
    return p2fma(a.z, b.z, p2fma(a.y, b.y, p2mul(a.x, b.x)));
}

// a.e with e the same for both sites
__device__ __forceinline__ float2 pdot_axis(const P3& a, const float e[3]) {
    return p2fma(a.z, p2(e[2]), p2fma(a.y, p2(e[1]), p2mul(a.x, p2(e[0]))));
}

__device__ __forceinline__ float2 pcubic(const P3& s) {
    const float2 x2 = p2mul(s.x, s.x), y2 = p2mul(s.y, s.y), z2 = p2mul(s.z, s.z);
    return p2fma(y2, z2, p2fma(x2, z2, p2mul(x2, y2)));
}

// -------------------------------------------------------------- trial point
// The cap point at z' = 1 - s c, azimuth phi, of both sites (the FP32 trial
// move of Table A1: uniform on the cap of half-angle theta about S), built
// about -sigma z and carried onto S by the Householder reflection of
// v = S + sigma z, sigma = sign S_z; renormalised.
__device__ __forceinline__ P3 pair_cap_point(const P3& S, float c, float2 s, float2 cp, float2 sp) {
    const float2 sc = p2mul(s, p2(c));
    const float2 r2 = p2mul(sc, p2fma(sc, p2(-1.0f), p2(2.0f)));  // sc (2 - sc)
    const float2 r = make_float2(sqrtf(r2.x), sqrtf(r2.y));
    const float2 sgn = make_float2(copysignf(1.0f, S.z.x), copysignf(1.0f, S.z.y));
    const float2 px = p2mul(r, cp), py = p2mul(r, sp);
    const float2 pz = p2mul(p2mul(sgn, p2(-1.0f)), p2fma(sc, p2(-1.0f), p2(1.0f)));  // -sgn (1 - sc)
    const float2 vz = p2add(S.z, sgn);
    const float2 d = p2fma(vz, pz, p2fma(S.y, py, p2mul(S.x, px)));
    const float2 den = p2fma(sgn, S.z, p2(1.0f));  // 1 + sgn S_z >= 1
    const float2 mk = p2mul(p2mul(d, make_float2(rcp_approx(den.x), rcp_approx(den.y))), p2(-1.0f));
    P3 n{p2fma(mk, S.x, px), p2fma(mk, S.y, py), p2fma(mk, vz, pz)};
    const float2 n2 = pdot(n, n);
    const float2 inv = make_float2(rsqrtf(n2.x), rsqrtf(n2.y));
    return P3{p2mul(n.x, inv), p2mul(n.y, inv), p2mul(n.z, inv)};
}

// Energy change of Eq. 2 for both sites, h the neighbour sums, e the easy
// axes (e == nullptr: the lattice's axis par.e for both):
// dE = -J d.h - K_u((Sn.e)^2 - (S.e)^2) + K_c(q(Sn) - q(S)) - H.d, d = Sn - S;
// the cubic and Zeeman terms are skipped when their constants are zero.
__device__ __forceinline__ float2 pair_delta_e(const Par<float>& par, const P3& S, const P3& Sn, const P3& h,
                                               const P3* e) {
    const P3 d{p2sub(Sn.x, S.x), p2sub(Sn.y, S.y), p2sub(Sn.z, S.z)};
    const float2 pn = e ? pdot(Sn, *e) : pdot_axis(Sn, par.e), po = e ? pdot(S, *e) : pdot_axis(S, par.e);
    const float2 du = p2fma(pn, pn, p2mul(p2mul(po, po), p2(-1.0f)));  // pn^2 - po^2
    float2 dE = p2fma(pdot(d, h), p2(-par.J), p2mul(du, p2(-par.Ku)));
    if (par.Kc != 0.0f) dE = p2fma(p2sub(pcubic(Sn), pcubic(S)), p2(par.Kc), dE);
    if (par.H[0] != 0.0f || par.H[1] != 0.0f || par.H[2] != 0.0f) dE = p2sub(dE, pdot_axis(d, par.H));
    return dE;
}

// The draws of both sites from one Philox call (direct_draw_two's bits: P
// 22 bits, s 21 bits, phi 21 bits per site), the trial points, Eq. 2 and the
// Metropolis test of Eq. 1 (accept iff dE <= 0 or P < 2^(dE beta2)); mov[v]
// = site v may move; e as for pair_delta_e.  Returns the new spins in Sf and
// the accepted count.
__device__ __forceinline__ unsigned pair_move(const Par<float>& par, float c, uint4 w, const P3& S, const P3& h,
                                              const bool mov[2], const P3* e, P3& Sf) {
    float P[2], sd[2], cp[2], sp[2];
    direct_draw_two(w, P, sd, cp, sp);
    const P3 Sn = pair_cap_point(S, c, make_float2(sd[0], sd[1]), make_float2(cp[0], cp[1]),
                                 make_float2(sp[0], sp[1]));
    const float2 dE = pair_delta_e(par, S, Sn, h, e);
    const float2 xb = p2mul(dE, p2(par.beta2));
    const bool a0 = mov[0] && (dE.x <= 0.0f || P[0] < exp2f(xb.x));
    const bool a1 = mov[1] && (dE.y <= 0.0f || P[1] < exp2f(xb.y));
    Sf.x = make_float2(a0 ? Sn.x.x : S.x.x, a1 ? Sn.x.y : S.x.y);
    Sf.y = make_float2(a0 ? Sn.y.x : S.y.x, a1 ? Sn.y.y : S.y.y);
    Sf.z = make_float2(a0 ? Sn.z.x : S.z.x, a1 ? Sn.z.y : S.z.y);
    return (a0 ? 1u : 0u) + (a1 ? 1u : 0u);
}

// ------------------------------------------------------------- sample sums
// The sample sums of a lane's part of a warp tile: its two sites (spins Sf,
// fields h, easy axes e) and the two sites of the other colour at the same
// indices (spins O, axes eo), packed; the lane's part of each sum is the
// sum of the two packed halves.  LEVEL 2 adds the torque sums.  Returns the
// per-lane FP32 values in kSum* order (the caller turns them into fixed
// point per warp tile).
template <int LEVEL>
__device__ __forceinline__ void pair_site_sums(P3 s, P3 e, bool nu, bool nc, float2 acc[kNumSums]) {
    acc[kSumMx] = p2add(acc[kSumMx], s.x);
    acc[kSumMy] = p2add(acc[kSumMy], s.y);
    acc[kSumMz] = p2add(acc[kSumMz], s.z);
    const float2 pe = pdot(s, e);
    if (nu) acc[kSumU] = p2fma(pe, pe, acc[kSumU]);
    if (nc) acc[kSumC] = p2add(acc[kSumC], pcubic(s));
    if constexpr (LEVEL >= 2) {
        // (S.e)(S x e) and S x c(S), c = (Sx(Sy^2 + Sz^2), Sy(Sx^2 + Sz^2), Sz(Sx^2 + Sy^2))
        const float2 cx = p2sub(p2mul(s.y, e.z), p2mul(s.z, e.y));
        const float2 cy = p2sub(p2mul(s.z, e.x), p2mul(s.x, e.z));
        const float2 cz = p2sub(p2mul(s.x, e.y), p2mul(s.y, e.x));
        acc[kSumTux] = p2fma(pe, cx, acc[kSumTux]);
        acc[kSumTuy] = p2fma(pe, cy, acc[kSumTuy]);
        acc[kSumTuz] = p2fma(pe, cz, acc[kSumTuz]);
        const float2 x2 = p2mul(s.x, s.x), y2 = p2mul(s.y, s.y), z2 = p2mul(s.z, s.z);
        const float2 c0 = p2mul(s.x, p2add(y2, z2)), c1 = p2mul(s.y, p2add(x2, z2)), c2 = p2mul(s.z, p2add(x2, y2));
        acc[kSumTcx] = p2add(acc[kSumTcx], p2sub(p2mul(s.y, c2), p2mul(s.z, c1)));
        acc[kSumTcy] = p2add(acc[kSumTcy], p2sub(p2mul(s.z, c0), p2mul(s.x, c2)));
        acc[kSumTcz] = p2add(acc[kSumTcz], p2sub(p2mul(s.x, c1), p2mul(s.y, c0)));
    }
}

// Fixed point of one warp tile from the packed per-lane parts (lane i
// receives sum i), as warp_tile_fix does for the scalar parts: each lane
// rounds its part (the two halves added) at 2^22, the warp adds integers.
template <int NS>
__device__ __forceinline__ long long pair_tile_fix(const float2 acc[kNumSums], int lane) {
    int mine = 0;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        const int t = __reduce_add_sync(0xffffffffu, __float2int_rn((acc[i].x + acc[i].y) * float(kFixScaleF32)));
        if (lane == i) mine = t;
    }
    return (long long)mine;
}

// The sample of one warp tile: own sites Sf with fields h and axes e, the
// other colour's sites O with axes eo.
template <int MEASURE, int NS>
__device__ __forceinline__ long long pair_tile_sample(const Par<float>& par, const P3& Sf, const P3& h, const P3& e,
                                                      const P3& O, const P3& eo, int lane) {
    float2 acc[kNumSums];
#pragma unroll
    for (int i = 0; i < kNumSums; ++i) acc[i] = make_float2(0.0f, 0.0f);
    const bool nu = par.Ku != 0.0f, nc = par.Kc != 0.0f;
    pair_site_sums<MEASURE>(Sf, e, nu, nc, acc);
    acc[kSumEx] = pdot(Sf, h);
    pair_site_sums<MEASURE>(O, eo, nu, nc, acc);
    return pair_tile_fix<NS>(acc, lane);
}

// The same parts added into each lane's own accumulators (lf[i] for sum i)
// instead of reduced per tile: the sums are exact integers, so reducing the
// accumulators once per run of tiles (pair_parts_flush) gives the totals of
// pair_tile_sample's per-tile reductions.  A lane's part of a tile is below
// 2^26 in magnitude (at most 12 at scale 2^22), so an int32 holds the parts
// of kPartTiles = 16 tiles.
constexpr int kPartTiles = 16;

template <int MEASURE, int NS>
__device__ __forceinline__ void pair_tile_parts(const Par<float>& par, const P3& Sf, const P3& h, const P3& e,
                                                const P3& O, const P3& eo, int lf[NS]) {
    float2 acc[kNumSums];
#pragma unroll
    for (int i = 0; i < kNumSums; ++i) acc[i] = make_float2(0.0f, 0.0f);
    const bool nu = par.Ku != 0.0f, nc = par.Kc != 0.0f;
    pair_site_sums<MEASURE>(Sf, e, nu, nc, acc);
    acc[kSumEx] = pdot(Sf, h);
    pair_site_sums<MEASURE>(O, eo, nu, nc, acc);
#pragma unroll
    for (int i = 0; i < NS; ++i) lf[i] += __float2int_rn((acc[i].x + acc[i].y) * float(kFixScaleF32));
}

// Warp totals of the accumulated parts: lane i receives sum i.  Each part
// is split into a signed high and an unsigned low 16-bit half, so that
// neither warp sum can overflow an int32; the accumulators are cleared.
template <int NS>
__device__ __forceinline__ long long pair_parts_flush(int lf[NS], int lane) {
    long long mine = 0;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        const int hi = __reduce_add_sync(0xffffffffu, lf[i] >> 16);
        const int lo = __reduce_add_sync(0xffffffffu, lf[i] & 0xFFFF);
        if (lane == i) mine = (long long)hi * 65536 + (long long)lo;
        lf[i] = 0;
    }
    return mine;
}

}  // namespace mcgb
