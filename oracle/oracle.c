/*
 * oracle.c -- serial FP64 CPU oracle of the parallel checkerboard Metropolis
 * sweep and the parallel constrained (pair-move) sweep of Lepadatu et al.,
 * "Computation of magnetization, exchange stiffness, anisotropy, and
 * susceptibilities in large-scale systems using GPU-accelerated atomistic
 * parallel Monte Carlo algorithms" (arXiv:2103.03517).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py may load this library.  The product path (the
 * CUDA library) never calls it, and this file shares no code, header, table
 * or constant with the CUDA sources: everything below is written out here
 * from the paper and from the published definitions it names.
 *
 * Compile with -O2 -ffp-contract=off -fno-fast-math so that every floating
 * point operation is one IEEE double operation in source order (no fused
 * multiply-add, no reassociation).  The GPU FP64 mode follows the same
 * operation order and must reproduce the spin trajectory of this file bit
 * for bit.
 *
 * Units are reduced: J, K_u, K_c, H and T are energies (k_B = 1, mu_S = 1,
 * h = mu0 mu_S H of Eq. 2 is written H).
 *
 * Parity pins (tests/test_oracle_*.py): Philox against an independent
 * Philox4x32-10 implementation; exp against libm within 2 ulp; the cone
 * sampler against its closed-form marginals; the energy change against a
 * brute-force total-energy difference; the chain against the Langevin law,
 * the two-spin closed form and quadratures, the T -> 0 energy, the
 * harmonic spin-wave magnetization, the Binder-cumulant Curie point, the
 * serial random-order chain, constrained invariants and the low-T torque.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_EXPORT __attribute__((visibility("default")))

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* --------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random      */
/* numbers: as easy as 1, 2, 3").  Ten rounds of the 4x32 Philox S-box      */
/* with the published multipliers and Weyl key increments.  The paper only  */
/* names UniformRandom (Table A1); the counter layout used here is          */
/* ctr = (site or pair, sweep, tag, draw), key = (seed_lo, seed_hi).        */
/* --------------------------------------------------------------------- */
static void philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                   uint32_t k0, uint32_t k1, uint32_t out[4]) {
    for (int round = 0; round < 10; ++round) {
        const uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        const uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        const uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        const uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

OR_EXPORT void or_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    philox(ctr[0], ctr[1], ctr[2], ctr[3], key[0], key[1], out);
}

/* Tag of a Philox stream: bit 0 = colour, bits 1.. = purpose. */
enum { PURPOSE_MOVE = 0, PURPOSE_PAIR = 1, PURPOSE_PERM = 2, PURPOSE_SERIAL = 3 };
static uint32_t tag_of(int colour, int purpose) { return (uint32_t)colour | ((uint32_t)purpose << 1); }

/* --------------------------------------------------------------------- */
/* exp for the Metropolis test of Eq. 1, FP64, identical bits on every      */
/* IEEE machine: Cody & Waite (1980) range reduction x = k ln2 + r with a   */
/* two-part ln2 (32-bit head, so k*LN2_HI is exact for |k| < 2^21), then    */
/* the degree-13 Taylor polynomial of e^r by Horner's rule (truncation      */
/* error < 5e-18 relative for |r| <= ln2/2), then scaling by 2^k as two     */
/* exact powers of two so that the only rounding is the final product.      */
/* Constants: nearest doubles to ln2 (split), 1/ln2 and 1/n!.               */
/* --------------------------------------------------------------------- */
static const double EXP_LN2_HI = 0x1.62e42ff000000p-1;
static const double EXP_LN2_LO = -0x1.718432a1b0e26p-35;
static const double EXP_INV_LN2 = 0x1.71547652b82fep+0;
static const double EXP_INV_FACT[14] = {
    0x1.0000000000000p+0,  0x1.0000000000000p+0,  0x1.0000000000000p-1,
    0x1.5555555555555p-3,  0x1.5555555555555p-5,  0x1.1111111111111p-7,
    0x1.6c16c16c16c17p-10, 0x1.a01a01a01a01ap-13, 0x1.a01a01a01a01ap-16,
    0x1.71de3a556c734p-19, 0x1.27e4fb7789f5cp-22, 0x1.ae64567f544e4p-26,
    0x1.1eed8eff8d898p-29, 0x1.6124613a86d09p-33};

static double pow2i(int k) { /* 2^k for -1022 <= k <= 1023, built from its bits */
    uint64_t bits = (uint64_t)(k + 1023) << 52;
    double d;
    memcpy(&d, &bits, sizeof d);
    return d;
}

static double exp_own(double x) {
    if (x != x) return x;
    if (x < -746.0) return 0.0;
    if (x > 709.79) return INFINITY;
    const double kf = floor(x * EXP_INV_LN2 + 0.5);
    const int k = (int)kf;
    const double r = (x - kf * EXP_LN2_HI) - kf * EXP_LN2_LO;
    double p = EXP_INV_FACT[13];
    for (int n = 12; n >= 0; --n) p = p * r + EXP_INV_FACT[n];
    const int k1 = k / 2;
    const int k2 = k - k1;
    return (p * pow2i(k1)) * pow2i(k2);
}

OR_EXPORT double or_exp(double x) { return exp_own(x); }

/* exp_own over an array (for pinning it against a library exp on many
   points): y[i] = exp_own(x[i]), i < n. */
OR_EXPORT void or_exp_array(const double* x, double* y, int64_t n) {
    for (int64_t i = 0; i < n; ++i) y[i] = exp_own(x[i]);
}

/* --------------------------------------------------------------------- */
/* Cone table: c(theta) = 1 - cos(theta) = 2 sin^2(theta/2) for integer     */
/* degrees 0..180 (theta is the cone half-angle, Table A1                   */
/* "UniformRandom_RotateSpin(S, theta)").                                   */
/* --------------------------------------------------------------------- */
static double cone_c(int deg) {
    const double h = sin((double)deg * (M_PI / 360.0));
    return 2.0 * (h * h);
}

/* Orthonormal basis {b1, b2, n} for a unit vector n, from Duff, Burgess,    */
/* Christensen, Hery, Kensler, Liani, Villemin, "Building an Orthonormal    */
/* Basis, Revisited", JCGT 6(1) 2017.                                       */
static void onb(const double n[3], double b1[3], double b2[3]) {
    const double sgn = copysign(1.0, n[2]);
    const double a = -1.0 / (sgn + n[2]);
    const double b = n[0] * n[1] * a;
    b1[0] = 1.0 + sgn * n[0] * n[0] * a;
    b1[1] = sgn * b;
    b1[2] = -sgn * n[0];
    b2[0] = b;
    b2[1] = sgn + n[1] * n[1] * a;
    b2[2] = -n[1];
}

/*
 * Trial move "UniformRandom_RotateSpin(S, theta)" (Table A1, Sec. 2): a
 * direction uniform by solid angle on the spherical cap of half-angle
 * theta about S.  Marsaglia's disk method (Ann. Math. Stat. 43, 1972)
 * generalised to a cap: (u1, u2) uniform in the unit disk, s = u1^2 + u2^2
 * uniform on [0, 1), z' = 1 - s c, (x', y') = (u1, u2) sqrt(c (2 - s c)),
 * which puts z' uniform on [cos theta, 1] with a uniform azimuth.  The point
 * is mapped through the basis of S and renormalised.  Attempt a uses the
 * words (w0, w1) of draw a; after 16 rejected disk points the move is
 * rejected (probability ~2e-11).  P of Eq. 1 is w2 of draw 0.
 * Returns 1 and the trial in out[] on success, 0 otherwise.
 */
static int cone_trial(const double S[3], double c, uint32_t idx, uint32_t sweep,
                      uint32_t tag, uint32_t k0, uint32_t k1, double out[3], double* P) {
    uint32_t w[4];
    philox(idx, sweep, tag, 0u, k0, k1, w);
    *P = (double)w[2] * 0x1p-32;
    double u1 = (double)w[0] * 0x1p-31 - 1.0;
    double u2 = (double)w[1] * 0x1p-31 - 1.0;
    double s = u1 * u1 + u2 * u2;
    uint32_t draw = 0;
    while (!(s < 1.0)) {
        if (++draw == 16u) return 0;
        philox(idx, sweep, tag, draw, k0, k1, w);
        u1 = (double)w[0] * 0x1p-31 - 1.0;
        u2 = (double)w[1] * 0x1p-31 - 1.0;
        s = u1 * u1 + u2 * u2;
    }
    const double sc = s * c;
    const double zp = 1.0 - sc;
    const double r = sqrt(c * (2.0 - sc));
    const double xp = u1 * r;
    const double yp = u2 * r;
    double b1[3], b2[3];
    onb(S, b1, b2);
    double n[3];
    for (int a = 0; a < 3; ++a) n[a] = xp * b1[a] + yp * b2[a] + zp * S[a];
    const double norm = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    for (int a = 0; a < 3; ++a) out[a] = n[a] / norm;
    return 1;
}

OR_EXPORT int or_cone_trial(const double S[3], int theta_deg, uint32_t idx, uint32_t sweep,
                            uint32_t tag, const uint32_t key[2], double out[3], double* P) {
    return cone_trial(S, cone_c(theta_deg), idx, sweep, tag, key[0], key[1], out, P);
}

/* --------------------------------------------------------------------- */
/* Lattice.  Sites are (x, y, z) with index x + Lx (y + Ly z); colour       */
/* (x + y + z) mod 2, 0 = red (Sec. 2, checkerboard).  Boundary per axis:   */
/* 0 periodic, 1 open, 2 pinned (open, and the two end planes are never    */
/* updated).  Optional per-site bond mask (films: bit d set = bond in       */
/* direction d present, d = -x,+x,-y,+y,-z,+z) and per-site easy axis via   */
/* a grain-id table.                                                        */
/* --------------------------------------------------------------------- */
typedef struct {
    int L[3];
    int bc[3];
    int64_t N;
    int64_t n_mov;
    double J, Ku, axis[3], Kc, H[3], T;
    uint32_t key0, key1;
    int theta;
    int adapt_in_measure;
    uint32_t sweep;
    double* S;          /* N x 3 */
    uint8_t* pinned;    /* N */
    uint8_t* bonds;     /* N, or NULL: full bonds from the boundary modes */
    int32_t* grain;     /* N, or NULL: uniform axis */
    double* grain_axis; /* n_grains x 3 */
    int n_grains;
    int64_t last_accepted;
    /* measurement accumulators (Sec. 3) */
    int64_t n_samples;
    double acc_m[3], acc_m2[3], acc_mabs[3];
    double acc_ml, acc_ml2, acc_ml4;
    double acc_e, acc_e2, acc_parts[4];
    double acc_tq[3], acc_tq2[3];
    double* profile; /* Lx: sums over samples of sum_{y,z} S_z */
    int64_t n_profile;
    /* per-sample series (ring) */
    double* ring;
    int ring_cap;
    int64_t ring_count;
} or_lattice;

enum { SAMPLE_WORDS = 14 }; /* sweep, theta, accepted, m[3], e_ex, e_u, e_c, e_z, tq[3], unused */

static int64_t site_of(const or_lattice* L, int x, int y, int z) {
    return (int64_t)x + (int64_t)L->L[0] * ((int64_t)y + (int64_t)L->L[1] * z);
}

/* neighbour in direction d (0..5 = -x,+x,-y,+y,-z,+z); -1 if absent.
 * Boundary modes: 0 periodic, 1 open, 2 pinned (open), 3 anti-periodic: the
 * axis wraps and the spin across the face enters as -S, *flip = 1. */
static int64_t neighbour(const or_lattice* L, int64_t i, int x, int y, int z, int d, int* flip) {
    int c[3] = {x, y, z};
    const int ax = d / 2;
    const int step = (d & 1) ? 1 : -1;
    int v = c[ax] + step;
    *flip = 0;
    if (v < 0 || v >= L->L[ax]) {
        if (L->bc[ax] != 0 && L->bc[ax] != 3) return -1;
        v = (v + L->L[ax]) % L->L[ax];
        *flip = L->bc[ax] == 3;
    }
    if (L->bonds && !((L->bonds[i] >> d) & 1u)) return -1;
    c[ax] = v;
    return site_of(L, c[0], c[1], c[2]);
}

static const double* easy_axis(const or_lattice* L, int64_t i) {
    if (L->grain) return &L->grain_axis[3 * (int64_t)L->grain[i]];
    return L->axis;
}

static double cubic_q(const double s[3]) {
    const double x2 = s[0] * s[0], y2 = s[1] * s[1], z2 = s[2] * s[2];
    return x2 * y2 + x2 * z2 + y2 * z2;
}

/*
 * Energy change of Eq. 2 for site i going from S to Sn, with the
 * neighbours held fixed:  dE = -J d.h - K_u((Sn.e)^2 - (S.e)^2)
 *                               + K_c(q(Sn) - q(S)) - H.d,  d = Sn - S,
 * h = sum of the present nearest neighbours, accumulated in the order
 * -x, +x, -y, +y, -z, +z (a neighbour across an anti-periodic face as -S).
 */
static double delta_e(const or_lattice* L, int64_t i, const double S[3], const double Sn[3]) {
    const int x = (int)(i % L->L[0]);
    const int y = (int)((i / L->L[0]) % L->L[1]);
    const int z = (int)(i / ((int64_t)L->L[0] * L->L[1]));
    double h[3] = {0.0, 0.0, 0.0};
    for (int d = 0; d < 6; ++d) {
        int flip;
        const int64_t j = neighbour(L, i, x, y, z, d, &flip);
        if (j < 0) continue;
        for (int a = 0; a < 3; ++a) h[a] = flip ? h[a] - L->S[3 * j + a] : h[a] + L->S[3 * j + a];
    }
    const double d0 = Sn[0] - S[0], d1 = Sn[1] - S[1], d2 = Sn[2] - S[2];
    const double e_ex = -(L->J * (d0 * h[0] + d1 * h[1] + d2 * h[2]));
    const double* e = easy_axis(L, i);
    const double pn = Sn[0] * e[0] + Sn[1] * e[1] + Sn[2] * e[2];
    const double po = S[0] * e[0] + S[1] * e[1] + S[2] * e[2];
    const double e_u = -(L->Ku * (pn * pn - po * po));
    const double e_c = L->Kc * (cubic_q(Sn) - cubic_q(S));
    const double e_z = -(L->H[0] * d0 + L->H[1] * d1 + L->H[2] * d2);
    return e_ex + e_u + e_c + e_z;
}

OR_EXPORT double or_delta_e(const or_lattice* L, int64_t i, const double Sn[3]) {
    return delta_e(L, i, &L->S[3 * i], Sn);
}

/* Metropolis acceptance of Eq. 1 / Table A1: accept iff P < exp(-dE/T). */
static int metropolis(double dE, double T, double P) {
    if (dE <= 0.0) return 1; /* exp(-dE/T) >= 1 > P */
    return P < exp_own(-(dE / T));
}

OR_EXPORT or_lattice* or_create(const int dims[3], const int bc[3], double J, double Ku,
                                const double axis[3], double Kc, const double H[3], double T,
                                uint64_t seed, int theta0, int adapt_in_measure, int ring_cap) {
    or_lattice* L = (or_lattice*)calloc(1, sizeof(or_lattice));
    if (!L) return NULL;
    for (int a = 0; a < 3; ++a) { L->L[a] = dims[a]; L->bc[a] = bc[a]; }
    L->N = (int64_t)dims[0] * dims[1] * dims[2];
    L->J = J; L->Ku = Ku; L->Kc = Kc; L->T = T;
    const double an = sqrt(axis[0] * axis[0] + axis[1] * axis[1] + axis[2] * axis[2]);
    for (int a = 0; a < 3; ++a) { L->axis[a] = axis[a] / an; L->H[a] = H[a]; }
    L->key0 = (uint32_t)seed;
    L->key1 = (uint32_t)(seed >> 32);
    L->theta = theta0;
    L->adapt_in_measure = adapt_in_measure;
    L->S = (double*)calloc((size_t)L->N * 3, sizeof(double));
    L->pinned = (uint8_t*)calloc((size_t)L->N, 1);
    L->profile = (double*)calloc((size_t)dims[0], sizeof(double));
    L->ring_cap = ring_cap > 0 ? ring_cap : 1;
    L->ring = (double*)calloc((size_t)L->ring_cap * SAMPLE_WORDS, sizeof(double));
    L->n_mov = 0;
    for (int64_t i = 0; i < L->N; ++i) {
        L->S[3 * i + 2] = 1.0;
        const int c[3] = {(int)(i % dims[0]), (int)((i / dims[0]) % dims[1]),
                          (int)(i / ((int64_t)dims[0] * dims[1]))};
        int pin = 0;
        for (int a = 0; a < 3; ++a)
            if (bc[a] == 2 && (c[a] == 0 || c[a] == dims[a] - 1)) pin = 1;
        L->pinned[i] = (uint8_t)pin;
        L->n_mov += !pin;
    }
    return L;
}

OR_EXPORT void or_destroy(or_lattice* L) {
    if (!L) return;
    free(L->S); free(L->pinned); free(L->bonds); free(L->grain); free(L->grain_axis);
    free(L->profile); free(L->ring); free(L);
}

OR_EXPORT void or_set_spins(or_lattice* L, const double* xyz) { memcpy(L->S, xyz, sizeof(double) * 3 * (size_t)L->N); }
OR_EXPORT void or_get_spins(const or_lattice* L, double* xyz) { memcpy(xyz, L->S, sizeof(double) * 3 * (size_t)L->N); }
OR_EXPORT void or_set_temperature(or_lattice* L, double T) { L->T = T; }
OR_EXPORT int or_theta(const or_lattice* L) { return L->theta; }
OR_EXPORT uint32_t or_sweep_count(const or_lattice* L) { return L->sweep; }
OR_EXPORT int64_t or_last_accepted(const or_lattice* L) { return L->last_accepted; }
OR_EXPORT int64_t or_n_mov(const or_lattice* L) { return L->n_mov; }

OR_EXPORT void or_set_bonds(or_lattice* L, const uint8_t* mask) {
    free(L->bonds);
    L->bonds = (uint8_t*)malloc((size_t)L->N);
    memcpy(L->bonds, mask, (size_t)L->N);
}

OR_EXPORT void or_set_grains(or_lattice* L, const int32_t* gid, const double* axes, int n_grains) {
    free(L->grain); free(L->grain_axis);
    L->grain = (int32_t*)malloc(sizeof(int32_t) * (size_t)L->N);
    memcpy(L->grain, gid, sizeof(int32_t) * (size_t)L->N);
    L->grain_axis = (double*)malloc(sizeof(double) * 3 * (size_t)n_grains);
    for (int g = 0; g < n_grains; ++g) {
        const double* v = &axes[3 * g];
        const double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        for (int a = 0; a < 3; ++a) L->grain_axis[3 * g + a] = v[a] / n;
    }
    L->n_grains = n_grains;
}

/* Cone-angle adaptation after a full iteration (Sec. 2, Table A1): the      */
/* acceptance rate is accepted/N_mov; strictly above 0.5 widens the cone    */
/* by one degree (up to 180), otherwise narrows it (down to 1).             */
static void adapt_theta(or_lattice* L, int64_t accepted) {
    if (2 * accepted > L->n_mov) {
        if (L->theta < 180) L->theta += 1;
    } else {
        if (L->theta > 1) L->theta -= 1;
    }
}

/* --------------------------------------------------------------------- */
/* Measurements (Sec. 3).  Per sample: M = sum S; exchange sum over bonds    */
/* (each bond once, via the +x, +y, +z neighbours); uniaxial, cubic and     */
/* Zeeman sums; torque sum S x (-dE_anis,Z/dS); slice sums of S_z per x.    */
/* --------------------------------------------------------------------- */
static void measure(or_lattice* L, int64_t accepted) {
    double M[3] = {0, 0, 0}, sex = 0, su = 0, sc = 0, tu[3] = {0, 0, 0}, tc[3] = {0, 0, 0};
    for (int64_t i = 0; i < L->N; ++i) {
        const double* s = &L->S[3 * i];
        const int x = (int)(i % L->L[0]);
        const int y = (int)((i / L->L[0]) % L->L[1]);
        const int z = (int)(i / ((int64_t)L->L[0] * L->L[1]));
        for (int a = 0; a < 3; ++a) M[a] += s[a];
        for (int d = 1; d < 6; d += 2) {
            int flip;
            const int64_t j = neighbour(L, i, x, y, z, d, &flip);
            if (j < 0) continue;
            const double* t = &L->S[3 * j];
            const double b = s[0] * t[0] + s[1] * t[1] + s[2] * t[2];
            sex += flip ? -b : b;
        }
        const double* e = easy_axis(L, i);
        const double pe = s[0] * e[0] + s[1] * e[1] + s[2] * e[2];
        su += pe * pe;
        sc += cubic_q(s);
        /* (S.e)(S x e) */
        tu[0] += pe * (s[1] * e[2] - s[2] * e[1]);
        tu[1] += pe * (s[2] * e[0] - s[0] * e[2]);
        tu[2] += pe * (s[0] * e[1] - s[1] * e[0]);
        /* S x c(S), c(S) = (Sx(Sy^2+Sz^2), Sy(Sx^2+Sz^2), Sz(Sx^2+Sy^2)) */
        const double x2 = s[0] * s[0], y2 = s[1] * s[1], z2 = s[2] * s[2];
        const double c0 = s[0] * (y2 + z2), c1 = s[1] * (x2 + z2), c2 = s[2] * (x2 + y2);
        tc[0] += s[1] * c2 - s[2] * c1;
        tc[1] += s[2] * c0 - s[0] * c2;
        tc[2] += s[0] * c1 - s[1] * c0;
        L->profile[x] += s[2];
    }
    L->n_profile += 1;
    const double N = (double)L->N;
    double m[3], ml2 = 0;
    for (int a = 0; a < 3; ++a) { m[a] = M[a] / N; ml2 += m[a] * m[a]; }
    const double ml = sqrt(ml2);
    const double e_ex = -L->J * sex / N, e_u = -L->Ku * su / N, e_c = L->Kc * sc / N;
    const double e_z = -(L->H[0] * M[0] + L->H[1] * M[1] + L->H[2] * M[2]) / N;
    const double e = e_ex + e_u + e_c + e_z;
    double tq[3];
    tq[0] = (2.0 * L->Ku * tu[0] - 2.0 * L->Kc * tc[0] + (M[1] * L->H[2] - M[2] * L->H[1])) / N;
    tq[1] = (2.0 * L->Ku * tu[1] - 2.0 * L->Kc * tc[1] + (M[2] * L->H[0] - M[0] * L->H[2])) / N;
    tq[2] = (2.0 * L->Ku * tu[2] - 2.0 * L->Kc * tc[2] + (M[0] * L->H[1] - M[1] * L->H[0])) / N;
    L->n_samples += 1;
    for (int a = 0; a < 3; ++a) {
        L->acc_m[a] += m[a]; L->acc_m2[a] += m[a] * m[a]; L->acc_mabs[a] += fabs(m[a]);
        L->acc_tq[a] += tq[a]; L->acc_tq2[a] += tq[a] * tq[a];
    }
    L->acc_ml += ml; L->acc_ml2 += ml2; L->acc_ml4 += ml2 * ml2;
    L->acc_e += e; L->acc_e2 += e * e;
    L->acc_parts[0] += e_ex; L->acc_parts[1] += e_u; L->acc_parts[2] += e_c; L->acc_parts[3] += e_z;
    double* r = &L->ring[(L->ring_count % L->ring_cap) * SAMPLE_WORDS];
    r[0] = (double)L->sweep; r[1] = (double)L->theta; r[2] = (double)accepted;
    r[3] = m[0]; r[4] = m[1]; r[5] = m[2];
    r[6] = e_ex; r[7] = e_u; r[8] = e_c; r[9] = e_z;
    r[10] = tq[0]; r[11] = tq[1]; r[12] = tq[2]; r[13] = 0.0;
    L->ring_count += 1;
}

/* Sums of the per-sample observables, in this order:
 * n, m[3], m2[3], mabs[3], ml, ml2, ml4, e, e2, parts[4], tq[3], tq2[3]  (26 words). */
OR_EXPORT void or_stats(const or_lattice* L, double* out) {
    int k = 0;
    out[k++] = (double)L->n_samples;
    for (int a = 0; a < 3; ++a) out[k++] = L->acc_m[a];
    for (int a = 0; a < 3; ++a) out[k++] = L->acc_m2[a];
    for (int a = 0; a < 3; ++a) out[k++] = L->acc_mabs[a];
    out[k++] = L->acc_ml; out[k++] = L->acc_ml2; out[k++] = L->acc_ml4;
    out[k++] = L->acc_e; out[k++] = L->acc_e2;
    for (int a = 0; a < 4; ++a) out[k++] = L->acc_parts[a];
    for (int a = 0; a < 3; ++a) out[k++] = L->acc_tq[a];
    for (int a = 0; a < 3; ++a) out[k++] = L->acc_tq2[a];
}

/* Eq. 4 (Sec. 3): temperature scaling of the anisotropy from the mean
 * easy-axis anisotropy energy of the standard algorithm.  K_easy is the mean
 * anisotropy energy per spin above its T = 0 value (all spins on the easy
 * direction); K_0,hard is the T = 0 energy per spin of the hard direction
 * above the easy one.  Uniaxial, E_u = -K_u (S.e)^2: K_easy = <E_u/N> + K_u,
 * K_0,hard = K_u, k_u = 1 - 3 K_easy / (2 K_0,hard).  Cubic, E_c = K_c q(S)
 * with K_c > 0 (easy <100>, q = 0; hard <111>, q = 1/3): K_easy = <E_c/N>,
 * K_0,hard = K_c / 3, k_c = 1 - 5 K_easy / (3 K_0,hard).  out[0] = k_u,
 * out[1] = k_c; NaN where the constant is zero or no sample was taken. */
OR_EXPORT void or_anisotropy_scaling(const or_lattice* L, double* out) {
    out[0] = NAN;
    out[1] = NAN;
    if (L->n_samples == 0) return;
    const double n = (double)L->n_samples;
    if (L->Ku != 0.0) {
        const double k_easy = L->acc_parts[1] / n + L->Ku;
        const double k0_hard = L->Ku;
        out[0] = 1.0 - 3.0 * k_easy / (2.0 * k0_hard);
    }
    if (L->Kc != 0.0) {
        const double k_easy = L->acc_parts[2] / n;
        const double k0_hard = L->Kc / 3.0;
        out[1] = 1.0 - 5.0 * k_easy / (3.0 * k0_hard);
    }
}

/* The most recent min(max, kept) samples, oldest first. */
OR_EXPORT int64_t or_samples(const or_lattice* L, double* out, int64_t max) {
    int64_t n = L->ring_count < L->ring_cap ? L->ring_count : L->ring_cap;
    if (n > max) n = max;
    const int64_t first = L->ring_count - n;
    int64_t k = 0;
    for (int64_t s = first; s < L->ring_count && k < max; ++s, ++k)
        memcpy(&out[k * SAMPLE_WORDS], &L->ring[(s % L->ring_cap) * SAMPLE_WORDS], sizeof(double) * SAMPLE_WORDS);
    return k;
}

OR_EXPORT void or_profile(const or_lattice* L, double* out) {
    const double denom = (double)L->n_profile * (double)L->L[1] * (double)L->L[2];
    for (int x = 0; x < L->L[0]; ++x) out[x] = L->n_profile ? L->profile[x] / denom : 0.0;
}

OR_EXPORT void or_reset_stats(or_lattice* L) {
    L->n_samples = 0;
    memset(L->acc_m, 0, sizeof L->acc_m); memset(L->acc_m2, 0, sizeof L->acc_m2);
    memset(L->acc_mabs, 0, sizeof L->acc_mabs);
    L->acc_ml = L->acc_ml2 = L->acc_ml4 = L->acc_e = L->acc_e2 = 0;
    memset(L->acc_parts, 0, sizeof L->acc_parts);
    memset(L->acc_tq, 0, sizeof L->acc_tq); memset(L->acc_tq2, 0, sizeof L->acc_tq2);
    memset(L->profile, 0, sizeof(double) * (size_t)L->L[0]);
    L->n_profile = 0;
    L->ring_count = 0;
}

/* --------------------------------------------------------------------- */
/* Parallel (checkerboard) Metropolis iteration, Table A1: the red pass     */
/* over every movable red site, then the black pass; within a colour the    */
/* sites do not interact, so the oracle simply visits them in index order.  */
/* The RNG is keyed by site, so the order inside a pass is immaterial.      */
/* --------------------------------------------------------------------- */
static int64_t colour_pass_planes(or_lattice* L, int colour, int z0, int z1) {
    const double c = cone_c(L->theta);
    const uint32_t tag = tag_of(colour, PURPOSE_MOVE);
    int64_t accepted = 0;
    for (int z = z0; z < z1; ++z)
        for (int y = 0; y < L->L[1]; ++y)
            for (int x = 0; x < L->L[0]; ++x) {
                if (((x + y + z) & 1) != colour) continue;
                const int64_t i = site_of(L, x, y, z);
                if (L->pinned[i]) continue;
                double* S = &L->S[3 * i];
                double Sn[3], P;
                if (!cone_trial(S, c, (uint32_t)i, L->sweep, tag, L->key0, L->key1, Sn, &P)) continue;
                const double dE = delta_e(L, i, S, Sn);
                if (metropolis(dE, L->T, P)) {
                    S[0] = Sn[0]; S[1] = Sn[1]; S[2] = Sn[2];
                    ++accepted;
                }
            }
    return accepted;
}

static int64_t colour_pass(or_lattice* L, int colour) { return colour_pass_planes(L, colour, 0, L->L[2]); }

/* One colour pass restricted to the planes z0 <= z < z1: the part of a      */
/* Table A1 pass that one slab of a lattice split along z performs.  The    */
/* per-site update is colour_pass's; the caller supplies the neighbouring   */
/* planes.  Returns the accepted moves.                                     */
OR_EXPORT int64_t or_colour_pass_planes(or_lattice* L, int colour, int z0, int z1) {
    if (colour < 0 || colour > 1 || z0 < 0 || z1 > L->L[2] || z0 > z1) return -1;
    return colour_pass_planes(L, colour, z0, z1);
}

/* The end of an unmeasured iteration of Table A1 given the accepted moves  */
/* of the whole lattice (summed over slabs): cone adaptation, sweep count.  */
OR_EXPORT void or_end_sweep(or_lattice* L, int64_t accepted) {
    L->last_accepted = accepted;
    adapt_theta(L, accepted);
    L->sweep += 1;
}

OR_EXPORT int or_sweep(or_lattice* L, int n_sweeps, int measure_flag) {
    for (int s = 0; s < n_sweeps; ++s) {
        int64_t acc = colour_pass(L, 0);
        acc += colour_pass(L, 1);
        L->last_accepted = acc;
        if (!measure_flag || L->adapt_in_measure) adapt_theta(L, acc);
        if (measure_flag) measure(L, acc);
        L->sweep += 1;
    }
    return 0;
}

/* Serial Metropolis in random site order (Sec. 2, the algorithm the paper   */
/* parallelises): each iteration visits every movable site once, in the    */
/* order of a Fisher-Yates shuffle drawn from Philox (purpose 3).  A        */
/* statistical second oracle only: its chain differs from the checkerboard  */
/* chain, its ensemble averages must not.                                   */
OR_EXPORT int or_sweep_serial(or_lattice* L, int n_sweeps, int measure_flag) {
    int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)L->N);
    if (!order) return -1;
    for (int s = 0; s < n_sweeps; ++s) {
        int64_t n = 0;
        for (int64_t i = 0; i < L->N; ++i)
            if (!L->pinned[i]) order[n++] = i;
        for (int64_t k = n - 1; k > 0; --k) {
            uint32_t w[4];
            philox((uint32_t)k, L->sweep, tag_of(0, PURPOSE_SERIAL), 0xFFFFFFFFu, L->key0, L->key1, w);
            const uint64_t r = (((uint64_t)w[0] << 32) | w[1]) % (uint64_t)(k + 1);
            const int64_t t = order[k]; order[k] = order[r]; order[r] = t;
        }
        const double c = cone_c(L->theta);
        int64_t acc = 0;
        for (int64_t k = 0; k < n; ++k) {
            const int64_t i = order[k];
            double* S = &L->S[3 * i];
            double Sn[3], P;
            if (!cone_trial(S, c, (uint32_t)i, L->sweep, tag_of(1, PURPOSE_SERIAL), L->key0, L->key1, Sn, &P)) continue;
            if (metropolis(delta_e(L, i, S, Sn), L->T, P)) {
                S[0] = Sn[0]; S[1] = Sn[1]; S[2] = Sn[2];
                ++acc;
            }
        }
        L->last_accepted = acc;
        if (!measure_flag || L->adapt_in_measure) adapt_theta(L, acc);
        if (measure_flag) measure(L, acc);
        L->sweep += 1;
    }
    free(order);
    return 0;
}

/* --------------------------------------------------------------------- */
/* Constrained Monte Carlo (Asselin et al., PRB 82, 054415 (2010)), in the  */
/* parallel form of Sec. 2 and Table A2.                                    */
/* --------------------------------------------------------------------- */

/* Exact, order-independent M_L = sum_i S_i . e_C: every FP64 term t is      */
/* written as q = trunc(t 2^52) (exact int64), split q = hi 2^26 + lo with  */
/* 0 <= lo < 2^26, and the two parts are summed as integers.               */
static double fixed_sum_value(int64_t hi, int64_t lo) {
    return (double)hi * 0x1p-26 + (double)lo * 0x1p-52;
}
static void fixed_add(double t, int64_t* hi, int64_t* lo) {
    const int64_t q = (int64_t)(t * 0x1p52);
    const int64_t h = q >> 26; /* arithmetic shift: floor(q / 2^26) */
    *hi += h;
    *lo += q - h * ((int64_t)1 << 26);
}

OR_EXPORT double or_fixed_sum(const double* t, int64_t n) {
    int64_t hi = 0, lo = 0;
    for (int64_t i = 0; i < n; ++i) fixed_add(t[i], &hi, &lo);
    return fixed_sum_value(hi, lo);
}

/* Frame with its x-axis along e_C (Table A2 RotateCoordinateSystem): rows   */
/* e1 = e_C = (sin th cos ph, sin th sin ph, cos th), e2 = (-sin ph,         */
/* cos ph, 0), e3 = e1 x e2 = (-cos th cos ph, -cos th sin ph, sin th).     */
static void constraint_frame(double theta_deg, double phi_deg, double R[9]) {
    const double th = theta_deg * (M_PI / 180.0), ph = phi_deg * (M_PI / 180.0);
    const double st = sin(th), ct = cos(th), sp = sin(ph), cp = cos(ph);
    R[0] = st * cp;  R[1] = st * sp;  R[2] = ct;
    R[3] = -sp;      R[4] = cp;       R[5] = 0.0;
    R[6] = -ct * cp; R[7] = -ct * sp; R[8] = st;
}

OR_EXPORT void or_constraint_frame(double theta_deg, double phi_deg, double R[9]) {
    constraint_frame(theta_deg, phi_deg, R);
}

static void rotate(const double R[9], const double s[3], double out[3]) {
    for (int r = 0; r < 3; ++r) out[r] = R[3 * r] * s[0] + R[3 * r + 1] * s[1] + R[3 * r + 2] * s[2];
}
static void rotate_back(const double R[9], const double h[3], double out[3]) {
    for (int a = 0; a < 3; ++a) out[a] = h[0] * R[a] + h[1] * R[3 + a] + h[2] * R[6 + a];
}

/* M_L of Table A2: sum of S . e_C over the lattice, exact. */
static double m_long(const or_lattice* L, const double R[9]) {
    int64_t hi = 0, lo = 0;
    for (int64_t i = 0; i < L->N; ++i) {
        const double* s = &L->S[3 * i];
        fixed_add(R[0] * s[0] + R[1] * s[1] + R[2] * s[2], &hi, &lo);
    }
    return fixed_sum_value(hi, lo);
}

OR_EXPORT double or_m_long(const or_lattice* L, double theta_deg, double phi_deg) {
    double R[9];
    constraint_frame(theta_deg, phi_deg, R);
    return m_long(L, R);
}

/* ShuffleRedBlackSpins (Sec. 2, Table A2) as a keyed bijection of the       */
/* colour indices [0, n): a 4-round alternating Feistel network on b-bit    */
/* words, b the least width with 2^b >= n (the alternating splits of the    */
/* FFX mode, Bellare, Rogaway & Spies 2010, for odd b), with cycle-walking  */
/* (Black & Rogaway, CT-RSA 2002).  Round k takes the low w bits R and the  */
/* high b - w bits L of the word to (R, L ^ F_k(R)), R now on top; w is     */
/* ceil(b/2) in rounds 0 and 2, floor(b/2) in rounds 1 and 3, so that for   */
/* even b every round is a balanced one.  F_k(R) is the "lowbias32" integer */
/* hash (C. Wellons, 2018) of R xor round key k, cut to b - w bits; the     */
/* round keys are the four words of Philox(0, sweep, colour | purpose 2, 0).*/
static uint32_t hash32(uint32_t v) {
    v ^= v >> 16; v *= 0x7feb352du;
    v ^= v >> 15; v *= 0x846ca68bu;
    v ^= v >> 16;
    return v;
}
static int domain_bits(uint32_t n) {
    int b = 1;
    while (((uint64_t)1 << b) < (uint64_t)n) ++b;
    return b;
}
static uint32_t low_mask(int w) { return w >= 32 ? 0xFFFFFFFFu : ((1u << w) - 1u); }
static uint32_t feistel_once(uint32_t v, int b, const uint32_t rk[4]) {
    for (int k = 0; k < 4; ++k) {
        const int w = (k % 2 == 0) ? (b + 1) / 2 : b / 2;
        const uint32_t r = v & low_mask(w);
        const uint32_t l = v >> w;
        const uint32_t f = hash32(r ^ rk[k]) & low_mask(b - w);
        v = (r << (b - w)) | (l ^ f);
    }
    return v;
}
static uint32_t permute(uint32_t i, uint32_t n, int b, const uint32_t rk[4]) {
    uint32_t v = i;
    do { v = feistel_once(v, b, rk); } while (v >= n);
    return v;
}

OR_EXPORT void or_permutation(uint32_t n, uint32_t sweep, int colour, const uint32_t key[2], uint32_t* out) {
    uint32_t rk[4];
    philox(0u, sweep, tag_of(colour, PURPOSE_PERM), 0u, key[0], key[1], rk);
    const int b = domain_bits(n);
    for (uint32_t i = 0; i < n; ++i) out[i] = permute(i, n, b, rk);
}

/* Site of colour index q = k + (Lx/2)(y + Ly z) of colour c. */
static int64_t colour_site(const or_lattice* L, int colour, uint32_t q) {
    const int lh = L->L[0] / 2;
    const int k = (int)(q % (uint32_t)lh);
    const uint32_t row = q / (uint32_t)lh;
    const int y = (int)(row % (uint32_t)L->L[1]);
    const int z = (int)(row / (uint32_t)L->L[1]);
    const int x = ((y + z + colour) & 1) + 2 * k;
    return site_of(L, x, y, z);
}

/*
 * One pair move of Table A2 for the spins i (cone move) and j (partner),
 * both of the same colour.  Rotated-frame components are written ^.
 * Readings of the paper fixed here: a rejected disk point (16 tries), a
 * non-positive t = |S_j|^2 - y'_j^2 - z'_j^2, or M^_L <= 0 reject the pair;
 * sign(0) = +1; the Boltzmann factor is exp(-(E'_i + E'_j - E_i - E_j)/T).
 * Returns 1 if accepted (and writes both spins).
 */
static int pair_move(or_lattice* L, const double R[9], double ML, double c, int64_t si, int64_t sj,
                     uint32_t pair, uint32_t tag) {
    double* Si = &L->S[3 * si];
    double* Sj = &L->S[3 * sj];
    double hi[3], hj[3];
    rotate(R, Si, hi);
    rotate(R, Sj, hj);
    double hni[3], P;
    if (!cone_trial(hi, c, pair, L->sweep, tag, L->key0, L->key1, hni, &P)) return 0;
    const double ynj = (hj[1] + hi[1]) - hni[1];
    const double znj = (hj[2] + hi[2]) - hni[2];
    const double t = (hj[0] * hj[0] + hj[1] * hj[1] + hj[2] * hj[2]) - ynj * ynj - znj * znj;
    if (!(t > 0.0)) return 0;
    double xnj = sqrt(t);
    if (hj[0] < 0.0) xnj = -xnj;
    const double MLn = ML + hni[0] + xnj - hi[0] - hj[0];
    if (!(MLn > 0.0)) return 0;
    const double hnj[3] = {xnj, ynj, znj};
    double Sni[3], Snj[3];
    rotate_back(R, hni, Sni);
    rotate_back(R, hnj, Snj);
    /* E(S'_i) - E(S_i) with the old neighbours, then E(S'_j) - E(S_j) with
     * S_i already moved: exact even when i and j are neighbours (serial
     * form); for a same-colour pair the second term does not see S_i. */
    const double dEi = delta_e(L, si, Si, Sni);
    const double keep[3] = {Si[0], Si[1], Si[2]};
    Si[0] = Sni[0]; Si[1] = Sni[1]; Si[2] = Sni[2];
    const double dEj = delta_e(L, sj, Sj, Snj);
    Si[0] = keep[0]; Si[1] = keep[1]; Si[2] = keep[2];
    const double dE = dEi + dEj;
    const double ratio = MLn / ML;
    double r = ratio * ratio;
    r = r * (fabs(hj[0]) / fabs(xnj));
    r = r * exp_own(-(dE / L->T));
    if (P < r) {
        Si[0] = Sni[0]; Si[1] = Sni[1]; Si[2] = Sni[2];
        Sj[0] = Snj[0]; Sj[1] = Snj[1]; Sj[2] = Snj[2];
        return 1;
    }
    return 0;
}

/* Parallel constrained iteration (Table A2): M_L once from the state at the */
/* start of the iteration, then the red and the black pass with that same   */
/* M_L; pairs (pi(2p), pi(2p+1)); accepted pairs count 2 towards the        */
/* acceptance rate; cone angle adapted as in Table A1.                       */
OR_EXPORT int or_constrained_sweep(or_lattice* L, double theta_deg, double phi_deg, int n_sweeps, int measure_flag) {
    double R[9];
    constraint_frame(theta_deg, phi_deg, R);
    for (int s = 0; s < n_sweeps; ++s) {
        const double ML = m_long(L, R);
        if (!(ML > 0.0)) return -5;
        const double c = cone_c(L->theta);
        int64_t acc = 0;
        for (int colour = 0; colour < 2; ++colour) {
            const uint32_t nc = (uint32_t)(L->N / 2);
            uint32_t rk[4];
            philox(0u, L->sweep, tag_of(colour, PURPOSE_PERM), 0u, L->key0, L->key1, rk);
            const int b = domain_bits(nc);
            const uint32_t tag = tag_of(colour, PURPOSE_PAIR);
            for (uint32_t p = 0; p < nc / 2; ++p) {
                const int64_t si = colour_site(L, colour, permute(2 * p, nc, b, rk));
                const int64_t sj = colour_site(L, colour, permute(2 * p + 1, nc, b, rk));
                acc += 2 * pair_move(L, R, ML, c, si, sj, p, tag);
            }
        }
        L->last_accepted = acc;
        if (!measure_flag || L->adapt_in_measure) adapt_theta(L, acc);
        if (measure_flag) measure(L, acc);
        L->sweep += 1;
    }
    return 0;
}

/* Serial constrained MC as introduced by Asselin et al.: pairs of distinct  */
/* random sites drawn from the whole lattice, M_L updated after every       */
/* accepted pair, N/2 pair attempts per iteration.  Statistical second      */
/* oracle for the parallel form (the paper's own check, Sec. 2).            */
OR_EXPORT int or_constrained_sweep_serial(or_lattice* L, double theta_deg, double phi_deg, int n_sweeps, int measure_flag) {
    double R[9];
    constraint_frame(theta_deg, phi_deg, R);
    for (int s = 0; s < n_sweeps; ++s) {
        double ML = m_long(L, R);
        if (!(ML > 0.0)) return -5;
        const double c = cone_c(L->theta);
        int64_t acc = 0;
        for (uint32_t p = 0; p < (uint32_t)(L->N / 2); ++p) {
            uint32_t w[4];
            philox(p, L->sweep, tag_of(1, PURPOSE_SERIAL), 0xFFFFFFFEu, L->key0, L->key1, w);
            const int64_t si = (int64_t)((((uint64_t)w[0] << 32) | w[1]) % (uint64_t)L->N);
            int64_t sj = (int64_t)((((uint64_t)w[2] << 32) | w[3]) % (uint64_t)(L->N - 1));
            if (sj >= si) sj += 1;
            double hi0 = 0, hj0 = 0;
            const double* a = &L->S[3 * si];
            const double* b = &L->S[3 * sj];
            hi0 = R[0] * a[0] + R[1] * a[1] + R[2] * a[2];
            hj0 = R[0] * b[0] + R[1] * b[1] + R[2] * b[2];
            if (pair_move(L, R, ML, c, si, sj, p, tag_of(0, PURPOSE_SERIAL))) {
                acc += 2;
                const double* a2 = &L->S[3 * si];
                const double* b2 = &L->S[3 * sj];
                ML = ML + (R[0] * a2[0] + R[1] * a2[1] + R[2] * a2[2]) + (R[0] * b2[0] + R[1] * b2[1] + R[2] * b2[2]) - hi0 - hj0;
            }
        }
        L->last_accepted = acc;
        if (!measure_flag || L->adapt_in_measure) adapt_theta(L, acc);
        if (measure_flag) measure(L, acc);
        L->sweep += 1;
    }
    return 0;
}

/* --------------------------------------------------------------------- */
/* Crystal structures (Sec. 2): bcc as 2 interleaved simple cubic          */
/* sub-lattices, fcc as 4, hcp as 4 simple tetragonal ones.  Each sub-lattice is split red/black by the      */
/* parity of its cell (x + y + z), and the sub-sets are visited in turn:    */
/* sub-lattice 0 red, 0 black, 1 red, 1 black, ...  J1 couples nearest      */
/* neighbours (other sub-lattices), J2 next-nearest neighbours (the same    */
/* sub-lattice, one cell away along an axis), so every sub-set is free of   */
/* internal bonds.  Cells: L[0] x L[1] x L[2], all periodic, even sizes.     */
/* Site index i = s + nsub (x + L0 (y + L1 z)) for sub-lattice s, cell      */
/* (x, y, z).  Lengths in units of the cubic cell.                          */
/* --------------------------------------------------------------------- */
enum { XTAL_MAX_SUB = 4, XTAL_MAX_NB = 24 };

typedef struct {
    int nsub;
    int L[3];
    int64_t N;
    int nnb[XTAL_MAX_SUB];                  /* neighbour entries per sub-lattice */
    int nb_sub[XTAL_MAX_SUB][XTAL_MAX_NB];  /* neighbour's sub-lattice            */
    int nb_d[XTAL_MAX_SUB][XTAL_MAX_NB][3]; /* its cell offset                    */
    double nb_J[XTAL_MAX_SUB][XTAL_MAX_NB]; /* its coupling (J1 or J2)            */
    double Ku, axis[3], Kc, H[3], T;
    uint32_t key0, key1;
    int theta, adapt_in_measure;
    uint32_t sweep;
    double* S;
    int64_t last_accepted;
    int64_t n_samples;
    double acc_m[3], acc_ml, acc_e, acc_parts[4], acc_tq[3];
} or_xtal;

/* Neighbour table from the basis positions (fractions of the cell, cell
 * lengths ell): entry (s', d) of sub-lattice s is a neighbour when
 * |(b_s' + d - b_s) ell|^2 equals the nearest-neighbour distance^2 (bcc 3/4,
 * fcc 1/2, hcp 1; coupling J1) or, for bcc and fcc with J2 != 0, 1 (the same
 * sub-lattice one cell away; coupling J2), for cell offsets d in
 * {-1, 0, 1}^3.  Entries are ordered by s' ascending, then d_z, d_y, d_x,
 * each from -1 to 1: the field h is accumulated in this order.
 * hcp: the orthohexagonal cell (a, sqrt(3) a, c), c/a = sqrt(8/3), with 4
 * simple tetragonal sub-lattices (0,0,0), (1/2,1/2,0), (1/2,1/6,1/2),
 * (0,2/3,1/2); a = 1. */
OR_EXPORT or_xtal* or_xtal_create(int type, const int cells[3], double J1, double J2, double Ku, const double axis[3],
                                  double Kc, const double H[3], double T, uint64_t seed, int theta0,
                                  int adapt_in_measure) {
    static const double bcc[2][3] = {{0, 0, 0}, {0.5, 0.5, 0.5}};
    static const double fcc[4][3] = {{0, 0, 0}, {0.5, 0.5, 0}, {0.5, 0, 0.5}, {0, 0.5, 0.5}};
    static const double hcp[4][3] = {{0, 0, 0}, {0.5, 0.5, 0}, {0.5, 1.0 / 6.0, 0.5}, {0, 2.0 / 3.0, 0.5}};
    if (type != 1 && type != 2 && type != 3) return NULL;
    or_xtal* X = (or_xtal*)calloc(1, sizeof(or_xtal));
    if (!X) return NULL;
    X->nsub = type == 1 ? 2 : 4;
    const double(*b)[3] = type == 1 ? bcc : (type == 2 ? fcc : hcp);
    const double ell[3] = {1.0, type == 3 ? sqrt(3.0) : 1.0, type == 3 ? sqrt(8.0 / 3.0) : 1.0};
    const double d1 = type == 1 ? 0.75 : (type == 2 ? 0.5 : 1.0);
    const int with_j2 = type != 3 && J2 != 0.0;
    for (int a = 0; a < 3; ++a) X->L[a] = cells[a];
    X->N = (int64_t)X->nsub * cells[0] * cells[1] * cells[2];
    for (int s = 0; s < X->nsub; ++s) {
        int n = 0;
        for (int t = 0; t < X->nsub; ++t)
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const double r[3] = {(b[t][0] + dx - b[s][0]) * ell[0], (b[t][1] + dy - b[s][1]) * ell[1],
                                             (b[t][2] + dz - b[s][2]) * ell[2]};
                        const double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
                        double J;
                        if (fabs(r2 - d1) < 1e-9) J = J1;
                        else if (with_j2 && fabs(r2 - 1.0) < 1e-9) J = J2;
                        else continue;
                        X->nb_sub[s][n] = t;
                        X->nb_d[s][n][0] = dx; X->nb_d[s][n][1] = dy; X->nb_d[s][n][2] = dz;
                        X->nb_J[s][n] = J;
                        ++n;
                    }
        X->nnb[s] = n;
    }
    X->Ku = Ku; X->Kc = Kc; X->T = T;
    const double an = sqrt(axis[0] * axis[0] + axis[1] * axis[1] + axis[2] * axis[2]);
    for (int a = 0; a < 3; ++a) { X->axis[a] = axis[a] / an; X->H[a] = H[a]; }
    X->key0 = (uint32_t)seed;
    X->key1 = (uint32_t)(seed >> 32);
    X->theta = theta0;
    X->adapt_in_measure = adapt_in_measure;
    X->S = (double*)calloc((size_t)X->N * 3, sizeof(double));
    for (int64_t i = 0; i < X->N; ++i) X->S[3 * i + 2] = 1.0;
    return X;
}

OR_EXPORT void or_xtal_destroy(or_xtal* X) {
    if (!X) return;
    free(X->S);
    free(X);
}

OR_EXPORT void or_xtal_set_spins(or_xtal* X, const double* xyz) { memcpy(X->S, xyz, sizeof(double) * 3 * (size_t)X->N); }
OR_EXPORT void or_xtal_get_spins(const or_xtal* X, double* xyz) { memcpy(xyz, X->S, sizeof(double) * 3 * (size_t)X->N); }
OR_EXPORT int or_xtal_theta(const or_xtal* X) { return X->theta; }
OR_EXPORT int64_t or_xtal_last_accepted(const or_xtal* X) { return X->last_accepted; }

static int64_t xtal_site(const or_xtal* X, int s, int x, int y, int z) {
    return (int64_t)s + (int64_t)X->nsub * ((int64_t)x + (int64_t)X->L[0] * ((int64_t)y + (int64_t)X->L[1] * z));
}

/* h_i = sum over the neighbour entries of J_e S_j, in table order. */
static void xtal_field(const or_xtal* X, int64_t i, double h[3]) {
    const int s = (int)(i % X->nsub);
    const int64_t cell = i / X->nsub;
    const int x = (int)(cell % X->L[0]), y = (int)((cell / X->L[0]) % X->L[1]),
              z = (int)(cell / ((int64_t)X->L[0] * X->L[1]));
    h[0] = h[1] = h[2] = 0.0;
    for (int e = 0; e < X->nnb[s]; ++e) {
        const int xx = (x + X->nb_d[s][e][0] + X->L[0]) % X->L[0];
        const int yy = (y + X->nb_d[s][e][1] + X->L[1]) % X->L[1];
        const int zz = (z + X->nb_d[s][e][2] + X->L[2]) % X->L[2];
        const double* t = &X->S[3 * xtal_site(X, X->nb_sub[s][e], xx, yy, zz)];
        const double J = X->nb_J[s][e];
        for (int a = 0; a < 3; ++a) h[a] = h[a] + J * t[a];
    }
}

/* Eq. 2 single-site energy change with the couplings inside h:
 * dE = -(d.h) - K_u((Sn.e)^2 - (S.e)^2) + K_c(q(Sn) - q(S)) - H.d. */
static double xtal_delta_e(const or_xtal* X, int64_t i, const double S[3], const double Sn[3]) {
    double h[3];
    xtal_field(X, i, h);
    const double d0 = Sn[0] - S[0], d1 = Sn[1] - S[1], d2 = Sn[2] - S[2];
    const double e_ex = -(d0 * h[0] + d1 * h[1] + d2 * h[2]);
    const double* e = X->axis;
    const double pn = Sn[0] * e[0] + Sn[1] * e[1] + Sn[2] * e[2];
    const double po = S[0] * e[0] + S[1] * e[1] + S[2] * e[2];
    const double e_u = -(X->Ku * (pn * pn - po * po));
    const double e_c = X->Kc * (cubic_q(Sn) - cubic_q(S));
    const double e_z = -(X->H[0] * d0 + X->H[1] * d1 + X->H[2] * d2);
    return e_ex + e_u + e_c + e_z;
}

OR_EXPORT double or_xtal_delta_e(const or_xtal* X, int64_t i, const double Sn[3]) {
    return xtal_delta_e(X, i, &X->S[3 * i], Sn);
}

/* One sub-set pass: every site of sub-lattice s whose cell parity is
 * colour, in index order; the draws are keyed by the site index. */
static int64_t xtal_pass(or_xtal* X, int s, int colour) {
    const double c = cone_c(X->theta);
    const uint32_t tag = tag_of(colour, PURPOSE_MOVE);
    int64_t accepted = 0;
    for (int z = 0; z < X->L[2]; ++z)
        for (int y = 0; y < X->L[1]; ++y)
            for (int x = 0; x < X->L[0]; ++x) {
                if (((x + y + z) & 1) != colour) continue;
                const int64_t i = xtal_site(X, s, x, y, z);
                double* S = &X->S[3 * i];
                double Sn[3], P;
                if (!cone_trial(S, c, (uint32_t)i, X->sweep, tag, X->key0, X->key1, Sn, &P)) continue;
                if (metropolis(xtal_delta_e(X, i, S, Sn), X->T, P)) {
                    S[0] = Sn[0]; S[1] = Sn[1]; S[2] = Sn[2];
                    ++accepted;
                }
            }
    return accepted;
}

/* Sample (Sec. 3): m = mean spin; exchange energy -1/2 sum_i S_i.h_i (every
 * bond seen from both ends); uniaxial, cubic and Zeeman energies; per spin. */
static void xtal_measure(or_xtal* X) {
    double M[3] = {0, 0, 0}, sh = 0, su = 0, sc = 0, tu[3] = {0, 0, 0}, tc[3] = {0, 0, 0};
    for (int64_t i = 0; i < X->N; ++i) {
        const double* s = &X->S[3 * i];
        double h[3];
        xtal_field(X, i, h);
        for (int a = 0; a < 3; ++a) M[a] += s[a];
        sh += s[0] * h[0] + s[1] * h[1] + s[2] * h[2];
        const double* e = X->axis;
        const double pe = s[0] * e[0] + s[1] * e[1] + s[2] * e[2];
        su += pe * pe;
        sc += cubic_q(s);
        /* torque sums as for the simple cubic sample: (S.e)(S x e), S x c(S) */
        tu[0] += pe * (s[1] * e[2] - s[2] * e[1]);
        tu[1] += pe * (s[2] * e[0] - s[0] * e[2]);
        tu[2] += pe * (s[0] * e[1] - s[1] * e[0]);
        const double x2 = s[0] * s[0], y2 = s[1] * s[1], z2 = s[2] * s[2];
        const double c0 = s[0] * (y2 + z2), c1 = s[1] * (x2 + z2), c2 = s[2] * (x2 + y2);
        tc[0] += s[1] * c2 - s[2] * c1;
        tc[1] += s[2] * c0 - s[0] * c2;
        tc[2] += s[0] * c1 - s[1] * c0;
    }
    const double N = (double)X->N;
    double ml2 = 0;
    for (int a = 0; a < 3; ++a) {
        X->acc_m[a] += M[a] / N;
        ml2 += (M[a] / N) * (M[a] / N);
    }
    const double e_ex = -0.5 * sh / N, e_u = -X->Ku * su / N, e_c = X->Kc * sc / N;
    const double e_z = -(X->H[0] * M[0] + X->H[1] * M[1] + X->H[2] * M[2]) / N;
    X->acc_ml += sqrt(ml2);
    X->acc_e += e_ex + e_u + e_c + e_z;
    X->acc_parts[0] += e_ex; X->acc_parts[1] += e_u; X->acc_parts[2] += e_c; X->acc_parts[3] += e_z;
    X->acc_tq[0] += (2.0 * X->Ku * tu[0] - 2.0 * X->Kc * tc[0] + (M[1] * X->H[2] - M[2] * X->H[1])) / N;
    X->acc_tq[1] += (2.0 * X->Ku * tu[1] - 2.0 * X->Kc * tc[1] + (M[2] * X->H[0] - M[0] * X->H[2])) / N;
    X->acc_tq[2] += (2.0 * X->Ku * tu[2] - 2.0 * X->Kc * tc[2] + (M[0] * X->H[1] - M[1] * X->H[0])) / N;
    X->n_samples += 1;
}

/* One iteration: every sub-set in turn, then the cone adaptation of Table
 * A1 over all N spins and, if measuring, the sample. */
OR_EXPORT void or_xtal_sweep(or_xtal* X, int n_sweeps, int measure_flag) {
    for (int k = 0; k < n_sweeps; ++k) {
        int64_t acc = 0;
        for (int s = 0; s < X->nsub; ++s)
            for (int colour = 0; colour < 2; ++colour) acc += xtal_pass(X, s, colour);
        X->last_accepted = acc;
        if (!measure_flag || X->adapt_in_measure) {
            if (2 * acc > X->N) { if (X->theta < 180) X->theta += 1; }
            else { if (X->theta > 1) X->theta -= 1; }
        }
        if (measure_flag) xtal_measure(X);
        X->sweep += 1;
    }
}

/* n, <m_x>, <m_y>, <m_z>, <|m|>, <E/N>, <E_ex/N>, <E_u/N>, <E_c/N>, <E_Z/N>,
 * <tau_x/N>, <tau_y/N>, <tau_z/N> */
OR_EXPORT void or_xtal_stats(const or_xtal* X, double* out) {
    const double n = X->n_samples ? (double)X->n_samples : 1.0;
    out[0] = (double)X->n_samples;
    for (int a = 0; a < 3; ++a) out[1 + a] = X->acc_m[a] / n;
    out[4] = X->acc_ml / n;
    out[5] = X->acc_e / n;
    for (int a = 0; a < 4; ++a) out[6 + a] = X->acc_parts[a] / n;
    for (int a = 0; a < 3; ++a) out[10 + a] = X->acc_tq[a] / n;
}

/* Constrained Monte Carlo (Table A2) on a crystal: the same iteration as the
 * simple cubic one, with the sub-sets of Sec. 2 in place of the two colours.
 * M_L once per iteration over all N spins; then for every sub-lattice s and
 * colour c in turn, the sub-set's colour indices q in [0, N_c) (cell (x, y,
 * z) of parity c, q = (x >> 1) + (L0/2)(y + L1 z)) are shuffled and taken in
 * pairs (pi(2p), pi(2p+1)).  The sub-set's draws carry s in bits 4.. of the
 * Philox tag (round keys Philox(0, sweep, c | 2<<1 | s<<4, 0); pair draws
 * keyed (p, sweep, c | 1<<1 | s<<4, attempt)), so sub-lattice 0 draws what a
 * simple cubic lattice does.  A sub-set has no internal bonds, so the
 * partners of a pair are never neighbours. */
static int64_t xtal_colour_site(const or_xtal* X, int s, int colour, uint32_t q) {
    const int lh = X->L[0] / 2;
    const int k = (int)(q % (uint32_t)lh);
    const uint32_t row = q / (uint32_t)lh;
    const int y = (int)(row % (uint32_t)X->L[1]);
    const int z = (int)(row / (uint32_t)X->L[1]);
    return xtal_site(X, s, ((y + z + colour) & 1) + 2 * k, y, z);
}

static int xtal_pair_move(or_xtal* X, const double R[9], double ML, double c, int64_t si, int64_t sj,
                          uint32_t pair, uint32_t tag) {
    double* Si = &X->S[3 * si];
    double* Sj = &X->S[3 * sj];
    double hi[3], hj[3];
    rotate(R, Si, hi);
    rotate(R, Sj, hj);
    double hni[3], P;
    if (!cone_trial(hi, c, pair, X->sweep, tag, X->key0, X->key1, hni, &P)) return 0;
    const double ynj = (hj[1] + hi[1]) - hni[1];
    const double znj = (hj[2] + hi[2]) - hni[2];
    const double t = (hj[0] * hj[0] + hj[1] * hj[1] + hj[2] * hj[2]) - ynj * ynj - znj * znj;
    if (!(t > 0.0)) return 0;
    double xnj = sqrt(t);
    if (hj[0] < 0.0) xnj = -xnj;
    const double MLn = ML + hni[0] + xnj - hi[0] - hj[0];
    if (!(MLn > 0.0)) return 0;
    const double hnj[3] = {xnj, ynj, znj};
    double Sni[3], Snj[3];
    rotate_back(R, hni, Sni);
    rotate_back(R, hnj, Snj);
    const double dE = xtal_delta_e(X, si, Si, Sni) + xtal_delta_e(X, sj, Sj, Snj);
    const double ratio = MLn / ML;
    double r = ratio * ratio;
    r = r * (fabs(hj[0]) / fabs(xnj));
    r = r * exp_own(-(dE / X->T));
    if (P < r) {
        Si[0] = Sni[0]; Si[1] = Sni[1]; Si[2] = Sni[2];
        Sj[0] = Snj[0]; Sj[1] = Snj[1]; Sj[2] = Snj[2];
        return 1;
    }
    return 0;
}

OR_EXPORT int or_xtal_constrained_sweep(or_xtal* X, double theta_deg, double phi_deg, int n_sweeps, int measure_flag) {
    double R[9];
    constraint_frame(theta_deg, phi_deg, R);
    const uint32_t nc = (uint32_t)((int64_t)X->L[0] * X->L[1] * X->L[2] / 2);
    for (int k = 0; k < n_sweeps; ++k) {
        int64_t hi = 0, lo = 0;
        for (int64_t i = 0; i < X->N; ++i) {
            const double* s = &X->S[3 * i];
            fixed_add(R[0] * s[0] + R[1] * s[1] + R[2] * s[2], &hi, &lo);
        }
        const double ML = fixed_sum_value(hi, lo);
        if (!(ML > 0.0)) return -5;
        const double c = cone_c(X->theta);
        int64_t acc = 0;
        for (int s = 0; s < X->nsub; ++s)
            for (int colour = 0; colour < 2; ++colour) {
                uint32_t rk[4];
                philox(0u, X->sweep, tag_of(colour, PURPOSE_PERM) | ((uint32_t)s << 4), 0u, X->key0, X->key1, rk);
                const int b = domain_bits(nc);
                const uint32_t tag = tag_of(colour, PURPOSE_PAIR) | ((uint32_t)s << 4);
                for (uint32_t p = 0; p < nc / 2; ++p) {
                    const int64_t si = xtal_colour_site(X, s, colour, permute(2 * p, nc, b, rk));
                    const int64_t sj = xtal_colour_site(X, s, colour, permute(2 * p + 1, nc, b, rk));
                    acc += 2 * xtal_pair_move(X, R, ML, c, si, sj, p, tag);
                }
            }
        X->last_accepted = acc;
        if (!measure_flag || X->adapt_in_measure) {
            if (2 * acc > X->N) { if (X->theta < 180) X->theta += 1; }
            else { if (X->theta > 1) X->theta -= 1; }
        }
        if (measure_flag) xtal_measure(X);
        X->sweep += 1;
    }
    return 0;
}
