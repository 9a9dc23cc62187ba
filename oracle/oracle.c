/*
 * oracle.c -- plain, slow FP64 CPU oracle of the PHAST multicanonical sweep.
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, the package smoke check and the
 * benchmark's CPU-baseline leg; never by the product path.  Independent of the
 * CUDA library: no shared headers, helpers, tables or constants.
 *
 * Every routine is written for a reader holding the paper: loops run in the
 * order of the sums as printed, nothing is blocked, fused or reordered.  Where
 * the paper is silent, the reading taken is stated at the routine.
 * Parity pins (tests/test_oracle_*.py): closed-form energies of hand-built
 * conformations, rigid-motion / periodic-shift / relabelling invariances,
 * E_after - E_before = dE, the trimer's exact density of states, the reduction
 * of Berg's recursion to the paper's naive recursion, and finite-difference
 * exactness on quadratic entropies.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Philox4x32-10, Salmon et al., "Parallel random numbers: as easy as 1, 2, 3", */
/* SC'11.  Round: two 32x32->64 products of counter words 0 and 2 with the     */
/* published multipliers, words recombined with the key, key bumped by the     */
/* published Weyl constants between rounds.  Stands in for the cuRAND vectors  */
/* of Sec. 3.2 (RANDOM.f / cudaRandom.cu).                                     */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Stream layout: key = (seed low, seed high); block b of move t uses counter
 * (t low, t high, b, 0x4D554341).  Blocks: 0 selection, 1 and 2 uniforms,
 * 3 + j Marsaglia attempt j (j < 64). */
#define ORC_STREAM_TAG 0x4D554341u

static void orc_block(uint64_t seed, uint64_t t, uint32_t b, uint32_t out[4]) {
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)t, (uint32_t)(t >> 32), b, ORC_STREAM_TAG};
    orc_philox4x32_10(ctr, key, out);
}

/* Uniform in (0,1) from 52 random bits, exact in FP64: ((a>>6) 2^26 + (b>>6) + 1/2) 2^-52. */
static double orc_u52(uint32_t a, uint32_t b) {
    double n = (double)(a >> 6) * 67108864.0 + (double)(b >> 6);
    return (n + 0.5) * (1.0 / 4503599627370496.0);
}

/* ------------------------------------------------------------------------- */
/* Move geometry (Sec. 3.2, UPDATE_ENGINE: pivots, Galilean updates; plus the  */
/* crankshaft).  sin and cos by their Taylor series (|a| <= 1), coefficients   */
/* (-1)^i/(2i+1)! and (-1)^i/(2i)! as correctly rounded quotients of exact     */
/* factorials; evaluated by Horner in a^2, each step one fused multiply-add    */
/* (C99 fma: a single rounding).  The paper fixes no evaluation order; this    */
/* one, written out below, is the one both implementations follow.           */
/* ------------------------------------------------------------------------- */
static double orc_factorial(int n) {
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f = f * (double)i;   /* exact for n <= 18 */
    return f;
}

static void orc_sincos(double a, double* s, double* c) {
    double x2 = a * a;
    double ps = 0.0, pc = 0.0;
    /* sin a = a * sum_{i=0..8} (-1)^i a^{2i}/(2i+1)! */
    for (int i = 8; i >= 0; --i) {
        double coef = (i % 2 ? -1.0 : 1.0) / orc_factorial(2 * i + 1);
        ps = (i == 8) ? coef : fma(ps, x2, coef);
    }
    /* cos a = sum_{i=0..9} (-1)^i a^{2i}/(2i)! */
    for (int i = 9; i >= 0; --i) {
        double coef = (i % 2 ? -1.0 : 1.0) / orc_factorial(2 * i);
        pc = (i == 9) ? coef : fma(pc, x2, coef);
    }
    *s = a * ps;
    *c = pc;
}

/* Rodrigues' rotation matrix about unit axis k by the angle with sine s and
 * cosine c: R = c I + s [k]x + (1 - c) k k^T, entry (i, j) as
 * fma((1 - c) k_i, k_j, d_ij) with d_ij = c on the diagonal and +-s k_l off it. */
static void orc_rotation(const double k[3], double s, double c, double R[3][3]) {
    double t = 1.0 - c;
    double tk[3] = {t * k[0], t * k[1], t * k[2]};
    double sk[3] = {s * k[0], s * k[1], s * k[2]};
    R[0][0] = fma(tk[0], k[0], c);
    R[0][1] = fma(tk[0], k[1], -sk[2]);
    R[0][2] = fma(tk[0], k[2], sk[1]);
    R[1][0] = fma(tk[1], k[0], sk[2]);
    R[1][1] = fma(tk[1], k[1], c);
    R[1][2] = fma(tk[1], k[2], -sk[0]);
    R[2][0] = fma(tk[2], k[0], -sk[1]);
    R[2][1] = fma(tk[2], k[1], sk[0]);
    R[2][2] = fma(tk[2], k[2], c);
}

/* x' = p + R (x - p): v = x - p, then x'_i = fma(R_i2, v_2, fma(R_i1, v_1, fma(R_i0, v_0, p_i))). */
static void orc_rotate_about(const double R[3][3], const double p[3], const double x[3], double out[3]) {
    double v[3] = {x[0] - p[0], x[1] - p[1], x[2] - p[2]};
    for (int i = 0; i < 3; ++i) out[i] = fma(R[i][2], v[2], fma(R[i][1], v[1], fma(R[i][0], v[0], p[i])));
}

/* Isotropic unit axis by Marsaglia (1972): (v1, v2) uniform in the unit disc,
 * axis = (2 v1 sqrt(1-s), 2 v2 sqrt(1-s), 1 - 2 s), s = v1^2 + v2^2. */
static void orc_axis(uint64_t seed, uint64_t t, double axis[3]) {
    for (uint32_t j = 0; j < 64; ++j) {
        uint32_t r[4];
        orc_block(seed, t, 3u + j, r);
        double v1 = 2.0 * orc_u52(r[0], r[1]) - 1.0;
        double v2 = 2.0 * orc_u52(r[2], r[3]) - 1.0;
        double s = v1 * v1 + v2 * v2;
        if (s < 1.0 && s > 0.0) {
            double q = sqrt(1.0 - s);
            axis[0] = 2.0 * v1 * q;
            axis[1] = 2.0 * v2 * q;
            axis[2] = 1.0 - 2.0 * s;
            return;
        }
    }
    axis[0] = 0.0; axis[1] = 0.0; axis[2] = 1.0;   /* probability (1 - pi/4)^64 */
}

static int orc_chain_offset(const orc_model* m, int c) {
    int o = 0;
    for (int i = 0; i < c; ++i) o += m->chain_len[i];
    return o;
}

static int orc_total(const orc_model* m) { return orc_chain_offset(m, m->n_chains); }

/* Draw move t of a walker.  Readings: the move type is chosen by comparing one
 * uniform with the running sum of the type probabilities; the chain is uniform;
 * pivot and crankshaft act on an interior monomer 1..n-2, a bond-length move
 * on a bond 0..n-2, a spherical cap on any monomer; angles and steps are
 * uniform in [-max, max]; the axis is isotropic. */
void orc_propose(const orc_model* m, const orc_muca* mu, uint64_t seed, uint64_t t,
                 orc_move* mv, double* u_acc) {
    uint32_t b0[4], b1[4], b2[4];
    orc_block(seed, t, 0u, b0);
    orc_block(seed, t, 1u, b1);
    orc_block(seed, t, 2u, b2);
    double u_type = orc_u52(b0[0], b0[1]);
    double u_a = orc_u52(b1[0], b1[1]);
    double u_b = orc_u52(b1[2], b1[3]);
    double u_c = orc_u52(b2[0], b2[1]);
    *u_acc = orc_u52(b2[2], b2[3]);

    int type = -1, last = 0;
    double cum = 0.0;
    for (int i = 0; i < 6; ++i) {
        cum = cum + mu->p[i];
        if (mu->p[i] > 0.0) {
            last = i;
            if (type < 0 && u_type < cum) type = i;
        }
    }
    if (type < 0) type = last;

    memset(mv, 0, sizeof(*mv));
    mv->type = type;
    mv->chain = (int32_t)(((uint64_t)b0[2] * (uint64_t)m->n_chains) >> 32);
    int n = m->chain_len[mv->chain];
    if (type == ORC_PIVOT || type == ORC_CRANK)
        mv->index = 1 + (int32_t)(((uint64_t)b0[3] * (uint64_t)(n - 2)) >> 32);
    if (type == ORC_BOND)   /* a bond 0..n-2 */
        mv->index = (int32_t)(((uint64_t)b0[3] * (uint64_t)(n - 1)) >> 32);
    if (type == ORC_CAP)    /* any monomer */
        mv->index = (int32_t)(((uint64_t)b0[3] * (uint64_t)n) >> 32);
    if (type == ORC_TRANS) {
        mv->disp[0] = (2.0 * u_a - 1.0) * mu->amax[ORC_TRANS];
        mv->disp[1] = (2.0 * u_b - 1.0) * mu->amax[ORC_TRANS];
        mv->disp[2] = (2.0 * u_c - 1.0) * mu->amax[ORC_TRANS];
    } else {
        mv->angle = (2.0 * u_a - 1.0) * mu->amax[type];   /* the length step for a bond move */
        if (type == ORC_PIVOT || type == ORC_ROT || type == ORC_CAP) orc_axis(seed, t, mv->axis);
    }
}

/* Hastings factor of a move: 1, except for a bond-length move, whose map
 * b -> b (r + delta) / r of the stretched bond vector (length r, every other
 * bond vector of the moved side unchanged) has Jacobian determinant
 * ((r + delta) / r)^2 in Cartesian coordinates.  Reading: the density of
 * states of Eq. 4 counts configuration-space volume in the bead coordinates,
 * in which pivot, crankshaft, rigid and cap moves are symmetric proposals;
 * a uniform dilation step delta is not, so the acceptance carries this
 * factor (Metropolis-Hastings).  r is computed as in orc_apply_move. */
double orc_move_jacobian(const orc_model* m, const double* xyz, const orc_move* mv) {
    if (mv->type != ORC_BOND) return 1.0;
    int o = orc_chain_offset(m, mv->chain), l = mv->index;
    double b[3];
    for (int d = 0; d < 3; ++d) b[d] = xyz[3 * (o + l + 1) + d] - xyz[3 * (o + l) + d];
    double r = sqrt((b[0] * b[0] + b[1] * b[1]) + b[2] * b[2]);
    double q = (r + mv->angle) / r;
    return q * q;
}

/* Centroid of monomers o..o+n-1 (the rotation centre of a rigid rotation).
 * Reading: the paper names the centre of mass but not the floating-point order
 * of its sum; it is fixed here so that every implementation reproduces the
 * coordinates bit for bit: 32 strided partial sums s_l = sum over j = l, l+32,
 * l+64, ... (increasing j) of x_{o+j}, combined by halving, s_l += s_{l+w} for
 * w = 16, 8, 4, 2, 1 and l < w, then s_0 / n. */
static void orc_centroid(const double* xyz, int o, int n, double center[3]) {
    for (int d = 0; d < 3; ++d) {
        double part[32];
        for (int l = 0; l < 32; ++l) {
            part[l] = 0.0;
            for (int j = l; j < n; j += 32) part[l] = part[l] + xyz[3 * (o + j) + d];
        }
        for (int w = 16; w >= 1; w /= 2)
            for (int l = 0; l < w; ++l) part[l] = part[l] + part[l + w];
        center[d] = part[0] / (double)n;
    }
}

/* Apply a move.  Pivot (Sec. 3.2 "pivotings"): rotate the shorter side of the
 * chain about an axis through the pivot monomer k; on a tie the tail j > k.
 * Translation / rotation (Sec. 3.2 "Galilean-group updates"): the whole chain,
 * rotation about its centroid (see orc_centroid for the order of the sum).
 * Crankshaft: monomer i about the axis through monomers i-1 and i+1. */
int orc_apply_move(const orc_model* m, const orc_move* mv, const double* xyz, double* xyz_new) {
    int N = orc_total(m);
    memcpy(xyz_new, xyz, sizeof(double) * 3 * (size_t)N);
    int o = orc_chain_offset(m, mv->chain);
    int n = m->chain_len[mv->chain];
    int lo, hi;
    double center[3], axis[3], R[3][3], s, c;

    if (mv->type == ORC_TRANS) {
        for (int j = o; j < o + n; ++j)
            for (int d = 0; d < 3; ++d) xyz_new[3 * j + d] = xyz[3 * j + d] + mv->disp[d];
        return n;
    }
    if (mv->type == ORC_BOND) {
        /* bond l between monomers l and l+1 changes length by delta: the shorter
         * side (head 0..l or tail l+1..n-1; on a tie the tail) slides along the
         * unit bond vector u = (x_{l+1} - x_l) / |x_{l+1} - x_l|, by +delta u (tail)
         * or -delta u (head). */
        int l = mv->index;
        double b[3], u[3], step[3];
        for (int d = 0; d < 3; ++d) b[d] = xyz[3 * (o + l + 1) + d] - xyz[3 * (o + l) + d];
        double len = sqrt((b[0] * b[0] + b[1] * b[1]) + b[2] * b[2]);
        if (!(len > 1e-12)) return 0;
        if (!(len + mv->angle > 0.0)) return 0;   /* the bond would pass through zero length */
        int head = (l + 1) < (n - 1 - l);
        double delta = head ? -mv->angle : mv->angle;
        for (int d = 0; d < 3; ++d) { u[d] = b[d] / len; step[d] = delta * u[d]; }
        if (head) { lo = o; hi = o + l; }
        else { lo = o + l + 1; hi = o + n - 1; }
        for (int j = lo; j <= hi; ++j)
            for (int d = 0; d < 3; ++d) xyz_new[3 * j + d] = xyz[3 * j + d] + step[d];
        return hi - lo + 1;
    }
    if (mv->type == ORC_PIVOT) {
        int k = mv->index;
        if (k < n - 1 - k) { lo = o; hi = o + k - 1; }
        else { lo = o + k + 1; hi = o + n - 1; }
        for (int d = 0; d < 3; ++d) { center[d] = xyz[3 * (o + k) + d]; axis[d] = mv->axis[d]; }
    } else if (mv->type == ORC_ROT) {
        lo = o; hi = o + n - 1;
        orc_centroid(xyz, o, n, center);
        for (int d = 0; d < 3; ++d) axis[d] = mv->axis[d];
    } else if (mv->type == ORC_CAP) {
        /* spherical cap: monomer i rotated about an isotropic axis through its
         * bonded neighbour i-1 (monomer 1 for i = 0), keeping that bond */
        int i = o + mv->index;
        int c = mv->index > 0 ? i - 1 : i + 1;
        for (int d = 0; d < 3; ++d) { center[d] = xyz[3 * c + d]; axis[d] = mv->axis[d]; }
        lo = hi = i;
    } else {   /* crankshaft */
        int i = o + mv->index;
        double e[3];
        for (int d = 0; d < 3; ++d) e[d] = xyz[3 * (i + 1) + d] - xyz[3 * (i - 1) + d];
        double len = sqrt((e[0] * e[0] + e[1] * e[1]) + e[2] * e[2]);
        if (!(len > 1e-12)) return 0;
        for (int d = 0; d < 3; ++d) { axis[d] = e[d] / len; center[d] = xyz[3 * (i - 1) + d]; }
        lo = hi = i;
    }
    orc_sincos(mv->angle, &s, &c);
    orc_rotation(axis, s, c, R);
    for (int j = lo; j <= hi; ++j) orc_rotate_about(R, center, &xyz[3 * j], &xyz_new[3 * j]);
    return hi - lo + 1;
}

/* ------------------------------------------------------------------------- */
/* Energy, Eq. 2 (kappa_F = 0) per chain and the inter-chain term of Eq. 3.    */
/* ------------------------------------------------------------------------- */

/* Lennard-Jones term of Eq. 2/3 without its coupling: r^-12 - C r^-6. */
static double orc_lj(double r2, double C) {
    double r6 = r2 * r2 * r2;
    return 1.0 / (r6 * r6) - C / r6;
}

/* Squared distance; between different chains of a periodic system the minimum
 * image d - L rint(d / L) per component (reading: the paper's spherical
 * container is replaced by a periodic cube; chains are never wrapped, so
 * intra-chain distances are direct). */
static double orc_dist2(const orc_model* m, const double* a, const double* b, int periodic) {
    double r2 = 0.0;
    for (int d = 0; d < 3; ++d) {
        double x = a[d] - b[d];
        if (periodic && m->box_L > 0.0) x = x - m->box_L * rint(x / m->box_L);
        r2 = r2 + x * x;
    }
    return r2;
}

/* Bending (kappa_C sum_k (1 - cos theta_k), theta_k the angle between bonds
 * k-1 and k, so a straight chain costs 0) and torsion (-kappa sum cos tau_j,
 * tau_j the dihedral of monomers j..j+3 from the normals b_j x b_{j+1} and
 * b_{j+1} x b_{j+2}; a dihedral whose normals have |n1|^2 |n2|^2 < 1e-20
 * contributes 0) of one chain starting at monomer o with n monomers. */
static void orc_chain_local(const orc_model* m, const double* xyz, int o, int n,
                            double* e_bend, double* e_tors) {
    double bend = 0.0, tors = 0.0;
    for (int k = 1; k <= n - 2; ++k) {
        const double* x0 = &xyz[3 * (o + k - 1)];
        const double* x1 = &xyz[3 * (o + k)];
        const double* x2 = &xyz[3 * (o + k + 1)];
        double a[3], b[3];
        for (int d = 0; d < 3; ++d) { a[d] = x1[d] - x0[d]; b[d] = x2[d] - x1[d]; }
        double ab = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
        double aa = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
        double bb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
        double cos_theta = ab / (sqrt(aa) * sqrt(bb));
        bend = bend + (1.0 - cos_theta);
    }
    for (int j = 0; j <= n - 4; ++j) {
        double b[3][3];
        for (int q = 0; q < 3; ++q)
            for (int d = 0; d < 3; ++d)
                b[q][d] = xyz[3 * (o + j + q + 1) + d] - xyz[3 * (o + j + q) + d];
        double n1[3] = {b[0][1] * b[1][2] - b[0][2] * b[1][1],
                        b[0][2] * b[1][0] - b[0][0] * b[1][2],
                        b[0][0] * b[1][1] - b[0][1] * b[1][0]};
        double n2[3] = {b[1][1] * b[2][2] - b[1][2] * b[2][1],
                        b[1][2] * b[2][0] - b[1][0] * b[2][2],
                        b[1][0] * b[2][1] - b[1][1] * b[2][0]};
        double n12 = n1[0] * n2[0] + n1[1] * n2[1] + n1[2] * n2[2];
        double n11 = n1[0] * n1[0] + n1[1] * n1[1] + n1[2] * n1[2];
        double n22 = n2[0] * n2[0] + n2[1] * n2[1] + n2[2] * n2[2];
        if (n11 * n22 < 1e-20) continue;
        tors = tors + n12 / (sqrt(n11) * sqrt(n22));
    }
    *e_bend = m->k_bend * bend;
    *e_tors = -m->k_tors * tors;
}

/* FENE bond term of Eq. 2, as printed, for the chain at o with n monomers:
 * k_fene R^2 sum_l C_F(s_l, s_{l+1}) ln(1 - ((r_{l,l+1} - r0) / R)^2); +inf for a
 * bond with |r - r0| >= R (outside the potential's range); 0 in the AB limit
 * k_fene = 0 of Sec. 4, where bonds keep their length. */
static double orc_chain_fene(const orc_model* m, const double* xyz, int o, int n) {
    if (m->k_fene == 0.0) return 0.0;
    double sum = 0.0;
    for (int l = o; l < o + n - 1; ++l) {
        double d[3];
        for (int q = 0; q < 3; ++q) d[q] = xyz[3 * (l + 1) + q] - xyz[3 * l + q];
        double r = sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
        double x = (r - m->fene_r0) / m->fene_R;
        double x2 = x * x;
        if (!(x2 < 1.0)) return INFINITY;
        sum = sum + m->C_F[2 * m->seq[l] + m->seq[l + 1]] * log(1.0 - x2);
    }
    return (m->k_fene * (m->fene_R * m->fene_R)) * sum;
}

/* Steric spherical container (Sec. 3.2, box_size.h), a hard wall about the
 * origin: 1 if every monomer lo..hi lies at (x^2 + y^2) + z^2 <= R^2 (or there
 * is no container), else 0. */
static int orc_inside(const orc_model* m, const double* xyz, int lo, int hi) {
    if (!(m->sphere_R > 0.0)) return 1;
    double R2 = m->sphere_R * m->sphere_R;
    for (int j = lo; j <= hi; ++j) {
        const double* x = &xyz[3 * j];
        if ((x[0] * x[0] + x[1] * x[1]) + x[2] * x[2] > R2) return 0;
    }
    return 1;
}

static int orc_chain_of(const orc_model* m, int j) {
    int o = 0;
    for (int c = 0; c < m->n_chains; ++c) {
        if (j < o + m->chain_len[c]) return c;
        o += m->chain_len[c];
    }
    return -1;
}

double orc_energy(const orc_model* m, const double* xyz, double* terms) {
    int N = orc_total(m);
    double bend = 0.0, tors = 0.0, intra = 0.0, inter = 0.0, fene = 0.0;
    for (int c = 0, o = 0; c < m->n_chains; o += m->chain_len[c], ++c) {
        double eb, et;
        orc_chain_local(m, xyz, o, m->chain_len[c], &eb, &et);
        bend = bend + eb;
        tors = tors + et;
        fene = fene + orc_chain_fene(m, xyz, o, m->chain_len[c]);
    }
    /* Eq. 2: pairs i < j - 1 of one chain.  Eq. 3: all pairs of different chains. */
    for (int i = 0; i < N; ++i) {
        int ci = orc_chain_of(m, i);
        for (int j = i + 1; j < N; ++j) {
            int cj = orc_chain_of(m, j);
            double C = m->C[2 * m->seq[i] + m->seq[j]];
            if (ci == cj) {
                if (j < i + 2) continue;
                intra = intra + orc_lj(orc_dist2(m, &xyz[3 * i], &xyz[3 * j], 0), C);
            } else {
                inter = inter + orc_lj(orc_dist2(m, &xyz[3 * i], &xyz[3 * j], 1), C);
            }
        }
    }
    intra = m->k_lj_intra * intra;
    inter = m->k_lj_inter * inter;
    if (terms) { terms[0] = bend; terms[1] = tors; terms[2] = intra; terms[3] = inter; terms[4] = fene; }
    if (!orc_inside(m, xyz, 0, N - 1)) return INFINITY;
    double E = ((bend + tors) + intra) + inter;
    return m->k_fene == 0.0 ? E : E + fene;
}

/* Moved monomer range of a move, [lo, hi] (global indices). */
static void orc_moved_range(const orc_model* m, const orc_move* mv, int* lo, int* hi) {
    int o = orc_chain_offset(m, mv->chain);
    int n = m->chain_len[mv->chain];
    if (mv->type == ORC_TRANS || mv->type == ORC_ROT) { *lo = o; *hi = o + n - 1; return; }
    if (mv->type == ORC_CRANK || mv->type == ORC_CAP) { *lo = *hi = o + mv->index; return; }
    if (mv->type == ORC_BOND) {
        int l = mv->index;
        if ((l + 1) < (n - 1 - l)) { *lo = o; *hi = o + l; }
        else { *lo = o + l + 1; *hi = o + n - 1; }
        return;
    }
    int k = mv->index;
    if (k < n - 1 - k) { *lo = o; *hi = o + k - 1; }
    else { *lo = o + k + 1; *hi = o + n - 1; }
}

/* dE of a move: the bending and torsion of the moved chain before and after,
 * plus every Lennard-Jones pair (moved monomer, unmoved monomer) before and
 * after.  Pairs of two moved monomers keep their distance (the moved set moves
 * rigidly) and are left out.  Returns NaN for a degenerate move. */
double orc_delta_energy(const orc_model* m, const double* xyz, const orc_move* mv, double* xyz_new) {
    int N = orc_total(m);
    double* xn = xyz_new ? xyz_new : (double*)malloc(sizeof(double) * 3 * (size_t)N);
    int moved = orc_apply_move(m, mv, xyz, xn);
    double dE;
    int lo, hi;
    orc_moved_range(m, mv, &lo, &hi);
    if (moved == 0) {
        dE = NAN;
    } else if (!orc_inside(m, xn, lo, hi)) {
        dE = INFINITY;   /* the hard wall of the container */
    } else {
        int o = orc_chain_offset(m, mv->chain);
        int n = m->chain_len[mv->chain];
        double eb0, et0, eb1, et1;
        orc_chain_local(m, xyz, o, n, &eb0, &et0);
        orc_chain_local(m, xn, o, n, &eb1, &et1);
        dE = (eb1 + et1) - (eb0 + et0);
        if (m->k_fene != 0.0) dE = dE + (orc_chain_fene(m, xn, o, n) - orc_chain_fene(m, xyz, o, n));
        for (int i = lo; i <= hi; ++i) {
            int ci = orc_chain_of(m, i);
            for (int j = 0; j < N; ++j) {
                if (j >= lo && j <= hi) continue;
                int cj = orc_chain_of(m, j);
                double C = m->C[2 * m->seq[i] + m->seq[j]];
                double e_old, e_new;
                if (ci == cj) {
                    if (abs(i - j) < 2) continue;
                    e_old = m->k_lj_intra * orc_lj(orc_dist2(m, &xyz[3 * i], &xyz[3 * j], 0), C);
                    e_new = m->k_lj_intra * orc_lj(orc_dist2(m, &xn[3 * i], &xn[3 * j], 0), C);
                } else {
                    e_old = m->k_lj_inter * orc_lj(orc_dist2(m, &xyz[3 * i], &xyz[3 * j], 1), C);
                    e_new = m->k_lj_inter * orc_lj(orc_dist2(m, &xn[3 * i], &xn[3 * j], 1), C);
                }
                dE = dE + (e_new - e_old);
            }
        }
    }
    if (!xyz_new) free(xn);
    return dE;
}

/* Magnitude of the terms a move changes: sum over the changed Lennard-Jones
 * pairs of |term before| + |term after|, plus the bending and torsion energy of
 * the moved chain before and after in absolute value.  Not part of the method:
 * the scale against which a reduced-precision dE is judged. */
double orc_delta_scale(const orc_model* m, const double* xyz, const orc_move* mv) {
    int N = orc_total(m);
    double* xn = (double*)malloc(sizeof(double) * 3 * (size_t)N);
    double scale = 0.0;
    if (orc_apply_move(m, mv, xyz, xn) > 0) {
        int o = orc_chain_offset(m, mv->chain), n = m->chain_len[mv->chain];
        double eb0, et0, eb1, et1;
        orc_chain_local(m, xyz, o, n, &eb0, &et0);
        orc_chain_local(m, xn, o, n, &eb1, &et1);
        scale = fabs(eb0) + fabs(et0) + fabs(eb1) + fabs(et1);
        if (m->k_fene != 0.0) scale += fabs(orc_chain_fene(m, xyz, o, n)) + fabs(orc_chain_fene(m, xn, o, n));
        int lo, hi;
        orc_moved_range(m, mv, &lo, &hi);
        for (int i = lo; i <= hi; ++i) {
            int ci = orc_chain_of(m, i);
            for (int j = 0; j < N; ++j) {
                if (j >= lo && j <= hi) continue;
                int cj = orc_chain_of(m, j);
                if (ci == cj && abs(i - j) < 2) continue;
                double C = m->C[2 * m->seq[i] + m->seq[j]];
                double k = ci == cj ? m->k_lj_intra : m->k_lj_inter;
                scale += fabs(k * orc_lj(orc_dist2(m, &xyz[3 * i], &xyz[3 * j], ci != cj), C));
                scale += fabs(k * orc_lj(orc_dist2(m, &xn[3 * i], &xn[3 * j], ci != cj), C));
            }
        }
    }
    free(xn);
    return scale;
}

/* Pair evaluations of a move: 2 (before and after) for every Lennard-Jones pair
 * (moved i, unmoved j) whose distance the move can change -- the pivot monomer
 * keeps its distance to the rotated side and is not counted. */
int64_t orc_pair_evals(const orc_model* m, const orc_move* mv) {
    int N = orc_total(m);
    int lo, hi;
    orc_moved_range(m, mv, &lo, &hi);
    int pivot = (mv->type == ORC_PIVOT) ? orc_chain_offset(m, mv->chain) + mv->index : -1;
    int64_t count = 0;
    for (int i = lo; i <= hi; ++i) {
        int ci = orc_chain_of(m, i);
        for (int j = 0; j < N; ++j) {
            if ((j >= lo && j <= hi) || j == pivot) continue;
            if (orc_chain_of(m, j) == ci && abs(i - j) < 2) continue;
            count += 2;
        }
    }
    return count;
}

/* Energy bin: floor((E - e_min) / width) on [e_min, e_min + K width); -1 outside
 * or for a non-finite E.  (Reading of Sec. 2.2: E_k in [E_0, E_max], half-open bins.) */
int32_t orc_bin(const orc_muca* mu, double E) {
    if (!isfinite(E)) return -1;
    double q = (E - mu->e_min) / mu->bin_width;
    if (!(q >= 0.0 && q < (double)mu->n_bins)) return -1;
    return (int32_t)floor(q);
}

/* ------------------------------------------------------------------------- */
/* The multicanonical Metropolis sweep of one walker (Sec. 2.2 and Sec. 3.2,   */
/* MONTE_CARLO.f): accept with min(1, J W(E')/W(E)), W = exp(lnW[bin]) piecewise*/
/* constant per bin (Eq. 8 tabulated), and count the current bin into the      */
/* histogram after every attempt, accepted or not.  Readings: one sweep is      */
/* N_tot attempts; a proposal out of the bin range or with non-finite dE is     */
/* rejected; every recompute_every sweeps the running energy is replaced by a   */
/* full FP64 energy and the drift recorded; the bin follows, the nearest edge  */
/* bin for an energy just past a range edge.                                    */
/* ------------------------------------------------------------------------- */
int orc_sweep_walker(const orc_model* m, const orc_muca* mu, const double* lnW,
                     uint64_t seed, int64_t n_moves,
                     double* xyz, double* E, int32_t* bin, uint64_t* t,
                     uint64_t* hist, const int8_t* force, orc_record* rec, double* stats) {
    int N = orc_total(m);
    const int32_t b0 = orc_bin(mu, *E);
    const int edge = (b0 < 0) && ((*E < mu->e_min && *bin == 0) || (*E >= mu->e_min && *bin == mu->n_bins - 1));
    if (*bin < 0 || *bin >= mu->n_bins || (b0 != *bin && !edge)) return -1;
    double* xn = (double*)malloc(sizeof(double) * 3 * (size_t)N);
    uint64_t attempts[6] = {0, 0, 0, 0, 0, 0}, accepts[6] = {0, 0, 0, 0, 0, 0};
    int64_t pair_evals = 0, n_recompute = 0, mismatches = 0;
    double drift_max = 0.0;
    uint64_t period = (uint64_t)N * (uint64_t)(mu->recompute_every > 0 ? mu->recompute_every : 0);

    for (int64_t it = 0; it < n_moves; ++it) {
        orc_move mv;
        double u_acc;
        orc_propose(m, mu, seed, *t, &mv, &u_acc);
        double dE = orc_delta_energy(m, xyz, &mv, xn);
        double E_new = *E + dE;
        int32_t b_new = orc_bin(mu, E_new);
        int own = 0;
        if (b_new >= 0) {
            /* min(1, J W(E') / W(E)); J = 1 except for bond-length moves */
            double dlnW = lnW[b_new] - lnW[*bin];
            double J = orc_move_jacobian(m, xyz, &mv);
            own = (dlnW >= 0.0 && J >= 1.0) || (u_acc < J * exp(dlnW));
        }
        int acc = own;
        if (force && force[it] >= 0) {
            acc = force[it];
            if (acc != own) mismatches++;
            if (acc && b_new < 0)   /* imposed acceptance at a range-edge near-tie */
                b_new = (E_new < mu->e_min) ? 0 : mu->n_bins - 1;
        }
        attempts[mv.type]++;
        pair_evals += orc_pair_evals(m, &mv);
        if (acc) {
            memcpy(xyz, xn, sizeof(double) * 3 * (size_t)N);
            *E = E_new;
            *bin = b_new;
            accepts[mv.type]++;
        }
        hist[*bin] += 1;
        if (rec) {
            rec[it].dE = dE;
            rec[it].E_after = *E;
            rec[it].bin_after = *bin;
            rec[it].accepted = acc;
        }
        *t += 1;
        if (period > 0 && (*t % period) == 0) {
            double Ef = orc_energy(m, xyz, NULL);
            double drift = fabs(*E - Ef);
            if (drift > drift_max) drift_max = drift;
            if (isfinite(Ef)) {
                int32_t bf = orc_bin(mu, Ef);
                *E = Ef;
                *bin = bf >= 0 ? bf : (Ef < mu->e_min ? 0 : mu->n_bins - 1);
            }
            n_recompute++;
        }
    }
    free(xn);
    if (stats) {
        for (int i = 0; i < 6; ++i) { stats[i] = (double)attempts[i]; stats[6 + i] = (double)accepts[i]; }
        stats[12] = (double)pair_evals;
        stats[13] = (double)n_recompute;
        stats[14] = drift_max;
        stats[15] = (double)mismatches;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Berg's multicanonical recursion with accumulated error weights (Sec. 2.2,    */
/* cited there to Berg).  With beta_k = (lnW_k - lnW_{k+1}) / eps (so that       */
/* S = -lnW and beta = dS/dE):                                                   */
/*   g0_k  = H_k H_{k+1} / (H_k + H_{k+1})   (0 unless both bins are visited)    */
/*   ghat  = g0_k / (g_acc_k + g0_k),  g_acc_k += g0_k                           */
/*   beta_k += ghat (ln H_{k+1} - ln H_k) / eps                                  */
/* and lnW re-integrated from lnW_0 = 0.  With g_acc = 0 this is the naive       */
/* recursion W^{n+1} = W^n / H^n on every pair of visited bins.                  */
/* Flatness (Sec. 4.1): c_Var = sigma_H / mu_H and the largest |H - mu_H| / mu_H */
/* over visited bins.                                                            */
/* ------------------------------------------------------------------------- */
void orc_berg_update(int32_t K, double bin_width, const double* H, double* lnW,
                     double* g_acc, double* flat_out) {
    (void)bin_width;   /* beta_k eps is carried as a difference; eps cancels */
    double* d = (double*)malloc(sizeof(double) * (size_t)(K > 1 ? K - 1 : 1));
    for (int k = 0; k + 1 < K; ++k) {
        double g0 = 0.0;
        if (H[k] > 0.0 && H[k + 1] > 0.0) g0 = H[k] * H[k + 1] / (H[k] + H[k + 1]);
        double den = g_acc[k] + g0;
        double ghat = den > 0.0 ? g0 / den : 0.0;
        g_acc[k] = den;
        d[k] = lnW[k] - lnW[k + 1];
        if (g0 > 0.0) d[k] = d[k] + ghat * (log(H[k + 1]) - log(H[k]));
    }
    if (K > 0) lnW[0] = 0.0;
    for (int k = 0; k + 1 < K; ++k) lnW[k + 1] = lnW[k] - d[k];
    free(d);
    if (flat_out) {
        double n = 0.0, sum = 0.0;
        for (int k = 0; k < K; ++k) if (H[k] > 0.0) { n = n + 1.0; sum = sum + H[k]; }
        double mean = n > 0.0 ? sum / n : 0.0;
        double var = 0.0, maxdev = 0.0;
        for (int k = 0; k < K; ++k) {
            if (!(H[k] > 0.0)) continue;
            var = var + (H[k] - mean) * (H[k] - mean);
            double dev = fabs(H[k] - mean) / mean;
            if (dev > maxdev) maxdev = dev;
        }
        var = n > 0.0 ? var / n : 0.0;
        flat_out[0] = n;
        flat_out[1] = mean;
        flat_out[2] = mean > 0.0 ? sqrt(var) / mean : 0.0;
        flat_out[3] = maxdev;
    }
}

/* ------------------------------------------------------------------------- */
/* Microcanonical analysis (Sec. 2.2 Eq. 4-6, Sec. 3.3 ANALYST).               */
/* S_k = -lnW_k + ln H_k on visited bins (the multicanonical reweighting; with */
/* H omitted S = -lnW, i.e. S_muca of Eq. 8), shifted so max S = 0.            */
/* beta_k = (S_{k+h} - S_{k-h}) / (2 h eps)            (Eq. 5, central)        */
/* S''_k  = (S_{k+h} - 2 S_k + S_{k-h}) / (h eps)^2                            */
/* C_V,k  = -beta_k^2 / S''_k                          (Eq. 6)                 */
/* Canonical: p_k(T) ~ exp(S_k - E_k / T), E_k the bin centre; <E>_T and       */
/* c_V(T) = var_T(E) / (N T^2); peak by a parabola through the grid maximum     */
/* and its neighbours.                                                          */
/* ------------------------------------------------------------------------- */
void orc_micro_analysis(int32_t K, double e_min, double bin_width, const double* lnW,
                        const double* H, int32_t h, int32_t n_monomers,
                        int32_t n_T, const double* T,
                        double* S, double* beta, double* CV,
                        double* E_T, double* cV_T, double* peak) {
    double smax = -INFINITY;
    for (int k = 0; k < K; ++k) {
        if (H && !(H[k] > 0.0)) { S[k] = NAN; continue; }
        S[k] = -lnW[k] + (H ? log(H[k]) : 0.0);
        if (S[k] > smax) smax = S[k];
    }
    for (int k = 0; k < K; ++k) if (!isnan(S[k])) S[k] = S[k] - smax;

    double he = (double)h * bin_width;
    for (int k = 0; k < K; ++k) {
        beta[k] = NAN;
        CV[k] = NAN;
        if (k - h < 0 || k + h >= K) continue;
        if (isnan(S[k - h]) || isnan(S[k + h])) continue;
        beta[k] = (S[k + h] - S[k - h]) / (2.0 * he);
        if (isnan(S[k])) continue;
        double s2 = (S[k + h] - 2.0 * S[k] + S[k - h]) / (he * he);
        CV[k] = -(beta[k] * beta[k]) / s2;
    }

    for (int i = 0; i < n_T; ++i) {
        double lmax = -INFINITY;
        for (int k = 0; k < K; ++k) {
            if (isnan(S[k])) continue;
            double Ek = e_min + ((double)k + 0.5) * bin_width;
            double lp = S[k] - Ek / T[i];
            if (lp > lmax) lmax = lp;
        }
        double Z = 0.0, sE = 0.0;
        for (int k = 0; k < K; ++k) {
            if (isnan(S[k])) continue;
            double Ek = e_min + ((double)k + 0.5) * bin_width;
            double w = exp(S[k] - Ek / T[i] - lmax);
            Z = Z + w;
            sE = sE + w * Ek;
        }
        double mean = sE / Z, var = 0.0;
        for (int k = 0; k < K; ++k) {
            if (isnan(S[k])) continue;
            double Ek = e_min + ((double)k + 0.5) * bin_width;
            double w = exp(S[k] - Ek / T[i] - lmax);
            var = var + w * (Ek - mean) * (Ek - mean);
        }
        var = var / Z;
        E_T[i] = mean;
        cV_T[i] = var / ((double)n_monomers * T[i] * T[i]);
    }

    if (n_T > 0) {
        int im = 0;
        for (int i = 1; i < n_T; ++i) if (cV_T[i] > cV_T[im]) im = i;
        peak[0] = T[im];
        peak[1] = cV_T[im];
        if (im > 0 && im < n_T - 1) {
            double x0 = T[im - 1], x1 = T[im], x2 = T[im + 1];
            double y0 = cV_T[im - 1], y1 = cV_T[im], y2 = cV_T[im + 1];
            double num = (x1 - x0) * (x1 - x0) * (y1 - y2) - (x1 - x2) * (x1 - x2) * (y1 - y0);
            double den = (x1 - x0) * (y1 - y2) - (x1 - x2) * (y1 - y0);
            if (den != 0.0) {
                double xs = x1 - 0.5 * num / den;
                /* value of the interpolating parabola at xs (Lagrange form) */
                double ys = y0 * (xs - x1) * (xs - x2) / ((x0 - x1) * (x0 - x2))
                          + y1 * (xs - x0) * (xs - x2) / ((x1 - x0) * (x1 - x2))
                          + y2 * (xs - x0) * (xs - x1) / ((x2 - x0) * (x2 - x1));
                peak[0] = xs;
                peak[1] = ys;
            }
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Jackknife error over data blocks (Sec. 4.1: error bars from blocks of the    */
/* data; here the blocks are groups of walkers).  The caller computes each      */
/* estimate once more with block b left out (replicate v_b, b < n); the error   */
/* of the estimate is sqrt((n - 1)/n * sum_b (v_b - vbar)^2), vbar the mean of  */
/* the replicates.  rep is [n][m] (m observables per replicate), err [m].  NaN  */
/* for n < 2; a NaN replicate makes that observable's error NaN.                */
/* ------------------------------------------------------------------------- */
void orc_jackknife(int32_t n, int32_t m, const double* rep, double* err) {
    for (int q = 0; q < m; ++q) {
        if (n < 2) {
            err[q] = NAN;
            continue;
        }
        double mean = 0.0;
        for (int b = 0; b < n; ++b) mean = mean + rep[(size_t)b * (size_t)m + (size_t)q];
        mean = mean / (double)n;
        double ss = 0.0;
        for (int b = 0; b < n; ++b) {
            const double d = rep[(size_t)b * (size_t)m + (size_t)q] - mean;
            ss = ss + d * d;
        }
        err[q] = sqrt((double)(n - 1) / (double)n * ss);
    }
}

/* ------------------------------------------------------------------------- */
/* Error bars by binning over iterations (Sec. 4.1, ANALYST: data blocks of     */
/* dN iterations of the range [N_S, N_E], the binning method).  Iteration i     */
/* (row i of lnW and, if given, of H) is analysed alone as orc_micro_analysis   */
/* does; each observable is averaged over n_b = n_it / block consecutive        */
/* blocks of `block` iterations (a remainder at the end is left out).  The      */
/* value is the mean of the block means B_b, the error                          */
/* sqrt(sum_b (B_b - mean)^2 / (n_b (n_b - 1))), NaN for n_b < 2.  A bin left   */
/* unvisited by any iteration of the range stays NaN.                           */
/* ------------------------------------------------------------------------- */
static void orc_binning(const double* v, size_t stride, int n_it, int block, double* val, double* err) {
    int n_b = n_it / block;
    double* bm = (double*)malloc(sizeof(double) * (size_t)(n_b > 0 ? n_b : 1));
    double mean = 0.0;
    for (int b = 0; b < n_b; ++b) {
        double s = 0.0;
        for (int i = b * block; i < (b + 1) * block; ++i) s = s + v[(size_t)i * stride];
        bm[b] = s / (double)block;
        mean = mean + bm[b];
    }
    mean = mean / (double)n_b;
    *val = mean;
    if (n_b < 2) {
        *err = NAN;
    } else {
        double q = 0.0;
        for (int b = 0; b < n_b; ++b) q = q + (bm[b] - mean) * (bm[b] - mean);
        *err = sqrt(q / ((double)n_b * (double)(n_b - 1)));
    }
    free(bm);
}

void orc_micro_binned(int32_t K, double e_min, double bin_width, const double* lnW, const double* H,
                      int32_t n_it, int32_t block, int32_t h, int32_t n_monomers, int32_t n_T, const double* T,
                      double* S, double* beta, double* CV, double* E_T, double* cV_T, double* peak,
                      double* S_err, double* beta_err, double* CV_err, double* E_T_err, double* cV_T_err,
                      double* peak_err) {
    size_t nk = (size_t)n_it * (size_t)K, nt = (size_t)n_it * (size_t)(n_T > 0 ? n_T : 1);
    double* s = (double*)malloc(sizeof(double) * nk);
    double* b = (double*)malloc(sizeof(double) * nk);
    double* c = (double*)malloc(sizeof(double) * nk);
    double* et = (double*)malloc(sizeof(double) * nt);
    double* cv = (double*)malloc(sizeof(double) * nt);
    double* pk = (double*)malloc(sizeof(double) * 2 * (size_t)n_it);
    for (int i = 0; i < n_it; ++i) {
        size_t o = (size_t)i * (size_t)K, ot = (size_t)i * (size_t)(n_T > 0 ? n_T : 1);
        pk[2 * i] = pk[2 * i + 1] = NAN;
        orc_micro_analysis(K, e_min, bin_width, lnW + o, H ? H + o : NULL, h, n_monomers, n_T, T,
                           s + o, b + o, c + o, et + ot, cv + ot, pk + 2 * i);
    }
    for (int k = 0; k < K; ++k) {
        orc_binning(s + k, (size_t)K, n_it, block, &S[k], &S_err[k]);
        orc_binning(b + k, (size_t)K, n_it, block, &beta[k], &beta_err[k]);
        orc_binning(c + k, (size_t)K, n_it, block, &CV[k], &CV_err[k]);
    }
    for (int i = 0; i < n_T; ++i) {
        orc_binning(et + i, (size_t)n_T, n_it, block, &E_T[i], &E_T_err[i]);
        orc_binning(cv + i, (size_t)n_T, n_it, block, &cV_T[i], &cV_T_err[i]);
    }
    for (int q = 0; q < 2; ++q) orc_binning(pk + q, 2, n_it, block, &peak[q], &peak_err[q]);
    free(s); free(b); free(c); free(et); free(cv); free(pk);
}

/* ------------------------------------------------------------------------- */
/* Derivatives of the energy of Eq. 2/3 (with the torsion term), for the      */
/* force-field sensitivities: every term differentiated by hand, in the same  */
/* loops as orc_energy.  Parameters p = (C_AA, C_BB, C_AB, kappa, kappa_C):   */
/* the energy is linear in each, so dE/dp is the sum of the terms it          */
/* multiplies.  Between different chains of a periodic system the minimum     */
/* image d - L rint(d / L) has derivative 1 in d (rint is piecewise constant).*/
/* ------------------------------------------------------------------------- */
static void orc_cross(const double a[3], const double b[3], double out[3]) {
    out[0] = a[1] * b[2] - a[2] * b[1];
    out[1] = a[2] * b[0] - a[0] * b[2];
    out[2] = a[0] * b[1] - a[1] * b[0];
}

static double orc_dot(const double a[3], const double b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

double orc_energy_grad(const orc_model* m, const double* xyz, double* gx, double* gp) {
    int N = orc_total(m);
    double g_local[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    double E = 0.0;
    if (gx) for (int q = 0; q < 3 * N; ++q) gx[q] = 0.0;
    for (int c = 0, o = 0; c < m->n_chains; o += m->chain_len[c], ++c) {
        int n = m->chain_len[c];
        /* bending: kappa_C (1 - cos theta), cos theta = a.b / (|a| |b|), a = x1 - x0, b = x2 - x1 */
        for (int k = 1; k <= n - 2; ++k) {
            int i0 = o + k - 1, i1 = o + k, i2 = o + k + 1;
            double a[3], b[3];
            for (int d = 0; d < 3; ++d) {
                a[d] = xyz[3 * i1 + d] - xyz[3 * i0 + d];
                b[d] = xyz[3 * i2 + d] - xyz[3 * i1 + d];
            }
            double la = sqrt(orc_dot(a, a)), lb = sqrt(orc_dot(b, b));
            double cs = orc_dot(a, b) / (la * lb);
            E = E + m->k_bend * (1.0 - cs);
            g_local[4] = g_local[4] + (1.0 - cs);
            if (!gx) continue;
            for (int d = 0; d < 3; ++d) {
                double dca = b[d] / (la * lb) - cs * a[d] / (la * la);   /* d cos / d a */
                double dcb = a[d] / (la * lb) - cs * b[d] / (lb * lb);   /* d cos / d b */
                /* E = kappa_C (1 - cos): dE/da = -kappa_C dca, a = x1 - x0, b = x2 - x1 */
                gx[3 * i0 + d] = gx[3 * i0 + d] + m->k_bend * dca;
                gx[3 * i1 + d] = gx[3 * i1 + d] - m->k_bend * (dca - dcb);
                gx[3 * i2 + d] = gx[3 * i2 + d] - m->k_bend * dcb;
            }
        }
        /* torsion: -kappa cos tau, cos tau = n1.n2 / (|n1| |n2|), n1 = u x v, n2 = v x w */
        for (int j = 0; j <= n - 4; ++j) {
            int i0 = o + j;
            double u[3], v[3], w[3], n1[3], n2[3];
            for (int d = 0; d < 3; ++d) {
                u[d] = xyz[3 * (i0 + 1) + d] - xyz[3 * i0 + d];
                v[d] = xyz[3 * (i0 + 2) + d] - xyz[3 * (i0 + 1) + d];
                w[d] = xyz[3 * (i0 + 3) + d] - xyz[3 * (i0 + 2) + d];
            }
            orc_cross(u, v, n1);
            orc_cross(v, w, n2);
            double n11 = orc_dot(n1, n1), n22 = orc_dot(n2, n2);
            if (n11 * n22 < 1e-20) continue;   /* degenerate dihedral: no term, no derivative */
            double l1 = sqrt(n11), l2 = sqrt(n22);
            double cs = orc_dot(n1, n2) / (l1 * l2);
            E = E - m->k_tors * cs;
            g_local[3] = g_local[3] - cs;
            if (!gx) continue;
            double g1[3], g2[3];   /* d cos / d n1, d cos / d n2 */
            for (int d = 0; d < 3; ++d) {
                g1[d] = n2[d] / (l1 * l2) - cs * n1[d] / n11;
                g2[d] = n1[d] / (l1 * l2) - cs * n2[d] / n22;
            }
            /* d(g1.(u x v))/du = v x g1, /dv = g1 x u; d(g2.(v x w))/dv = w x g2, /dw = g2 x v */
            double du[3], dv1[3], dv2[3], dw[3];
            orc_cross(v, g1, du);
            orc_cross(g1, u, dv1);
            orc_cross(w, g2, dv2);
            orc_cross(g2, v, dw);
            for (int d = 0; d < 3; ++d) {
                double eu = -m->k_tors * du[d], ev = -m->k_tors * (dv1[d] + dv2[d]), ew = -m->k_tors * dw[d];
                gx[3 * i0 + d] = gx[3 * i0 + d] - eu;
                gx[3 * (i0 + 1) + d] = gx[3 * (i0 + 1) + d] + eu - ev;
                gx[3 * (i0 + 2) + d] = gx[3 * (i0 + 2) + d] + ev - ew;
                gx[3 * (i0 + 3) + d] = gx[3 * (i0 + 3) + d] + ew;
            }
        }
    }
    /* FENE bonds: phi = k R^2 C_F ln(1 - x^2), x = (r - r0) / R, dphi/dr = -2 k R C_F x / (1 - x^2) */
    if (m->k_fene != 0.0) {
        for (int c = 0, o = 0; c < m->n_chains; o += m->chain_len[c], ++c) {
            for (int l = o; l < o + m->chain_len[c] - 1; ++l) {
                double d[3];
                for (int q = 0; q < 3; ++q) d[q] = xyz[3 * (l + 1) + q] - xyz[3 * l + q];
                double r = sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
                double x = (r - m->fene_r0) / m->fene_R;
                double cf = m->C_F[2 * m->seq[l] + m->seq[l + 1]];
                E = E + (m->k_fene * (m->fene_R * m->fene_R)) * (cf * log(1.0 - x * x));
                if (!gx) continue;
                double dphi = -2.0 * m->k_fene * m->fene_R * cf * x / (1.0 - x * x);
                for (int q = 0; q < 3; ++q) {
                    gx[3 * (l + 1) + q] = gx[3 * (l + 1) + q] + dphi * d[q] / r;
                    gx[3 * l + q] = gx[3 * l + q] - dphi * d[q] / r;
                }
            }
        }
    }
    /* Lennard-Jones pairs (Eq. 2: i < j - 1 of one chain; Eq. 3: all pairs of different chains):
     * phi = k (s^6 - C s^3), s = 1 / r^2, dphi / d(r^2) = k s (3 C s^3 - 6 s^6), dphi/dC = -k s^3 */
    for (int i = 0; i < N; ++i) {
        int ci = orc_chain_of(m, i);
        for (int j = i + 1; j < N; ++j) {
            int cj = orc_chain_of(m, j);
            if (ci == cj && j < i + 2) continue;
            double dv[3], r2 = 0.0;
            for (int d = 0; d < 3; ++d) {
                double x = xyz[3 * i + d] - xyz[3 * j + d];
                if (ci != cj && m->box_L > 0.0) x = x - m->box_L * rint(x / m->box_L);
                dv[d] = x;
                r2 = r2 + x * x;
            }
            int si = m->seq[i], sj = m->seq[j];
            double C = m->C[2 * si + sj];
            double k = (ci == cj) ? m->k_lj_intra : m->k_lj_inter;
            double s = 1.0 / r2, s3 = s * s * s, s6 = s3 * s3;
            E = E + k * (s6 - C * s3);
            int pidx = (si == sj) ? (si == 0 ? 0 : 1) : 2;
            g_local[pidx] = g_local[pidx] - k * s3;
            if (!gx) continue;
            double f = 2.0 * k * s * (3.0 * C * s3 - 6.0 * s6);   /* 2 dphi/d(r^2) */
            for (int d = 0; d < 3; ++d) {
                gx[3 * i + d] = gx[3 * i + d] + f * dv[d];
                gx[3 * j + d] = gx[3 * j + d] - f * dv[d];
            }
        }
    }
    if (gp) for (int q = 0; q < 5; ++q) gp[q] = g_local[q];
    return E;
}

/* Canonical averages and their parameter derivatives from multicanonical
 * samples (Sec. 2.2: reweighting the multicanonical ensemble to temperature T).
 * Sample n has energy E_n, derivative D_n = dE/dlambda and was drawn with
 * log-weight lnW_n, so its canonical weight at T is w_n ~ exp(-E_n / T - lnW_n)
 * (the sampling weights do not depend on lambda).  With beta = 1 / T and
 * centred moments over the w_n:
 *   <E>, c_V = <(E - <E>)^2> / (N T^2),
 *   d<E>/dlambda = <D> - beta <(E - <E>)(D - <D>)>,
 *   d c_V/dlambda = [2 <(E - <E>)(D - <D>)> - beta <(E - <E>)^2 (D - <D>)>] / (N T^2),
 * the last from d<O>/dlambda = <dO/dlambda> - beta Cov(O, D) for O = E and E^2. */
void orc_reweight_sensitivity(int64_t n, const double* E, const double* D, const double* lnW, int32_t n_monomers,
                              int32_t n_T, const double* T, double* E_T, double* cV_T, double* dE_T, double* dcV_T) {
    for (int i = 0; i < n_T; ++i) {
        double beta = 1.0 / T[i];
        double amax = -INFINITY;
        for (int64_t q = 0; q < n; ++q) {
            double a = -beta * E[q] - lnW[q];
            if (a > amax) amax = a;
        }
        double Z = 0.0, sE = 0.0, sD = 0.0;
        for (int64_t q = 0; q < n; ++q) {
            double w = exp(-beta * E[q] - lnW[q] - amax);
            Z = Z + w;
            sE = sE + w * E[q];
            sD = sD + w * D[q];
        }
        double mE = sE / Z, mD = sD / Z;
        double vE = 0.0, cED = 0.0, m3 = 0.0;
        for (int64_t q = 0; q < n; ++q) {
            double w = exp(-beta * E[q] - lnW[q] - amax);
            double e = E[q] - mE, dd = D[q] - mD;
            vE = vE + w * e * e;
            cED = cED + w * e * dd;
            m3 = m3 + w * e * e * dd;
        }
        vE = vE / Z;
        cED = cED / Z;
        m3 = m3 / Z;
        double nT2 = (double)n_monomers * T[i] * T[i];
        E_T[i] = mE;
        cV_T[i] = vE / nT2;
        dE_T[i] = mD - beta * cED;
        dcV_T[i] = (2.0 * cED - beta * m3) / nT2;
    }
}

/* ------------------------------------------------------------------------- */
/* Free energy (Eq. 7) and the Maxwell construction on the caloric curve      */
/* (Sec. 3.3, ANALYST: Tol_Beta, Tol_L).  Reading: the equal-area line on     */
/* beta(E) is the common tangent of S(E), i.e. an edge of the upper concave   */
/* hull of the points (E_k, S_k) over visited bins that spans bins lying      */
/* below it (a convex intruder).  Among intruders with a positive slope      */
/* (beta_c = 1/T_c > 0: a transition at a positive temperature), a latent    */
/* heat (E_b - E_a)/N of at least tol_L, and across which beta_k = (S_{k+h} - */
/* S_{k-h})/(2 h w) rises by at least tol_beta (the S-bend), the one with the */
/* largest latent heat is taken: beta_c its slope, eps_1 = E_a/N,             */
/* eps_2 = E_b/N, and the barrier of f = (E - S/beta_c)/N between the two     */
/* coexisting states, max (hull(E_k) - S_k) / (beta_c N) over the bins inside.*/
/* ------------------------------------------------------------------------- */
void orc_maxwell(int32_t K, double e_min, double bin_width, const double* S, int32_t n_monomers,
                 int32_t fd_half_width, double beta_c_in, double tol_beta, double tol_L, double* f_out,
                 double* res) {
    double N = (double)n_monomers;
    int h = fd_half_width;
    for (int q = 0; q < 6; ++q) res[q] = NAN;
    res[5] = 0.0;
    /* upper hull by Andrew's monotone chain over visited bins (S finite), left to right */
    int* hull = (int*)malloc(sizeof(int) * (size_t)(K > 0 ? K : 1));
    int nh = 0;
    for (int k = 0; k < K; ++k) {
        if (!isfinite(S[k])) continue;
        double ek = e_min + ((double)k + 0.5) * bin_width;
        while (nh >= 2) {
            int i = hull[nh - 2], j = hull[nh - 1];
            double ei = e_min + ((double)i + 0.5) * bin_width, ej = e_min + ((double)j + 0.5) * bin_width;
            /* drop j if it lies on or below the chord from i to k */
            if ((S[j] - S[i]) * (ek - ei) <= (S[k] - S[i]) * (ej - ei)) --nh;
            else break;
        }
        hull[nh++] = k;
    }
    double best_L = -1.0;
    int best_a = -1, best_b = -1;
    if (beta_c_in <= 0.0) {
        for (int q = 0; q + 1 < nh; ++q) {
            int a = hull[q], b = hull[q + 1];
            int inside = 0;
            for (int k = a + 1; k < b; ++k) if (isfinite(S[k])) inside = 1;
            if (!inside) continue;
            double ea = e_min + ((double)a + 0.5) * bin_width, eb = e_min + ((double)b + 0.5) * bin_width;
            /* the common tangent's slope is beta_c = 1/T_c: a transition needs beta_c > 0 */
            if (!((S[b] - S[a]) / (eb - ea) > 0.0)) continue;
            double L = (eb - ea) / N;
            /* largest rise of beta across [a, b]: max over k <= j of beta_j - beta_k */
            double rise = 0.0, bmin = INFINITY;
            for (int k = a; k <= b; ++k) {
                if (k - h < 0 || k + h >= K || !isfinite(S[k - h]) || !isfinite(S[k + h])) continue;
                double bk = (S[k + h] - S[k - h]) / (2.0 * h * bin_width);
                if (bk - bmin > rise) rise = bk - bmin;
                if (bk < bmin) bmin = bk;
            }
            if (L >= tol_L && rise >= tol_beta && L > best_L) {
                best_L = L;
                best_a = a;
                best_b = b;
            }
        }
    }
    double beta_c = beta_c_in;
    if (best_a >= 0) {
        double ea = e_min + ((double)best_a + 0.5) * bin_width, eb = e_min + ((double)best_b + 0.5) * bin_width;
        beta_c = (S[best_b] - S[best_a]) / (eb - ea);
        double gap = 0.0;
        for (int k = best_a + 1; k < best_b; ++k) {
            if (!isfinite(S[k])) continue;
            double ek = e_min + ((double)k + 0.5) * bin_width;
            double line = S[best_a] + beta_c * (ek - ea);
            if (line - S[k] > gap) gap = line - S[k];
        }
        res[0] = beta_c;
        res[1] = ea / N;
        res[2] = eb / N;
        res[3] = (eb - ea) / N;
        res[4] = gap / (beta_c * N);
        res[5] = 1.0;
    } else if (beta_c_in > 0.0) {
        res[0] = beta_c_in;
    }
    if (f_out) {
        for (int k = 0; k < K; ++k) {
            double ek = e_min + ((double)k + 0.5) * bin_width;
            f_out[k] = (isfinite(S[k]) && beta_c > 0.0) ? (ek - S[k] / beta_c) / N : NAN;
        }
    }
    free(hull);
}
