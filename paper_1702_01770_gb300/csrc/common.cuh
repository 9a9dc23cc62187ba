// common.cuh -- device building blocks shared by the PHAST kernels (sm_103a):
// system descriptors, the Philox4x32-10 walker stream, FP64 move geometry with
// explicitly rounded operations, FP64 bending/torsion terms, the bin map, and
// host-side error reporting.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "phast.h"

#define PHAST_STREAM_TAG 0x4D554341u   // counter word 3 of every walker-stream block
#define PHAST_MARSAGLIA_TRIES 64

// ---------------------------------------------------------------------------
// Host-side errors (thread-local message; every entry point returns a code).
// ---------------------------------------------------------------------------
int phast_set_error(int code, const char* fmt, ...);
#define PHAST_CUDA_TRY(call)                                                            \
    do {                                                                                \
        cudaError_t err_ = (call);                                                      \
        if (err_ != cudaSuccess)                                                        \
            return phast_set_error(PHAST_ECUDA, "%s: %s (%s:%d)", #call,               \
                                   cudaGetErrorString(err_), __FILE__, __LINE__);       \
    } while (0)

// ---------------------------------------------------------------------------
// System descriptor: one system type with its force field and MUCA set-up,
// flattened for the device.  Built once on the host from the ABI structs.
// ---------------------------------------------------------------------------
struct SysDesc {
    int32_t n_chains, N, n_bins, recompute_every;
    int32_t walker_off, n_walkers, lnw_off, max_chain;
    int32_t pair_precision, n_tiles, tile_off, pad0;
    int64_t xyz_off;      // offset of walker 0's coordinates in the concatenated xyz (doubles)
    int64_t hw_off;       // offset of walker 0's histogram in hist_walker (bins)
    double box_L, inv_L;  // inv_L = 0 for open systems
    double k_bend, k_tors, k_lj_intra, k_lj_inter;
    double C[4];
    double e_min, bin_width;
    double p[PHAST_N_MOVES], amax[PHAST_N_MOVES];
    uint64_t thr[PHAST_N_MOVES];   // move-type thresholds: type i if 2n+1 < thr[i] (n the 52-bit uniform), see propose_select
    int32_t last_type, type_mask;   // type_mask: bit i set when p[i] > 0
    int32_t has_sphere, pad2;       // has_sphere: a steric container (sphere_R2 > 0)
    double sphere_R2;     // sphere_R * sphere_R of the steric container (0: none)
    double k_fene, fene_r0, fene_R, fene_kR2;   // FENE term of Eq. 2; fene_kR2 = k_fene * (R * R)
    double C_F[4];
    float C32[4];         // FP32 copies for the FP32 working precision
    float L32, iL32, kin32, kout32, kbend32, ktors32, iw32, sphere_R2_32;
    float amax32[PHAST_N_MOVES], pad3[2];
    float fene_r0_32, fene_iR32, fene_kR2_32, pad4;
    float C_F32[4];
    int32_t chain_off[PHAST_MAX_CHAINS + 1];
    int32_t pad1[3];
    uint8_t seq[PHAST_MAX_MONOMERS];
    uint8_t chain_of[PHAST_MAX_MONOMERS];
    uint16_t n_a_before[PHAST_MAX_MONOMERS + 8];   // number of A monomers with index < j
    int32_t pad5[2];
};
static_assert(sizeof(SysDesc) % 16 == 0, "SysDesc must be 16-byte sized for vector copies");

// Validates the ABI structs and fills a descriptor (offsets left at 0).
// Berg step on stream st (weights.cu); set_attr: set the kernel's shared-memory
// limit first (not allowed while a stream is being captured).
int phast_launch_berg(int32_t K, double bin_width, const uint64_t* hist, int32_t n_blocks, double* lnW,
                      double* g_acc, double* beta_out, double* flat_out, cudaStream_t st, bool set_attr);

int phast_build_desc(const phast_system* sys, const phast_ff* ff, const phast_muca_params* mp,
                     SysDesc* d, const char* what);

// ---------------------------------------------------------------------------
// Explicitly rounded FP64 arithmetic: the geometry below must round exactly
// as the specification states (fused multiply-adds only where written, no
// other contraction), so that coordinates are reproducible bit for bit by any
// IEEE-754 implementation of it.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double xadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double xsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double xmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double xdiv(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double xsqrt(double a) { return __dsqrt_rn(a); }
__device__ __forceinline__ double xfma(double a, double b, double c) { return __fma_rn(a, b, c); }

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// The same rounds kept out of line and not unrolled: one short copy of the
// code.  Small systems, whose per-move path does not stay in the instruction
// cache, run faster with it; the one-warp-per-walker build keeps the unrolled
// rounds inline.
static __device__ __noinline__ uint4 philox4x32_10_outline(uint4 c, uint2 k) {
#pragma unroll 1
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// Block b of move t of the walker keyed by `seed` (OUTLINE: the out-of-line rounds).
template <bool OUTLINE = false>
__device__ __forceinline__ uint4 stream_block(uint64_t seed, uint64_t t, uint32_t b) {
    const uint4 c = make_uint4((uint32_t)t, (uint32_t)(t >> 32), b, PHAST_STREAM_TAG);
    const uint2 k = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    if constexpr (OUTLINE) return philox4x32_10_outline(c, k);
    else return philox4x32_10(c, k);
}

// Uniform in (0,1) from 52 bits, exact: ((a>>6) 2^26 + (b>>6) + 1/2) 2^-52.
__device__ __forceinline__ double u52(uint32_t a, uint32_t b) {
    double n = xadd(xmul((double)(a >> 6), 67108864.0), (double)(b >> 6));
    return xmul(xadd(n, 0.5), 2.220446049250313080847263336181640625e-16);
}

// 52-bit integer n of a uniform u = (n + 1/2) 2^-52 drawn from words a, b.
__device__ __forceinline__ uint64_t u52_bits(uint32_t a, uint32_t b) {
    return ((uint64_t)(a >> 6) << 26) | (uint64_t)(b >> 6);
}
// 2u - 1 = (2n + 1 - 2^52) 2^-52, exact.
__device__ __forceinline__ double sym_unit(uint32_t a, uint32_t b) {
    int64_t k = (int64_t)(2 * u52_bits(a, b) + 1) - (int64_t)(1ull << 52);
    return xmul((double)k, 2.220446049250313080847263336181640625e-16);
}

// sin and cos of |a| <= 1 by their Taylor series, Horner in a^2 with separately
// rounded operations; coefficients are the correctly rounded (-1)^i/(2i+1)! and
// (-1)^i/(2i)!.
__device__ __forceinline__ void taylor_sincos(double a, double* s, double* c) {
    const double S[9] = {1.0, -1.0 / 6.0, 1.0 / 120.0, -1.0 / 5040.0, 1.0 / 362880.0,
                         -1.0 / 39916800.0, 1.0 / 6227020800.0, -1.0 / 1307674368000.0,
                         1.0 / 355687428096000.0};
    const double Cc[10] = {1.0, -1.0 / 2.0, 1.0 / 24.0, -1.0 / 720.0, 1.0 / 40320.0,
                           -1.0 / 3628800.0, 1.0 / 479001600.0, -1.0 / 87178291200.0,
                           1.0 / 20922789888000.0, -1.0 / 6402373705728000.0};
    double x2 = xmul(a, a);
    double ps = S[8];
#pragma unroll
    for (int i = 7; i >= 0; --i) ps = xfma(ps, x2, S[i]);
    double pc = Cc[9];
#pragma unroll
    for (int i = 8; i >= 0; --i) pc = xfma(pc, x2, Cc[i]);
    *s = xmul(a, ps);
    *c = pc;
}

// Rodrigues' matrix about unit axis k, angle with sine s and cosine c:
// entry (i, j) = fma((1 - c) k_i, k_j, d_ij), d_ij = c on the diagonal, +-s k_l off it.
struct Rot3 { double m[9]; };
__device__ __forceinline__ Rot3 rodrigues(double kx, double ky, double kz, double s, double c) {
    double t = xsub(1.0, c);
    double tx = xmul(t, kx), ty = xmul(t, ky), tz = xmul(t, kz);
    double sx = xmul(s, kx), sy = xmul(s, ky), sz = xmul(s, kz);
    Rot3 R;
    R.m[0] = xfma(tx, kx, c);
    R.m[1] = xfma(tx, ky, -sz);
    R.m[2] = xfma(tx, kz, sy);
    R.m[3] = xfma(ty, kx, sz);
    R.m[4] = xfma(ty, ky, c);
    R.m[5] = xfma(ty, kz, -sx);
    R.m[6] = xfma(tz, kx, -sy);
    R.m[7] = xfma(tz, ky, sx);
    R.m[8] = xfma(tz, kz, c);
    return R;
}

// x' = p + R (x - p): v = x - p, x'_i = fma(R_i2, v_2, fma(R_i1, v_1, fma(R_i0, v_0, p_i))).
__device__ __forceinline__ double3 rotate_about(const Rot3& R, double3 p, double3 x) {
    double v0 = xsub(x.x, p.x), v1 = xsub(x.y, p.y), v2 = xsub(x.z, p.z);
    return make_double3(xfma(R.m[2], v2, xfma(R.m[1], v1, xfma(R.m[0], v0, p.x))),
                        xfma(R.m[5], v2, xfma(R.m[4], v1, xfma(R.m[3], v0, p.y))),
                        xfma(R.m[8], v2, xfma(R.m[7], v1, xfma(R.m[6], v0, p.z))));
}

// One Marsaglia (1972) attempt from block r: (v1, v2) uniform in the square,
// kept if inside the unit disc (0 < s < 1); the axis is then
// (2 v1 sqrt(1-s), 2 v2 sqrt(1-s), 1 - 2 s), isotropic on the sphere.
__device__ __forceinline__ bool marsaglia_in_disc(uint4 r, double* v1, double* v2, double* s) {
    *v1 = sym_unit(r.x, r.y);
    *v2 = sym_unit(r.z, r.w);
    *s = xadd(xmul(*v1, *v1), xmul(*v2, *v2));
    return *s < 1.0 && *s > 0.0;
}
__device__ __forceinline__ double3 marsaglia_axis(double v1, double v2, double s) {
    double q = xsqrt(xsub(1.0, s));
    return make_double3(xmul(xmul(2.0, v1), q), xmul(xmul(2.0, v2), q), xsub(1.0, xmul(2.0, s)));
}
__device__ __forceinline__ bool marsaglia_try(uint4 r, double3* axis) {
    double v1, v2, s;
    if (!marsaglia_in_disc(r, &v1, &v2, &s)) return false;
    *axis = marsaglia_axis(v1, v2, s);
    return true;
}

// Centroid of monomers o..o+n-1 in the fixed summation order of the move's
// specification: 32 strided partial sums s_l over j = l, l+32, ... (increasing
// j), halved by s_l += s_{l+w} for w = 16, 8, 4, 2, 1, then s_0 / n.  One thread.
__device__ __forceinline__ double3 centroid_serial(const double* x64, int o, int n) {
    double c[3];
    for (int d = 0; d < 3; ++d) {
        double part[32];
        for (int l = 0; l < 32; ++l) {
            part[l] = 0.0;
            for (int j = l; j < n; j += 32) part[l] = xadd(part[l], x64[3 * (o + j) + d]);
        }
        for (int w = 16; w >= 1; w /= 2)
            for (int l = 0; l < w; ++l) part[l] = xadd(part[l], part[l + w]);
        c[d] = xdiv(part[0], (double)n);
    }
    return make_double3(c[0], c[1], c[2]);
}

// A proposed move, drawn from the walker stream.
struct Proposal {
    int type, chain, index;
    int attempt;            // winning Marsaglia attempt (-1: none won, axis (0, 0, 1))
    double angle;           // exact amplitude, axis and step (FP64 mode and exact replay)
    double3 axis, disp;
    float angle32;          // their FP32 images (FP32 trial moves)
    float3 axis32, disp32;
    uint32_t uz, uw;        // words of the acceptance uniform (block 2 z, w)
};

// Monomer or bond a move acts on, from block 0's last word: an interior
// monomer 1..n-2 (pivot, crankshaft), a bond 0..n-2 (bond length), any
// monomer 0..n-1 (spherical cap); 0 for whole-chain moves.
__host__ __device__ __forceinline__ int move_index(int type, int n, uint32_t w) {
    if (type == PHAST_PIVOT || type == PHAST_CRANK) return 1 + (int)(((uint64_t)w * (uint64_t)(n - 2)) >> 32);
    if (type == PHAST_BOND) return (int)(((uint64_t)w * (uint64_t)(n - 1)) >> 32);
    if (type == PHAST_CAP) return (int)(((uint64_t)w * (uint64_t)n) >> 32);
    return 0;
}

// Selection part of move t (blocks 0-2): the type is the first one with p > 0
// whose running probability sum exceeds the uniform (the last type with p > 0
// catches the rounding remainder) -- compared exactly in integers, since
// u < cum  <=>  2n + 1 < cum 2^53  <=>  2n + 1 < ceil(cum 2^53) = thr;
// uniform chain; interior monomer 1..n-2 for pivot and crankshaft; amplitude
// uniform in [-amax, amax].  The axis is set separately.
__device__ __forceinline__ void propose_select(const SysDesc& d, uint4 b0, uint4 b1, uint4 b2,
                                               Proposal* P) {
    const uint64_t v = 2 * u52_bits(b0.x, b0.y) + 1;
    int type = d.last_type;
#pragma unroll
    for (int i = PHAST_N_MOVES - 1; i >= 0; --i)
        if (((d.type_mask >> i) & 1) && v < d.thr[i]) type = i;
    P->uz = b2.z;
    P->uw = b2.w;
    P->attempt = -1;
    P->type = type;
    P->chain = (int)(((uint64_t)b0.z * (uint64_t)d.n_chains) >> 32);
    int n = d.chain_off[P->chain + 1] - d.chain_off[P->chain];
    P->index = move_index(type, n, b0.w);
    P->angle = 0.0;
    P->disp = make_double3(0.0, 0.0, 0.0);
    P->axis = make_double3(0.0, 0.0, 1.0);
    if (type == PHAST_TRANS) {
        double a = d.amax[PHAST_TRANS];
        P->disp = make_double3(xmul(sym_unit(b1.x, b1.y), a), xmul(sym_unit(b1.z, b1.w), a),
                               xmul(sym_unit(b2.x, b2.y), a));
    } else {   // rotation angle, or the signed length step of a bond move
        P->angle = xmul(sym_unit(b1.x, b1.y), d.amax[type]);
    }
}

// Moved monomer range [lo, hi] (system indices) and the fixed point excluded
// from the pair set (the pivot; -1 otherwise) of a move.
__device__ __forceinline__ void moved_range(const SysDesc& d, int type, int chain, int index,
                                            int* lo, int* hi, int* fixed) {
    int o = d.chain_off[chain], n = d.chain_off[chain + 1] - o;
    *fixed = -1;
    if (type == PHAST_TRANS || type == PHAST_ROT) { *lo = o; *hi = o + n - 1; return; }
    if (type == PHAST_CRANK || type == PHAST_CAP) { *lo = *hi = o + index; return; }
    if (type == PHAST_BOND) {   // the shorter side of bond index (on a tie the tail)
        if (index + 1 < n - 1 - index) { *lo = o; *hi = o + index; }
        else { *lo = o + index + 1; *hi = o + n - 1; }
        return;
    }
    *fixed = o + index;
    if (index < n - 1 - index) { *lo = o; *hi = o + index - 1; }
    else { *lo = o + index + 1; *hi = o + n - 1; }
}

// Energy bin of E: floor((E - e_min) / w) or -1 (out of range / non-finite).
__device__ __forceinline__ int bin_of(const SysDesc& d, double E) {
    if (!isfinite(E)) return -1;
    double q = xdiv(xsub(E, d.e_min), d.bin_width);
    if (!(q >= 0.0 && q < (double)d.n_bins)) return -1;
    return (int)floor(q);
}

// ---------------------------------------------------------------------------
// FP64 local terms.  Positions come from a functor pos(j) -> double3.
// ---------------------------------------------------------------------------
template <class Pos>
__device__ __forceinline__ double bend_term(const Pos& pos, int o, int k) {
    // 1 - cos(theta_k), theta_k between bonds (k-1 -> k) and (k -> k+1) of the chain at o
    double3 x0 = pos(o + k - 1), x1 = pos(o + k), x2 = pos(o + k + 1);
    double ax = x1.x - x0.x, ay = x1.y - x0.y, az = x1.z - x0.z;
    double bx = x2.x - x1.x, by = x2.y - x1.y, bz = x2.z - x1.z;
    double ab = ax * bx + ay * by + az * bz;
    double aa = ax * ax + ay * ay + az * az, bb = bx * bx + by * by + bz * bz;
    return 1.0 - ab / (sqrt(aa) * sqrt(bb));
}

template <class Pos>
__device__ __forceinline__ double torsion_term(const Pos& pos, int o, int j) {
    // cos(tau_j) of monomers j..j+3; 0 when a normal degenerates
    double3 x0 = pos(o + j), x1 = pos(o + j + 1), x2 = pos(o + j + 2), x3 = pos(o + j + 3);
    double b0x = x1.x - x0.x, b0y = x1.y - x0.y, b0z = x1.z - x0.z;
    double b1x = x2.x - x1.x, b1y = x2.y - x1.y, b1z = x2.z - x1.z;
    double b2x = x3.x - x2.x, b2y = x3.y - x2.y, b2z = x3.z - x2.z;
    double n1x = b0y * b1z - b0z * b1y, n1y = b0z * b1x - b0x * b1z, n1z = b0x * b1y - b0y * b1x;
    double n2x = b1y * b2z - b1z * b2y, n2y = b1z * b2x - b1x * b2z, n2z = b1x * b2y - b1y * b2x;
    double n12 = n1x * n2x + n1y * n2y + n1z * n2z;
    double n11 = n1x * n1x + n1y * n1y + n1z * n1z, n22 = n2x * n2x + n2y * n2y + n2z * n2z;
    if (n11 * n22 < 1e-20) return 0.0;
    return n12 / (sqrt(n11) * sqrt(n22));
}

// Local (bending + torsion) items a move changes.  Items 0..nb-1 are bends at
// vertices vb0.., items nb.. are dihedrals starting at jt0..; returns the count.
__device__ __forceinline__ void local_window(const SysDesc& d, int type, int chain, int index,
                                             int* vb0, int* nb, int* jt0, int* nt, int* fb0, int* nf) {
    int n = d.chain_off[chain + 1] - d.chain_off[chain];
    *nb = 0; *nt = 0; *vb0 = 0; *jt0 = 0; *fb0 = 0; *nf = 0;
    if (type == PHAST_PIVOT) {
        *vb0 = index; *nb = 1;
        int a = max(index - 2, 0), b = min(index - 1, n - 4);
        *jt0 = a; *nt = max(b - a + 1, 0);
    } else if (type == PHAST_CRANK || type == PHAST_CAP) {
        int a = max(index - 1, 1), b = min(index + 1, n - 2);
        *vb0 = a; *nb = max(b - a + 1, 0);
        int c = max(index - 3, 0), e = min(index, n - 4);
        *jt0 = c; *nt = max(e - c + 1, 0);
        // a cap keeps the bond to its rotation centre; the other bond changes length
        if (type == PHAST_CAP && d.k_fene != 0.0 && index >= 1 && index <= n - 2) { *fb0 = index; *nf = 1; }
    } else if (type == PHAST_BOND) {   // bend and torsion angles keep; one bond's length changes
        if (d.k_fene != 0.0) { *fb0 = index; *nf = 1; }
    }
}

// FENE term of bond l (monomers l, l+1 of the chain at o):
// k_fene R^2 C_F ln(1 - ((r - r0) / R)^2), +inf outside |r - r0| < R (FP64).
template <class Pos>
__device__ __forceinline__ double fene_term(const SysDesc& d, const Pos& pos, int o, int l) {
    double3 a = pos(o + l), b = pos(o + l + 1);
    double dx = b.x - a.x, dy = b.y - a.y, dz = b.z - a.z;
    double r = sqrt((dx * dx + dy * dy) + dz * dz);
    double x = (r - d.fene_r0) / d.fene_R;
    double x2 = x * x;
    if (!(x2 < 1.0)) return INFINITY;
    return d.fene_kR2 * (d.C_F[2 * d.seq[o + l] + d.seq[o + l + 1]] * log(1.0 - x2));
}

__device__ __forceinline__ double3 ld3(const double* p) { return make_double3(p[0], p[1], p[2]); }

// Exact step of a bond-length move on bond l of the chain at o (n monomers):
// the shorter side slides by +delta u (tail) or -delta u (head), u the unit
// bond vector (x_{l+1} - x_l) / |x_{l+1} - x_l|; false for coincident monomers
// or a step through zero length.  *jac: the move's Hastings factor
// ((r + delta) / r)^2, the Jacobian determinant of the radial map of the bond
// vector (bead coordinates are the sampled measure).
__device__ __forceinline__ bool bond_step(const double* x64, int o, int n, int l, double delta, double3* step,
                                          double* jac) {
    const double3 a = ld3(x64 + 3 * (o + l)), b = ld3(x64 + 3 * (o + l + 1));
    const double bx = xsub(b.x, a.x), by = xsub(b.y, a.y), bz = xsub(b.z, a.z);
    const double len = xsqrt(xadd(xadd(xmul(bx, bx), xmul(by, by)), xmul(bz, bz)));
    if (!(len > 1e-12) || !(xadd(len, delta) > 0.0)) return false;
    const double q = xdiv(xadd(len, delta), len);
    *jac = xmul(q, q);
    const double dl = (l + 1 < n - 1 - l) ? -delta : delta;
    *step = make_double3(xmul(dl, xdiv(bx, len)), xmul(dl, xdiv(by, len)), xmul(dl, xdiv(bz, len)));
    return true;
}

// Steric container (hard wall about the origin): true if (x^2 + y^2) + z^2 <= R^2.
__device__ __forceinline__ bool inside64(const SysDesc& d, double3 x) {
    return !(d.sphere_R2 > 0.0) || xadd(xadd(xmul(x.x, x.x), xmul(x.y, x.y)), xmul(x.z, x.z)) <= d.sphere_R2;
}

// Lennard-Jones pair of Eq. 2/3 without its coupling: r^-12 - C r^-6 (FP64).
__device__ __forceinline__ double lj64(double r2, double C) {
    double ir2 = 1.0 / r2;
    double ir6 = ir2 * ir2 * ir2;
    return ir6 * (ir6 - C);
}

// Minimum-image component (FP64); inv_L = 0 leaves d unchanged.
__device__ __forceinline__ double mimage64(double dx, double L, double inv_L) {
    return dx - L * rint(dx * inv_L);
}

// Block-wide FP64 sum; every thread gets the result.  red: >= 32 doubles of shared.
__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        v = (l < nw) ? red[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (l == 0) red[0] = v;
    }
    __syncthreads();
    double r = red[0];
    __syncthreads();
    return r;
}
