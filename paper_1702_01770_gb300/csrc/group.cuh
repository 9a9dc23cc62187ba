// group.cuh -- the per-walker machinery of the sweep, written for a group of
// TPW lanes of one warp (TPW in {4, 8, 16, 32}) that owns one walker:
//   * working positions in shared memory: FP32 coordinates relative to the
//     FP64 centroid of their chain plus an FP32 table of minimum-imaged
//     centroid differences (so every FP32 distance is formed from small
//     numbers), or plain FP64 copies in the FP64-pair mode;
//   * the walker's Philox stream drawn by the lanes in parallel (selection
//     blocks and Marsaglia attempts side by side);
//   * FP64 move geometry into group scratch; scalar FP64 work (selection,
//     sin/cos, rotation matrix, bin, acceptance) on one lane only -- FP64 is
//     the scarce pipe of this chip, so no lane repeats another's FP64 work;
//   * dE = (bending + torsion window) + (moved x unmoved Lennard-Jones pairs,
//     R unmoved partners held in registers per lane), in the working
//     precision, summed per lane and across the group in FP64;
//   * full FP64 energies for the drift recompute.
#pragma once

#include "common.cuh"

template <typename T> struct P4;
template <> struct __align__(16) P4<float> { float x, y, z; int tag; };
template <> struct __align__(16) P4<double> { double x, y, z; int tag; int pad; };
// tag = sequence letter (bit 0) | chain index << 1

template <int TPW>
struct Group {
    int lane;
    int base;        // first lane of the group inside the warp
    unsigned mask;
    __device__ __forceinline__ Group() {
        int l = threadIdx.x & 31;
        lane = l & (TPW - 1);
        base = l - lane;
        mask = (TPW == 32) ? 0xffffffffu : (((1u << TPW) - 1u) << base);
    }
    __device__ __forceinline__ void sync() const { __syncwarp(mask); }
    __device__ __forceinline__ uint32_t bcast(uint32_t v, int src) const { return __shfl_sync(mask, v, src, TPW); }
    __device__ __forceinline__ double bcastd(double v, int src) const { return __shfl_sync(mask, v, src, TPW); }
    // Tree sum; every lane receives lane 0's total (one value for the whole group).
    __device__ __forceinline__ double sum(double v) const {
#pragma unroll
        for (int o = TPW / 2; o > 0; o >>= 1) v += __shfl_down_sync(mask, v, o, TPW);
        return __shfl_sync(mask, v, 0, TPW);
    }
    // Tree sum valid on lane 0 only.
    __device__ __forceinline__ double sum0(double v) const {
#pragma unroll
        for (int o = TPW / 2; o > 0; o >>= 1) v += __shfl_down_sync(mask, v, o, TPW);
        return v;
    }
};

// Shared-memory layout of one walker slot.
struct SlotLayout {
    int r_off, d_off, newr_off, orig_off, new64_off, geo_off, bytes;
};
__host__ __device__ inline int align16(int x) { return (x + 15) & ~15; }
template <typename PT>
__host__ __device__ inline SlotLayout slot_layout(int N, int nc, int mc) {
    SlotLayout L;
    int o = 0;
    L.r_off = o;     o = align16(o + (int)sizeof(P4<PT>) * N);
    L.d_off = o;     o = align16(o + (int)sizeof(P4<PT>) * nc * nc);
    L.newr_off = o;  o = align16(o + (int)sizeof(P4<PT>) * mc);
    L.orig_off = o;  o = align16(o + 8 * 3 * nc);
    L.new64_off = o; o = align16(o + 8 * 3 * mc);
    L.geo_off = o;   o = align16(o + 8 * 16);
    L.bytes = o;
    return L;
}

template <typename PT>
struct Slot {
    P4<PT>* r;      // [N] working positions
    P4<PT>* D;      // [nc * nc] origin differences (FP32 mode)
    P4<PT>* newr;   // [max_chain] working positions of the moved monomers after the move
    double* orig;   // [nc * 3] chain origins (FP32 mode; zero in FP64 mode)
    double* new64;  // [max_chain * 3] FP64 positions of the moved monomers after the move
    double* geo;    // [16] rotation matrix, centre, flags of the current move
    __device__ __forceinline__ Slot(unsigned char* p, const SlotLayout& L)
        : r((P4<PT>*)(p + L.r_off)), D((P4<PT>*)(p + L.d_off)), newr((P4<PT>*)(p + L.newr_off)),
          orig((double*)(p + L.orig_off)), new64((double*)(p + L.new64_off)), geo((double*)(p + L.geo_off)) {}
};

__device__ __forceinline__ double3 ld3(const double* p) { return make_double3(p[0], p[1], p[2]); }

// Minimum-imaged difference of the origins of chains a and b, in the working precision.
template <typename PT>
__device__ __forceinline__ P4<PT> origin_shift(const SysDesc& d, const double* orig, int a, int b) {
    P4<PT> q;
    q.x = (PT)mimage64(orig[3 * a + 0] - orig[3 * b + 0], d.box_L, d.inv_L);
    q.y = (PT)mimage64(orig[3 * a + 1] - orig[3 * b + 1], d.box_L, d.inv_L);
    q.z = (PT)mimage64(orig[3 * a + 2] - orig[3 * b + 2], d.box_L, d.inv_L);
    q.tag = 0;
    return q;
}

// Working copy of a walker: chain origins (FP64 centroid, FP32 mode), relative
// coordinates, origin-difference table.  x64 is the walker's FP64 [N][3].
template <int TPW, typename PT>
__device__ void build_working(const SysDesc& d, const double* x64, Slot<PT>& s, const Group<TPW>& g) {
    const bool rel = sizeof(PT) == 4;
    const int nc = d.n_chains;
    for (int c = g.lane; c < nc; c += TPW) {
        double sx = 0.0, sy = 0.0, sz = 0.0;
        const int o = d.chain_off[c], n = d.chain_off[c + 1] - o;
        if (rel) {
            for (int j = o; j < o + n; ++j) { sx += x64[3 * j]; sy += x64[3 * j + 1]; sz += x64[3 * j + 2]; }
            sx /= n; sy /= n; sz /= n;
        }
        s.orig[3 * c + 0] = sx;
        s.orig[3 * c + 1] = sy;
        s.orig[3 * c + 2] = sz;
    }
    g.sync();
    for (int j = g.lane; j < d.N; j += TPW) {
        int c = d.chain_of[j];
        P4<PT> q;
        q.x = (PT)(x64[3 * j + 0] - s.orig[3 * c + 0]);
        q.y = (PT)(x64[3 * j + 1] - s.orig[3 * c + 1]);
        q.z = (PT)(x64[3 * j + 2] - s.orig[3 * c + 2]);
        q.tag = (int)d.seq[j] | (c << 1);
        s.r[j] = q;
    }
    for (int p = g.lane; p < nc * nc; p += TPW) s.D[p] = origin_shift<PT>(d, s.orig, p / nc, p % nc);
    g.sync();
}

// After an accepted rigid translation by disp of chain c (FP32 mode): move the
// chain's origin with it, so its relative coordinates stay unchanged and small.
template <int TPW, typename PT>
__device__ void rebase_translated(const SysDesc& d, int c, double3 disp, Slot<PT>& s, const Group<TPW>& g) {
    if (g.lane == 0) {
        s.orig[3 * c + 0] += disp.x;
        s.orig[3 * c + 1] += disp.y;
        s.orig[3 * c + 2] += disp.z;
    }
    g.sync();
    const int nc = d.n_chains;
    for (int b = g.lane; b < nc; b += TPW) {
        s.D[c * nc + b] = origin_shift<PT>(d, s.orig, c, b);
        s.D[b * nc + c] = origin_shift<PT>(d, s.orig, b, c);
    }
}

// Draw move t: lanes compute Philox blocks 0..TPW-1 at once (blocks 0-2 are the
// selection, block 3+j is Marsaglia attempt j); lane 0 turns the selection
// blocks into the move and broadcasts it; further rounds of attempts follow
// only when the first round found no point in the disc.  u_acc is valid on
// lane 0 only.
template <int TPW>
__device__ Proposal propose_group(const SysDesc& d, uint64_t seed, uint64_t t, const Group<TPW>& g) {
    const uint4 blk = stream_block(seed, t, (uint32_t)g.lane);
    uint4 b[3];
#pragma unroll
    for (int i = 1; i < 3; ++i)
        b[i] = make_uint4(g.bcast(blk.x, i), g.bcast(blk.y, i), g.bcast(blk.z, i), g.bcast(blk.w, i));
    b[0] = blk;
    Proposal P;
    int packed = 0;
    double amp = 0.0, dy = 0.0, dz = 0.0;
    if (g.lane == 0) {
        propose_select(d, b[0], b[1], b[2], &P);
        packed = P.type | (P.chain << 2) | (P.index << 8);
        amp = P.type == PHAST_TRANS ? P.disp.x : P.angle;
        dy = P.disp.y;
        dz = P.disp.z;
    }
    packed = (int)g.bcast((uint32_t)packed, 0);
    P.type = packed & 3;
    P.chain = (packed >> 2) & 63;
    P.index = packed >> 8;
    amp = g.bcastd(amp, 0);
    P.angle = 0.0;
    P.disp = make_double3(0.0, 0.0, 0.0);
    P.axis = make_double3(0.0, 0.0, 1.0);
    if (P.type == PHAST_TRANS) {
        P.disp = make_double3(amp, g.bcastd(dy, 0), g.bcastd(dz, 0));
    } else {
        P.angle = amp;
    }
    if (P.type == PHAST_PIVOT || P.type == PHAST_ROT) {
        const unsigned gm = TPW == 32 ? 0xffffffffu : ((1u << TPW) - 1u);
        double v1 = 0.0, v2 = 0.0, sq = 0.0;
        bool ok = (g.lane >= 3) && marsaglia_in_disc(blk, &v1, &v2, &sq);
        unsigned bits = (__ballot_sync(g.mask, ok) >> g.base) & gm;
        for (int round = 1; bits == 0 && round * TPW <= 2 + PHAST_MARSAGLIA_TRIES; ++round) {
            const uint32_t blkid = (uint32_t)(round * TPW + g.lane);
            ok = blkid <= 2 + PHAST_MARSAGLIA_TRIES && marsaglia_in_disc(stream_block(seed, t, blkid), &v1, &v2, &sq);
            bits = (__ballot_sync(g.mask, ok) >> g.base) & gm;
        }
        if (bits) {
            const int src = __ffs(bits) - 1;
            double3 ax = make_double3(0.0, 0.0, 1.0);
            if (g.lane == src) ax = marsaglia_axis(v1, v2, sq);
            P.axis = make_double3(g.bcastd(ax.x, src), g.bcastd(ax.y, src), g.bcastd(ax.z, src));
        }
    }
    return P;
}

// Moved range and the unmoved monomers whose pair with a moved one is left
// out (the pivot keeps its distances; a crankshaft's bonded neighbours).
struct MoveSet { int lo, hi, ex0, ex1, ex2; };
__device__ __forceinline__ MoveSet move_set(const SysDesc& d, int type, int chain, int index) {
    MoveSet M;
    int fixed;
    moved_range(d, type, chain, index, &M.lo, &M.hi, &fixed);
    M.ex0 = fixed;
    M.ex1 = (type == PHAST_CRANK) ? M.lo - 1 : -1;
    M.ex2 = (type == PHAST_CRANK) ? M.hi + 1 : -1;
    return M;
}

// Pair evaluations of a move between different chains (2 per pair).
__device__ __forceinline__ uint64_t move_pair_evals_inter(const SysDesc& d, int type, int chain, const MoveSet& M) {
    const int nc = d.chain_off[chain + 1] - d.chain_off[chain];
    const int m = (type == PHAST_CRANK) ? 1 : M.hi - M.lo + 1;
    return 2ull * m * (d.N - nc);
}

// Pair evaluations a move costs (2 per changed Lennard-Jones pair).
__device__ __forceinline__ uint64_t move_pair_evals(const SysDesc& d, int type, const MoveSet& M) {
    int m = M.hi - M.lo + 1;
    if (type == PHAST_PIVOT) return 2ull * m * (d.N - m - 1);
    if (type == PHAST_CRANK) return 2ull * (d.N - 3);
    return 2ull * m * (d.N - m);
}

// FP64 positions (new64) and working positions (newr) of the moved monomers.
// Lane 0 builds the centre and rotation (into the slot's geo scratch); every
// lane then moves its share of the monomers.  Returns false for a degenerate
// crankshaft axis.
template <int TPW, typename PT>
__device__ bool make_new_positions(const SysDesc& d, const double* x64, const Proposal& P, const MoveSet& M,
                                   Slot<PT>& s, const Group<TPW>& g) {
    const int m = M.hi - M.lo + 1;
    const int c = P.chain, o = d.chain_off[c], n = d.chain_off[c + 1] - o;
    if (P.type != PHAST_TRANS && g.lane == 0) {
        double3 axis = P.axis, center;
        double ok = 1.0;
        if (P.type == PHAST_PIVOT) {
            center = ld3(x64 + 3 * (o + P.index));
        } else if (P.type == PHAST_ROT) {   // centroid: running sum j = 0..n-1, then / n
            double sx = 0.0, sy = 0.0, sz = 0.0;
            for (int j = o; j < o + n; ++j) {
                sx = xadd(sx, x64[3 * j + 0]);
                sy = xadd(sy, x64[3 * j + 1]);
                sz = xadd(sz, x64[3 * j + 2]);
            }
            center = make_double3(xdiv(sx, (double)n), xdiv(sy, (double)n), xdiv(sz, (double)n));
        } else {   // crankshaft about the axis through monomers i-1 and i+1
            const int i = o + P.index;
            const double3 a = ld3(x64 + 3 * (i - 1)), b = ld3(x64 + 3 * (i + 1));
            const double ex = xsub(b.x, a.x), ey = xsub(b.y, a.y), ez = xsub(b.z, a.z);
            const double len = xsqrt(xadd(xadd(xmul(ex, ex), xmul(ey, ey)), xmul(ez, ez)));
            if (!(len > 1e-12)) ok = 0.0;
            else axis = make_double3(xdiv(ex, len), xdiv(ey, len), xdiv(ez, len));
            center = a;
        }
        double sn, cs;
        taylor_sincos(P.angle, &sn, &cs);
        const Rot3 R = rodrigues(axis.x, axis.y, axis.z, sn, cs);
#pragma unroll
        for (int k = 0; k < 9; ++k) s.geo[k] = R.m[k];
        s.geo[9] = center.x;
        s.geo[10] = center.y;
        s.geo[11] = center.z;
        s.geo[12] = ok;
    }
    g.sync();
    if (P.type != PHAST_TRANS && s.geo[12] == 0.0) return false;
    Rot3 R;
    double3 center = make_double3(0.0, 0.0, 0.0);
    if (P.type != PHAST_TRANS) {
#pragma unroll
        for (int k = 0; k < 9; ++k) R.m[k] = s.geo[k];
        center = make_double3(s.geo[9], s.geo[10], s.geo[11]);
    }
    const bool rel = sizeof(PT) == 4;
    const double ox = rel ? s.orig[3 * c + 0] : 0.0, oy = rel ? s.orig[3 * c + 1] : 0.0,
                 oz = rel ? s.orig[3 * c + 2] : 0.0;
    for (int q = g.lane; q < m; q += TPW) {
        const int j = M.lo + q;
        const double3 x = ld3(x64 + 3 * j);
        double3 y;
        if (P.type == PHAST_TRANS)
            y = make_double3(xadd(x.x, P.disp.x), xadd(x.y, P.disp.y), xadd(x.z, P.disp.z));
        else
            y = rotate_about(R, center, x);
        s.new64[3 * q + 0] = y.x;
        s.new64[3 * q + 1] = y.y;
        s.new64[3 * q + 2] = y.z;
        P4<PT> w;
        w.x = (PT)(y.x - ox);
        w.y = (PT)(y.y - oy);
        w.z = (PT)(y.z - oz);
        w.tag = (int)d.seq[j] | (c << 1);
        s.newr[q] = w;
    }
    g.sync();
    return true;
}

// Bending and torsion terms from working positions (any precision; positions
// of one chain share an origin, so bond vectors are plain differences).
__device__ __forceinline__ float rsqrt_w(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_w(double x) { return 1.0 / sqrt(x); }

template <typename PT, class Pos>
__device__ __forceinline__ PT bend_w(const Pos& pos, int o, int k) {
    const P4<PT> x0 = pos(o + k - 1), x1 = pos(o + k), x2 = pos(o + k + 1);
    const PT ax = x1.x - x0.x, ay = x1.y - x0.y, az = x1.z - x0.z;
    const PT bx = x2.x - x1.x, by = x2.y - x1.y, bz = x2.z - x1.z;
    const PT ab = ax * bx + ay * by + az * bz;
    const PT aa = ax * ax + ay * ay + az * az, bb = bx * bx + by * by + bz * bz;
    if (sizeof(PT) == 8) return (PT)1 - ab / (sqrt(aa) * sqrt(bb));
    return (PT)1 - ab * rsqrt_w(aa * bb);
}

template <typename PT, class Pos>
__device__ __forceinline__ PT torsion_w(const Pos& pos, int o, int j) {
    const P4<PT> x0 = pos(o + j), x1 = pos(o + j + 1), x2 = pos(o + j + 2), x3 = pos(o + j + 3);
    const PT b0x = x1.x - x0.x, b0y = x1.y - x0.y, b0z = x1.z - x0.z;
    const PT b1x = x2.x - x1.x, b1y = x2.y - x1.y, b1z = x2.z - x1.z;
    const PT b2x = x3.x - x2.x, b2y = x3.y - x2.y, b2z = x3.z - x2.z;
    const PT n1x = b0y * b1z - b0z * b1y, n1y = b0z * b1x - b0x * b1z, n1z = b0x * b1y - b0y * b1x;
    const PT n2x = b1y * b2z - b1z * b2y, n2y = b1z * b2x - b1x * b2z, n2z = b1x * b2y - b1y * b2x;
    const PT n12 = n1x * n2x + n1y * n2y + n1z * n2z;
    const PT n11 = n1x * n1x + n1y * n1y + n1z * n1z, n22 = n2x * n2x + n2y * n2y + n2z * n2z;
    if (n11 * n22 < (PT)1e-20) return (PT)0;
    if (sizeof(PT) == 8) return n12 / (sqrt(n11) * sqrt(n22));
    return n12 * rsqrt_w(n11 * n22);
}

// This lane's share of the bending/torsion change, in the working precision.
template <int TPW, typename PT>
__device__ double local_delta(const SysDesc& d, const Proposal& P, const MoveSet& M, const Slot<PT>& s,
                              const Group<TPW>& g) {
    int vb0, nb, jt0, nt;
    local_window(d, P.type, P.chain, P.index, &vb0, &nb, &jt0, &nt);
    const int o = d.chain_off[P.chain];
    const int items = 2 * (nb + nt);
    PT part = (PT)0;
    for (int it = g.lane; it < items; it += TPW) {
        const bool after = it & 1;
        const int k = it >> 1;
        auto pos = [&](int j) -> P4<PT> {
            if (after && j >= M.lo && j <= M.hi) return s.newr[j - M.lo];
            return s.r[j];
        };
        const PT term = (k < nb) ? (PT)d.k_bend * bend_w<PT>(pos, o, vb0 + k)
                                 : -(PT)d.k_tors * torsion_w<PT>(pos, o, jt0 + (k - nb));
        part += after ? term : -term;
    }
    return (double)part;
}

__device__ __forceinline__ float fast_rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float pair_rcp(float x) { return fast_rcp(x); }
__device__ __forceinline__ double pair_rcp(double x) { return 1.0 / x; }

// Nearest integer to x * iL on the FMA pipe: adding 1.5 * 2^23 to the exact
// product rounds it to an integer (round to nearest even) for |x iL| < 2^22;
// the special-function unit (where cvt.rni runs) stays free for the reciprocal.
__device__ __forceinline__ float image_count(float x, float iL) {
    const float M = 12582912.0f;   // 1.5 * 2^23
    return __fsub_rn(__fmaf_rn(x, iL, M), M);
}
__device__ __forceinline__ double image_count(double x, double iL) { return rint(x * iL); }

// r^-12 - C r^-6 of one displacement with the per-partner minimum image
// (Lj = iLj = 0 leaves the displacement unchanged).
template <typename PT>
__device__ __forceinline__ PT lj_pair(PT dx, PT dy, PT dz, PT Lj, PT iLj, PT C) {
    dx -= Lj * image_count(dx, iLj);
    dy -= Lj * image_count(dy, iLj);
    dz -= Lj * image_count(dz, iLj);
    PT r2 = dx * dx + dy * dy + dz * dz;
    PT ir2 = pair_rcp(r2);
    PT ir6 = ir2 * ir2 * ir2;
    return ir6 * (ir6 - C);
}

// This lane's share of the Lennard-Jones change: unmoved partners t = lane,
// lane + TPW, ... (skipping the moved range), R of them in registers at a
// time, each swept against every moved monomer before and after the move.
template <int TPW, typename PT, int R>
__device__ double pair_delta(const SysDesc& d, const MoveSet& M, int mchain, const Slot<PT>& s,
                             const Group<TPW>& g) {
    const int m = M.hi - M.lo + 1;
    const int U = d.N - m;
    const int nc = d.n_chains;
    const PT L = (PT)d.box_L, iL = (PT)d.inv_L;
    const PT kin = (PT)d.k_lj_intra, kout = (PT)d.k_lj_inter;
    const PT far = (PT)1.0e4;
    PT part = (PT)0;
    for (int t0 = g.lane; t0 < U; t0 += TPW * R) {
        PT qx[R], qy[R], qz[R], Lj[R], iLj[R], C0[R], C1[R], kap[R], acc[R];
#pragma unroll
        for (int u = 0; u < R; ++u) {
            int t = t0 + u * TPW;
            qx[u] = qy[u] = qz[u] = far;
            Lj[u] = iLj[u] = C0[u] = C1[u] = kap[u] = (PT)0;
            acc[u] = (PT)0;
            if (t < U) {
                int j = t < M.lo ? t : t + m;
                P4<PT> p = s.r[j];
                int cj = p.tag >> 1, tj = p.tag & 1;
                bool same = cj == mchain;
                bool ex = (j == M.ex0) | (j == M.ex1) | (j == M.ex2);
                if (!ex) {
                    if (same) {
                        qx[u] = p.x; qy[u] = p.y; qz[u] = p.z;
                        kap[u] = kin;
                    } else {
                        P4<PT> sh = s.D[mchain * nc + cj];
                        qx[u] = p.x - sh.x; qy[u] = p.y - sh.y; qz[u] = p.z - sh.z;
                        Lj[u] = L; iLj[u] = iL;
                        kap[u] = kout;
                    }
                    C0[u] = (PT)d.C[tj];
                    C1[u] = (PT)d.C[2 + tj];
                }
            }
        }
        for (int i = 0; i < m; ++i) {
            const P4<PT> a = s.r[M.lo + i];
            const P4<PT> b = s.newr[i];
            const bool ib = a.tag & 1;
#pragma unroll
            for (int u = 0; u < R; ++u) {
                PT C = ib ? C1[u] : C0[u];
                PT e0 = lj_pair<PT>(a.x - qx[u], a.y - qy[u], a.z - qz[u], Lj[u], iLj[u], C);
                PT e1 = lj_pair<PT>(b.x - qx[u], b.y - qy[u], b.z - qz[u], Lj[u], iLj[u], C);
                acc[u] += e1 - e0;
            }
        }
#pragma unroll
        for (int u = 0; u < R; ++u) part += kap[u] * acc[u];
    }
    return (double)part;
}

// Full FP64 energy (Eq. 2 per chain + inter-chain term of Eq. 3) of the
// walker at x64; every lane of the group receives the total.
template <int TPW>
__device__ double full_energy64(const SysDesc& d, const double* x64, const Group<TPW>& g) {
    double part = 0.0;
    auto pos = [&](int j) -> double3 { return ld3(x64 + 3 * j); };
    for (int c = 0; c < d.n_chains; ++c) {
        int o = d.chain_off[c], n = d.chain_off[c + 1] - o;
        for (int k = 1 + g.lane; k <= n - 2; k += TPW) part += d.k_bend * bend_term(pos, o, k);
        for (int j = g.lane; j <= n - 4; j += TPW) part -= d.k_tors * torsion_term(pos, o, j);
    }
    for (int i = 0; i < d.N; ++i) {
        const double3 xi = pos(i);
        const int ci = d.chain_of[i], si = d.seq[i];
        for (int j = i + 1 + g.lane; j < d.N; j += TPW) {
            const int cj = d.chain_of[j];
            if (ci == cj && j < i + 2) continue;
            const double3 xj = pos(j);
            double dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
            if (ci != cj) {
                dx = mimage64(dx, d.box_L, d.inv_L);
                dy = mimage64(dy, d.box_L, d.inv_L);
                dz = mimage64(dz, d.box_L, d.inv_L);
            }
            double e = lj64(dx * dx + dy * dy + dz * dz, d.C[2 * si + d.seq[j]]);
            part += (ci == cj ? d.k_lj_intra : d.k_lj_inter) * e;
        }
    }
    return g.sum(part);
}

// Full energy with the Lennard-Jones pairs in the working precision (from the
// working copy) and the local terms in FP64 (from x64).
template <int TPW, typename PT>
__device__ double full_energy_working(const SysDesc& d, const Slot<PT>& s, const Group<TPW>& g) {
    double part = 0.0;
    auto pos = [&](int j) -> P4<PT> { return s.r[j]; };
    for (int c = 0; c < d.n_chains; ++c) {
        int o = d.chain_off[c], n = d.chain_off[c + 1] - o;
        for (int k = 1 + g.lane; k <= n - 2; k += TPW) part += (double)((PT)d.k_bend * bend_w<PT>(pos, o, k));
        for (int j = g.lane; j <= n - 4; j += TPW) part -= (double)((PT)d.k_tors * torsion_w<PT>(pos, o, j));
    }
    const PT L = (PT)d.box_L, iL = (PT)d.inv_L;
    for (int i = 0; i < d.N; ++i) {
        const P4<PT> a = s.r[i];
        const int ci = a.tag >> 1, si = a.tag & 1;
        PT row = (PT)0;
        for (int j = i + 1 + g.lane; j < d.N; j += TPW) {
            const P4<PT> b = s.r[j];
            const int cj = b.tag >> 1;
            if (ci == cj && j < i + 2) continue;
            PT dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z, Lj = 0, iLj = 0;
            if (ci != cj) {
                P4<PT> sh = s.D[ci * d.n_chains + cj];
                dx += sh.x; dy += sh.y; dz += sh.z;
                Lj = L; iLj = iL;
            }
            PT e = lj_pair<PT>(dx, dy, dz, Lj, iLj, (PT)d.C[2 * si + (b.tag & 1)]);
            row += (ci == cj ? (PT)d.k_lj_intra : (PT)d.k_lj_inter) * e;
        }
        part += (double)row;
    }
    return g.sum(part);
}
