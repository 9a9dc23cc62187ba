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
    template <typename T>
    __device__ __forceinline__ T sum0(T v) const {
#pragma unroll
        for (int o = TPW / 2; o > 0; o >>= 1) v += __shfl_down_sync(mask, v, o, TPW);
        return v;
    }
};

// Double-float value hi + lo carried in two FP32 numbers; additions keep each
// rounding error (Knuth's TwoSum), so a sum of FP32 terms loses nothing but
// the final rounding of lo.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF df_add(DF a, DF b) {
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb);
    return DF{s, e + (a.lo + b.lo)};
}
// An FP64 value as a double-float (hi its FP32 rounding, lo the rest).
__device__ __forceinline__ DF df_of(double x) {
    const float h = (float)x;
    return DF{h, (float)(x - (double)h)};
}
// Tree sum of the group's DF values; every lane receives lane 0's total.
template <int TPW>
__device__ __forceinline__ DF group_sum_df(DF v, const Group<TPW>& g) {
#pragma unroll
    for (int o = TPW / 2; o > 0; o >>= 1)
        v = df_add(v, DF{__shfl_down_sync(g.mask, v.hi, o, TPW), __shfl_down_sync(g.mask, v.lo, o, TPW)});
    return DF{__shfl_sync(g.mask, v.hi, 0, TPW), __shfl_sync(g.mask, v.lo, 0, TPW)};
}

// Shared-memory layout of one walker slot.
// An accepted move waiting for its exact FP64 replay (FP32 mode).
// Its exact amplitude and step are regenerated from the counter-based stream.
struct QEntry {
    int32_t packed;      // type | chain << 3 | index << 9
    int32_t attempt;     // winning Marsaglia attempt
    uint64_t t;          // move index (the walker stream's counter)
};
static_assert(sizeof(QEntry) == 16, "QEntry layout");
constexpr int kQueue = 32;   // accepted moves replayed per batch (at most the group's lanes)

struct SlotLayout {
    int r_off, d_off, newr_off, orig_off, new64_off, geo_off, q_off, st_off, bytes;
};
__host__ __device__ inline int align16(int x) { return (x + 15) & ~15; }
template <typename PT>
__host__ __device__ inline SlotLayout slot_layout(int N, int nc, int mc) {
    SlotLayout L;
    int o = 0;
    L.r_off = o;     o = align16(o + (int)sizeof(P4<PT>) * N);
    L.d_off = o;     o = align16(o + (int)sizeof(P4<PT>) * nc * nc);
    L.newr_off = o;  o = align16(o + 32 * mc);   // FP64: P4<double>; FP32: two float4 per moved monomer
    L.orig_off = o;  o = align16(o + 8 * 3 * nc);
    L.new64_off = o; o = align16(o + (sizeof(PT) == 8 ? 8 * 3 * mc : 0));
    L.geo_off = o;   o = align16(o + 8 * 32);
    L.q_off = o;     o = align16(o + (sizeof(PT) == 4 ? (int)sizeof(QEntry) * kQueue : 0));
    L.st_off = o;    o = align16(o + (int)sizeof(phast_walker_stats));
    L.bytes = o;
    return L;
}

// The one-walker-per-thread form's per-warp layout (lane.cuh).

// Per-warp shared-memory layout of the one-walker-per-thread sweep (bytes).
struct LaneLayout {
    int r_off, w_off, org_off, bytes;
};
template <typename PT>
__host__ __device__ inline LaneLayout lane_layout(int N, int nc, int mc) {
    LaneLayout L;
    int o = 0;
    (void)mc;
    L.r_off = o;    o += 32 * (int)sizeof(P4<PT>) * N;
    L.w_off = o;    o += 32 * 16 * nc;
    L.org_off = o;  o += 32 * 16 * nc;
    L.bytes = o;
    return L;
}

template <typename PT>
struct Slot {
    P4<PT>* r;      // [N] working positions
    P4<PT>* D;      // [nc * nc] origin differences (FP32 mode)
    P4<PT>* newr;   // [max_chain] moved monomers after the move (FP64 mode); in FP32 mode the same bytes
                    // hold two float4 per moved monomer, old and new interleaved: (xo, xn, yo, yn), (zo, zn, tag, 0),
                    // in rec_slot order (A monomers first)
    double* orig;   // [nc * 3] chain origins (FP32 mode; zero in FP64 mode)
    double* new64;  // [max_chain * 3] FP64 positions of the moved monomers after the move (FP64 mode)
    double* geo;    // [32] FP64 rotation matrix, centre, flag of a move being made exactly
    QEntry* queue;  // [kQueue] accepted moves not yet replayed in FP64 (FP32 mode)
    phast_walker_stats* st;   // this launch's counters of the walker (lane 0 writes them)
    __device__ __forceinline__ Slot(unsigned char* p, const SlotLayout& L)
        : r((P4<PT>*)(p + L.r_off)), D((P4<PT>*)(p + L.d_off)), newr((P4<PT>*)(p + L.newr_off)),
          orig((double*)(p + L.orig_off)), new64((double*)(p + L.new64_off)), geo((double*)(p + L.geo_off)),
          queue((QEntry*)(p + L.q_off)), st((phast_walker_stats*)(p + L.st_off)) {}
};


// Force-field constants in the working precision (FP32 copies live in the descriptor).
template <typename PT> struct FF;
template <> struct FF<float> {
    const SysDesc& d;
    __device__ __forceinline__ float C(int i) const { return d.C32[i]; }
    __device__ __forceinline__ float L() const { return d.L32; }
    __device__ __forceinline__ float iL() const { return d.iL32; }
    __device__ __forceinline__ float kin() const { return d.kin32; }
    __device__ __forceinline__ float kout() const { return d.kout32; }
    __device__ __forceinline__ float kbend() const { return d.kbend32; }
    __device__ __forceinline__ float ktors() const { return d.ktors32; }
};
template <> struct FF<double> {
    const SysDesc& d;
    __device__ __forceinline__ double C(int i) const { return d.C[i]; }
    __device__ __forceinline__ double L() const { return d.box_L; }
    __device__ __forceinline__ double iL() const { return d.inv_L; }
    __device__ __forceinline__ double kin() const { return d.k_lj_intra; }
    __device__ __forceinline__ double kout() const { return d.k_lj_inter; }
    __device__ __forceinline__ double kbend() const { return d.k_bend; }
    __device__ __forceinline__ double ktors() const { return d.k_tors; }
};

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

// FP32 image of the Marsaglia coordinate v = 2u - 1 from block words (a, b):
// v = ((a >> 6) - 2^25) 2^-25 + (2 (b >> 6) + 1) 2^-52, kept to within 6e-8.
__device__ __forceinline__ float sym_unit32(uint32_t a) {
    return __int2float_rn((int)(a >> 6) - (1 << 25)) * 2.98023223876953125e-8f;
}

// Disc test of one Marsaglia attempt, decided exactly as the FP64 test
// s = v1^2 + v2^2 < 1 decides it: the FP32 estimate settles every case outside
// a 1e-6 band around s = 1 (its error is below 5e-7); inside the band the FP64
// test runs.  In FP32 mode the winner's FP32 axis serves the trial move.
__device__ __forceinline__ bool disc_test(uint4 r, float* v1f, float* v2f, float* sf) {
    *v1f = sym_unit32(r.x);
    *v2f = sym_unit32(r.z);
    *sf = *v1f * *v1f + *v2f * *v2f;
    if (*sf < 1.0f - 1e-6f) return true;
    if (*sf > 1.0f + 1e-6f) return false;
    double v1, v2, sd;
    return marsaglia_in_disc(r, &v1, &v2, &sd);
}

// Draw move t: lanes compute Philox blocks 0..TPW-1 at once (blocks 0-2 are the
// selection, block 3+j is Marsaglia attempt j); lane 0 turns the selection
// blocks into the move and broadcasts it; further rounds of attempts follow
// only when the first round found no point in the disc.  The winning attempt
// index is kept; the axis is exact FP64 in FP64 mode and the FP32 image of the
// same axis in FP32 mode (whose exact axis is rebuilt at commit from the
// winning block).  The acceptance words uz, uw are valid on lane 0 only
// (u = u52(uz, uw) is formed only when the acceptance test needs it).
template <int TPW, typename PT, bool GEOM = true>
__device__ Proposal propose_group(const SysDesc& d, uint64_t seed, uint64_t t, uint4 blk, const Group<TPW>& g) {
    // blk: this lane's stream block (block index = lane) of move t
    Proposal P;
    P.angle = 0.0;
    P.disp = make_double3(0.0, 0.0, 0.0);
    P.axis = make_double3(0.0, 0.0, 1.0);
    P.angle32 = 0.0f;
    P.disp32 = make_float3(0.0f, 0.0f, 0.0f);
    P.axis32 = make_float3(0.0f, 0.0f, 1.0f);
    if constexpr (sizeof(PT) == 8) {
        uint4 b[3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
            b[i] = make_uint4(g.bcast(blk.x, i), g.bcast(blk.y, i), g.bcast(blk.z, i), g.bcast(blk.w, i));
        propose_select(d, b[0], b[1], b[2], &P);
    } else {   // selection in integers, amplitudes in FP32, on every lane: no FP64 on the trial path
        const uint32_t w0x = g.bcast(blk.x, 0), w0y = g.bcast(blk.y, 0), w0z = g.bcast(blk.z, 0),
                       w0w = g.bcast(blk.w, 0), w1x = g.bcast(blk.x, 1), w1z = g.bcast(blk.z, 1),
                       w2x = g.bcast(blk.x, 2);
        P.uz = g.bcast(blk.z, 2);
        P.uw = g.bcast(blk.w, 2);
        const uint64_t v = 2 * u52_bits(w0x, w0y) + 1;
        int type = d.last_type;
#pragma unroll
        for (int i = (GEOM ? PHAST_N_MOVES : 4) - 1; i >= 0; --i)
            if (((d.type_mask >> i) & 1) && v < d.thr[i]) type = i;
        P.type = type;
        P.chain = (int)(((uint64_t)w0z * (uint64_t)d.n_chains) >> 32);
        const int n = d.chain_off[P.chain + 1] - d.chain_off[P.chain];
        P.index = move_index(type, n, w0w);
        const float am = d.amax32[type];
        const float a0 = sym_unit32(w1x) * am;
        if (type == PHAST_TRANS) P.disp32 = make_float3(a0, sym_unit32(w1z) * am, sym_unit32(w2x) * am);
        else P.angle32 = a0;
    }
    P.attempt = -1;
    if (P.type == PHAST_PIVOT || P.type == PHAST_ROT || (GEOM && P.type == PHAST_CAP)) {
        const unsigned gm = TPW == 32 ? 0xffffffffu : ((1u << TPW) - 1u);
        uint4 mine = blk;
        int round = 0;
        float v1f = 0.f, v2f = 0.f, sf = 0.f;
        bool ok = (g.lane >= 3) && disc_test(mine, &v1f, &v2f, &sf);
        unsigned bits = (__ballot_sync(g.mask, ok) >> g.base) & gm;
        while (bits == 0 && (round + 1) * TPW <= 2 + PHAST_MARSAGLIA_TRIES) {
            ++round;
            const uint32_t blkid = (uint32_t)(round * TPW + g.lane);
            mine = stream_block<(TPW < 32 || GEOM)>(seed, t, blkid);
            ok = blkid <= 2 + PHAST_MARSAGLIA_TRIES && disc_test(mine, &v1f, &v2f, &sf);
            bits = (__ballot_sync(g.mask, ok) >> g.base) & gm;
        }
        if (bits) {
            const int src = __ffs(bits) - 1;
            P.attempt = round * TPW + src - 3;
            if (sizeof(PT) == 8) {
                double3 ax = make_double3(0.0, 0.0, 1.0);
                if (g.lane == src) {
                    double v1, v2, sd;
                    marsaglia_in_disc(mine, &v1, &v2, &sd);
                    ax = marsaglia_axis(v1, v2, sd);
                }
                P.axis = make_double3(g.bcastd(ax.x, src), g.bcastd(ax.y, src), g.bcastd(ax.z, src));
            } else {
                float q = sqrtf(fmaxf(1.0f - sf, 0.0f));
                float ax = 2.0f * v1f * q, ay = 2.0f * v2f * q, az = 1.0f - 2.0f * sf;
                ax = __shfl_sync(g.mask, ax, src, TPW);
                ay = __shfl_sync(g.mask, ay, src, TPW);
                az = __shfl_sync(g.mask, az, src, TPW);
                P.axis32 = make_float3(ax, ay, az);
            }
        }
    }
    return P;
}

// Centroid of monomers o..o+n-1 by the group, in the same summation order as
// centroid_serial (32 strided partial sums, halved by w = 16 .. 1); every lane
// receives it.
template <int TPW>
__device__ double3 centroid_tree(const double* x64, int o, int n, const Group<TPW>& g) {
    constexpr int V = 32 / TPW;   // partials l = lane + v TPW held by this lane
    double c[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double part[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            part[v] = 0.0;
            for (int j = g.lane + v * TPW; j < n; j += 32) part[v] = xadd(part[v], x64[3 * (o + j) + d]);
        }
#pragma unroll
        for (int w = 16; w >= TPW; w /= 2)
#pragma unroll
            for (int v = 0; v < w / TPW; ++v) part[v] = xadd(part[v], part[v + w / TPW]);
        double sum = part[0];
#pragma unroll
        for (int w = (TPW < 32 ? TPW : 32) / 2; w >= 1; w /= 2) sum = xadd(sum, __shfl_down_sync(g.mask, sum, w, TPW));
        c[d] = g.bcastd(xdiv(sum, (double)n), 0);
    }
    return make_double3(c[0], c[1], c[2]);
}

// Exact FP64 axis of a pivot or rotation: the winning Marsaglia attempt replayed.
template <bool OUTLINE = false>
__device__ __forceinline__ double3 exact_axis(uint64_t seed, uint64_t t, int attempt) {
    if (attempt < 0) return make_double3(0.0, 0.0, 1.0);
    double v1, v2, s;
    marsaglia_in_disc(stream_block<OUTLINE>(seed, t, 3u + (uint32_t)attempt), &v1, &v2, &s);
    return marsaglia_axis(v1, v2, s);
}

// Moved range and the unmoved monomers whose pair with a moved one is left
// out (the pivot keeps its distances; a crankshaft's bonded neighbours).
// Moved range [lo, hi], up to three excluded partners, and the A monomers of
// the range: a_lo of them before lo in the system, n_a inside it.
struct MoveSet { int lo, hi, ex0, ex1, ex2, a_lo, n_a; };
__device__ __forceinline__ MoveSet move_set(const SysDesc& d, int type, int chain, int index) {
    MoveSet M;
    int fixed;
    moved_range(d, type, chain, index, &M.lo, &M.hi, &fixed);
    // partners left out: the pivot (its distances to the rotated side keep) and,
    // for one moved monomer (crankshaft, cap), its bonded neighbours.  A
    // bond-length move keeps every partner; its one bonded pair is taken back
    // out in local_delta.
    const int o = d.chain_off[chain], e = d.chain_off[chain + 1] - 1;
    const bool single = type == PHAST_CRANK || type == PHAST_CAP;
    M.ex0 = fixed;
    M.ex1 = (single && M.lo - 1 >= o) ? M.lo - 1 : -1;
    M.ex2 = (single && M.hi + 1 <= e) ? M.hi + 1 : -1;
    M.a_lo = d.n_a_before[M.lo];
    M.n_a = d.n_a_before[M.hi + 1] - M.a_lo;
    return M;
}

// Record slot of moved monomer j in the FP32 trial records: the A monomers of
// the moved range first, then the B monomers, each in chain order, so that the
// pair loop runs over each type with its Lennard-Jones constants fixed.
__device__ __forceinline__ int rec_slot(const SysDesc& d, const MoveSet& M, int j) {
    const int a = d.n_a_before[j] - M.a_lo;
    return d.seq[j] ? M.n_a + (j - M.lo - a) : a;
}

// Pair evaluations of a move between different chains (2 per pair).
__device__ __forceinline__ uint64_t move_pair_evals_inter(const SysDesc& d, int type, int chain, const MoveSet& M) {
    const int nc = d.chain_off[chain + 1] - d.chain_off[chain];
    const int m = M.hi - M.lo + 1;
    return 2ull * m * (d.N - nc);
}

// Pair evaluations a move costs (2 per changed Lennard-Jones pair).
__device__ __forceinline__ uint64_t move_pair_evals(const SysDesc& d, int type, const MoveSet& M) {
    const int m = M.hi - M.lo + 1;
    if (type == PHAST_BOND) return 2ull * ((uint64_t)m * (d.N - m) - 1);   // all but the bonded pair
    const int excluded = (M.ex0 >= 0) + (M.ex1 >= 0) + (M.ex2 >= 0);
    return 2ull * m * (d.N - m - excluded);
}

// Lane 0 builds the move's exact centre and rotation (FP64, bit-reproducible)
// into the slot's geo scratch: geo[0..8] R, geo[9..11] centre, geo[12] 1 (0 for
// a degenerate crankshaft axis or bond step); for a bond-length move geo[13..15]
// the step and geo[16] its Hastings factor.  axis64 is the exact axis of a
// pivot or rotation.
template <int TPW, typename PT>
__device__ bool prepare_exact(const SysDesc& d, const double* x64, const Proposal& P, double3 axis64, Slot<PT>& s,
                              const Group<TPW>& g) {
    const int c = P.chain, o = d.chain_off[c], n = d.chain_off[c + 1] - o;
    double3 rot_center = make_double3(0.0, 0.0, 0.0);
    if (P.type == PHAST_ROT) rot_center = centroid_tree<TPW>(x64, o, n, g);
    if (P.type == PHAST_BOND && g.lane == 0) {   // the slide of the moved side
        double3 step = make_double3(0.0, 0.0, 0.0);
        double jac = 1.0;
        s.geo[12] = bond_step(x64, o, n, P.index, P.angle, &step, &jac) ? 1.0 : 0.0;
        s.geo[13] = step.x;
        s.geo[14] = step.y;
        s.geo[15] = step.z;
        s.geo[16] = jac;
    } else if (P.type != PHAST_TRANS && g.lane == 0) {
        double3 axis = axis64, center;
        double ok = 1.0;
        if (P.type == PHAST_PIVOT) {
            center = ld3(x64 + 3 * (o + P.index));
        } else if (P.type == PHAST_CAP) {   // about the bonded neighbour i-1 (monomer 1 for i = 0)
            center = ld3(x64 + 3 * (o + (P.index > 0 ? P.index - 1 : 1)));
        } else if (P.type == PHAST_ROT) {
            center = rot_center;
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
    return P.type == PHAST_TRANS || s.geo[12] != 0.0;
}

// Exact FP64 position of a moved monomer after the move (the geometry every
// implementation of the method reproduces bit for bit).
__device__ __forceinline__ double3 exact_position(const Proposal& P, const double* geo, double3 x) {
    if (P.type == PHAST_TRANS)
        return make_double3(xadd(x.x, P.disp.x), xadd(x.y, P.disp.y), xadd(x.z, P.disp.z));
    if (P.type == PHAST_BOND)
        return make_double3(xadd(x.x, geo[13]), xadd(x.y, geo[14]), xadd(x.z, geo[15]));
    Rot3 R;
#pragma unroll
    for (int k = 0; k < 9; ++k) R.m[k] = geo[k];
    return rotate_about(R, make_double3(geo[9], geo[10], geo[11]), x);
}

// sin and cos of |a| <= 1 in FP32 (Taylor to a^13 / a^12), for trial moves.
__device__ __forceinline__ void sincos32(float a, float* s, float* c) {
    const float x2 = a * a;
    float ps = fmaf(x2, 1.6059043836821614e-10f, -2.5052108385441720e-8f);
    ps = fmaf(x2, ps, 2.7557319223985893e-6f);
    ps = fmaf(x2, ps, -1.9841269841269841e-4f);
    ps = fmaf(x2, ps, 8.3333333333333333e-3f);
    ps = fmaf(x2, ps, -1.6666666666666667e-1f);
    *s = fmaf(a * x2, ps, a);
    float pc = fmaf(x2, 2.0876756987868099e-9f, -2.7557319223985893e-7f);
    pc = fmaf(x2, pc, 2.4801587301587302e-5f);
    pc = fmaf(x2, pc, -1.3888888888888889e-3f);
    pc = fmaf(x2, pc, 4.1666666666666667e-2f);
    pc = fmaf(x2, pc, -0.5f);
    *c = fmaf(x2, pc, 1.0f);
}

// Trial positions of the moved monomers in the working precision (newr).
// FP64 mode: the exact FP64 positions (also kept in new64).  FP32 mode: the
// FP32 relative coordinates moved by an FP32 rotation or translation built
// from FP32 data only; the exact FP64 move is made only when it is accepted
// (commit_move).  Returns false for a degenerate crankshaft axis or bond step.
// *jac (bond-length moves, when given): the Hastings factor ((r + delta) / r)^2,
// exact in FP64 mode, from the FP32 bond length in FP32 mode.
template <int TPW, typename PT, bool GEOM = true>
__device__ bool make_new_positions(const SysDesc& d, const double* x64, const Proposal& P, const MoveSet& M,
                                   Slot<PT>& s, const Group<TPW>& g, double* jac = nullptr) {
    const int m = M.hi - M.lo + 1;
    const int c = P.chain, o = d.chain_off[c], n = d.chain_off[c + 1] - o;
    if constexpr (sizeof(PT) == 8) {
        if (!prepare_exact<TPW, PT>(d, x64, P, P.axis, s, g)) return false;
        if (GEOM && jac && P.type == PHAST_BOND) *jac = s.geo[16];
        for (int q = g.lane; q < m; q += TPW) {
            const int j = M.lo + q;
            const double3 y = exact_position(P, s.geo, ld3(x64 + 3 * j));
            s.new64[3 * q + 0] = y.x;
            s.new64[3 * q + 1] = y.y;
            s.new64[3 * q + 2] = y.z;
            P4<PT> w;
            w.x = y.x;
            w.y = y.y;
            w.z = y.z;
            w.tag = (int)d.seq[j] | (c << 1);
            s.newr[q] = w;
        }
        g.sync();
        return true;
    } else {
        float4* mv = reinterpret_cast<float4*>(s.newr);
        if (P.type == PHAST_TRANS || (GEOM && P.type == PHAST_BOND)) {
            float dx = P.disp32.x, dy = P.disp32.y, dz = P.disp32.z;
            if (GEOM && P.type == PHAST_BOND) {   // slide along the FP32 unit bond vector
                const P4<PT> a = s.r[o + P.index], b = s.r[o + P.index + 1];
                const float bx = b.x - a.x, by = b.y - a.y, bz = b.z - a.z;
                const float len = sqrtf(bx * bx + by * by + bz * bz);
                if (!(len > 1e-12f) || !(len + P.angle32 > 0.0f)) return false;
                if (jac) {
                    const float q = (len + P.angle32) / len;
                    *jac = (double)(q * q);
                }
                const float dl = (P.index + 1 < n - 1 - P.index) ? -P.angle32 : P.angle32;
                dx = dl * (bx / len);
                dy = dl * (by / len);
                dz = dl * (bz / len);
            }
            for (int q = g.lane; q < m; q += TPW) {
                const P4<PT> w = s.r[M.lo + q];
                const float nx = w.x + dx, ny = w.y + dy, nz = w.z + dz;
                const int k = rec_slot(d, M, M.lo + q);
                mv[2 * k] = make_float4(w.x, nx, w.y, ny);
                mv[2 * k + 1] = make_float4(w.z, nz, __int_as_float(w.tag), 0.0f);
            }
        } else {
            float kx = P.axis32.x, ky = P.axis32.y, kz = P.axis32.z, cx, cy, cz;
            if (P.type == PHAST_PIVOT || (GEOM && P.type == PHAST_CAP)) {
                const P4<PT> p = s.r[o + (P.type == PHAST_PIVOT ? P.index : (P.index > 0 ? P.index - 1 : 1))];
                cx = p.x; cy = p.y; cz = p.z;
            } else if (P.type == PHAST_ROT) {
                cx = cy = cz = 0.0f;
                for (int j = o + g.lane; j < o + n; j += TPW) {
                    const P4<PT> p = s.r[j];
                    cx += p.x; cy += p.y; cz += p.z;
                }
#pragma unroll
                for (int w = TPW / 2; w > 0; w >>= 1) {
                    cx += __shfl_xor_sync(g.mask, cx, w, TPW);
                    cy += __shfl_xor_sync(g.mask, cy, w, TPW);
                    cz += __shfl_xor_sync(g.mask, cz, w, TPW);
                }
                const float inv = 1.0f / (float)n;
                cx *= inv; cy *= inv; cz *= inv;
            } else {
                const P4<PT> a = s.r[o + P.index - 1], b = s.r[o + P.index + 1];
                const float ex = b.x - a.x, ey = b.y - a.y, ez = b.z - a.z;
                const float len = sqrtf(ex * ex + ey * ey + ez * ez);
                if (!(len > 1e-12f)) return false;
                kx = ex / len; ky = ey / len; kz = ez / len;
                cx = a.x; cy = a.y; cz = a.z;
            }
            float sn, cs;
            sincos32(P.angle32, &sn, &cs);
            const float tt = 1.0f - cs;
            const float r0 = tt * kx * kx + cs, r1 = tt * kx * ky - sn * kz, r2 = tt * kx * kz + sn * ky;
            const float r3 = tt * ky * kx + sn * kz, r4 = tt * ky * ky + cs, r5 = tt * ky * kz - sn * kx;
            const float r6 = tt * kz * kx - sn * ky, r7 = tt * kz * ky + sn * kx, r8 = tt * kz * kz + cs;
            for (int q = g.lane; q < m; q += TPW) {
                const P4<PT> w = s.r[M.lo + q];
                const float vx = w.x - cx, vy = w.y - cy, vz = w.z - cz;
                const float nx = cx + (r0 * vx + r1 * vy + r2 * vz);
                const float ny = cy + (r3 * vx + r4 * vy + r5 * vz);
                const float nz = cz + (r6 * vx + r7 * vy + r8 * vz);
                const int k = rec_slot(d, M, M.lo + q);
                mv[2 * k] = make_float4(w.x, nx, w.y, ny);
                mv[2 * k + 1] = make_float4(w.z, nz, __int_as_float(w.tag), 0.0f);
            }
        }
        g.sync();
        return true;
    }
}

// Steric container: every moved monomer's trial position inside the sphere,
// decided as the FP64 test (x^2 + y^2) + z^2 <= R^2 on the exact position.
// FP32 mode estimates |origin + r|^2 from the trial record (error far below
// 1e-5 R^2) and builds the exact positions only when a monomer is that close
// to the wall.  The same value on every lane of the group.
// exact: P carries the exact FP64 move (else it is regenerated from the
// walker's stream, key seed and move index t, as the replay does).
// queued (FP32 sweep): accepted moves not yet replayed on x64; they are
// replayed first, so that the exact test sees the current coordinates.
// Kept out of line: the check runs only with a container, and its code stays
// out of the instruction stream of the moves that need none.
template <int TPW, bool GEOM = true>
__device__ __noinline__ void flush_queue(const SysDesc& d, double* x64, uint64_t seed, Slot<float>& s, const Group<TPW>& g,
                                         int count);

template <int TPW, typename PT>
__device__ __noinline__ bool container_ok(const SysDesc& d, double* x64, const Proposal& P, const MoveSet& M,
                                          Slot<PT>& s, const Group<TPW>& g, bool exact, uint64_t seed, uint64_t t,
                                          int* queued) {
    if (!d.has_sphere) return true;
    const int m = M.hi - M.lo + 1;
    const unsigned gm = TPW == 32 ? 0xffffffffu : ((1u << TPW) - 1u);
    bool out = false, unsure = false;
    if constexpr (sizeof(PT) == 8) {
        for (int q = g.lane; q < m; q += TPW)
            out |= !inside64(d, make_double3(s.new64[3 * q], s.new64[3 * q + 1], s.new64[3 * q + 2]));
    } else {
        const float4* mv = reinterpret_cast<const float4*>(s.newr);
        const int c = P.chain;
        const float ox = (float)s.orig[3 * c], oy = (float)s.orig[3 * c + 1], oz = (float)s.orig[3 * c + 2];
        const float R2 = d.sphere_R2_32, band = 1e-5f * R2;
        for (int q = g.lane; q < m; q += TPW) {
            const int k = rec_slot(d, M, M.lo + q);
            const float4 A = mv[2 * k], B = mv[2 * k + 1];
            const float x = ox + A.y, y = oy + A.w, z = oz + B.y;
            // one difference decides both tests (exact for r2 near R2), so the two
            // cover the line without a gap: a separately rounded R2 + band could
            // leave r2 - R2 just above band counted neither out nor unsure
            const float e = (x * x + y * y + z * z) - R2;
            out |= e > band;
            unsure |= fabsf(e) <= band;
        }
        if ((__ballot_sync(g.mask, unsure) >> g.base) & gm) {   // near the wall: the exact positions decide
            if (queued && *queued > 0) {
                flush_queue<TPW, true>(d, x64, seed, s, g, *queued);
                *queued = 0;
            }
            Proposal E = P;
            if (!exact) {
                propose_select(d, stream_block(seed, t, 0u), stream_block(seed, t, 1u), stream_block(seed, t, 2u), &E);
                if (E.type == PHAST_PIVOT || E.type == PHAST_ROT || E.type == PHAST_CAP)
                    E.axis = exact_axis(seed, t, P.attempt);
            }
            const bool ok_geo = prepare_exact<TPW, PT>(d, x64, E, E.axis, s, g);
            if (ok_geo)
                for (int q = g.lane; q < m; q += TPW)
                    out |= !inside64(d, exact_position(E, s.geo, ld3(x64 + 3 * (M.lo + q))));
        }
    }
    return ((__ballot_sync(g.mask, out) >> g.base) & gm) == 0u;
}

// Local terms of a move in FP64 on the exact positions, for FP32 mode: the
// FENE change (fene; when one of its terms lies in the band of fene_w) and the
// torsion change of the move's window (tors; when a dihedral lies in the band of
// torsion_w), summed (+inf for a bond beyond its range, NaN for an exact
// geometry that is no move).  exact, seed, t and queued as for container_ok:
// the queued moves are replayed first, so that x64 holds the current
// coordinates.  The same value on every lane of the group.  Out of line, as
// container_ok.
template <int TPW, bool GEOM>
__device__ __noinline__ double local_delta_exact(const SysDesc& d, double* x64, const Proposal& P, const MoveSet& M,
                                                 Slot<float>& s, const Group<TPW>& g, bool exact, uint64_t seed,
                                                 uint64_t t, int* queued, bool fene, bool tors) {
    if (queued && *queued > 0) {
        flush_queue<TPW, GEOM>(d, x64, seed, s, g, *queued);
        *queued = 0;
    }
    Proposal E = P;
    if (!exact) {
        propose_select(d, stream_block(seed, t, 0u), stream_block(seed, t, 1u), stream_block(seed, t, 2u), &E);
        if (E.type == PHAST_PIVOT || E.type == PHAST_ROT || E.type == PHAST_CAP)
            E.axis = exact_axis(seed, t, P.attempt);
    }
    const bool ok = prepare_exact<TPW, float>(d, x64, E, E.axis, s, g);
    int vb0, nb, jt0, nt, fb0, nf;
    local_window(d, P.type, P.chain, P.index, &vb0, &nb, &jt0, &nt, &fb0, &nf);
    const int o = d.chain_off[P.chain];
    const int nF = fene ? 2 * nf : 0, nT = tors ? 2 * nt : 0;
    double part = 0.0;
    if (ok)
        for (int k = g.lane; k < nF + nT; k += TPW) {
            const bool after = k & 1;
            auto pos = [&](int j) -> double3 {
                const double3 x = ld3(x64 + 3 * j);
                return (after && j >= M.lo && j <= M.hi) ? exact_position(E, s.geo, x) : x;
            };
            const double v = k < nF ? fene_term(d, pos, o, fb0 + (k >> 1))
                                    : -d.k_tors * torsion_term(pos, o, jt0 + ((k - nF) >> 1));
            part += after ? v : -v;
        }
    const double dX = g.sum(part);
    return ok ? dX : __longlong_as_double(0x7ff8000000000000ll);
}

// Commit an accepted move in FP64 mode: the exact positions computed for the
// trial become the master coordinates and the working copy.
template <int TPW>
__device__ void commit_move64(double* x64, const MoveSet& M, Slot<double>& s, const Group<TPW>& g) {
    const int m = M.hi - M.lo + 1;
    for (int q = g.lane; q < m; q += TPW) {
        const int j = M.lo + q;
        x64[3 * j + 0] = s.new64[3 * q + 0];
        x64[3 * j + 1] = s.new64[3 * q + 1];
        x64[3 * j + 2] = s.new64[3 * q + 2];
        s.r[j] = s.newr[q];
    }
}

// Accept a move in FP32 mode: the working copy takes the trial positions at
// once (a translated chain keeps them and moves its origin instead), and the
// move joins the queue whose exact FP64 replay flush_queue makes later.
template <int TPW>
__device__ void accept_move32(const SysDesc& d, const Proposal& P, uint64_t t, const MoveSet& M, Slot<float>& s,
                              const Group<TPW>& g, int count) {
    if (g.lane == 0) {
        QEntry e;
        e.packed = P.type | (P.chain << 3) | (P.index << 9);
        e.attempt = P.attempt;
        e.t = t;
        s.queue[count] = e;
    }
    if (P.type == PHAST_TRANS) {   // the origin moves by the FP32 step the trial used
        rebase_translated<TPW, float>(d, P.chain, make_double3(P.disp32.x, P.disp32.y, P.disp32.z), s, g);
        return;
    }
    const int m = M.hi - M.lo + 1;
    const float4* mv = reinterpret_cast<const float4*>(s.newr);
    for (int q = g.lane; q < m; q += TPW) {
        const int k = rec_slot(d, M, M.lo + q);
        const float4 A = mv[2 * k], B = mv[2 * k + 1];
        P4<float> w = s.r[M.lo + q];
        w.x = A.y;
        w.y = A.w;
        w.z = B.y;
        s.r[M.lo + q] = w;
    }
}

// Replay the queued accepted moves exactly, in order, on the FP64 master
// coordinates.  The state-independent part of each rotation (the winning
// Marsaglia axis, sin/cos, Rodrigues' matrix) is built for all queued moves at
// once, one move per lane; centres are read from the coordinates as each move
// is made.  Then the working copy of the chains they moved is refreshed from
// the exact coordinates.
template <int TPW, bool GEOM>
__device__ __noinline__ void flush_queue(const SysDesc& d, double* x64, uint64_t seed, Slot<float>& s, const Group<TPW>& g,
                            int count) {
    if (count == 0) return;
    g.sync();
    Rot3 Rl;
    double3 dl = make_double3(0.0, 0.0, 0.0);   // exact step (translations) or angle in .x (crankshafts)
    if (g.lane < count) {   // the exact proposal of queued move `lane`, regenerated from its stream blocks
        const QEntry e = s.queue[g.lane];
        Proposal Q;
        constexpr bool OUT = TPW < 32 || GEOM;
        propose_select(d, stream_block<OUT>(seed, e.t, 0u), stream_block<OUT>(seed, e.t, 1u),
                       stream_block<OUT>(seed, e.t, 2u), &Q);
        if constexpr (!GEOM) __builtin_assume(Q.type >= 0 && Q.type < PHAST_BOND);
        if (Q.type == PHAST_PIVOT || Q.type == PHAST_ROT || Q.type == PHAST_CAP) {
            const double3 ax = exact_axis<OUT>(seed, e.t, e.attempt);
            double sn, cs;
            taylor_sincos(Q.angle, &sn, &cs);
            Rl = rodrigues(ax.x, ax.y, ax.z, sn, cs);
        } else if (Q.type == PHAST_TRANS) {
            dl = Q.disp;
        } else {   // crankshaft angle, bond-length step
            dl.x = Q.angle;
        }
    }
    for (int k = 0; k < count; ++k) {
        const QEntry e = s.queue[k];
        Proposal P;
        P.type = e.packed & 7;
        P.chain = (e.packed >> 3) & 63;
        P.index = e.packed >> 9;
        if constexpr (!GEOM) __builtin_assume(P.type < PHAST_BOND);
        P.attempt = e.attempt;
        P.angle = 0.0;
        P.disp = make_double3(0.0, 0.0, 0.0);
        P.axis = make_double3(0.0, 0.0, 1.0);
        if (P.type == PHAST_TRANS) P.disp = make_double3(g.bcastd(dl.x, k), g.bcastd(dl.y, k), g.bcastd(dl.z, k));
        if (P.type == PHAST_CRANK || P.type == PHAST_BOND) P.angle = g.bcastd(dl.x, k);
        const MoveSet M = move_set(d, P.type, P.chain, P.index);
        const int m = M.hi - M.lo + 1;
        const int o = d.chain_off[P.chain], n = d.chain_off[P.chain + 1] - o;
        Rot3 R;
        double3 center = make_double3(0.0, 0.0, 0.0);
        bool ok = true;
        double3 step = P.disp;
        if (P.type == PHAST_PIVOT || P.type == PHAST_ROT || P.type == PHAST_CAP) {
#pragma unroll
            for (int q = 0; q < 9; ++q) R.m[q] = g.bcastd(Rl.m[q], k);
            if (P.type == PHAST_ROT) center = centroid_tree<TPW>(x64, o, n, g);
            else center = ld3(x64 + 3 * (o + (P.type == PHAST_PIVOT ? P.index : (P.index > 0 ? P.index - 1 : 1))));
        } else if (P.type == PHAST_CRANK || P.type == PHAST_BOND) {   // axis / slide depend on the coordinates
            ok = prepare_exact<TPW, float>(d, x64, P, P.axis, s, g);
#pragma unroll
            for (int q = 0; q < 9; ++q) R.m[q] = s.geo[q];
            center = make_double3(s.geo[9], s.geo[10], s.geo[11]);
            step = make_double3(s.geo[13], s.geo[14], s.geo[15]);
        }
        if (ok) {
            for (int q = g.lane; q < m; q += TPW) {
                const int j = M.lo + q;
                const double3 x = ld3(x64 + 3 * j);
                double3 y;
                if (P.type == PHAST_TRANS || P.type == PHAST_BOND)
                    y = make_double3(xadd(x.x, step.x), xadd(x.y, step.y), xadd(x.z, step.z));
                else
                    y = rotate_about(R, center, x);
                x64[3 * j + 0] = y.x;
                x64[3 * j + 1] = y.y;
                x64[3 * j + 2] = y.z;
            }
        }
        g.sync();
    }
    uint32_t touched = 0;   // only the chains the replayed moves changed
    for (int k = 0; k < count; ++k) touched |= 1u << ((s.queue[k].packed >> 3) & 63);
    for (int j = g.lane; j < d.N; j += TPW) {
        const int c = d.chain_of[j];
        if (!((touched >> c) & 1)) continue;
        P4<float> w = s.r[j];
        w.x = (float)(x64[3 * j + 0] - s.orig[3 * c + 0]);
        w.y = (float)(x64[3 * j + 1] - s.orig[3 * c + 1]);
        w.z = (float)(x64[3 * j + 2] - s.orig[3 * c + 2]);
        s.r[j] = w;
    }
    g.sync();
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

// An FP32 dihedral whose normals FP32 cannot resolve.  The FP64 term is 0 for a
// degenerate dihedral (n1^2 n2^2 < 1e-20, so one normal has n^2 < 1e-10: collinear
// bonds, as in a chain that started straight and keeps straight stretches under
// pivot moves), but FP32 coordinates carry rounding of half an ulp of their
// magnitude (a few ulp for the FP32 trial positions of a rotation), which leaves
// the normal of a collinear pair of unit bonds with a length of a few to some
// tens of ulp and a meaningless direction, and an FP32 cos tau of a normal n
// carries an error of about that noise over |n|.  A normal with n^2 below
// max((32 ulp)^2, floor), the ulp that of the largest coordinate of the four
// monomers, marks the term: wide (the builds with an exact FP64 path) takes the
// floor 1e-6 (bonds within ~0.06 degrees of collinear), narrow (the build
// without it, where a marked term counts as degenerate) 1e-10.  A dihedral that is that close to degenerate
// without being degenerate (a bend under ~6e-5 rad for a 55-mer) has a
// probability of order 1e-9 under continuous moves of a chain that did not start
// straight; the host runs contexts whose chains start straight in a build with
// the exact path.
__device__ __forceinline__ bool torsion_unresolved32(float n11, float n22, float mx, bool wide) {
    const float u = __int_as_float(((__float_as_int(fmaxf(mx, 1.0f)) >> 23) - 23) << 23);   // ulp of mx
    const float tau = fmaxf(1024.0f * u * u, wide ? 1e-6f : 1e-10f);
    return fminf(n11, n22) < tau;
}

// cos tau_j in the working precision.  near (FP32 only): a dihedral FP32 cannot
// resolve (torsion_unresolved32) sets *near and counts 0, for the caller to
// replace by the exact FP64 term or to take as degenerate.
template <typename PT, class Pos>
__device__ __forceinline__ PT torsion_w(const Pos& pos, int o, int j, bool* near = nullptr, bool wide = true) {
    const P4<PT> x0 = pos(o + j), x1 = pos(o + j + 1), x2 = pos(o + j + 2), x3 = pos(o + j + 3);
    const PT b0x = x1.x - x0.x, b0y = x1.y - x0.y, b0z = x1.z - x0.z;
    const PT b1x = x2.x - x1.x, b1y = x2.y - x1.y, b1z = x2.z - x1.z;
    const PT b2x = x3.x - x2.x, b2y = x3.y - x2.y, b2z = x3.z - x2.z;
    const PT n1x = b0y * b1z - b0z * b1y, n1y = b0z * b1x - b0x * b1z, n1z = b0x * b1y - b0y * b1x;
    const PT n2x = b1y * b2z - b1z * b2y, n2y = b1z * b2x - b1x * b2z, n2z = b1x * b2y - b1y * b2x;
    const PT n12 = n1x * n2x + n1y * n2y + n1z * n2z;
    const PT n11 = n1x * n1x + n1y * n1y + n1z * n1z, n22 = n2x * n2x + n2y * n2y + n2z * n2z;
    if constexpr (sizeof(PT) == 4) {
        if (near) {
            float mx = fmaxf(fmaxf(fabsf(x0.x), fabsf(x0.y)), fabsf(x0.z));
            mx = fmaxf(mx, fmaxf(fmaxf(fabsf(x1.x), fabsf(x1.y)), fabsf(x1.z)));
            mx = fmaxf(mx, fmaxf(fmaxf(fabsf(x2.x), fabsf(x2.y)), fabsf(x2.z)));
            mx = fmaxf(mx, fmaxf(fmaxf(fabsf(x3.x), fabsf(x3.y)), fabsf(x3.z)));
            if (torsion_unresolved32(n11, n22, mx, wide)) {
                *near = true;
                return (PT)0;
            }
        }
    }
    if (n11 * n22 < (PT)1e-20) return (PT)0;
    if (sizeof(PT) == 8) return n12 / (sqrt(n11) * sqrt(n22));
    return n12 * rsqrt_w(n11 * n22);
}

// Band of x^2 = ((r - r0) / R)^2 where an FP32 FENE term is not trusted: the
// FP32 working copy carries ~1e-5 of error in x^2, against a divergence at
// x^2 = 1 that FP64 resolves to ~1e-16, and each term's error grows as
// 1 / (1 - x^2).  Inside the band the exact positions decide (and give the term).
constexpr float kFeneExactLo = 0.99f, kFeneExactHi = 1.01f;

// FENE term of bond l in the working precision:
// k_fene R^2 C_F ln(1 - ((r - r0) / R)^2), +inf outside |r - r0| < R.
// near (FP32 only): a term inside the band [kFeneExactLo, kFeneExactHi) of x^2
// sets *near and counts 0, for the caller to replace by the exact FP64 term.
template <typename PT, class Pos>
__device__ __forceinline__ PT fene_w(const SysDesc& d, const Pos& pos, int o, int l, bool* near = nullptr) {
    const P4<PT> a = pos(o + l), b = pos(o + l + 1);
    const PT dx = b.x - a.x, dy = b.y - a.y, dz = b.z - a.z;
    const PT r = sqrt(dx * dx + dy * dy + dz * dz);
    if constexpr (sizeof(PT) == 8) {   // one FP64 implementation for every FP64 path
        (void)r;
        return fene_term(d, [&](int j) { const P4<PT> p = pos(j); return make_double3(p.x, p.y, p.z); }, o, l);
    } else {
        const float x = (r - d.fene_r0_32) * d.fene_iR32;
        const float x2 = x * x;
        if (near && x2 >= kFeneExactLo) {
            if (!(x2 < kFeneExactHi)) return INFINITY;   // beyond the range by far more than the FP32 error
            *near = true;
            return 0.0f;
        }
        if (!(x2 < 1.0f)) return INFINITY;
        return d.fene_kR2_32 * (d.C_F32[2 * d.seq[o + l] + d.seq[o + l + 1]] * log1pf(-x2));
    }
}

// This lane's share of the bending/torsion change, in the working precision.
template <typename PT>
__device__ __forceinline__ PT lj_pair(PT dx, PT dy, PT dz, PT Lj, PT iLj, PT C);

// A FENE bond term of monomers (l, l + 1) at positions a, b (fene), or minus
// the Lennard-Jones term of that pair (the bonded pair of a bond move).
// near: as for fene_w.
template <typename PT>
__device__ __noinline__ PT bond_item(const SysDesc& d, bool fene, P4<PT> a, P4<PT> b, int l, bool* near = nullptr) {
    const FF<PT> f{d};
    if (fene) {
        auto pos2 = [&](int j) -> P4<PT> { return j == l ? a : b; };
        return fene_w<PT>(d, pos2, l, 0, near);
    }
    return -f.kin() * lj_pair<PT>(a.x - b.x, a.y - b.y, a.z - b.z, (PT)0, (PT)0, f.C(2 * d.seq[l] + d.seq[l + 1]));
}

// fene (FP32): the FENE terms go to *fene rather than into the returned part,
// and *near is set where one of them lies in the band of fene_w.  tors (FP32):
// likewise the torsion terms go to *tors, and *tnear is set where a dihedral
// lies in the band of torsion_w.
template <int TPW, typename PT, bool GEOM = true>
__device__ PT local_delta(const SysDesc& d, const Proposal& P, const MoveSet& M, const Slot<PT>& s,
                              const Group<TPW>& g, PT* fene = nullptr, bool* near = nullptr, PT* tors = nullptr,
                              bool* tnear = nullptr) {
    int vb0, nb, jt0, nt, fb0, nf;
    local_window(d, P.type, P.chain, P.index, &vb0, &nb, &jt0, &nt, &fb0, &nf);
    const int o = d.chain_off[P.chain];
    if (!GEOM) nf = 0;
    const int nc = GEOM && P.type == PHAST_BOND;   // the stretched bond's pair, counted by the pair loop, taken back
    const int items = 2 * (nb + nt + nf + nc);
    PT part = (PT)0;
    for (int it = g.lane; it < items; it += TPW) {
        const bool after = it & 1;
        const int k = it >> 1;
        auto pos = [&](int j) -> P4<PT> {
            if (after && j >= M.lo && j <= M.hi) {
                if constexpr (sizeof(PT) == 4) {
                    const float4* mv = reinterpret_cast<const float4*>(s.newr) + 2 * rec_slot(d, M, j);
                    const float4 a = mv[0], b = mv[1];
                    P4<PT> w;
                    w.x = a.y; w.y = a.w; w.z = b.y; w.tag = __float_as_int(b.z);
                    return w;
                } else {
                    return s.newr[j - M.lo];
                }
            }
            return s.r[j];
        };
        const FF<PT> f{d};
        PT term;
        if (k < nb) term = f.kbend() * bend_w<PT>(pos, o, vb0 + k);
        else if (k < nb + nt) {
            if (sizeof(PT) == 4 && tors) {
                const PT v = -f.ktors() * torsion_w<PT>(pos, o, jt0 + (k - nb), tnear, GEOM);
                *tors += after ? v : -v;
                continue;
            }
            term = -f.ktors() * torsion_w<PT>(pos, o, jt0 + (k - nb));
        } else {   // a FENE bond or the bond move's pair: out of line (most workloads have neither)
            const bool is_fene = k < nb + nt + nf;
            const int l = o + (is_fene ? fb0 + (k - nb - nt) : P.index);   // the bond's first monomer
            term = bond_item<PT>(d, is_fene, pos(l), pos(l + 1), l, fene ? near : nullptr);
            if (is_fene && fene) {
                *fene += after ? term : -term;
                continue;
            }
        }
        part += after ? term : -term;
    }
    return part;
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

// FP32 pair loop.  Old and new evaluations of a pair travel together as the
// two halves of one paired FP32 instruction (add/mul/fma .f32x2), from the
// interleaved (old, new) records of the moved monomers, A monomers first.
// Partners t = lane, lane + TPW, ... (skipping the moved range) are held RR at
// a time in registers; the ragged tail runs one at a time so no register slot
// idles.  PBC: partners on other chains take the minimum image by the nearest
// integer count of box lengths, rounded on the FMA pipe by the 1.5 * 2^23
// constant (three paired instructions per component; the special-function unit
// keeps only the reciprocal).
template <int RR, bool PBC>
__device__ __forceinline__ float pair_chunk32(const SysDesc& d, const MoveSet& M, int mchain, int m, int t0,
                                              int stride, const P4<float>* __restrict__ r,
                                              const P4<float>* __restrict__ D, const float4* __restrict__ mv,
                                              int sub = 0, int step = 1) {
    // moved monomers i = sub, sub + step, ... of each type segment (step > 1: a
    // partner shared by `step` lanes in the ragged tail)
    const int nc = d.n_chains;
    float2 nqx[RR], nqy[RR], nqz[RR], nC0[RR], nC1[RR], nL[RR], iL[RR], acc[RR];
    float kap[RR];
#pragma unroll
    for (int u = 0; u < RR; ++u) {
        const int t = t0 + u * stride;
        const int j = t < M.lo ? t : t + m;
        const P4<float> p = r[j];
        const int cj = p.tag >> 1, tj = p.tag & 1;
        const bool ex = (j == M.ex0) | (j == M.ex1) | (j == M.ex2);
        float qx = p.x, qy = p.y, qz = p.z, Lj = 0.0f, iLj = 0.0f;
        kap[u] = d.kin32;
        if (cj != mchain) {   // into the moved chain's frame
            const P4<float> sh = D[mchain * nc + cj];
            qx -= sh.x; qy -= sh.y; qz -= sh.z;
            Lj = d.L32;
            iLj = d.iL32;
            kap[u] = d.kout32;
        }
        if (ex) { qx = qy = qz = 1.0e4f; kap[u] = 0.0f; Lj = iLj = 0.0f; }
        nqx[u] = make_float2(-qx, -qx);
        nqy[u] = make_float2(-qy, -qy);
        nqz[u] = make_float2(-qz, -qz);
        nL[u] = make_float2(-Lj, -Lj);
        iL[u] = make_float2(iLj, iLj);
        nC0[u] = make_float2(-d.C32[tj], -d.C32[tj]);
        nC1[u] = make_float2(-d.C32[2 + tj], -d.C32[2 + tj]);
        acc[u] = make_float2(0.0f, 0.0f);
    }
    const float2 Mg = make_float2(12582912.0f, 12582912.0f), nMg = make_float2(-12582912.0f, -12582912.0f);
    // records [0, n_a) are A monomers, [n_a, m) B monomers
    auto sweep = [&](int i0, int i1, const float2* nC) {
#pragma unroll 1
        for (int i = i0 + ((sub - i0) % step + step) % step; i < i1; i += step) {
            const float4 A = mv[2 * i], B = mv[2 * i + 1];
            const float2 x2 = make_float2(A.x, A.y), y2 = make_float2(A.z, A.w), z2 = make_float2(B.x, B.y);
            // stage-major: each stage for all RR partners before the next, so the
            // independent chains sit next to each other for the scheduler
            float2 dx[RR], dy[RR], dz[RR], r2[RR];
#pragma unroll
            for (int u = 0; u < RR; ++u) {
                dx[u] = __fadd2_rn(x2, nqx[u]);
                dy[u] = __fadd2_rn(y2, nqy[u]);
                dz[u] = __fadd2_rn(z2, nqz[u]);
            }
            if (PBC) {
#pragma unroll
                for (int u = 0; u < RR; ++u) {
                    dx[u] = __ffma2_rn(nL[u], __fadd2_rn(__ffma2_rn(dx[u], iL[u], Mg), nMg), dx[u]);
                    dy[u] = __ffma2_rn(nL[u], __fadd2_rn(__ffma2_rn(dy[u], iL[u], Mg), nMg), dy[u]);
                    dz[u] = __ffma2_rn(nL[u], __fadd2_rn(__ffma2_rn(dz[u], iL[u], Mg), nMg), dz[u]);
                }
            }
#pragma unroll
            for (int u = 0; u < RR; ++u) r2[u] = __fmul2_rn(dx[u], dx[u]);
#pragma unroll
            for (int u = 0; u < RR; ++u) r2[u] = __ffma2_rn(dy[u], dy[u], r2[u]);
#pragma unroll
            for (int u = 0; u < RR; ++u) r2[u] = __ffma2_rn(dz[u], dz[u], r2[u]);
#pragma unroll
            for (int u = 0; u < RR; ++u) r2[u] = make_float2(fast_rcp(r2[u].x), fast_rcp(r2[u].y));
#pragma unroll
            for (int u = 0; u < RR; ++u) {
                const float2 i6 = __fmul2_rn(__fmul2_rn(r2[u], r2[u]), r2[u]);
                acc[u] = __ffma2_rn(i6, __fadd2_rn(i6, nC[u]), acc[u]);   // (old, new) sums
            }
        }
    };
    sweep(0, M.n_a, nC0);
    sweep(M.n_a, m, nC1);
    float part = 0.0f;
#pragma unroll
    for (int u = 0; u < RR; ++u) part += kap[u] * (acc[u].y - acc[u].x);
    return part;
}

// This lane's share, summed over its partner chunks in double-float.
template <int TPW, int R, bool PBC>
__device__ DF pair_delta32(const SysDesc& d, const MoveSet& M, int mchain, const Slot<float>& s,
                               const Group<TPW>& g) {
    const int m = M.hi - M.lo + 1;
    const int U = d.N - m;
    const float4* mv = reinterpret_cast<const float4*>(s.newr);
    const int full = U / (TPW * R) * (TPW * R);       // partners in chunks of R per lane
    const int full1 = U / TPW * TPW;                    // then one per lane
    DF sum{0.0f, 0.0f};
    if constexpr (TPW < 32) {   // small systems: one partner per lane, the shortest code
        for (int t = g.lane; t < U; t += TPW)
            sum = df_add(sum, DF{pair_chunk32<1, PBC>(d, M, mchain, m, t, TPW, s.r, s.D, mv), 0.0f});
        return sum;
    }
    int t0 = g.lane;
    for (; t0 < full; t0 += TPW * R) sum = df_add(sum, DF{pair_chunk32<R, PBC>(d, M, mchain, m, t0, TPW, s.r, s.D, mv), 0.0f});
    for (; t0 < full1; t0 += TPW) sum = df_add(sum, DF{pair_chunk32<1, PBC>(d, M, mchain, m, t0, TPW, s.r, s.D, mv), 0.0f});
    // the last P < TPW partners: each shared by TPW / P' lanes (P' the power of two
    // >= P), which split its moved monomers between them
    const int P = U - full1;
    if (P > 0) {
        int Pp = 1;
        while (Pp < P) Pp <<= 1;
        const int p = g.lane & (Pp - 1), sub = g.lane / Pp;
        if (p < P)
            sum = df_add(sum, DF{pair_chunk32<1, PBC>(d, M, mchain, m, full1 + p, TPW, s.r, s.D, mv, sub, TPW / Pp), 0.0f});
    }
    return sum;
}

// This lane's share of the Lennard-Jones change in the working precision
// (FP64 mode): unmoved partners t = lane, lane + TPW, ... (skipping the moved
// range), R of them in registers at a time, each swept against every moved
// monomer before and after the move, with the nearest-integer minimum image
// between chains.
template <int TPW, typename PT, int R>
__device__ PT pair_delta(const SysDesc& d, const MoveSet& M, int mchain, const Slot<PT>& s,
                         const Group<TPW>& g) {
    const int m = M.hi - M.lo + 1;
    const int U = d.N - m;
    const int nc = d.n_chains;
    const FF<PT> f{d};
    const PT L = f.L(), iL = f.iL();
    const PT kin = f.kin(), kout = f.kout();
    const PT far = (PT)1.0e4;
    PT part = (PT)0;
    for (int t0 = g.lane; t0 < U; t0 += TPW * R) {
        PT qx[R], qy[R], qz[R], Lj[R], iLj[R], C0[R], C1[R], kap[R], acc[R];
#pragma unroll
        for (int u = 0; u < R; ++u) {
            const int t = t0 + u * TPW;
            qx[u] = qy[u] = qz[u] = far;
            Lj[u] = iLj[u] = C0[u] = C1[u] = kap[u] = (PT)0;
            acc[u] = (PT)0;
            if (t < U) {
                const int j = t < M.lo ? t : t + m;
                const P4<PT> p = s.r[j];
                const int cj = p.tag >> 1, tj = p.tag & 1;
                const bool ex = (j == M.ex0) | (j == M.ex1) | (j == M.ex2);
                if (!ex) {
                    if (cj == mchain) {
                        qx[u] = p.x; qy[u] = p.y; qz[u] = p.z;
                        kap[u] = kin;
                    } else {
                        const P4<PT> sh = s.D[mchain * nc + cj];
                        qx[u] = p.x - sh.x; qy[u] = p.y - sh.y; qz[u] = p.z - sh.z;
                        Lj[u] = L; iLj[u] = iL;
                        kap[u] = kout;
                    }
                    C0[u] = f.C(tj);
                    C1[u] = f.C(2 + tj);
                }
            }
        }
#pragma unroll 2
        for (int i = 0; i < m; ++i) {
            const P4<PT> a = s.r[M.lo + i];
            const P4<PT> b = s.newr[i];
            const bool ib = a.tag & 1;
#pragma unroll
            for (int u = 0; u < R; ++u) {
                const PT C = ib ? C1[u] : C0[u];
                const PT e0 = lj_pair<PT>(a.x - qx[u], a.y - qy[u], a.z - qz[u], Lj[u], iLj[u], C);
                const PT e1 = lj_pair<PT>(b.x - qx[u], b.y - qy[u], b.z - qz[u], Lj[u], iLj[u], C);
                acc[u] += e1 - e0;
            }
        }
#pragma unroll
        for (int u = 0; u < R; ++u) part += kap[u] * acc[u];
    }
    return part;
}

// Bin of E + dE, the group's total dE = hi + lo (double-float) given with
// erel = FP32 image of E - e_min.  The FP32 estimate of (E + dE - e_min) / w
// decides unless it lies within its error bound of a bin edge: erel carries
// half an ulp, the two FP32 additions one each, the scaling by 1/w two more,
// all within 4e-7 (|erel| + |hi| + |lo|) / w.  Near an edge, bin_of decides on
// the FP64 sum E + (hi + lo) -- so the bin always equals bin_of's.
__device__ __forceinline__ int bin_after(const SysDesc& d, double E, float erel, DF dE) {
    const float x = ((erel + dE.hi) + dE.lo) * d.iw32;
    const float fl = floorf(x);
    const float fr = x - fl;
    const float mg = 4e-7f * (fabsf(erel) + fabsf(dE.hi) + fabsf(dE.lo)) * d.iw32 + 1e-6f;
    if (fr > mg && fr < 1.0f - mg) return (fl < 0.0f || fl >= (float)d.n_bins) ? -1 : (int)fl;
    return bin_of(d, E + ((double)dE.hi + (double)dE.lo));
}

// The acceptance test for dlnW < 0: u < exp(dlnW), decided exactly as in
// FP64.  FP32 mode settles it with an FP32 exponential and the top 24 bits of
// u whenever they are further apart than their error bounds (|u - u24| <=
// 2^-24; expf within 2 ulp; the FP32 rounding of dlnW adds |dlnW| 2^-24
// relative), and falls back to FP64 in the rare near-tie.
template <typename PT>
__device__ __forceinline__ bool accept_below(double dl, const Proposal& P) {
    if constexpr (sizeof(PT) == 4) {
        const float dlf = (float)dl;
        const float e = expf(dlf);
        const float u24 = ((float)(P.uz >> 8) + 0.5f) * 5.9604644775390625e-8f;
        const float rel = 5e-7f + fabsf(dlf) * 1.2e-7f;
        if (u24 + 6e-8f < e * (1.0f - rel)) return true;
        if (u24 - 6e-8f > e * (1.0f + rel)) return false;
    }
    return u52(P.uz, P.uw) < exp(dl);
}

// Acceptance of a bond-length move: min(1, J W(E')/W(E)) with its Hastings
// factor J; one FP64 test (bond moves are a small share of the moves).
__device__ __forceinline__ bool accept_stretch(double dl, double J, const Proposal& P) {
    if (dl >= 0.0 && J >= 1.0) return true;
    return u52(P.uz, P.uw) < J * exp(dl);
}

// Full FP64 energy (Eq. 2 per chain + inter-chain term of Eq. 3) of the
// walker at x64; every lane of the group receives the total.
template <int TPW>
__device__ double full_energy64(const SysDesc& d, const double* x64, const Group<TPW>& g) {
    double part = 0.0;
    auto pos = [&](int j) -> double3 { return ld3(x64 + 3 * j); };
    bool out = false;   // a monomer outside the steric container: infinite energy
    for (int c = 0; c < d.n_chains; ++c) {
        int o = d.chain_off[c], n = d.chain_off[c + 1] - o;
        for (int k = 1 + g.lane; k <= n - 2; k += TPW) part += d.k_bend * bend_term(pos, o, k);
        for (int j = g.lane; j <= n - 4; j += TPW) part -= d.k_tors * torsion_term(pos, o, j);
        if (d.k_fene != 0.0)
            for (int l = g.lane; l <= n - 2; l += TPW) part += fene_term(d, pos, o, l);
    }
    for (int j = g.lane; j < d.N; j += TPW) out |= !inside64(d, pos(j));
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
    const double E = g.sum(part);
    return __any_sync(g.mask, out) ? INFINITY : E;
}

// Full energy with the Lennard-Jones pairs in the working precision (from the
// working copy) and the local terms in FP64 (from x64).
template <int TPW, typename PT>
__device__ double full_energy_working(const SysDesc& d, const double* x64, const Slot<PT>& s, const Group<TPW>& g) {
    double part = 0.0;
    auto pos = [&](int j) -> double3 { return ld3(x64 + 3 * j); };
    for (int c = 0; c < d.n_chains; ++c) {
        int o = d.chain_off[c], n = d.chain_off[c + 1] - o;
        for (int k = 1 + g.lane; k <= n - 2; k += TPW) part += d.k_bend * bend_term(pos, o, k);
        for (int j = g.lane; j <= n - 4; j += TPW) part -= d.k_tors * torsion_term(pos, o, j);
        if (d.k_fene != 0.0)
            for (int l = g.lane; l <= n - 2; l += TPW) part += fene_term(d, pos, o, l);
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
