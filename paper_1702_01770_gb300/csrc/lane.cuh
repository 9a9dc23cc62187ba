// lane.cuh -- the multicanonical sweep with one walker per thread, for small
// systems (the paper's own: a few chains of 9-13 monomers, Sec. 4.1-4.2).
//
// A move of a small system has tens to a few hundred pair evaluations, too
// few to spread over the lanes of a warp: a group of lanes per walker spends
// most of its issue slots on the per-move control path.  Here each thread runs
// its own walker through the whole move, so one warp instruction serves 32
// walkers:
//   * the trial positions are the exact FP64 positions of the move (the
//     geometry every implementation reproduces bit for bit), rounded to FP32
//     relative to their chain's origin for the pair terms; an accepted move
//     commits them as they are, so the FP32 working copy always equals the
//     rounded master coordinates and the running energy carries no geometric
//     drift;
//   * Lennard-Jones pairs (moved x unmoved, old and new positions side by side
//     in paired FP32 instructions) in FP32 with the minimum image, local terms
//     in FP32, totals in FP64 (PT = float), or everything in FP64 (PT = double,
//     the mode whose decisions equal the oracle's);
//   * walker arrays in shared memory are lane-interleaved (element e of lane l
//     at e * 32 + l), so the lanes of a warp reach theirs without bank
//     conflicts whatever indices they use; the FP64 master coordinates stay in
//     global memory (L2-resident for these sizes), the trial positions (FP64
//     and their working-precision records) in a per-walker global scratch, so
//     that shared memory holds only the working copy and more warps fit.
#pragma once

#include "group.cuh"

// One lane's view of its walker's shared arrays.
template <typename PT>
struct LaneSlot {
    P4<PT>* r;       // [N][32] working positions (FP32: relative to the chain origin; FP64: absolute)
    P4<PT>* newr;    // [mc] trial positions of the moved monomers (the walker's global scratch)
    float4* w;       // [nc][32] shift of each chain's origin from chain 0's, wrapped into the box (FP32 mode)
    float4* org;     // [nc][32] chain origins (FP32 values, exact in FP64)
    int lane;
    __device__ __forceinline__ LaneSlot(unsigned char* warp_base, const LaneLayout& L, int lane_)
        : r((P4<PT>*)(warp_base + L.r_off)), newr(nullptr),
          w((float4*)(warp_base + L.w_off)), org((float4*)(warp_base + L.org_off)), lane(lane_) {}
    __device__ __forceinline__ P4<PT>& R(int j) const { return r[j * 32 + lane]; }
    __device__ __forceinline__ P4<PT>& NR(int q) const { return newr[q]; }
    __device__ __forceinline__ float4& W(int c) const { return w[c * 32 + lane]; }
    __device__ __forceinline__ float4& O(int c) const { return org[c * 32 + lane]; }
};

// Full FP64 energy (Eq. 2 per chain + the inter-chain term of Eq. 3, torsion,
// FENE bonds and the container) of one walker by one thread.
__device__ double lane_energy64(const SysDesc& d, const double* x64) {
    auto pos = [&](int j) -> double3 { return ld3(x64 + 3 * j); };
    double e = 0.0;
    bool out = false;
    for (int c = 0; c < d.n_chains; ++c) {
        const int o = d.chain_off[c], n = d.chain_off[c + 1] - o;
        for (int k = 1; k <= n - 2; ++k) e += d.k_bend * bend_term(pos, o, k);
        for (int j = 0; j <= n - 4; ++j) e -= d.k_tors * torsion_term(pos, o, j);
        if (d.k_fene != 0.0)
            for (int l = 0; l <= n - 2; ++l) e += fene_term(d, pos, o, l);
    }
    for (int j = 0; j < d.N; ++j) out |= !inside64(d, pos(j));
    for (int i = 0; i < d.N; ++i) {
        const double3 xi = pos(i);
        const int ci = d.chain_of[i];
        for (int j = i + 1; j < d.N; ++j) {
            const int cj = d.chain_of[j];
            if (ci == cj && j < i + 2) continue;
            const double3 xj = pos(j);
            double dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
            if (ci != cj) {
                dx = mimage64(dx, d.box_L, d.inv_L);
                dy = mimage64(dy, d.box_L, d.inv_L);
                dz = mimage64(dz, d.box_L, d.inv_L);
            }
            e += (ci == cj ? d.k_lj_intra : d.k_lj_inter) * lj64(dx * dx + dy * dy + dz * dz, d.C[2 * d.seq[i] + d.seq[j]]);
        }
    }
    return out ? INFINITY : e;
}

// Chain origin of the FP32 working copy: the chain's centroid rounded to FP32,
// so that the origin is exact in both precisions.
__device__ __forceinline__ double3 lane_origin(const double* x64, int o, int n) {
    double sx = 0.0, sy = 0.0, sz = 0.0;
    for (int j = o; j < o + n; ++j) { sx += x64[3 * j]; sy += x64[3 * j + 1]; sz += x64[3 * j + 2]; }
    return make_double3((double)(float)(sx / n), (double)(float)(sy / n), (double)(float)(sz / n));
}

// Working copy of one walker.  FP32 mode: per chain c the origin o_c, the
// shift w_c = o_c - o_0 (wrapped into the box for a periodic system, exact in
// FP64 and then rounded) and positions x - o_c rounded to FP32; FP64 mode:
// the absolute positions.
template <typename PT>
__device__ void lane_build(const SysDesc& d, const double* x64, const LaneSlot<PT>& s) {
    if constexpr (sizeof(PT) == 4) {
        const double3 o0 = lane_origin(x64, d.chain_off[0], d.chain_off[1] - d.chain_off[0]);
        for (int c = 0; c < d.n_chains; ++c) {
            const int o = d.chain_off[c], n = d.chain_off[c + 1] - o;
            const double3 oc = c == 0 ? o0 : lane_origin(x64, o, n);
            double wx = oc.x - o0.x, wy = oc.y - o0.y, wz = oc.z - o0.z;
            if (d.box_L > 0.0) {
                wx = mimage64(wx, d.box_L, d.inv_L);
                wy = mimage64(wy, d.box_L, d.inv_L);
                wz = mimage64(wz, d.box_L, d.inv_L);
            }
            s.W(c) = make_float4((float)wx, (float)wy, (float)wz, 0.0f);   // enters differences between chains
            s.O(c) = make_float4((float)oc.x, (float)oc.y, (float)oc.z, 0.0f);   // exact: oc is an FP32 value
            for (int j = o; j < o + n; ++j) {
                P4<PT> q;
                q.x = (float)(x64[3 * j + 0] - oc.x);
                q.y = (float)(x64[3 * j + 1] - oc.y);
                q.z = (float)(x64[3 * j + 2] - oc.z);
                q.tag = (int)d.seq[j] | (c << 1);
                s.R(j) = q;
            }
        }
    } else {
        for (int j = 0; j < d.N; ++j) {
            P4<PT> q;
            q.x = x64[3 * j + 0];
            q.y = x64[3 * j + 1];
            q.z = x64[3 * j + 2];
            q.tag = (int)d.seq[j] | ((int)d.chain_of[j] << 1);
            s.R(j) = q;
        }
    }
}

// The exact FP64 move: centre, rotation and step (geometry of Sec. 3.2 with
// the fixed evaluation order of the specification).  Returns false for a
// degenerate crankshaft axis or bond step (no move).  *jac: the Hastings
// factor of a bond-length move.
struct LaneGeo {
    Rot3 R;
    double3 c, step;
    bool rot;
};
template <bool GEOM>
__device__ __forceinline__ bool lane_geometry(const SysDesc& d, const double* x64, const Proposal& P, LaneGeo* G,
                                              double* jac) {
    const int o = d.chain_off[P.chain], n = d.chain_off[P.chain + 1] - o;
    G->c = make_double3(0.0, 0.0, 0.0);
    G->step = make_double3(0.0, 0.0, 0.0);
    G->rot = false;
    *jac = 1.0;
    if (P.type == PHAST_TRANS) {
        G->step = P.disp;
        return true;
    }
    if (GEOM && P.type == PHAST_BOND) return bond_step(x64, o, n, P.index, P.angle, &G->step, jac);
    double3 axis = P.axis;
    if (P.type == PHAST_PIVOT) {
        G->c = ld3(x64 + 3 * (o + P.index));
    } else if (GEOM && P.type == PHAST_CAP) {
        G->c = ld3(x64 + 3 * (o + (P.index > 0 ? P.index - 1 : 1)));
    } else if (P.type == PHAST_ROT) {
        G->c = centroid_serial(x64, o, n);
    } else {   // crankshaft about the axis through monomers i-1 and i+1
        const int i = o + P.index;
        const double3 a = ld3(x64 + 3 * (i - 1)), b = ld3(x64 + 3 * (i + 1));
        const double ex = xsub(b.x, a.x), ey = xsub(b.y, a.y), ez = xsub(b.z, a.z);
        const double len = xsqrt(xadd(xadd(xmul(ex, ex), xmul(ey, ey)), xmul(ez, ez)));
        if (!(len > 1e-12)) return false;
        axis = make_double3(xdiv(ex, len), xdiv(ey, len), xdiv(ez, len));
        G->c = a;
    }
    double sn, cs;
    taylor_sincos(P.angle, &sn, &cs);
    G->R = rodrigues(axis.x, axis.y, axis.z, sn, cs);
    G->rot = true;
    return true;
}

// Lennard-Jones change of the move: every (moved, unmoved) pair, old and new
// positions side by side in paired FP32 instructions, as one flat loop over the
// m x U pairs (the lanes of a warp then run max(m U) iterations rather than
// max(m) x max(U)).  Partners of other chains are taken into the moved chain's
// frame by the difference of the chains' wrapped origin shifts and get the
// per-pair minimum image; left-out partners contribute nothing.  Returns the
// change with the couplings k_lj_intra / k_lj_inter applied.
template <bool PBC>
__device__ __forceinline__ float lane_pairs32(const SysDesc& d, const MoveSet& M, int mchain, const LaneSlot<float>& s) {
    const int m = M.hi - M.lo + 1, U = d.N - m;
    const int total = m * U;
    const float2 Mg = make_float2(12582912.0f, 12582912.0f), nMg = make_float2(-12582912.0f, -12582912.0f);
    const float4 wm = s.W(mchain);
    float acc = 0.0f;
    int q = 0, t = 0;
    P4<float> ow = s.R(M.lo), nw = s.NR(0);
#pragma unroll 2
    for (int k = 0; k < total; ++k) {
        const int j = t < M.lo ? t : t + m;
        const bool skip = (j == M.ex0) | (j == M.ex1) | (j == M.ex2);
        const P4<float> p = s.R(j);
        const int cj = p.tag >> 1;
        const float C = d.C32[2 * (ow.tag & 1) + (p.tag & 1)];
        float qx = p.x, qy = p.y, qz = p.z;
        const bool inter = cj != mchain;
        if (inter) {   // into the moved chain's frame
            const float4 wc = s.W(cj);
            qx += wc.x - wm.x;
            qy += wc.y - wm.y;
            qz += wc.z - wm.z;
        }
        float2 dx = __fadd2_rn(make_float2(ow.x, nw.x), make_float2(-qx, -qx));
        float2 dy = __fadd2_rn(make_float2(ow.y, nw.y), make_float2(-qy, -qy));
        float2 dz = __fadd2_rn(make_float2(ow.z, nw.z), make_float2(-qz, -qz));
        if (PBC) {   // image counts of zero (same chain) leave the displacement unchanged
            const float Lj = inter ? d.L32 : 0.0f, iLj = inter ? d.iL32 : 0.0f;
            const float2 iL = make_float2(iLj, iLj), nL = make_float2(-Lj, -Lj);
            dx = __ffma2_rn(nL, __fadd2_rn(__ffma2_rn(dx, iL, Mg), nMg), dx);
            dy = __ffma2_rn(nL, __fadd2_rn(__ffma2_rn(dy, iL, Mg), nMg), dy);
            dz = __ffma2_rn(nL, __fadd2_rn(__ffma2_rn(dz, iL, Mg), nMg), dz);
        }
        float2 r2 = __fmul2_rn(dx, dx);
        r2 = __ffma2_rn(dy, dy, r2);
        r2 = __ffma2_rn(dz, dz, r2);
        const float2 i2 = make_float2(fast_rcp(r2.x), fast_rcp(r2.y));
        const float2 i6 = __fmul2_rn(__fmul2_rn(i2, i2), i2);
        const float2 e = __fmul2_rn(i6, __fadd2_rn(i6, make_float2(-C, -C)));
        const float kap = skip ? 0.0f : (inter ? d.kout32 : d.kin32);
        acc = __fmaf_rn(kap, e.y - e.x, acc);
        if (++t == U) {   // the next moved monomer
            t = 0;
            if (++q < m) {
                ow = s.R(M.lo + q);
                nw = s.NR(q);
            }
        }
    }
    return acc;
}

// The same in FP64 (absolute positions, per-pair minimum image between chains).
__device__ __forceinline__ double lane_pairs64(const SysDesc& d, const MoveSet& M, int mchain, const LaneSlot<double>& s) {
    const int m = M.hi - M.lo + 1, U = d.N - m;
    const int total = m * U;
    double acc = 0.0;
    int q = 0, t = 0;
    P4<double> ow = s.R(M.lo), nw = s.NR(0);
    for (int k = 0; k < total; ++k) {
        const int j = t < M.lo ? t : t + m;
        const bool skip = (j == M.ex0) | (j == M.ex1) | (j == M.ex2);
        const P4<double> p = s.R(j);
        const int cj = p.tag >> 1;
        const double C = d.C[2 * (ow.tag & 1) + (p.tag & 1)];
        double Lj = 0.0, iLj = 0.0, kap = d.k_lj_intra;
        if (cj != mchain) { Lj = d.box_L; iLj = d.inv_L; kap = d.k_lj_inter; }
        const double e0 = lj_pair<double>(ow.x - p.x, ow.y - p.y, ow.z - p.z, Lj, iLj, C);
        const double e1 = lj_pair<double>(nw.x - p.x, nw.y - p.y, nw.z - p.z, Lj, iLj, C);
        if (!skip) acc += kap * (e1 - e0);
        if (++t == U) {
            t = 0;
            if (++q < m) {
                ow = s.R(M.lo + q);
                nw = s.NR(q);
            }
        }
    }
    return acc;
}

// Sweeps between re-centrings of the FP32 working copy on the chain centroids.
constexpr int kLaneRebuildSweeps = 64;

// One walker, one thread: n_sweeps sweeps of the multicanonical Metropolis
// scheme (Sec. 2.2) -- the counterpart of run_walker for a group of one lane.
template <typename PT, bool GEOM>
__device__ void run_walker_lane(const SysDesc& sd, const SweepArgs& a, int s_id, int w_local, LaneSlot<PT> s,
                                uint32_t* hist, unsigned long long* hist_tile, unsigned long long* hist_g) {
    const int gw = sd.walker_off + w_local;
    double* x64 = a.xyz + sd.xyz_off + (int64_t)w_local * sd.N * 3;
    double* new64 = a.scratch + (int64_t)gw * a.scratch_stride;   // the trial's exact positions [mc][3]
    s.newr = reinterpret_cast<P4<PT>*>(new64 + 4 * sd.max_chain);   // their records [mc] (16-byte aligned)
    const double* lnW = a.lnW + sd.lnw_off;
    double E = a.E[gw];
    int bin = a.bin[gw];
    uint64_t t = a.t[gw];
    const uint64_t seed = a.seed[gw];
    phast_walker_stats* st = a.stats + gw;   // move counters go straight to it (one reduction each)
    unsigned long long n_recompute = 0, n_outside = 0;
    uint64_t pair_evals = 0, pair_evals_inter = 0;
    double drift_max = 0.0;
    uint32_t* hw = a.hist_walker ? a.hist_walker + sd.hw_off + (int64_t)w_local * sd.n_bins : nullptr;
    const bool tracing = a.trace && s_id == 0 && w_local < a.trace_walkers;
    const int64_t n_moves = a.n_sweeps * sd.N;
    const uint64_t period = (uint64_t)sd.recompute_every * (uint64_t)sd.N;
    const uint64_t rebuild = (uint64_t)kLaneRebuildSweeps * (uint64_t)sd.N;
    lane_build<PT>(sd, x64, s);
    double lnw_here = __ldg(lnW + bin);
    float erel = (float)(E - sd.e_min);
    for (int64_t it = 0; it < n_moves; ++it) {
        Proposal P;
        propose_select(sd, stream_block<true>(seed, t, 0u), stream_block<true>(seed, t, 1u),
                       stream_block<true>(seed, t, 2u), &P);
        if constexpr (!GEOM) __builtin_assume(P.type >= 0 && P.type < PHAST_BOND);
        if (P.type == PHAST_PIVOT || P.type == PHAST_ROT || (GEOM && P.type == PHAST_CAP)) {
            for (int j = 0; j < PHAST_MARSAGLIA_TRIES; ++j) {
                double3 ax;
                if (marsaglia_try(stream_block<true>(seed, t, 3u + (uint32_t)j), &ax)) { P.axis = ax; break; }
            }
        }
        const MoveSet M = move_set(sd, P.type, P.chain, P.index);
        const int m = M.hi - M.lo + 1;
        const int o = sd.chain_off[P.chain];
        LaneGeo G;
        double jac = 1.0;
        const bool ok = lane_geometry<GEOM>(sd, x64, P, &G, &jac);
        bool wall = false;
        double3 oc = make_double3(0.0, 0.0, 0.0);   // the moved chain's origin (FP32 mode)
        if constexpr (sizeof(PT) == 4) {
            const float4 og = s.O(P.chain);
            oc = make_double3((double)og.x, (double)og.y, (double)og.z);
        }
        if (ok) {
            for (int q = 0; q < m; ++q) {
                const double3 x = ld3(x64 + 3 * (M.lo + q));
                const double3 y = G.rot ? rotate_about(G.R, G.c, x)
                                        : make_double3(xadd(x.x, G.step.x), xadd(x.y, G.step.y), xadd(x.z, G.step.z));
                new64[3 * q + 0] = y.x;
                new64[3 * q + 1] = y.y;
                new64[3 * q + 2] = y.z;
                if (GEOM) wall |= !inside64(sd, y);
                P4<PT> w;
                if constexpr (sizeof(PT) == 4) {
                    w.x = (float)(y.x - oc.x);
                    w.y = (float)(y.y - oc.y);
                    w.z = (float)(y.z - oc.z);
                } else {
                    w.x = y.x; w.y = y.y; w.z = y.z;
                }
                w.tag = s.R(M.lo + q).tag;
                s.NR(q) = w;
            }
        }
        const bool eval = ok && !wall;
        // dE: local terms and Lennard-Jones pairs in the working precision
        DF dE32{0.0f, 0.0f};
        double dE64 = 0.0;
        if (eval) {
            auto pos = [&](int j, bool after) -> P4<PT> {
                return (after && j >= M.lo && j <= M.hi) ? s.NR(j - M.lo) : s.R(j);
            };
            int vb0, nb, jt0, nt, fb0, nf;
            local_window(sd, P.type, P.chain, P.index, &vb0, &nb, &jt0, &nt, &fb0, &nf);
            const int nc1 = GEOM && P.type == PHAST_BOND;
            const FF<PT> f{sd};
            PT loc = (PT)0;
            double fene = 0.0;   // the terms taken in FP64 on the exact positions
            for (int k = 0; k < nb + nt + nc1; ++k) {
#pragma unroll
                for (int after = 0; after < 2; ++after) {
                    auto p = [&](int j) -> P4<PT> { return pos(j, after); };
                    PT term;
                    if (k < nb) {
                        term = f.kbend() * bend_w<PT>(p, o, vb0 + k);
                    } else if (k < nb + nt) {
                        bool nr = false;   // FP32: a dihedral near degenerate is taken in FP64
                        term = -f.ktors() * torsion_w<PT>(p, o, jt0 + (k - nb), sizeof(PT) == 4 ? &nr : nullptr);
                        if (nr) {
                            auto ex = [&](int j) -> double3 {
                                return (after && j >= M.lo && j <= M.hi) ? ld3(new64 + 3 * (j - M.lo))
                                                                         : ld3(x64 + 3 * j);
                            };
                            const double v = -sd.k_tors * torsion_term(ex, o, jt0 + (k - nb));
                            fene += after ? v : -v;
                        }
                    } else {
                        term = bond_item<PT>(sd, false, p(o + P.index), p(o + P.index + 1), o + P.index);
                    }
                    loc += after ? term : -term;
                }
            }
            // FENE bonds in FP64 on the exact positions: FP32 records cannot resolve
            // 1 - ((r - r0) / R)^2 near the divergence
            if constexpr (GEOM)
                for (int k = 0; k < nf; ++k) {
                    auto before = [&](int j) -> double3 { return ld3(x64 + 3 * j); };
                    auto after = [&](int j) -> double3 {
                        return (j >= M.lo && j <= M.hi) ? ld3(new64 + 3 * (j - M.lo)) : ld3(x64 + 3 * j);
                    };
                    fene += fene_term(sd, after, o, fb0 + k) - fene_term(sd, before, o, fb0 + k);
                }
            if constexpr (sizeof(PT) == 4) {
                const float pr = sd.box_L > 0.0 ? lane_pairs32<true>(sd, M, P.chain, s)
                                                : lane_pairs32<false>(sd, M, P.chain, s);
                dE32 = df_add(DF{loc, 0.0f}, DF{pr, 0.0f});
                if (fene != 0.0) dE32 = df_add(dE32, df_of(fene));
            } else {
                dE64 = loc + fene + lane_pairs64(sd, M, P.chain, s);
            }
        }
        const bool finite = eval && (sizeof(PT) == 4 ? (isfinite(dE32.hi) && isfinite(dE32.lo)) : isfinite(dE64));
        int b_new = -1;
        if (finite) b_new = sizeof(PT) == 4 ? bin_after(sd, E, erel, dE32) : bin_of(sd, E + dE64);
        bool acc = false;
        double lnw_new = lnw_here;
        if (b_new >= 0) {
            lnw_new = __ldg(lnW + b_new);
            const double dl = lnw_new - lnw_here;
            if (GEOM && P.type == PHAST_BOND) acc = accept_stretch(dl, jac, P);
            else acc = (dl >= 0.0) || accept_below<PT>(dl, P);
        }
        if (acc) {
            E = E + (sizeof(PT) == 4 ? (double)dE32.hi + (double)dE32.lo : dE64);
            bin = b_new;
            lnw_here = lnw_new;
            erel = (float)(E - sd.e_min);
            for (int q = 0; q < m; ++q) {   // commit the exact positions and their working copy
                x64[3 * (M.lo + q) + 0] = new64[3 * q + 0];
                x64[3 * (M.lo + q) + 1] = new64[3 * q + 1];
                x64[3 * (M.lo + q) + 2] = new64[3 * q + 2];
                s.R(M.lo + q) = s.NR(q);
            }
        }
        if (hist_g) {
            atomicAdd(hist_g + bin, 1ull);
        } else if (!a.hist_flush_on) {
            atomicAdd(hist + bin, 1u);
        } else if (((atomicAdd(hist + bin, 1u) + 1u) & (a.hist_flush - 1u)) == 0u && hist_tile) {
            atomicSub(hist + bin, a.hist_flush);   // the flush of the 32-bit shared bin (see run_walker)
            atomicAdd(hist_tile + bin, (unsigned long long)a.hist_flush);
        }
        if (hw) atomicAdd(hw + bin, 1u);
        atomicAdd(reinterpret_cast<unsigned long long*>(&st->attempts[P.type]), 1ull);
        if (acc) atomicAdd(reinterpret_cast<unsigned long long*>(&st->accepts[P.type]), 1ull);
        pair_evals += move_pair_evals(sd, P.type, M);
        pair_evals_inter += move_pair_evals_inter(sd, P.type, P.chain, M);
        if (tracing) {
            phast_trace tr;
            tr.dE = !ok ? __longlong_as_double(0x7ff8000000000000ll)
                  : wall ? INFINITY
                         : (sizeof(PT) == 4 ? (isinf(dE32.hi) ? (double)dE32.hi : (double)dE32.hi + (double)dE32.lo)
                                            : dE64);
            tr.bin_after = bin;
            tr.accepted = (int32_t)acc;
            a.trace[(int64_t)w_local * n_moves + it] = tr;
        }
        ++t;
        if (period && (t % period) == 0) {   // the FP64 full energy replaces the running one
            const double Ef = lane_energy64(sd, x64);
            drift_max = fmax(drift_max, fabs(E - Ef));
            ++n_recompute;
            if (isfinite(Ef)) {
                const int bf = bin_of(sd, Ef);
                E = Ef;
                erel = (float)(E - sd.e_min);
                bin = bf >= 0 ? bf : (Ef < sd.e_min ? 0 : sd.n_bins - 1);
                lnw_here = __ldg(lnW + bin);
                if (bf < 0) ++n_outside;
            }
            lane_build<PT>(sd, x64, s);   // origins re-centred, working copy rounded afresh
        } else if (sizeof(PT) == 4 && (t % rebuild) == 0) {
            // translations carry a chain away from its origin, and its FP32 coordinates
            // lose digits: re-centre now and then even without an energy recompute
            lane_build<PT>(sd, x64, s);
        }
    }
    a.E[gw] = E;
    a.bin[gw] = bin;
    a.t[gw] = t;
    st->pair_evals += pair_evals;
    st->pair_evals_inter += pair_evals_inter;
    st->recomputes += n_recompute;
    st->recompute_outside += n_outside;
    st->drift_max = fmax(st->drift_max, drift_max);
}
