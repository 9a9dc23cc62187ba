// sweep.cu -- the multicanonical sweep (Sec. 2.2; MONTE_CARLO.f / UPDATE_ENGINE.f
// of Sec. 3.2) over many independent walkers, and the walker context.
//
//  * batched form: a persistent kernel; each CTA takes tiles of walkers of one
//    system type (one jackknife block) from an atomic work counter, a group of
//    TPW lanes runs one walker with its coordinates staged in shared memory,
//    FP32 (or FP64) pair terms and FP64 totals, and all walkers of the CTA
//    count into one shared-memory histogram flushed once per tile;
//  * plain form: one CTA per walker, everything in FP64 straight from global
//    memory, histogram atomics to global memory (the comparison form).
// Both draw the same Philox stream and apply the same FP64 geometry, so their
// decisions match the FP64 oracle move for move.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "group.cuh"

struct phast_ctx {
    int n_sys;
    int W;
    int device;
    SysDesc desc[PHAST_MAX_SYSTEMS];
    SysDesc* d_desc;
    int64_t xyz_total;    // doubles
    int64_t lnw_total;
    int64_t hw_total;     // bins of a per-walker histogram array
    int max_N, max_nc, max_chain, max_bins;
    double* xyz;
    double* E;
    int32_t* bin;
    uint64_t* t;
    uint64_t* seed;
    phast_walker_stats* stats;
    int32_t* tile_counter;
    double* plain_scratch;   // [W][8 max_chain] trial positions: [max_chain][3] FP64 (plain and lane forms),
                             // then [max_chain] working-precision records at 4 max_chain (lane form)
    int tpw, wpc;
    uint32_t hist_flush;     // count at which a shared histogram bin moves into hist_sum
    int order[PHAST_MAX_SYSTEMS];   // tile order: most expensive system types first
    bool near_straight;      // a type with torsion starts with a dihedral FP32 cannot resolve
};

namespace {

// ---------------------------------------------------------------------------
// Launch arguments (by value).
// ---------------------------------------------------------------------------
struct SweepArgs {
    const SysDesc* descs;
    int n_sys, n_jk, wpc, n_tiles;
    int64_t n_sweeps;
    int order[PHAST_MAX_SYSTEMS];
    int tile_start[PHAST_MAX_SYSTEMS + 1];
    int tiles[PHAST_MAX_SYSTEMS];        // tiles of each system, by enumeration position
    int64_t hs_off[PHAST_MAX_SYSTEMS];   // hist_sum offset of each system id
    double* xyz;
    double* E;
    int32_t* bin;
    uint64_t* t;
    const uint64_t* seed;
    phast_walker_stats* stats;
    const double* lnW;
    unsigned long long* hist_sum;
    uint32_t* hist_walker;
    phast_trace* trace;
    int trace_walkers;
    int32_t* tile_counter;
    double* scratch;
    int scratch_stride;                   // doubles per walker in scratch
    SlotLayout L;
    LaneLayout LL;                        // per-warp layout of the one-walker-per-thread form
    int hist_bins;                        // shared histogram capacity (max n_bins)
    uint32_t hist_flush;                  // a shared bin reaching this count moves it into hist_sum
    int hist_flush_on;                    // a tile's counts can reach hist_flush in this launch
};

}  // namespace

#include "lane.cuh"   // the one-walker-per-thread form (uses SweepArgs)

namespace {

__device__ __forceinline__ void copy_desc(SysDesc* dst, const SysDesc* src) {
    const int4* s = reinterpret_cast<const int4*>(src);
    int4* d = reinterpret_cast<int4*>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(SysDesc) / 16); i += blockDim.x) d[i] = s[i];
}

// Jackknife block of walker w of a type with W walkers split into n blocks
// [b W / n, (b+1) W / n).
__host__ __device__ __forceinline__ int jk_block(int w, int W, int n) {
    return (int)(((int64_t)(w + 1) * n - 1) / W);
}

// ---------------------------------------------------------------------------
// Initial energies: one warp per walker, FP64.
// ---------------------------------------------------------------------------
__global__ void init_energy_kernel(const SysDesc* __restrict__ descs, int n_sys, int W, const double* xyz,
                                   double* E, int32_t* bin) {
    Group<32> g;
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (gw >= W) return;
    int s = 0;
    while (s + 1 < n_sys && gw >= descs[s + 1].walker_off) ++s;
    const SysDesc& d = descs[s];
    const double* x64 = xyz + d.xyz_off + (int64_t)(gw - d.walker_off) * d.N * 3;
    double e = full_energy64<32>(d, x64, g);
    if (g.lane == 0) {
        E[gw] = e;
        bin[gw] = bin_of(d, e);
    }
}

// ---------------------------------------------------------------------------
// Batched form.
// ---------------------------------------------------------------------------

// The FP64 full energy replaces the running one (when in range) and the
// working copy is rebuilt.
template <int TPW, typename PT>
__device__ __forceinline__ void recompute_energy(const SysDesc& sd, const double* x64, const double* lnW, Slot<PT>& slot,
                                              const Group<TPW>& g, phast_walker_stats* ls, double& E, int& bin,
                                              double& lnw_here, float& erel) {
    const double Ef = full_energy64<TPW>(sd, x64, g);
    if (g.lane == 0) {
        ls->drift_max = fmax(ls->drift_max, fabs(E - Ef));
        ls->recomputes++;
    }
    // the running energy always takes the FP64 value (the drift is removed); a
    // value outside the bins (an FP32 rounding let the walker step just past a
    // range edge) counts in the nearest edge bin until a move brings it back
    if (isfinite(Ef)) {
        const int bf = bin_of(sd, Ef);
        E = Ef;
        erel = (float)(E - sd.e_min);
        bin = bf >= 0 ? bf : (Ef < sd.e_min ? 0 : sd.n_bins - 1);
        lnw_here = __ldg(lnW + bin);
        if (bf < 0 && g.lane == 0) ls->recompute_outside++;
    }
    g.sync();
    build_working<TPW, PT>(sd, x64, slot, g);
}
// GEOM: the system types use the paper's own geometry (FENE bonds, container,
// bond-length or cap moves); without it those branches are compiled out, which
// keeps the per-move loop short in the instruction cache.
template <int TPW, typename PT, bool GEOM>
__device__ void run_walker(const SysDesc& sd, const SweepArgs& a, int s_id, int w_local, Slot<PT>& slot,
                           uint32_t* hist, unsigned long long* const* hist_tile, unsigned long long* hist_g,
                           const Group<TPW>& g) {
    // hist: the tile's shared histogram, whose bins move into *hist_tile (the global
    // sums of the tile's jackknife block, or null; kept in shared memory, read only
    // when a bin reaches a multiple of a.hist_flush); hist_g (non-null): this
    // walker's jackknife block differs from the tile's, so its visits go straight to
    // the global sums
    const int gw = sd.walker_off + w_local;
    double* x64 = a.xyz + sd.xyz_off + (int64_t)w_local * sd.N * 3;
    const double* lnW = a.lnW + sd.lnw_off;
    double E = a.E[gw];
    int bin = a.bin[gw];
    uint64_t t = a.t[gw];
    const uint64_t seed = a.seed[gw];
    phast_walker_stats* ls = slot.st;   // counters of this launch, in shared memory
    if (g.lane == 0) memset(ls, 0, sizeof(*ls));
    uint32_t* hw = a.hist_walker ? a.hist_walker + sd.hw_off + (int64_t)w_local * sd.n_bins : nullptr;
    const bool tracing = a.trace && s_id == 0 && w_local < a.trace_walkers;
    const int64_t n_moves = a.n_sweeps * sd.N;
    const uint64_t period = (uint64_t)sd.recompute_every * (uint64_t)sd.N;

    build_working<TPW, PT>(sd, x64, slot, g);
    int queued = 0;                                         // accepted moves awaiting their FP64 replay
    const int qcap = TPW < kQueue ? TPW : kQueue;
    // Every lane holds the walker's scalar state and takes the same decision
    // from the same broadcast values; lane 0 alone writes histograms and counters.
    double lnw_here = __ldg(lnW + bin);
    float erel = (float)(E - sd.e_min);                     // FP32 image of E - e_min (FP32 mode)
    constexpr bool OUT = TPW < 32 || GEOM;                  // the Philox rounds out of line
    uint4 blk = stream_block<OUT>(seed, t, (uint32_t)g.lane);   // this lane's block of the current move
    for (int64_t it = 0; it < n_moves; ++it) {
        const Proposal P = propose_group<TPW, PT, GEOM>(sd, seed, t, blk, g);
        if constexpr (!GEOM) __builtin_assume(P.type >= 0 && P.type < PHAST_BOND);   // no bond or cap moves
        const MoveSet M = move_set(sd, P.type, P.chain, P.index);
        double jac = 1.0;   // Hastings factor (bond-length moves)
        const bool ok = make_new_positions<TPW, PT, GEOM>(sd, x64, P, M, slot, g, &jac);
        // a trial position beyond the container's wall: infinite energy, not evaluated
        bool wall = false;
        if constexpr (GEOM)
            wall = ok && sd.has_sphere &&
                   !container_ok<TPW, PT>(sd, x64, P, M, slot, g, sizeof(PT) == 8, seed, t, sizeof(PT) == 4 ? &queued : nullptr);
        const bool eval = ok && !wall;
        DF dE32{0.0f, 0.0f};
        double dE64 = 0.0;
        if constexpr (sizeof(PT) == 4) {   // this lane's share in double-float, the group total on every lane
            DF part{0.0f, 0.0f};
            if (eval) {
                part = sd.box_L > 0.0 ? pair_delta32<TPW, 3, true>(sd, M, P.chain, slot, g)
                                      : pair_delta32<TPW, 3, false>(sd, M, P.chain, slot, g);
                float fene = 0.0f, tors = 0.0f;
                bool near = false, tnear = false;
                part = df_add(part, DF{local_delta<TPW, PT, GEOM>(sd, P, M, slot, g, GEOM ? &fene : nullptr,
                                                                  &near, &tors, &tnear), 0.0f});
                if constexpr (GEOM) {
                    // a FENE bond near its divergence or a dihedral near degenerate: the
                    // exact positions give that kind of term's change
                    const bool fx = __ballot_sync(g.mask, near) & g.mask;
                    const bool tx = __ballot_sync(g.mask, tnear) & g.mask;
                    if (fx || tx) {
                        const double dX = local_delta_exact<TPW, GEOM>(sd, x64, P, M, slot, g, false, seed, t,
                                                                       &queued, fx, tx);
                        if (g.lane == 0) part = df_add(part, df_of(dX));
                    }
                    if (!fx) part = df_add(part, DF{fene, 0.0f});
                    if (!tx) part = df_add(part, DF{tors, 0.0f});
                } else {
                    // this build keeps the exact path (an out-of-line call) out of its move
                    // loop: a dihedral whose normals lie below FP32 resolution counts 0, the
                    // FP64 value of collinear bonds (in continuous sampling a dihedral that
                    // is near degenerate without being degenerate has probability ~1e-9, and
                    // the host runs contexts whose chains start straight in the general build)
                    part = df_add(part, DF{tors, 0.0f});
                }
            }
            dE32 = group_sum_df<TPW>(part, g);
        } else {
            double part = 0.0;
            if (eval) part = local_delta<TPW, PT, GEOM>(sd, P, M, slot, g) + pair_delta<TPW, PT, 4>(sd, M, P.chain, slot, g);
            dE64 = g.sum(part);
        }
        const bool finite = eval && (sizeof(PT) == 4 ? (isfinite(dE32.hi) && isfinite(dE32.lo)) : isfinite(dE64));
        int b_new = -1;
        if (finite) b_new = sizeof(PT) == 4 ? bin_after(sd, E, erel, dE32) : bin_of(sd, E + dE64);
        const double lnw_new = __ldg(lnW + (b_new >= 0 ? b_new : bin));
        blk = stream_block<OUT>(seed, t + 1, (uint32_t)g.lane);   // next move's block, while the load is in flight
        bool acc = false;
        if (b_new >= 0) {
            const double dl = lnw_new - lnw_here;
            if (GEOM && P.type == PHAST_BOND) acc = accept_stretch(dl, jac, P);
            else acc = (dl >= 0.0) || accept_below<PT>(dl, P);
        }
        if (acc) {
            E = E + (sizeof(PT) == 4 ? (double)dE32.hi + (double)dE32.lo : dE64);
            bin = b_new;
            lnw_here = lnw_new;
            erel = (float)(E - sd.e_min);
        }
        if (g.lane == 0) {   // histogram and bookkeeping on one lane
            if (hist_g) {
                atomicAdd(hist_g + bin, 1ull);
            } else if (!a.hist_flush_on) {   // the tile cannot count to the flush count in this launch
                atomicAdd(hist + bin, 1u);
            } else if (((atomicAdd(hist + bin, 1u) + 1u) & (a.hist_flush - 1u)) == 0u && *hist_tile) {
                // this increment took the bin to a multiple of the flush count (a power
                // of two): move that many into the 64-bit sums.  Each multiple is crossed
                // by one increment, so the bin stays below the flush count plus the
                // walkers of the tile.
                atomicSub(hist + bin, a.hist_flush);
                atomicAdd(*hist_tile + bin, (unsigned long long)a.hist_flush);
            }
            if (hw) atomicAdd(hw + bin, 1u);
            ls->attempts[P.type]++;
            ls->accepts[P.type] += acc;
            ls->pair_evals += move_pair_evals(sd, P.type, M);
            ls->pair_evals_inter += move_pair_evals_inter(sd, P.type, P.chain, M);
            if (tracing) {
                phast_trace tr;
                // an infinite FP32 term leaves NaN in the double-float's low word: report hi alone
                tr.dE = !ok ? __longlong_as_double(0x7ff8000000000000ll)
                      : wall ? INFINITY
                             : (sizeof(PT) == 4 ? (isinf(dE32.hi) ? (double)dE32.hi : (double)dE32.hi + (double)dE32.lo)
                                                : dE64);
                tr.bin_after = bin;
                tr.accepted = (int32_t)acc;
                a.trace[(int64_t)w_local * n_moves + it] = tr;
            }
        }
        if (acc) {
            if constexpr (sizeof(PT) == 4) {
                accept_move32<TPW>(sd, P, t, M, slot, g, queued);
                if (++queued == qcap) {
                    flush_queue<TPW, GEOM>(sd, x64, seed, slot, g, queued);
                    queued = 0;
                }
            } else {
                commit_move64<TPW>(x64, M, slot, g);
            }
        }
        g.sync();
        ++t;
        if (period && (t % period) == 0) {   // FP64 full energy kills the drift of the running sum
            if constexpr (sizeof(PT) == 4) {
                flush_queue<TPW, GEOM>(sd, x64, seed, slot, g, queued);
                queued = 0;
            }
            recompute_energy<TPW, PT>(sd, x64, lnW, slot, g, ls, E, bin, lnw_here, erel);
        }
    }
    if constexpr (sizeof(PT) == 4) flush_queue<TPW, GEOM>(sd, x64, seed, slot, g, queued);
    if (g.lane == 0) {
        a.E[gw] = E;
        a.bin[gw] = bin;
        a.t[gw] = t;
        phast_walker_stats* st = a.stats + gw;
        for (int i = 0; i < PHAST_N_MOVES; ++i) { st->attempts[i] += ls->attempts[i]; st->accepts[i] += ls->accepts[i]; }
        st->pair_evals += ls->pair_evals;
        st->pair_evals_inter += ls->pair_evals_inter;
        st->recomputes += ls->recomputes;
        st->recompute_outside += ls->recompute_outside;
        st->drift_max = fmax(st->drift_max, ls->drift_max);
    }
}

constexpr int kMaxTileThreads = 512;
constexpr uint32_t kHistFlushDefault = 1u << 31;   // shared histogram bins stay below 2^31 + wpc

// MINB: CTAs of kMaxTileThreads per SM the registers must allow.  Small systems
// run a build held to 64 registers (MINB = 2): their moves are short and
// latency-bound, and twice the warps per SM hide more of it than the spills cost.
template <int TPW, typename PT, bool GEOM, int MINB = 1>
__global__ void __launch_bounds__(kMaxTileThreads, MINB)
sweep_batched_kernel(const SweepArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_tile;
    __shared__ unsigned long long* s_hs_tile;   // the global sums of the tile's jackknife block
    SysDesc& sd = *reinterpret_cast<SysDesc*>(smem);
    uint32_t* hist = reinterpret_cast<uint32_t*>(smem + sizeof(SysDesc));
    unsigned char* slots = smem + sizeof(SysDesc) + align16(4 * a.hist_bins);
    const Group<TPW> g;
    const int slot_id = threadIdx.x / TPW;
    Slot<PT> slot(slots + (size_t)slot_id * a.L.bytes, a.L);

    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(a.tile_counter, 1);
        __syncthreads();
        const int tile = s_tile;
        if (tile >= a.n_tiles) break;
        int pos = 0;
        while (pos + 1 < a.n_sys && tile >= a.tile_start[pos + 1]) ++pos;
        const int s_id = a.order[pos];
        copy_desc(&sd, a.descs + s_id);
        __syncthreads();
        for (int k = threadIdx.x; k < sd.n_bins; k += blockDim.x) hist[k] = 0u;
        // tile k of this system: walkers [k W / nt, (k + 1) W / nt), at most wpc of them;
        // the shared histogram collects the jackknife block of the first one
        const int k = tile - a.tile_start[pos], nt = a.tiles[pos];
        const int W = sd.n_walkers;
        const int w_a = (int)((int64_t)k * W / nt), w_b = (int)((int64_t)(k + 1) * W / nt);
        const int w_local = w_a + slot_id;
        const int blk = jk_block(w_a, W, a.n_jk);
        __syncthreads();
        if (threadIdx.x == 0) s_hs_tile = a.hist_sum ? a.hist_sum + a.hs_off[s_id] + (int64_t)blk * sd.n_bins : nullptr;
        __syncthreads();
        if (w_local < w_b) {
            const int mine = jk_block(w_local, W, a.n_jk);
            unsigned long long* hg =
                (a.hist_sum && mine != blk) ? a.hist_sum + a.hs_off[s_id] + (int64_t)mine * sd.n_bins : nullptr;
            run_walker<TPW, PT, GEOM>(sd, a, s_id, w_local, slot, hist, &s_hs_tile, hg, g);
        }
        __syncthreads();
        unsigned long long* hs_tile = s_hs_tile;
        if (hs_tile) {
            for (int k = threadIdx.x; k < sd.n_bins; k += blockDim.x)
                if (hist[k]) atomicAdd(hs_tile + k, (unsigned long long)hist[k]);
        }
        __syncthreads();
    }
}

// One walker per thread (small systems): the same persistent tiles, a tile being
// the CTA's blockDim.x walkers, each warp's walkers in one lane-interleaved
// shared-memory slot.
constexpr int kLaneMaxThreads = 256;

template <typename PT, bool GEOM>
__global__ void __launch_bounds__(kLaneMaxThreads)
sweep_lane_kernel(const SweepArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_tile;
    SysDesc& sd = *reinterpret_cast<SysDesc*>(smem);
    uint32_t* hist = reinterpret_cast<uint32_t*>(smem + sizeof(SysDesc));
    unsigned char* warps = smem + sizeof(SysDesc) + align16(4 * a.hist_bins);
    const LaneSlot<PT> slot(warps + (size_t)(threadIdx.x >> 5) * a.LL.bytes, a.LL, threadIdx.x & 31);
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(a.tile_counter, 1);
        __syncthreads();
        const int tile = s_tile;
        if (tile >= a.n_tiles) break;
        int pos = 0;
        while (pos + 1 < a.n_sys && tile >= a.tile_start[pos + 1]) ++pos;
        const int s_id = a.order[pos];
        copy_desc(&sd, a.descs + s_id);
        __syncthreads();
        for (int k = threadIdx.x; k < sd.n_bins; k += blockDim.x) hist[k] = 0u;
        const int k = tile - a.tile_start[pos], nt = a.tiles[pos];
        const int W = sd.n_walkers;
        const int w_a = (int)((int64_t)k * W / nt), w_b = (int)((int64_t)(k + 1) * W / nt);
        const int w_local = w_a + (int)threadIdx.x;
        const int blk = jk_block(w_a, W, a.n_jk);
        __syncthreads();
        unsigned long long* hs_tile = a.hist_sum ? a.hist_sum + a.hs_off[s_id] + (int64_t)blk * sd.n_bins : nullptr;
        if (w_local < w_b) {
            const int mine = jk_block(w_local, W, a.n_jk);
            unsigned long long* hg =
                (a.hist_sum && mine != blk) ? a.hist_sum + a.hs_off[s_id] + (int64_t)mine * sd.n_bins : nullptr;
            run_walker_lane<PT, GEOM>(sd, a, s_id, w_local, slot, hist, hs_tile, hg);
        }
        __syncthreads();
        if (hs_tile) {
            for (int k = threadIdx.x; k < sd.n_bins; k += blockDim.x)
                if (hist[k]) atomicAdd(hs_tile + k, (unsigned long long)hist[k]);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Plain form: one CTA per walker, FP64, global memory.
// ---------------------------------------------------------------------------
constexpr int kPlainThreads = 128;

__device__ double block_full_energy64(const SysDesc& d, const double* x64, double* red) {
    double part = 0.0;
    auto pos = [&](int j) -> double3 { return ld3(x64 + 3 * j); };
    for (int c = 0; c < d.n_chains; ++c) {
        int o = d.chain_off[c], n = d.chain_off[c + 1] - o;
        for (int k = 1 + threadIdx.x; k <= n - 2; k += blockDim.x) part += d.k_bend * bend_term(pos, o, k);
        for (int j = threadIdx.x; j <= n - 4; j += blockDim.x) part -= d.k_tors * torsion_term(pos, o, j);
        if (d.k_fene != 0.0)
            for (int l = threadIdx.x; l <= n - 2; l += blockDim.x) part += fene_term(d, pos, o, l);
    }
    int out = 0;   // a monomer beyond the container's wall: infinite energy
    for (int j = threadIdx.x; j < d.N; j += blockDim.x) out |= !inside64(d, pos(j));
    out = __syncthreads_or(out);
    for (int i = 0; i < d.N; ++i) {
        const double3 xi = pos(i);
        const int ci = d.chain_of[i];
        for (int j = i + 1 + threadIdx.x; j < d.N; j += blockDim.x) {
            const int cj = d.chain_of[j];
            if (ci == cj && j < i + 2) continue;
            const double3 xj = pos(j);
            double dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
            if (ci != cj) {
                dx = mimage64(dx, d.box_L, d.inv_L);
                dy = mimage64(dy, d.box_L, d.inv_L);
                dz = mimage64(dz, d.box_L, d.inv_L);
            }
            part += (ci == cj ? d.k_lj_intra : d.k_lj_inter) *
                    lj64(dx * dx + dy * dy + dz * dz, d.C[2 * d.seq[i] + d.seq[j]]);
        }
    }
    const double E = block_sum(part, red);
    return out ? INFINITY : E;
}

__global__ void __launch_bounds__(kPlainThreads) sweep_plain_kernel(const SweepArgs a, int W_total) {
    __shared__ __align__(16) SysDesc sd;
    __shared__ double red[32];
    __shared__ Proposal sP;
    __shared__ double sR[9], sC[3], sD[3];
    __shared__ int s_ok, s_acc;
    const int gw = blockIdx.x;
    if (gw >= W_total) return;
    int s_id = 0;
    while (s_id + 1 < a.n_sys && gw >= a.descs[s_id + 1].walker_off) ++s_id;
    copy_desc(&sd, a.descs + s_id);
    __syncthreads();
    const int w_local = gw - sd.walker_off;
    double* x64 = a.xyz + sd.xyz_off + (int64_t)w_local * sd.N * 3;
    double* nx = a.scratch + (int64_t)gw * a.scratch_stride;
    const double* lnW = a.lnW + sd.lnw_off;
    double E = a.E[gw];
    int bin = a.bin[gw];
    uint64_t t = a.t[gw];
    const uint64_t seed = a.seed[gw];
    __shared__ phast_walker_stats s_st;   // counters of this launch
    phast_walker_stats* ls = &s_st;
    if (threadIdx.x == 0) memset(ls, 0, sizeof(*ls));
    unsigned long long* hs = a.hist_sum
        ? a.hist_sum + a.hs_off[s_id] + (int64_t)jk_block(w_local, sd.n_walkers, a.n_jk) * sd.n_bins : nullptr;
    uint32_t* hw = a.hist_walker ? a.hist_walker + sd.hw_off + (int64_t)w_local * sd.n_bins : nullptr;
    const bool tracing = a.trace && s_id == 0 && w_local < a.trace_walkers;
    const int64_t n_moves = a.n_sweeps * sd.N;
    const uint64_t period = (uint64_t)sd.recompute_every * (uint64_t)sd.N;

    for (int64_t it = 0; it < n_moves; ++it) {
        double jac = 1.0;   // Hastings factor of a bond-length move (thread 0)
        if (threadIdx.x == 0) {   // proposal, serial Marsaglia, centre and rotation
            Proposal P;
            propose_select(sd, stream_block(seed, t, 0), stream_block(seed, t, 1), stream_block(seed, t, 2), &P);
            if (P.type == PHAST_PIVOT || P.type == PHAST_ROT || P.type == PHAST_CAP) {
                double3 ax = make_double3(0.0, 0.0, 1.0);
                for (int j = 0; j < PHAST_MARSAGLIA_TRIES; ++j)
                    if (marsaglia_try(stream_block(seed, t, 3u + j), &ax)) break;
                P.axis = ax;
            }
            const int o = sd.chain_off[P.chain], n = sd.chain_off[P.chain + 1] - o;
            int ok = 1;
            double3 center = make_double3(0, 0, 0), axis = P.axis, step = P.disp;
            if (P.type == PHAST_PIVOT) {
                center = ld3(x64 + 3 * (o + P.index));
            } else if (P.type == PHAST_CAP) {
                center = ld3(x64 + 3 * (o + (P.index > 0 ? P.index - 1 : 1)));
            } else if (P.type == PHAST_BOND) {
                ok = bond_step(x64, o, n, P.index, P.angle, &step, &jac) ? 1 : 0;
            } else if (P.type == PHAST_ROT) {
                center = centroid_serial(x64, o, n);
            } else if (P.type == PHAST_CRANK) {
                const int i = o + P.index;
                double3 p0 = ld3(x64 + 3 * (i - 1)), p1 = ld3(x64 + 3 * (i + 1));
                double ex = xsub(p1.x, p0.x), ey = xsub(p1.y, p0.y), ez = xsub(p1.z, p0.z);
                double len = xsqrt(xadd(xadd(xmul(ex, ex), xmul(ey, ey)), xmul(ez, ez)));
                if (!(len > 1e-12)) ok = 0;
                else axis = make_double3(xdiv(ex, len), xdiv(ey, len), xdiv(ez, len));
                center = p0;
            }
            if (P.type != PHAST_TRANS && P.type != PHAST_BOND && ok) {
                double sn, cs;
                taylor_sincos(P.angle, &sn, &cs);
                Rot3 R = rodrigues(axis.x, axis.y, axis.z, sn, cs);
                for (int k = 0; k < 9; ++k) sR[k] = R.m[k];
            }
            sC[0] = center.x; sC[1] = center.y; sC[2] = center.z;
            sD[0] = step.x; sD[1] = step.y; sD[2] = step.z;
            sP = P;
            s_ok = ok;
        }
        __syncthreads();
        const Proposal P = sP;
        const MoveSet M = move_set(sd, P.type, P.chain, P.index);
        const int m = M.hi - M.lo + 1;
        const bool ok = s_ok;
        double dE = __longlong_as_double(0x7ff8000000000000ll);
        int wall = 0;
        if (ok) {
            Rot3 R;
            for (int k = 0; k < 9; ++k) R.m[k] = sR[k];
            const double3 center = make_double3(sC[0], sC[1], sC[2]), step = make_double3(sD[0], sD[1], sD[2]);
            int out = 0;
            for (int q = threadIdx.x; q < m; q += blockDim.x) {
                const double3 x = ld3(x64 + 3 * (M.lo + q));
                double3 y = (P.type == PHAST_TRANS || P.type == PHAST_BOND)
                    ? make_double3(xadd(x.x, step.x), xadd(x.y, step.y), xadd(x.z, step.z))
                    : rotate_about(R, center, x);
                nx[3 * q] = y.x; nx[3 * q + 1] = y.y; nx[3 * q + 2] = y.z;
                out |= !inside64(sd, y);
            }
            wall = __syncthreads_or(out);
        }
        if (ok && wall) dE = INFINITY;   // beyond the container's wall
        if (ok && !wall) {
            // local terms
            int vb0, nb, jt0, nt, fb0, nf;
            local_window(sd, P.type, P.chain, P.index, &vb0, &nb, &jt0, &nt, &fb0, &nf);
            const int o = sd.chain_off[P.chain];
            const int nc = P.type == PHAST_BOND;   // the stretched bond's pair, counted below, taken back
            double part = 0.0;
            for (int itm = threadIdx.x; itm < 2 * (nb + nt + nf + nc); itm += blockDim.x) {
                const bool after = itm & 1;
                const int k = itm >> 1;
                auto pos = [&](int j) -> double3 {
                    if (after && j >= M.lo && j <= M.hi) return ld3(nx + 3 * (j - M.lo));
                    return ld3(x64 + 3 * j);
                };
                double term;
                if (k < nb) term = sd.k_bend * bend_term(pos, o, vb0 + k);
                else if (k < nb + nt) term = -sd.k_tors * torsion_term(pos, o, jt0 + (k - nb));
                else if (k < nb + nt + nf) term = fene_term(sd, pos, o, fb0 + (k - nb - nt));
                else {
                    const double3 a = pos(o + P.index), b = pos(o + P.index + 1);
                    const double dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
                    term = -sd.k_lj_intra * lj64(dx * dx + dy * dy + dz * dz,
                                                 sd.C[2 * sd.seq[o + P.index] + sd.seq[o + P.index + 1]]);
                }
                part += after ? term : -term;
            }
            // pairs (moved i, unmoved j), before and after
            const int U = sd.N - m;
            for (int64_t p = threadIdx.x; p < (int64_t)m * U; p += blockDim.x) {
                const int q = (int)(p / U), tt = (int)(p % U);
                const int i = M.lo + q, j = tt < M.lo ? tt : tt + m;
                if (j == M.ex0 || j == M.ex1 || j == M.ex2) continue;
                const bool inter = sd.chain_of[j] != P.chain;
                const double C = sd.C[2 * sd.seq[i] + sd.seq[j]];
                const double kap = inter ? sd.k_lj_inter : sd.k_lj_intra;
                const double3 xj = ld3(x64 + 3 * j), xo = ld3(x64 + 3 * i), xn = ld3(nx + 3 * q);
                double dx = xo.x - xj.x, dy = xo.y - xj.y, dz = xo.z - xj.z;
                double ex = xn.x - xj.x, ey = xn.y - xj.y, ez = xn.z - xj.z;
                if (inter) {
                    dx = mimage64(dx, sd.box_L, sd.inv_L); dy = mimage64(dy, sd.box_L, sd.inv_L);
                    dz = mimage64(dz, sd.box_L, sd.inv_L); ex = mimage64(ex, sd.box_L, sd.inv_L);
                    ey = mimage64(ey, sd.box_L, sd.inv_L); ez = mimage64(ez, sd.box_L, sd.inv_L);
                }
                part += kap * (lj64(ex * ex + ey * ey + ez * ez, C) - lj64(dx * dx + dy * dy + dz * dz, C));
            }
            dE = block_sum(part, red);
        }
        if (threadIdx.x == 0) {
            const double E_new = E + dE;
            const int b_new = bin_of(sd, E_new);
            int acc = 0;
            if (b_new >= 0) {
                const double dl = lnW[b_new] - lnW[bin];
                acc = P.type == PHAST_BOND ? accept_stretch(dl, jac, P) : (dl >= 0.0) || (u52(P.uz, P.uw) < exp(dl));
            }
            s_acc = acc;
            if (acc) { E = E_new; bin = b_new; }
            if (hs) atomicAdd(hs + bin, 1ull);
            if (hw) atomicAdd(hw + bin, 1u);
            ls->attempts[P.type]++;
            ls->accepts[P.type] += acc;
            ls->pair_evals += move_pair_evals(sd, P.type, M);
            ls->pair_evals_inter += move_pair_evals_inter(sd, P.type, P.chain, M);
            if (tracing) {
                phast_trace tr;
                tr.dE = dE;
                tr.bin_after = bin;
                tr.accepted = acc;
                a.trace[(int64_t)w_local * n_moves + it] = tr;
            }
        }
        __syncthreads();
        if (s_acc)
            for (int q = threadIdx.x; q < 3 * m; q += blockDim.x) x64[3 * M.lo + q] = nx[q];
        ++t;
        __syncthreads();
        if (period && (t % period) == 0) {
            const double Ef = block_full_energy64(sd, x64, red);
            if (threadIdx.x == 0) {
                ls->drift_max = fmax(ls->drift_max, fabs(E - Ef));
                if (isfinite(Ef)) {   // as in the batched form: edge bin when just out of range
                    const int bf = bin_of(sd, Ef);
                    E = Ef;
                    bin = bf >= 0 ? bf : (Ef < sd.e_min ? 0 : sd.n_bins - 1);
                    if (bf < 0) ls->recompute_outside++;
                }
                ls->recomputes++;
            }
        }
    }
    if (threadIdx.x == 0) {
        a.E[gw] = E;
        a.bin[gw] = bin;
        a.t[gw] = t;
        phast_walker_stats* st = a.stats + gw;
        for (int i = 0; i < PHAST_N_MOVES; ++i) { st->attempts[i] += ls->attempts[i]; st->accepts[i] += ls->accepts[i]; }
        st->pair_evals += ls->pair_evals;
        st->pair_evals_inter += ls->pair_evals_inter;
        st->recomputes += ls->recomputes;
        st->recompute_outside += ls->recompute_outside;
        st->drift_max = fmax(st->drift_max, ls->drift_max);
    }
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
typedef void (*batched_fn)(const SweepArgs);

template <bool G>
batched_fn pick_batched_g(int tpw, bool fp32, bool lean) {
    switch (tpw) {
        case 4: return fp32 ? sweep_batched_kernel<4, float, G> : sweep_batched_kernel<4, double, G>;
        case 8: return fp32 ? sweep_batched_kernel<8, float, G> : sweep_batched_kernel<8, double, G>;
        case 16:
            if (fp32 && lean) return sweep_batched_kernel<16, float, G, 2>;
            return fp32 ? sweep_batched_kernel<16, float, G> : sweep_batched_kernel<16, double, G>;
        case 32: return fp32 ? sweep_batched_kernel<32, float, G> : sweep_batched_kernel<32, double, G>;
        default: return nullptr;
    }
}

// Systems below this size run the 16-lane FP32 tiles in the 64-register build
// (measured on GB300: 4 x 9-mers +28 %, 2 x 13-mers in a sphere +10 %; 72
// monomers -9 %).
constexpr int kLeanMaxN = 48;

batched_fn pick_batched(int tpw, bool fp32, bool geom, bool lean) {
    if (tpw == 1)
        return geom ? (fp32 ? sweep_lane_kernel<float, true> : sweep_lane_kernel<double, true>)
                    : (fp32 ? sweep_lane_kernel<float, false> : sweep_lane_kernel<double, false>);
    return geom ? pick_batched_g<true>(tpw, fp32, lean) : pick_batched_g<false>(tpw, fp32, lean);
}


size_t batched_smem(const phast_ctx* c, bool fp32, int wpc, SlotLayout* L) {
    *L = fp32 ? slot_layout<float>(c->max_N, c->max_nc, c->max_chain)
              : slot_layout<double>(c->max_N, c->max_nc, c->max_chain);
    return sizeof(SysDesc) + (size_t)align16(4 * c->max_bins) + (size_t)wpc * L->bytes;
}

// Shared memory of a one-walker-per-thread tile of wpc walkers (wpc / 32 warp slots).
size_t lane_smem(const phast_ctx* c, bool fp32, int wpc, LaneLayout* L) {
    *L = fp32 ? lane_layout<float>(c->max_N, c->max_nc, c->max_chain)
              : lane_layout<double>(c->max_N, c->max_nc, c->max_chain);
    return sizeof(SysDesc) + (size_t)align16(4 * c->max_bins) + (size_t)(wpc / 32) * L->bytes;
}

size_t tile_smem(const phast_ctx* c, bool fp32, int tpw, int wpc) {
    SlotLayout S;
    LaneLayout L;
    return tpw == 1 ? lane_smem(c, fp32, wpc, &L) : batched_smem(c, fp32, wpc, &S);
}

double system_cost(const SysDesc& d) {
    // expected pair evaluations per sweep and walker, for ordering the tiles
    double pv = 0.0, n = d.N;
    for (int c = 0; c < d.n_chains; ++c) {
        double nc = d.chain_off[c + 1] - d.chain_off[c];
        pv += (d.p[PHAST_PIVOT] * nc / 4.0 * (n - nc / 4.0) + (d.p[PHAST_TRANS] + d.p[PHAST_ROT]) * nc * (n - nc) +
               d.p[PHAST_CRANK] * n) / d.n_chains;
    }
    return pv * n * d.n_walkers + 1.0;
}

int fill_args(const phast_ctx* c, int64_t n_sweeps, const double* lnW, int n_jk, uint64_t* hist_sum,
              uint32_t* hist_walker, phast_trace* trace, int trace_walkers, int wpc, SweepArgs* a) {
    memset(a, 0, sizeof(*a));
    a->descs = c->d_desc;
    a->n_sys = c->n_sys;
    a->n_jk = n_jk;
    a->wpc = wpc;
    a->n_sweeps = n_sweeps;
    int64_t hs = 0;
    for (int s = 0; s < c->n_sys; ++s) { a->hs_off[s] = hs; hs += (int64_t)n_jk * c->desc[s].n_bins; }
    for (int p = 0; p < c->n_sys; ++p) a->order[p] = c->order[p];
    a->xyz = c->xyz;
    a->E = c->E;
    a->bin = c->bin;
    a->t = c->t;
    a->seed = c->seed;
    a->stats = c->stats;
    a->lnW = lnW;
    a->hist_sum = reinterpret_cast<unsigned long long*>(hist_sum);
    a->hist_walker = hist_walker;
    a->trace = trace;
    a->trace_walkers = trace_walkers;
    a->tile_counter = c->tile_counter;
    a->scratch = c->plain_scratch;
    a->scratch_stride = 8 * c->max_chain;   // keeps each walker's records 16-byte aligned
    a->hist_bins = c->max_bins;
    a->hist_flush = c->hist_flush;
    // the walkers of a tile add at most wpc n_sweeps N counts to its shared histogram
    a->hist_flush_on = (uint64_t)wpc * (uint64_t)n_sweeps * (uint64_t)c->max_N >= (uint64_t)c->hist_flush;
    return PHAST_OK;
}

// Tiles of at most wpc walkers, as many as make whole rounds of the grid: the
// last system in the order (the cheapest) is cut into smaller tiles so that no
// CTA idles through the final round while others finish theirs.
void layout_tiles(const phast_ctx* c, int wpc, int grid, SweepArgs* a) {
    int nt[PHAST_MAX_SYSTEMS], total = 0;
    for (int p = 0; p < c->n_sys; ++p) {
        nt[p] = (c->desc[a->order[p]].n_walkers + wpc - 1) / wpc;
        total += nt[p];
    }
    const int want = (total + grid - 1) / grid * grid;
    for (int p = c->n_sys - 1; p >= 0 && total < want; --p) {
        const int add = std::min(want - total, c->desc[a->order[p]].n_walkers - nt[p]);
        nt[p] += add;
        total += add;
    }
    int start = 0;
    for (int p = 0; p < c->n_sys; ++p) {
        a->tile_start[p] = start;
        a->tiles[p] = nt[p];
        start += nt[p];
    }
    a->tile_start[c->n_sys] = start;
    a->n_tiles = start;
}

// Whether a system type with a torsion term starts with a bend whose normal is
// under 1e-5 (bonds within ~1e-5 rad of collinear: a straight start, collinear
// up to FP64 rounding; a random start has such a bend with probability ~1e-11 per
// bend).  Pivot moves keep such stretches and keep making nearly collinear bonds
// with small angles; FP32 resolves none of them, so such contexts run the build
// that takes those dihedrals in FP64 on the exact positions.
bool starts_near_straight(const phast_ctx* c, const double* xyz0) {
    for (int s = 0; s < c->n_sys; ++s) {
        const SysDesc& d = c->desc[s];
        if (d.k_tors == 0.0) continue;
        for (int w = 0; w < d.n_walkers; ++w) {
            const double* x = xyz0 + d.xyz_off + (int64_t)w * d.N * 3;
            for (int ch = 0; ch < d.n_chains; ++ch)
                for (int j = d.chain_off[ch]; j + 2 < d.chain_off[ch + 1]; ++j) {
                    const double* a = x + 3 * j;
                    const double b0[3] = {a[3] - a[0], a[4] - a[1], a[5] - a[2]};
                    const double b1[3] = {a[6] - a[3], a[7] - a[4], a[8] - a[5]};
                    const double n[3] = {b0[1] * b1[2] - b0[2] * b1[1], b0[2] * b1[0] - b0[0] * b1[2],
                                         b0[0] * b1[1] - b0[1] * b1[0]};
                    if (n[0] * n[0] + n[1] * n[1] + n[2] * n[2] < 1e-10) return true;
                }
        }
    }
    return false;
}

// Whether the context runs the general build (the paper's own geometry, and the
// exact FP64 path of the local terms): a system type needs that geometry, or a
// type with torsion starts near straight.
bool uses_geometry(const phast_ctx* c) {
    if (c->near_straight) return true;
    for (int s = 0; s < c->n_sys; ++s) {
        const SysDesc& d = c->desc[s];
        if (d.has_sphere || d.k_fene != 0.0 || d.p[PHAST_BOND] > 0.0 || d.p[PHAST_CAP] > 0.0) return true;
    }
    return false;
}

struct BatchedLaunch {
    batched_fn fn;
    int grid, threads;
    size_t smem;
    SweepArgs a;
};

// Host-side part of a batched launch: kernel choice, shared-memory limit,
// occupancy and tile layout (nothing is queued on a stream).
int prepare_batched(phast_ctx* c, const SweepArgs& a0, int tpw, int wpc, bool fp32, BatchedLaunch* L) {
    L->a = a0;
    SlotLayout SL;
    LaneLayout LLay;
    L->smem = tpw == 1 ? lane_smem(c, fp32, wpc, &LLay) : batched_smem(c, fp32, wpc, &SL);
    L->a.L = SL;
    L->a.LL = LLay;
    L->fn = pick_batched(tpw, fp32, uses_geometry(c), c->max_N < kLeanMaxN);
    if (!L->fn) return phast_set_error(PHAST_EINVAL, "threads per walker %d not in {1, 4, 8, 16, 32}", tpw);
    L->threads = tpw * wpc;
    const int max_threads = tpw == 1 ? kLaneMaxThreads : kMaxTileThreads;
    if (L->threads < 32 || L->threads > max_threads || L->threads % 32)
        return phast_set_error(PHAST_EINVAL, "tile of %d x %d threads is not a whole number of warps <= %d", tpw, wpc,
                               max_threads);
    int max_sm = 0;
    PHAST_CUDA_TRY(cudaDeviceGetAttribute(&max_sm, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    if (L->smem + 64 > (size_t)max_sm)
        return phast_set_error(PHAST_EINVAL, "tile needs %zu bytes of shared memory (> %d)", L->smem, max_sm);
    PHAST_CUDA_TRY(cudaFuncSetAttribute(L->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L->smem));
    int per_sm = 0, n_sm = 0;
    PHAST_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, L->fn, L->threads, L->smem));
    const batched_fn full = pick_batched(tpw, fp32, uses_geometry(c), false);
    if (tpw != 1 && L->fn != full) {   // the 64-register build pays only if more CTAs then share an SM
        int per_sm_full = 0;
        PHAST_CUDA_TRY(cudaFuncSetAttribute(full, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L->smem));
        PHAST_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_full, full, L->threads, L->smem));
        if (per_sm <= per_sm_full) {
            L->fn = full;
            per_sm = per_sm_full;
        }
    }
    PHAST_CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, c->device));
    if (per_sm < 1) return phast_set_error(PHAST_EINVAL, "tile of %d x %d does not fit on an SM", tpw, wpc);
    L->grid = per_sm * n_sm;
    layout_tiles(c, wpc, L->grid, &L->a);
    if (L->grid > L->a.n_tiles) L->grid = L->a.n_tiles;
    return PHAST_OK;
}

// Stream part: reset the tile counter, launch.
int enqueue_batched(phast_ctx* c, const BatchedLaunch& L, cudaStream_t st) {
    PHAST_CUDA_TRY(cudaMemsetAsync(c->tile_counter, 0, sizeof(int32_t), st));
    L.fn<<<L.grid, L.threads, L.smem, st>>>(L.a);
    PHAST_CUDA_TRY(cudaGetLastError());
    return PHAST_OK;
}

int launch_batched(phast_ctx* c, const SweepArgs& a0, int tpw, int wpc, bool fp32, cudaStream_t st) {
    BatchedLaunch L;
    const int rc = prepare_batched(c, a0, tpw, wpc, fp32, &L);
    if (rc != PHAST_OK) return rc;
    return enqueue_batched(c, L, st);
}

void default_tile(const phast_ctx* c, int* tpw, int* wpc) {
    // one warp per walker for large systems, smaller groups for small ones;
    // as many walkers per CTA as 512 threads and the shared memory allow
    const int N = c->max_N;
    const bool fp32 = c->desc[0].pair_precision == 32;
    *tpw = N >= 128 ? 32 : (N >= 48 || (fp32 && N > 16) ? 16 : 8);
    int w = kMaxTileThreads / *tpw;
    SlotLayout L;
    while (w * *tpw > 32 && batched_smem(c, fp32, w, &L) > 220 * 1024) w >>= 1;
    *wpc = w;
}

uint32_t crc32(const unsigned char* p, size_t n, uint32_t crc) {
    crc = ~crc;
    for (size_t i = 0; i < n; ++i) {
        crc ^= p[i];
        for (int k = 0; k < 8; ++k) crc = (crc >> 1) ^ (0xEDB88320u & (0u - (crc & 1u)));
    }
    return ~crc;
}

struct CkptHeader {
    uint32_t magic, version;
    int32_t n_sys, W;
    int64_t xyz_total;
    int32_t N[PHAST_MAX_SYSTEMS];
    int32_t walkers[PHAST_MAX_SYSTEMS];
};

}  // namespace

// ---------------------------------------------------------------------------
// Entry points.
// ---------------------------------------------------------------------------
extern "C" int phast_ctx_create(phast_ctx** out, int32_t n_systems, const phast_system* sys, const phast_ff* ff,
                                const phast_muca_params* mp, const int32_t* walkers, const uint64_t* seeds,
                                const double* xyz0, void* stream) {
    if (!out) return phast_set_error(PHAST_EINVAL, "phast_ctx_create: NULL out");
    *out = nullptr;
    if (n_systems < 1 || n_systems > PHAST_MAX_SYSTEMS)
        return phast_set_error(PHAST_EINVAL, "phast_ctx_create: n_systems %d outside [1, %d]", n_systems, PHAST_MAX_SYSTEMS);
    if (!sys || !ff || !mp || !walkers || !seeds || !xyz0)
        return phast_set_error(PHAST_EINVAL, "phast_ctx_create: NULL argument");
    phast_ctx* c = (phast_ctx*)calloc(1, sizeof(phast_ctx));
    if (!c) return phast_set_error(PHAST_ENOMEM, "phast_ctx_create: host allocation");
    c->n_sys = n_systems;
    int64_t xyz_total = 0, lnw_total = 0, hw_total = 0;
    int W = 0;
    for (int s = 0; s < n_systems; ++s) {
        char what[64];
        snprintf(what, sizeof(what), "phast_ctx_create (system %d)", s);
        int rc = phast_build_desc(&sys[s], &ff[s], &mp[s], &c->desc[s], what);
        if (rc) { free(c); return rc; }
        if (walkers[s] < 1) { free(c); return phast_set_error(PHAST_EINVAL, "%s: walkers < 1", what); }
        SysDesc& d = c->desc[s];
        d.walker_off = W;
        d.n_walkers = walkers[s];
        d.xyz_off = xyz_total;
        d.lnw_off = (int32_t)lnw_total;
        d.hw_off = hw_total;
        W += walkers[s];
        xyz_total += (int64_t)walkers[s] * d.N * 3;
        lnw_total += d.n_bins;
        hw_total += (int64_t)walkers[s] * d.n_bins;
        c->max_N = std::max(c->max_N, d.N);
        c->max_nc = std::max(c->max_nc, d.n_chains);
        c->max_chain = std::max(c->max_chain, d.max_chain);
        c->max_bins = std::max(c->max_bins, d.n_bins);
    }
    for (int64_t i = 0; i < xyz_total; ++i)
        if (!isfinite(xyz0[i])) { free(c); return phast_set_error(PHAST_ENONFINITE, "phast_ctx_create: non-finite xyz0[%lld]", (long long)i); }
    c->W = W;
    c->xyz_total = xyz_total;
    c->lnw_total = lnw_total;
    c->hw_total = hw_total;
    c->near_straight = starts_near_straight(c, xyz0);
    // tile order: most expensive system types first
    std::vector<std::pair<double, int>> cost;
    for (int s = 0; s < n_systems; ++s) cost.push_back({-system_cost(c->desc[s]), s});
    std::sort(cost.begin(), cost.end());
    for (int p = 0; p < n_systems; ++p) c->order[p] = cost[p].second;

    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaGetDevice(&c->device);
    size_t bytes_stats = sizeof(phast_walker_stats) * (size_t)W;
    if (e == cudaSuccess) e = cudaMalloc(&c->d_desc, sizeof(SysDesc) * n_systems);
    if (e == cudaSuccess) e = cudaMalloc(&c->xyz, sizeof(double) * xyz_total);
    if (e == cudaSuccess) e = cudaMalloc(&c->E, sizeof(double) * W);
    if (e == cudaSuccess) e = cudaMalloc(&c->bin, sizeof(int32_t) * W);
    if (e == cudaSuccess) e = cudaMalloc(&c->t, sizeof(uint64_t) * W);
    if (e == cudaSuccess) e = cudaMalloc(&c->seed, sizeof(uint64_t) * W);
    if (e == cudaSuccess) e = cudaMalloc(&c->stats, bytes_stats);
    if (e == cudaSuccess) e = cudaMalloc(&c->tile_counter, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&c->plain_scratch, sizeof(double) * 8 * (size_t)c->max_chain * W);
    if (e != cudaSuccess) {
        phast_ctx_destroy(c);
        return phast_set_error(e == cudaErrorMemoryAllocation ? PHAST_ENOMEM : PHAST_ECUDA,
                               "phast_ctx_create: %s", cudaGetErrorString(e));
    }
    e = cudaMemcpyAsync(c->d_desc, c->desc, sizeof(SysDesc) * n_systems, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->xyz, xyz0, sizeof(double) * xyz_total, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->seed, seeds, sizeof(uint64_t) * W, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->t, 0, sizeof(uint64_t) * W, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->stats, 0, bytes_stats, st);
    if (e == cudaSuccess) {
        init_energy_kernel<<<(W + 3) / 4, 128, 0, st>>>(c->d_desc, n_systems, W, c->xyz, c->E, c->bin);
        e = cudaGetLastError();
    }
    std::vector<int32_t> bins(W);
    std::vector<double> Es(W);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bins.data(), c->bin, sizeof(int32_t) * W, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(Es.data(), c->E, sizeof(double) * W, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        phast_ctx_destroy(c);
        return phast_set_error(PHAST_ECUDA, "phast_ctx_create: %s", cudaGetErrorString(e));
    }
    for (int w = 0; w < W; ++w)
        if (bins[w] < 0) {
            phast_ctx_destroy(c);
            return phast_set_error(PHAST_ERANGE, "phast_ctx_create: walker %d starts at E = %.17g outside its bins", w, Es[w]);
        }
    default_tile(c, &c->tpw, &c->wpc);
    c->hist_flush = kHistFlushDefault;
    *out = c;
    return PHAST_OK;
}

extern "C" void phast_ctx_destroy(phast_ctx* c) {
    if (!c) return;
    cudaFree(c->d_desc);
    cudaFree(c->xyz);
    cudaFree(c->E);
    cudaFree(c->bin);
    cudaFree(c->t);
    cudaFree(c->seed);
    cudaFree(c->stats);
    cudaFree(c->tile_counter);
    cudaFree(c->plain_scratch);
    free(c);
}

extern "C" int phast_ctx_info(const phast_ctx* c, int32_t s, int64_t* info8) {
    if (!c || !info8) return phast_set_error(PHAST_EINVAL, "phast_ctx_info: NULL argument");
    if (s < 0 || s >= c->n_sys) return phast_set_error(PHAST_EINVAL, "phast_ctx_info: system %d of %d", s, c->n_sys);
    const SysDesc& d = c->desc[s];
    info8[0] = c->W;
    info8[1] = d.N;
    info8[2] = d.n_bins;
    info8[3] = d.walker_off;
    info8[4] = d.xyz_off;
    info8[5] = d.lnw_off;
    info8[6] = c->n_sys;
    info8[7] = d.n_walkers;
    return PHAST_OK;
}

extern "C" int phast_ctx_get_state(const phast_ctx* c, double* xyz, double* E, int32_t* bin, uint64_t* t,
                                   phast_walker_stats* stats, void* stream) {
    if (!c) return phast_set_error(PHAST_EINVAL, "phast_ctx_get_state: NULL context");
    cudaStream_t st = (cudaStream_t)stream;
    if (xyz) PHAST_CUDA_TRY(cudaMemcpyAsync(xyz, c->xyz, sizeof(double) * c->xyz_total, cudaMemcpyDefault, st));
    if (E) PHAST_CUDA_TRY(cudaMemcpyAsync(E, c->E, sizeof(double) * c->W, cudaMemcpyDefault, st));
    if (bin) PHAST_CUDA_TRY(cudaMemcpyAsync(bin, c->bin, sizeof(int32_t) * c->W, cudaMemcpyDefault, st));
    if (t) PHAST_CUDA_TRY(cudaMemcpyAsync(t, c->t, sizeof(uint64_t) * c->W, cudaMemcpyDefault, st));
    if (stats) PHAST_CUDA_TRY(cudaMemcpyAsync(stats, c->stats, sizeof(phast_walker_stats) * c->W, cudaMemcpyDefault, st));
    return PHAST_OK;
}

extern "C" int phast_ctx_set_state(phast_ctx* c, const double* xyz, const double* E, const int32_t* bin,
                                   const uint64_t* t, const phast_walker_stats* stats, void* stream) {
    if (!c) return phast_set_error(PHAST_EINVAL, "phast_ctx_set_state: NULL context");
    cudaStream_t st = (cudaStream_t)stream;
    if (xyz) PHAST_CUDA_TRY(cudaMemcpyAsync(c->xyz, xyz, sizeof(double) * c->xyz_total, cudaMemcpyDefault, st));
    if (E) PHAST_CUDA_TRY(cudaMemcpyAsync(c->E, E, sizeof(double) * c->W, cudaMemcpyDefault, st));
    if (bin) PHAST_CUDA_TRY(cudaMemcpyAsync(c->bin, bin, sizeof(int32_t) * c->W, cudaMemcpyDefault, st));
    if (t) PHAST_CUDA_TRY(cudaMemcpyAsync(c->t, t, sizeof(uint64_t) * c->W, cudaMemcpyDefault, st));
    if (stats) PHAST_CUDA_TRY(cudaMemcpyAsync(c->stats, stats, sizeof(phast_walker_stats) * c->W, cudaMemcpyDefault, st));
    return PHAST_OK;
}

extern "C" int phast_ctx_set_tile(phast_ctx* c, int32_t tpw, int32_t wpc) {
    if (!c) return phast_set_error(PHAST_EINVAL, "phast_ctx_set_tile: NULL context");
    int dt, dw;
    default_tile(c, &dt, &dw);
    if (tpw == 0) tpw = dt;
    if (wpc == 0) wpc = dw;
    if (tpw != 1 && tpw != 4 && tpw != 8 && tpw != 16 && tpw != 32)
        return phast_set_error(PHAST_EINVAL, "phast_ctx_set_tile: threads per walker %d not in {1, 4, 8, 16, 32}", tpw);
    const int max_threads = tpw == 1 ? kLaneMaxThreads : kMaxTileThreads;
    if (wpc < 1 || tpw * wpc > max_threads || (tpw * wpc) % 32)
        return phast_set_error(PHAST_EINVAL, "phast_ctx_set_tile: %d walkers of %d threads is not a whole number of warps <= %d",
                               wpc, tpw, max_threads);
    c->tpw = tpw;
    c->wpc = wpc;
    return PHAST_OK;
}

extern "C" int phast_ctx_set_hist_flush(phast_ctx* c, uint32_t count) {
    if (!c) return phast_set_error(PHAST_EINVAL, "phast_ctx_set_hist_flush: NULL context");
    if (count > kHistFlushDefault || (count & (count - 1u)))
        return phast_set_error(PHAST_EINVAL, "phast_ctx_set_hist_flush: %u is not a power of two <= 2^31", count);
    c->hist_flush = count ? count : kHistFlushDefault;
    return PHAST_OK;
}

extern "C" int phast_ctx_get_tile(const phast_ctx* c, int32_t* tpw, int32_t* wpc) {
    if (!c || !tpw || !wpc) return phast_set_error(PHAST_EINVAL, "phast_ctx_get_tile: NULL argument");
    *tpw = c->tpw;
    *wpc = c->wpc;
    return PHAST_OK;
}

extern "C" int phast_muca_sweep(phast_ctx* c, int64_t n_sweeps, const double* lnW, int32_t form, int32_t n_jk,
                                uint64_t* hist_sum, uint32_t* hist_walker, phast_trace* trace,
                                int32_t trace_walkers, void* stream) {
    if (!c) return phast_set_error(PHAST_EINVAL, "phast_muca_sweep: NULL context");
    if (n_sweeps < 0) return phast_set_error(PHAST_EINVAL, "phast_muca_sweep: n_sweeps < 0");
    if (!lnW) return phast_set_error(PHAST_EINVAL, "phast_muca_sweep: NULL lnW");
    if (form != PHAST_FORM_BATCHED && form != PHAST_FORM_PLAIN)
        return phast_set_error(PHAST_EINVAL, "phast_muca_sweep: unknown form %d", form);
    if (!hist_sum) n_jk = 1;
    if (n_jk < 1) return phast_set_error(PHAST_EINVAL, "phast_muca_sweep: n_jk < 1");
    for (int s = 0; s < c->n_sys; ++s)
        if (n_jk > c->desc[s].n_walkers)
            return phast_set_error(PHAST_EINVAL, "phast_muca_sweep: n_jk %d > walkers of system %d", n_jk, s);
    if (trace && (trace_walkers < 0 || trace_walkers > c->desc[0].n_walkers))
        return phast_set_error(PHAST_EINVAL, "phast_muca_sweep: trace_walkers outside [0, walkers of system 0]");
    if (hist_walker && (uint64_t)n_sweeps * (uint64_t)c->max_N >= (1ull << 32))
        return phast_set_error(PHAST_EINVAL,
                               "phast_muca_sweep: %lld sweeps x %d moves add >= 2^32 counts to a walker's uint32 "
                               "histogram (hist_walker); split the call", (long long)n_sweeps, c->max_N);
    if (n_sweeps == 0) return PHAST_OK;
    cudaStream_t st = (cudaStream_t)stream;
    SweepArgs a;
    if (form == PHAST_FORM_PLAIN) {
        fill_args(c, n_sweeps, lnW, n_jk, hist_sum, hist_walker, trace, trace_walkers, 1, &a);
        sweep_plain_kernel<<<c->W, kPlainThreads, 0, st>>>(a, c->W);
        PHAST_CUDA_TRY(cudaGetLastError());
        return PHAST_OK;
    }
    bool fp32 = c->desc[0].pair_precision == 32;
    for (int s = 1; s < c->n_sys; ++s)
        if ((c->desc[s].pair_precision == 32) != fp32)
            return phast_set_error(PHAST_EINVAL, "phast_muca_sweep: system types mix pair precisions");
    fill_args(c, n_sweeps, lnW, n_jk, hist_sum, hist_walker, trace, trace_walkers, c->wpc, &a);
    return launch_batched(c, a, c->tpw, c->wpc, fp32, st);
}

extern "C" int phast_ctx_autotune(phast_ctx* c, const double* lnW, int32_t sweeps, void* stream) {
    if (!c || !lnW) return phast_set_error(PHAST_EINVAL, "phast_ctx_autotune: NULL argument");
    if (sweeps < 1) sweeps = 1;
    cudaStream_t st = (cudaStream_t)stream;
    const bool fp32 = c->desc[0].pair_precision == 32;
    // run the candidates on a scratch copy so the walkers' trajectories are untouched
    phast_ctx tmp = *c;
    cudaError_t e = cudaMalloc(&tmp.xyz, sizeof(double) * c->xyz_total);
    if (e == cudaSuccess) e = cudaMalloc(&tmp.E, sizeof(double) * c->W);
    if (e == cudaSuccess) e = cudaMalloc(&tmp.bin, sizeof(int32_t) * c->W);
    if (e == cudaSuccess) e = cudaMalloc(&tmp.t, sizeof(uint64_t) * c->W);
    if (e == cudaSuccess) e = cudaMalloc(&tmp.stats, sizeof(phast_walker_stats) * c->W);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    int best_t = c->tpw, best_w = c->wpc;
    float best = 1e30f;
    const int cands[][2] = {{32, 4}, {32, 8}, {32, 16}, {16, 4}, {16, 8}, {16, 16}, {16, 32}, {8, 8}, {8, 16},
                            {8, 32}, {8, 64}, {4, 16}, {4, 32}, {4, 64}, {4, 128}, {1, 32}, {1, 64}, {1, 128},
                            {1, 256}};
    for (const auto& cd : cands) {
        if (e != cudaSuccess) break;
        if (tile_smem(c, fp32, cd[0], cd[1]) > 220 * 1024) continue;
        e = cudaMemcpyAsync(tmp.xyz, c->xyz, sizeof(double) * c->xyz_total, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tmp.E, c->E, sizeof(double) * c->W, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tmp.bin, c->bin, sizeof(int32_t) * c->W, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tmp.t, c->t, sizeof(uint64_t) * c->W, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) break;
        SweepArgs a;
        fill_args(&tmp, sweeps, lnW, 1, nullptr, nullptr, nullptr, 0, cd[1], &a);
        BatchedLaunch BL;
        if (prepare_batched(&tmp, a, cd[0], cd[1], fp32, &BL) != PHAST_OK) continue;
        // an untimed launch first (module loading, caches), then the timed one;
        // the host-side set-up stays outside the events
        if (enqueue_batched(&tmp, BL, st) != PHAST_OK) continue;
        cudaEventRecord(e0, st);
        if (enqueue_batched(&tmp, BL, st) != PHAST_OK) continue;
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < best) { best = ms; best_t = cd[0]; best_w = cd[1]; }
    }
    cudaFree(tmp.xyz);
    cudaFree(tmp.E);
    cudaFree(tmp.bin);
    cudaFree(tmp.t);
    cudaFree(tmp.stats);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return phast_set_error(PHAST_ECUDA, "phast_ctx_autotune: %s", cudaGetErrorString(e));
    c->tpw = best_t;
    c->wpc = best_w;
    return PHAST_OK;
}

extern "C" int phast_ctx_checkpoint(phast_ctx* c, void* buf, size_t* len, void* stream) {
    if (!c || !len) return phast_set_error(PHAST_EINVAL, "phast_ctx_checkpoint: NULL argument");
    const size_t W = c->W;
    const size_t need = sizeof(CkptHeader) + sizeof(double) * c->xyz_total + W * (sizeof(double) + sizeof(int32_t) +
                        sizeof(uint64_t) + sizeof(phast_walker_stats)) + sizeof(uint32_t);
    if (!buf) { *len = need; return PHAST_OK; }
    if (*len < need) return phast_set_error(PHAST_EINVAL, "phast_ctx_checkpoint: buffer of %zu < %zu bytes", *len, need);
    unsigned char* p = (unsigned char*)buf;
    CkptHeader h;
    memset(&h, 0, sizeof(h));
    h.magic = 0x4B434850u;   // "PHCK"
    h.version = PHAST_VERSION;
    h.n_sys = c->n_sys;
    h.W = c->W;
    h.xyz_total = c->xyz_total;
    for (int s = 0; s < c->n_sys; ++s) { h.N[s] = c->desc[s].N; h.walkers[s] = c->desc[s].n_walkers; }
    memcpy(p, &h, sizeof(h));
    unsigned char* q = p + sizeof(h);
    cudaStream_t st = (cudaStream_t)stream;
    double* xyz = (double*)q;                   q += sizeof(double) * c->xyz_total;
    double* E = (double*)q;                     q += sizeof(double) * W;
    int32_t* bin = (int32_t*)q;                 q += sizeof(int32_t) * W;
    uint64_t* t = (uint64_t*)q;                 q += sizeof(uint64_t) * W;
    phast_walker_stats* stt = (phast_walker_stats*)q; q += sizeof(phast_walker_stats) * W;
    int rc = phast_ctx_get_state(c, xyz, E, bin, t, stt, stream);
    if (rc) return rc;
    PHAST_CUDA_TRY(cudaStreamSynchronize(st));
    uint32_t crc = crc32(p, (size_t)(q - p), 0);
    memcpy(q, &crc, sizeof(crc));
    *len = need;
    return PHAST_OK;
}

extern "C" int phast_ctx_restore(phast_ctx* c, const void* buf, size_t len, void* stream) {
    if (!c || !buf) return phast_set_error(PHAST_EINVAL, "phast_ctx_restore: NULL argument");
    size_t need = 0;
    phast_ctx_checkpoint(c, nullptr, &need, stream);
    if (len != need) return phast_set_error(PHAST_EINVAL, "phast_ctx_restore: %zu bytes, expected %zu", len, need);
    const unsigned char* p = (const unsigned char*)buf;
    CkptHeader h;
    memcpy(&h, p, sizeof(h));
    if (h.magic != 0x4B434850u || h.n_sys != c->n_sys || h.W != c->W || h.xyz_total != c->xyz_total)
        return phast_set_error(PHAST_EINVAL, "phast_ctx_restore: checkpoint of a different context");
    for (int s = 0; s < c->n_sys; ++s)
        if (h.N[s] != c->desc[s].N || h.walkers[s] != c->desc[s].n_walkers)
            return phast_set_error(PHAST_EINVAL, "phast_ctx_restore: system %d differs", s);
    uint32_t crc;
    memcpy(&crc, p + need - sizeof(uint32_t), sizeof(crc));
    if (crc != crc32(p, need - sizeof(uint32_t), 0))
        return phast_set_error(PHAST_EINVAL, "phast_ctx_restore: CRC mismatch (corrupt checkpoint)");
    const size_t W = c->W;
    const unsigned char* q = p + sizeof(h);
    const double* xyz = (const double*)q;       q += sizeof(double) * c->xyz_total;
    const double* E = (const double*)q;         q += sizeof(double) * W;
    const int32_t* bin = (const int32_t*)q;     q += sizeof(int32_t) * W;
    const uint64_t* t = (const uint64_t*)q;     q += sizeof(uint64_t) * W;
    const phast_walker_stats* stt = (const phast_walker_stats*)q;
    int rc = phast_ctx_set_state(c, xyz, E, bin, t, stt, stream);
    if (rc) return rc;
    PHAST_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    return PHAST_OK;
}

// ---------------------------------------------------------------------------
// One multicanonical iteration (sweeps, then Berg's step per system type) as a
// CUDA graph, replayed by phast_graph_launch.
// ---------------------------------------------------------------------------
struct phast_graph {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

extern "C" int phast_ctx_capture_iteration(phast_ctx* c, int64_t n_sweeps, double* lnW, int32_t n_jk,
                                           uint64_t* hist_sum, double* g_acc, double* flat_out, phast_graph** out,
                                           void* stream) {
    if (out) *out = nullptr;
    if (!c || !lnW || !hist_sum || !g_acc || !out)
        return phast_set_error(PHAST_EINVAL, "phast_ctx_capture_iteration: NULL argument");
    if (!stream)
        return phast_set_error(PHAST_EINVAL, "phast_ctx_capture_iteration: the legacy default stream cannot be captured");
    if (n_sweeps < 1) return phast_set_error(PHAST_EINVAL, "phast_ctx_capture_iteration: n_sweeps < 1");
    if (n_jk < 1) return phast_set_error(PHAST_EINVAL, "phast_ctx_capture_iteration: n_jk < 1");
    const bool fp32 = c->desc[0].pair_precision == 32;
    int max_bins = 1;
    size_t hs_bytes = 0;
    for (int s = 0; s < c->n_sys; ++s) {
        if (n_jk > c->desc[s].n_walkers)
            return phast_set_error(PHAST_EINVAL, "phast_ctx_capture_iteration: n_jk %d > walkers of system %d", n_jk, s);
        if ((c->desc[s].pair_precision == 32) != fp32)
            return phast_set_error(PHAST_EINVAL, "phast_ctx_capture_iteration: system types mix pair precisions");
        max_bins = std::max(max_bins, (int)c->desc[s].n_bins);
        hs_bytes += sizeof(uint64_t) * (size_t)n_jk * (size_t)c->desc[s].n_bins;
    }
    SweepArgs a;
    fill_args(c, n_sweeps, lnW, n_jk, hist_sum, nullptr, nullptr, 0, c->wpc, &a);
    BatchedLaunch L;
    int rc = prepare_batched(c, a, c->tpw, c->wpc, fp32, &L);
    if (rc != PHAST_OK) return rc;
    // the Berg kernel's shared-memory limit is set outside the capture
    rc = phast_launch_berg(max_bins, 1.0, nullptr, 1, nullptr, nullptr, nullptr, nullptr, nullptr, true);
    if (rc != PHAST_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return phast_set_error(PHAST_ECUDA, "phast_ctx_capture_iteration: %s", cudaGetErrorString(e));
    rc = PHAST_OK;
    if (cudaMemsetAsync(hist_sum, 0, hs_bytes, st) != cudaSuccess) rc = PHAST_ECUDA;
    if (rc == PHAST_OK) rc = enqueue_batched(c, L, st);
    for (int s = 0; s < c->n_sys && rc == PHAST_OK; ++s) {
        const SysDesc& d = c->desc[s];
        rc = phast_launch_berg(d.n_bins, d.bin_width, hist_sum + a.hs_off[s], n_jk, lnW + d.lnw_off, g_acc + d.lnw_off,
                               nullptr, flat_out ? flat_out + 4 * s : nullptr, st, false);
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(st, &graph);
    if (rc != PHAST_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return rc != PHAST_OK ? rc : phast_set_error(PHAST_ECUDA, "phast_ctx_capture_iteration: %s", cudaGetErrorString(e));
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return phast_set_error(PHAST_ECUDA, "phast_ctx_capture_iteration: instantiate: %s", cudaGetErrorString(e));
    }
    phast_graph* g = (phast_graph*)malloc(sizeof(phast_graph));
    if (!g) {
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        return phast_set_error(PHAST_ENOMEM, "phast_ctx_capture_iteration: out of host memory");
    }
    g->graph = graph;
    g->exec = exec;
    *out = g;
    return PHAST_OK;
}

extern "C" int phast_graph_launch(phast_graph* g, void* stream) {
    if (!g) return phast_set_error(PHAST_EINVAL, "phast_graph_launch: NULL graph");
    PHAST_CUDA_TRY(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
    return PHAST_OK;
}

extern "C" void phast_graph_destroy(phast_graph* g) {
    if (!g) return;
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    free(g);
}
