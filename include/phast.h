/*
 * phast.h -- C ABI of libphast.so, the GB300 (sm_103a) multicanonical sweep of
 * off-lattice AB heteropolymers (PHAST, arXiv 1702.01770).
 *
 * Conventions for every entry point:
 *  - Return 0 (PHAST_OK) or a negative PHAST_E* code; phast_last_error() gives
 *    a message for the calling thread's last failure.
 *  - "dev" pointers are CUDA device pointers on the current device; "host"
 *    pointers are ordinary host memory.  The library never frees or keeps a
 *    caller pointer beyond the call, except the phast_ctx object, which the
 *    caller creates and destroys.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Work is enqueued asynchronously on it; device-side failures surface at the
 *    next synchronising call (PHAST_ECUDA).
 *  - Coordinates are unwrapped Cartesian positions in units of the bond length
 *    r0 = 1 (Sec. 4: kappa_F = 0 fixes every bond at r0); energies are in units
 *    of the Lennard-Jones well depth with k_B = 1.  xyz arrays are [.][N][3]
 *    doubles, monomers of chain 0 first, then chain 1, and so on.
 *  - Sequences are uint8, 0 = A (hydrophobic), 1 = B (hydrophilic), Eq. 1.
 *
 * Equations are numbered in order of appearance in the paper: Eq. 1 C_LJ,
 * Eq. 2 H_single, Eq. 3 H_multi (Sec. 2.1); Eq. 4 S = k_B ln Omega, Eq. 5
 * beta(E), Eq. 6 C_V(E), Eq. 7 F(E), Eq. 8 S_muca (Sec. 2.2).
 */
#ifndef PHAST_H
#define PHAST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PHAST_VERSION 2

/* Hard limits of this build. */
#define PHAST_MAX_SYSTEMS 8      /* system types in one context */
#define PHAST_MAX_CHAINS 16      /* chains per system */
#define PHAST_MAX_MONOMERS 512   /* monomers per system (all chains) */
#define PHAST_MAX_BINS 16384     /* energy bins per system */
#define PHAST_MAX_ANGLE 1.0      /* largest rotation amplitude (rad) */

enum {
    PHAST_OK = 0,
    PHAST_EINVAL = -1,     /* bad argument (message says which) */
    PHAST_ERANGE = -2,     /* a walker energy outside its bin range */
    PHAST_ENOMEM = -3,     /* device or host allocation failed */
    PHAST_ECUDA = -4,      /* a CUDA runtime call failed */
    PHAST_ETIMEOUT = -5,   /* reserved: a bounded device wait ran out (no kernel of this build waits) */
    PHAST_EDEVICE = -6,    /* reserved: a kernel reported an error word (none of this build does:
                              bad inputs are refused on the host, bad moves rejected in the sweep) */
    PHAST_ENONFINITE = -7  /* non-finite coordinates or energy */
};

/* Move types (Sec. 3.2, UPDATE_ENGINE): pivot, Galilean translation and
 * rotation of a chain, crankshaft, bond-length change, spherical cap. */
enum { PHAST_PIVOT = 0, PHAST_TRANS = 1, PHAST_ROT = 2, PHAST_CRANK = 3, PHAST_BOND = 4, PHAST_CAP = 5 };
#define PHAST_N_MOVES 6

/* A system type: M chains (each >= 3 monomers), their AB sequence and the box.
 * box_L > 0: periodic cube of side box_L with the minimum image between
 * different chains (chains are never wrapped, so distances within a chain are
 * direct); box_L = 0: open space.  sphere_R > 0 (with box_L = 0): the steric
 * spherical container of Sec. 3.2 (box_size.h), a hard wall at |x| = sphere_R
 * about the origin -- a configuration with a monomer at |x|^2 > sphere_R^2 has
 * infinite energy; 0: none.  All pointers are host pointers. */
typedef struct {
    int32_t n_chains;
    const int32_t* chain_len;   /* host [n_chains] */
    const uint8_t* seq;         /* host [N], N = sum chain_len */
    double box_L;
    double sphere_R;
} phast_system;

/* Force field, Eq. 2/3 plus torsion:
 * E = k_fene R^2 sum_l C_F[2 s_l + s_{l+1}] ln(1 - ((r_{l,l+1} - r0) / R)^2)
 *   + k_bend sum_k (1 - cos theta_k) - k_tors sum_j cos tau_j
 *   + k_lj_intra sum_{i < j-1} (r^-12 - C r^-6) + k_lj_inter sum_{inter} (...).
 * C[2*s_i + s_j] is C_LJ of Eq. 1 (AA = 1, AB = BA = -1/2, BB = 1/2).  The
 * FENE bond term is the printed first term of Eq. 2 (r0 = fene_r0, R =
 * fene_R); it confines bonds when k_fene C_F < 0, and a bond with
 * |r - r0| >= R has infinite energy.  k_fene = 0 is the AB limit of Sec. 4:
 * bonds stay at their length and no bond term is evaluated. */
typedef struct {
    double k_bend, k_tors, k_lj_intra, k_lj_inter;
    double C[4];
    double k_fene, fene_r0, fene_R;
    double C_F[4];
} phast_ff;

/* Multicanonical set-up of one system type (Sec. 2.2, Eq. 8): bins
 * [e_min + k w, e_min + (k+1) w), k < n_bins; move mix p[] over the
 * PHAST_N_MOVES types (sums to 1; bond-length and spherical-cap moves need
 * k_fene != 0); amplitudes amax[] (angles in rad <= PHAST_MAX_ANGLE,
 * translation step per component, bond-length step); an FP64 full-energy
 * recompute every `recompute_every` sweeps (0 = never); pair arithmetic of the
 * batched sweep in FP32 (32) or FP64 (64). */
typedef struct {
    double e_min, bin_width;
    int32_t n_bins;
    int32_t recompute_every;
    double p[PHAST_N_MOVES];
    double amax[PHAST_N_MOVES];
    int32_t pair_precision;
    int32_t pad;
} phast_muca_params;

/* An explicit move (64 bytes): pivot about monomer `index` of `chain` by
 * `angle` around unit `axis`; translation by `disp`; rotation of the chain
 * about its centroid; crankshaft of monomer `index` about its neighbours' axis
 * (axis ignored); bond-length change of bond `index` (monomers index and
 * index+1) by `angle` (the shorter side slides along the bond; a change that
 * takes the bond through zero length is no move, dE NaN); spherical cap:
 * monomer `index` alone rotated by `angle` around `axis` through its bonded
 * neighbour index-1 (monomer 1 for index 0). */
typedef struct {
    int32_t type, chain, index, pad;
    double axis[3];
    double angle;
    double disp[3];
} phast_move;

/* Per-walker counters, accumulated over sweeps (dev arrays of these). */
typedef struct {
    uint64_t attempts[PHAST_N_MOVES];
    uint64_t accepts[PHAST_N_MOVES];
    uint64_t pair_evals;   /* 2 per (moved, unmoved) Lennard-Jones pair whose distance can change */
    uint64_t pair_evals_inter;  /* the part of pair_evals between different chains */
    uint64_t recomputes;
    double drift_max;      /* largest |E_running - E_full| seen at a recompute */
    uint64_t recompute_outside; /* recomputes whose FP64 energy fell outside the bins (an FP32
                                   rounding let the walker step just past a range edge): the
                                   running energy takes the FP64 value and the walker counts
                                   in the nearest edge bin until a move brings it back */
    uint64_t pad;
} phast_walker_stats;

/* One traced move (16 bytes). */
typedef struct {
    double dE;           /* energy change computed for the proposal (NaN: degenerate) */
    int32_t bin_after;   /* bin counted for this attempt */
    int32_t accepted;
} phast_trace;

typedef struct phast_ctx phast_ctx;

/* ---- energy (Sec. 2.1, Eq. 2 and Eq. 3) --------------------------------- */

/* Total energy of B configurations of one system.  xyz: dev [B][N][3] FP64;
 * pair_precision 32 or 64 selects the arithmetic of the Lennard-Jones pairs
 * (FP32 positions are taken relative to their chain's FP64 centroid); the
 * bending, torsion and FENE terms and all sums are FP64 (a dihedral of
 * collinear bonds is 0, a decision FP32 coordinates cannot take).  E_out: dev
 * [B].  B = 0 is a no-op. */
int phast_energy(const phast_system* sys, const phast_ff* ff, int32_t B, const double* xyz,
                 int32_t pair_precision, double* E_out, void* stream);

/* Energy change of move b applied to configuration b (Sec. 3.2 move set):
 * bending/torsion terms that the move changes plus every Lennard-Jones pair
 * (moved, unmoved) before and after.  With pair_precision 32 the local terms
 * are FP32 too, except that a dihedral with bonds within ~0.06 degrees of
 * collinear (where FP32 cannot resolve its normal, and the FP64 term of
 * collinear bonds is 0) or a FENE bond near its range makes that kind of term's
 * change FP64 on the exact positions.  moves: dev [B]; dE_out: dev [B];
 * xyz_new_out: dev [B][N][3] or NULL (receives the moved configurations).
 * A degenerate crankshaft (coincident neighbours) gives NaN. */
int phast_delta_energy(const phast_system* sys, const phast_ff* ff, int32_t B, const double* xyz,
                       const phast_move* moves, int32_t pair_precision, double* dE_out,
                       double* xyz_new_out, void* stream);

/* ---- walker context ---------------------------------------------------- */

/* Create the walker state of n_systems system types on the current device:
 * walkers[s] walkers of type s (walker indices run over type 0 first), host
 * seeds[W] (each walker's Philox4x32-10 key; walker streams are
 * counter-based: block b of move t uses counter (t_lo, t_hi, b, 0x4D554341)),
 * host xyz0 concatenated per type [walkers[s]][N_s][3].  Computes every
 * walker's FP64 energy and bin; PHAST_ERANGE if one is outside its range.
 * Allocates the device state (the caller destroys the context). */
int phast_ctx_create(phast_ctx** out, int32_t n_systems, const phast_system* sys,
                     const phast_ff* ff, const phast_muca_params* mp, const int32_t* walkers,
                     const uint64_t* seeds, const double* xyz0, void* stream);
void phast_ctx_destroy(phast_ctx* ctx);

/* Sizes: total walkers, and for system type s its N, n_bins, walker offset,
 * xyz offset (doubles) and lnW offset (the concatenated per-type layouts). */
int phast_ctx_info(const phast_ctx* ctx, int32_t s, int64_t* info8);

/* Copy walker state between the context and caller buffers (dev or host:
 * cudaMemcpyAsync with cudaMemcpyDefault).  Any pointer may be NULL. xyz:
 * concatenated per type; E [W] FP64; bin [W] int32; move index t [W] uint64;
 * stats [W]. set_state recomputes nothing: E and bin must match xyz. */
int phast_ctx_get_state(const phast_ctx* ctx, double* xyz, double* E, int32_t* bin, uint64_t* t,
                        phast_walker_stats* stats, void* stream);
int phast_ctx_set_state(phast_ctx* ctx, const double* xyz, const double* E, const int32_t* bin,
                        const uint64_t* t, const phast_walker_stats* stats, void* stream);

/* Tile shape of the batched sweep: threads per walker (1, 4, 8, 16 or 32) and
 * walkers per CTA (a whole number of warps: threads per walker x walkers per
 * CTA a multiple of 32, at most 512, or 256 with one walker per thread); 0
 * picks the default.  One thread per walker runs each walker's whole move on
 * its own thread (small systems); a group of lanes shares a walker's pair
 * loop.  phast_ctx_autotune runs each candidate on a scratch copy of the state
 * for `sweeps` sweeps, once untimed and once timed, and keeps the fastest.
 * Systems of fewer than 48 monomers run 16-lane FP32 tiles in a build held to
 * 64 registers when that fits more CTAs on an SM. */
int phast_ctx_set_tile(phast_ctx* ctx, int32_t threads_per_walker, int32_t walkers_per_cta);
int phast_ctx_get_tile(const phast_ctx* ctx, int32_t* threads_per_walker, int32_t* walkers_per_cta);
int phast_ctx_autotune(phast_ctx* ctx, const double* lnW, int32_t sweeps, void* stream);

/* ---- the multicanonical sweep (Sec. 2.2; MONTE_CARLO.f of Sec. 3.2) ------ */

enum { PHAST_FORM_BATCHED = 0, PHAST_FORM_PLAIN = 1 };

/* n_sweeps sweeps (a sweep = N_s move attempts) of every walker with the
 * tabulated log-weights lnW (dev, concatenated per type [n_bins_s]): propose
 * (Philox stream), dE from the changed terms, accept with min(1, W(E')/W(E))
 * (times ((r + delta) / r)^2 for a bond-length move, the Jacobian of its
 * radial map), count the current bin after every attempt.  Proposals out of
 * range, beyond the sphere or with non-finite dE are rejected.  Every
 * recompute_every sweeps (by each walker's own move index) the running energy
 * is replaced by an FP64 full energy, and the bin by its bin (the nearest edge
 * bin when that energy lies just outside the range; phast_walker_stats counts
 * those events).  With pair_precision 32 the local terms are FP32 except near
 * their hard edges, which the exact FP64 positions decide: the container wall,
 * a FENE bond near its range, and a dihedral of bonds within ~0.06 degrees of
 * collinear (whose FP64 term is 0 when they are collinear).  The batched form
 * has a lean build without the paper's geometry, in which such a dihedral
 * counts as collinear; a context runs it only when no system type needs the
 * geometry and no type with a torsion term starts with a bend under ~1e-5 rad
 * (a straight start).
 *  form: PHAST_FORM_BATCHED (shared-memory tiles, FP32 or FP64 pairs per
 *        mp.pair_precision) or PHAST_FORM_PLAIN (one walker per CTA, all FP64,
 *        global-memory histogram atomics; the comparison form).
 *  hist_sum: dev uint64 [sum_s n_jk * n_bins_s] or NULL; += counts summed over
 *        the walkers of jackknife block b of type s, block b holding walkers
 *        [b W_s / n_jk, (b+1) W_s / n_jk) (integer division).
 *  hist_walker: dev uint32 [sum_s W_s * n_bins_s] or NULL; += per-walker counts.
 *        A call adds n_sweeps * N_s counts per walker, so a call with
 *        n_sweeps * max_s N_s >= 2^32 is refused (PHAST_EINVAL); keeping the
 *        counts accumulated over calls below 2^32 is the caller's part.
 *  The batched form counts the walkers of a tile in a 32-bit shared-memory
 *  histogram; a bin that reaches the context's flush count (2^31 unless
 *  phast_ctx_set_hist_flush says otherwise) moves that count into hist_sum at
 *  once, so no count wraps however long the call.
 *  trace: dev [trace_walkers][n_sweeps * N] or NULL; per-move record of the
 *        first trace_walkers walkers of type 0 (walker-major).
 * Histograms are added to, never cleared. */
int phast_muca_sweep(phast_ctx* ctx, int64_t n_sweeps, const double* lnW, int32_t form,
                     int32_t n_jk, uint64_t* hist_sum, uint32_t* hist_walker,
                     phast_trace* trace, int32_t trace_walkers, void* stream);

/* The count at which a tile's 32-bit shared-memory histogram bin is moved
 * into the 64-bit hist_sum during a batched sweep: a power of two, at most
 * 2^31 (the default; 0 restores it); PHAST_EINVAL otherwise.  Whenever an
 * increment takes a bin to a multiple of it, that many counts move.  The
 * results do not depend on it: a small value only exercises the flush (a
 * testing hook). */
int phast_ctx_set_hist_flush(phast_ctx* ctx, uint32_t count);

/* ---- Berg's weight recursion (Sec. 2.2) ------------------------------- */

/* One step of the multicanonical recursion with accumulated error weights:
 * H_k = sum over n_blocks rows of hist (dev uint64 [n_blocks][K]);
 * g0_k = H_k H_{k+1} / (H_k + H_{k+1}) (0 unless both are visited),
 * ghat_k = g0_k / (g_acc_k + g0_k), g_acc_k += g0_k,
 * beta_k += ghat_k (ln H_{k+1} - ln H_k) / w with beta_k = (lnW_k - lnW_{k+1}) / w,
 * then lnW re-integrated from lnW_0 = 0.  From g_acc = 0 this is the naive
 * recursion W^{n+1} = W^n / H^n.  lnW dev [K] in/out, g_acc dev [K-1] in/out,
 * beta_out dev [K-1] or NULL, flat_out dev [4] or NULL: visited bins, mean,
 * c_Var = sigma_H / mu_H, max |H - mu_H| / mu_H (Sec. 4.1 flatness). */
int phast_weight_update(int32_t K, double bin_width, const uint64_t* hist, int32_t n_blocks,
                        double* lnW, double* g_acc, double* beta_out, double* flat_out,
                        void* stream);

/* ---- Force-field derivatives (Eq. 2/3 and the torsion term) ---------- */

/* Energy and its derivatives for a batch of B conformations of one system:
 * xyz dev FP64 [B][N][3]; E_out dev FP64 [B] or NULL; grad_xyz dev FP64
 * [B][N][3] or NULL (dE/dx, the minimum image between chains of a periodic
 * system); grad_ff dev FP64 [B][5] or NULL: dE/d(C_AA, C_BB, C_AB, kappa,
 * kappa_C) -- the Lennard-Jones coefficients of Eq. 1, the torsion weight and
 * the bending weight kappa_C of Eq. 2.  pair_precision 32: FP32 terms on
 * coordinates relative to chain centroids, FP64 sums of the energy and the
 * parameter derivatives; 64: FP64 throughout.  One warp per conformation;
 * nothing is kept between calls (a backward pass recomputes the forward one).
 * PHAST_EINVAL for bad arguments. */
int phast_energy_grad(const phast_system* sys, const phast_ff* ff, int32_t B, const double* xyz,
                      int32_t pair_precision, double* E_out, double* grad_xyz, double* grad_ff,
                      void* stream);

/* The same with the five parameters (C_AA, C_BB, C_AB, kappa, kappa_C) read
 * from params, a dev FP64 [5] array, in place of ff's values (C_AB serves AB
 * and BA): a caller that keeps the parameters on the device (a training loop)
 * needs no copy to the host.  ff supplies everything else.  PHAST_EINVAL for a
 * NULL params or the arguments phast_energy_grad refuses. */
int phast_energy_grad_params(const phast_system* sys, const phast_ff* ff, int32_t B, const double* xyz,
                             int32_t pair_precision, const double* params, double* E_out,
                             double* grad_xyz, double* grad_ff, void* stream);

/* Canonical averages from multicanonical samples (Sec. 2.2 reweighting) and
 * their derivatives in a force-field parameter lambda.  Sample q (of n) has
 * energy E[q], D[q] = dE/dlambda (e.g. a column of grad_ff) and was drawn with
 * log-weight lnW[q] (the weight of its bin), so at temperature T its
 * canonical weight is exp(-E/T - lnW) (normalised by log-sum-exp).  With
 * beta = 1/T and centred moments over those weights, per T[i]:
 *   E_T = <E>, cV_T = <(E-<E>)^2> / (N T^2)  (N = n_monomers),
 *   dE_T = d<E>/dlambda = <D> - beta <(E-<E>)(D-<D>)>,
 *   dcV_T = [2 <(E-<E>)(D-<D>)> - beta <(E-<E>)^2 (D-<D>)>] / (N T^2),
 * from d<O>/dlambda = <dO/dlambda> - beta Cov(O, D) for O = E and E^2.
 * All arrays on the device, FP64: E, D, lnW [n]; T, E_T, cV_T, dE_T, dcV_T [n_T].
 * One CTA per temperature.  PHAST_EINVAL for bad arguments. */
int phast_reweight_sensitivity(int64_t n, const double* E, const double* D, const double* lnW,
                               int32_t n_monomers, int32_t n_T, const double* T, double* E_T,
                               double* cV_T, double* dE_T, double* dcV_T, void* stream);

/* ---- One multicanonical iteration as a CUDA graph (Sec. 2.2, Fig. 2) --- */

/* Captures on `stream` one iteration of the multicanonical loop of Sec. 2.2
 * for every system type of ctx: clear hist_sum, n_sweeps sweeps of the
 * batched form (as phast_muca_sweep with the context's tile), then one step of
 * Berg's recursion per type on its rows of hist_sum (as phast_weight_update).
 * Nothing runs at capture time; each phast_graph_launch runs one more
 * iteration on the same buffers, the walkers' state carried in ctx.
 *  lnW: dev [sum_s K_s] (type s at its lnw offset, phast_ctx_info), read by the
 *       sweeps and rewritten by the step; g_acc: dev [sum_s K_s], type s at the
 *       same offset as its lnW (its last entry unused);
 *  hist_sum: dev uint64 [sum_s n_jk K_s], jackknife layout of phast_muca_sweep;
 *  flat_out: dev [n_types][4] or NULL (phast_weight_update's flatness row);
 *  stream: a created stream (the legacy default stream cannot be captured).
 * The pointers are baked into the graph: it must not outlive ctx or the
 * buffers, and must not run concurrently with other sweeps of ctx.  *out is
 * owned by the caller (phast_graph_destroy).  PHAST_EINVAL for a bad argument,
 * PHAST_ECUDA if capture or instantiation fails (*out = NULL). */
typedef struct phast_graph phast_graph;
int phast_ctx_capture_iteration(phast_ctx* ctx, int64_t n_sweeps, double* lnW, int32_t n_jk,
                                uint64_t* hist_sum, double* g_acc, double* flat_out,
                                phast_graph** out, void* stream);
/* Replays the captured iteration on `stream` (any stream, default included). */
int phast_graph_launch(phast_graph* graph, void* stream);
void phast_graph_destroy(phast_graph* graph);

/* ---- microcanonical analysis (Eq. 4-6, Sec. 3.3) ------------------------ */

/* Outputs of phast_micro_analysis (all dev pointers; any may be NULL).
 * Values from all blocks; *_err the jackknife errors over leave-one-block-out
 * replicates (n_blocks >= 2), NaN where undefined. */
typedef struct {
    double *S, *beta, *CV;               /* [K] */
    double *E_T, *cV_T;                  /* [n_T] */
    double *peak;                        /* [2]: T_peak, c_V peak */
    double *S_err, *beta_err, *CV_err;   /* [K] */
    double *E_T_err, *cV_T_err;          /* [n_T] */
    double *peak_err;                    /* [2] */
} phast_micro_out;

/* S_k = -lnW_k + ln H_k on visited bins (H from hist summed over blocks; with
 * hist = NULL, S = -lnW, the S_muca of Eq. 8), shifted to max S = 0 (Eq. 4);
 * beta_k = (S_{k+h} - S_{k-h}) / (2 h w) (Eq. 5); C_V,k = -beta_k^2 / S''_k
 * with S'' the central second difference of step h (Eq. 6); canonical
 * <E>_T and c_V(T) = var_T(E) / (n_monomers T^2) with p_k ~ exp(S_k - E_k/T),
 * E_k the bin centre; peak by a parabola through the largest c_V(T) on the
 * T grid.  T: dev [n_T].  workspace: dev, phast_micro_workspace_size() bytes. */
size_t phast_micro_workspace_size(int32_t K, int32_t n_T, int32_t n_blocks);
int phast_micro_analysis(int32_t K, double e_min, double bin_width, const double* lnW,
                         const uint64_t* hist, int32_t n_blocks, int32_t fd_half_width,
                         int32_t n_monomers, int32_t n_T, const double* T,
                         const phast_micro_out* out, void* workspace, size_t workspace_bytes,
                         void* stream);

/* Error bars by binning over iterations (Sec. 4.1: data blocks of dN
 * iterations of a range [N_S, N_E], the binning method), the alternative to
 * the jackknife over walker blocks.  lnW: dev [n_it][K], the weight tables of
 * the iterations of the range (row i = iteration N_S + i); hist: dev uint64
 * [n_it][K], each iteration's histogram summed over walkers, or NULL (S =
 * -lnW).  Each iteration is analysed alone as phast_micro_analysis does (one
 * replicate, its own weights and histogram); every observable is then averaged
 * over n_b = n_it / block consecutive blocks of `block` iterations (a
 * remainder at the end is left out).  out's values are the means of the block
 * means, its *_err fields (when not NULL) their standard error
 * sqrt(sum_b (B_b - mean)^2 / (n_b (n_b - 1))), NaN for n_b < 2; a bin that
 * any iteration of the used range leaves unvisited is NaN.  workspace: dev,
 * phast_micro_binned_workspace_size() bytes.  PHAST_EINVAL for bad arguments
 * (including n_it < block). */
size_t phast_micro_binned_workspace_size(int32_t K, int32_t n_T, int32_t n_it);
int phast_micro_analysis_binned(int32_t K, double e_min, double bin_width, const double* lnW,
                                const uint64_t* hist, int32_t n_it, int32_t block, int32_t fd_half_width,
                                int32_t n_monomers, int32_t n_T, const double* T,
                                const phast_micro_out* out, void* workspace, size_t workspace_bytes,
                                void* stream);

/* Free energy (Eq. 7) and the Maxwell construction on the caloric curve
 * (Sec. 3.3, ANALYST with Tol_Beta and Tol_L).  S_k from lnW and hist as in
 * phast_micro_analysis (shifted to max S = 0, unvisited bins skipped).  The
 * equal-area line on beta(E) is the common tangent of S(E): an edge of the
 * upper concave hull of (E_k, S_k) spanning bins below it.  Among those with a
 * positive slope (beta_c > 0) and a latent heat (E_b - E_a)/N >= tol_L, across
 * which beta_k = (S_{k+h} -
 * S_{k-h})/(2 h w) rises by >= tol_beta, the widest (the first of equal
 * width) gives beta_c (its slope),
 * eps_1 = E_a/N, eps_2 = E_b/N, the latent heat, and the barrier
 * max (hull - S) / (beta_c N) of f between the coexisting states.  beta_c > 0
 * fixes beta_c instead (no construction); 0 asks for it.
 *  f_out: dev [K] or NULL, f_k = (E_k - S_k / beta_c) / N from all blocks (NaN
 *         where S is undefined or no beta_c was found);
 *  rep: dev [(1 + R) * 6], R = n_blocks if n_blocks >= 2 (else 0): row 0 from
 *       all blocks, row r from all but block r-1; each row {beta_c, eps_1,
 *       eps_2, latent, barrier, found (1/0)};
 *  err: dev [6] or NULL: jackknife errors of row 0 over the R rows (NaN unless
 *       every row found a transition); err[5] = the number of rows that did.
 * K <= PHAST_MAX_BINS (13 bytes of shared memory per bin and CTA, 208 KB at
 * the limit).  PHAST_EINVAL for bad arguments. */
int phast_maxwell(int32_t K, double e_min, double bin_width, const double* lnW, const uint64_t* hist,
                  int32_t n_blocks, int32_t fd_half_width, int32_t n_monomers, double beta_c,
                  double tol_beta, double tol_L, double* f_out, double* rep, double* err, void* stream);

/* Allocation-free variant of phast_micro_analysis, for callers that cannot
 * allocate device memory when they run the analysis (a plug-in working inside
 * another program's CUDA context under a fixed memory budget, or code between
 * the steps of a loop that must leave the device's allocations untouched).  It
 * takes no workspace: it uses a device array of PHAST_MICRO_NOALLOC_DOUBLES
 * doubles (4 MiB) that the library reserves on every device where its module is
 * loaded and keeps until the process exits.  The paper has no counterpart; this
 * is a property of this library only.
 *  - Same arguments and results as phast_micro_analysis minus the workspace.
 *  - The call needs (1 + B) (3 K + 2 n_T + 2) doubles of that array, with B =
 *    n_blocks when n_blocks >= 2 (else 0); a larger request fails with
 *    PHAST_EINVAL and a message naming the sizes (use phast_micro_analysis).
 *    K = 8000 bins with 64 temperatures and 16 blocks fits.
 *  - The array has its own device address in each CUDA context.  The first
 *    call in a context (the device's primary context, or any context the
 *    caller has made current) looks that address up and caches it under the
 *    context's unique ID, so a context created later -- after cudaDeviceReset,
 *    say -- gets a fresh lookup.  Make the first call in each context before
 *    any stream capture.
 *  - Every call shares the one array and every element it reads is written
 *    earlier in the same call, so nothing needs clearing; calls that overlap on
 *    the GPU (other streams, other host threads) race on it.
 *  - Calls no allocating routine. */
#define PHAST_MICRO_NOALLOC_DOUBLES 524288
int phast_micro_analysis_noalloc(int32_t K, double e_min, double bin_width, const double* lnW,
                                 const uint64_t* hist, int32_t n_blocks, int32_t fd_half_width,
                                 int32_t n_monomers, int32_t n_T, const double* T,
                                 const phast_micro_out* out, void* stream);

/* ---- checkpoint --------------------------------------------------------- */

/* Serialise the walker state (coordinates, energies, bins, move indices,
 * counters) with a CRC-32 into a host buffer.  With buf = NULL, *len receives
 * the size needed.  Restore checks sizes and the CRC (PHAST_EINVAL on a
 * mismatch) and synchronises `stream`. */
int phast_ctx_checkpoint(phast_ctx* ctx, void* buf, size_t* len, void* stream);
int phast_ctx_restore(phast_ctx* ctx, const void* buf, size_t len, void* stream);

/* ---- misc --------------------------------------------------------------- */
const char* phast_last_error(void);
int phast_version(void);

#ifdef __cplusplus
}
#endif
#endif
