/*
 * oracle.h -- plain, slow FP64 CPU oracle of the PHAST multicanonical sweep.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
 * its Python binding) may include, link or call this code; only the tests, the
 * package's smoke check and the benchmark's CPU-baseline leg use it.  It shares
 * no header, helper, table or constant with the CUDA path.
 *
 * Paper: R. B. Frigori, "PHAST: Protein-like heteropolymer analysis by
 * statistical thermodynamics" (arXiv 1702.01770).  Equations are numbered in
 * order of appearance: Eq. 1 C_LJ (Sec. 2.1), Eq. 2 H_single (Sec. 2.1),
 * Eq. 3 H_multi (Sec. 2.1), Eq. 4 S = k_B ln Omega, Eq. 5 beta(E),
 * Eq. 6 C_V(E), Eq. 7 F(E), Eq. 8 S_muca (all Sec. 2.2).
 *
 * Readings of the paper that the text leaves open are listed, one per item,
 * beside the function that takes them.  Everything is FP64 and single-threaded
 * per call; the library is built with -ffp-contract=off so that no a*b+c is
 * fused behind the reader's back.
 */
#ifndef PHAST_ORACLE_H
#define PHAST_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_CHAINS 64

/* The force field of Eq. 2/3 in the AB limit (kappa_F = 0, bonds fixed at
 * r0 = 1, Sec. 4 footnote) plus a torsion term -k_tors * sum cos(tau). */
typedef struct {
    int n_chains;
    const int32_t* chain_len;     /* [n_chains], each >= 3 */
    const uint8_t* seq;           /* [N_tot], 0 = A, 1 = B */
    double box_L;                 /* > 0: periodic cube, minimum image between chains; 0: open */
    double k_bend;                /* kappa_C */
    double k_tors;                /* kappa (torsion weight; energy is -kappa * sum cos tau) */
    double k_lj_intra;            /* kappa_LJ_INTRA */
    double k_lj_inter;            /* kappa_LJ_INTER */
    double C[4];                  /* C_LJ(s_i, s_j) at index 2*s_i + s_j (Eq. 1) */
    double sphere_R;              /* > 0: steric spherical container about the origin (hard wall) */
    double k_fene, fene_r0, fene_R;   /* FENE bond term of Eq. 2 (k_fene = 0: AB limit, rigid bonds) */
    double C_F[4];                /* C_F(s_l, s_{l+1}) at index 2*s_l + s_{l+1} */
} orc_model;

/* Multicanonical set-up: energy bins, move mix and step sizes. */
typedef struct {
    double e_min, bin_width;
    int32_t n_bins;
    double p[6];                  /* probabilities of pivot, translation, rotation, crankshaft,
                                     bond-length change, spherical cap */
    double amax[6];               /* pivot angle, translation step, rotation angle, crank angle,
                                     bond-length step, cap angle */
    int32_t recompute_every;      /* full FP64 energy every this many sweeps (0 = never) */
} orc_muca;

enum { ORC_PIVOT = 0, ORC_TRANS = 1, ORC_ROT = 2, ORC_CRANK = 3, ORC_BOND = 4, ORC_CAP = 5 };

typedef struct {
    int32_t type, chain, index, pad;
    double axis[3];
    double angle;
    double disp[3];
} orc_move;

/* Per-move record of a sweep (for lockstep comparison with another sampler). */
typedef struct {
    double dE;          /* energy change of the proposal (NaN if the move is degenerate) */
    double E_after;     /* running energy after the decision */
    int32_t bin_after;  /* histogram bin counted for this attempt */
    int32_t accepted;   /* 1 accepted, 0 rejected */
} orc_record;

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): out = philox(ctr, key). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Total energy, Eq. 2 summed per chain plus the inter-chain sum of Eq. 3;
 * +inf if a monomer is outside the spherical container or a bond outside the
 * FENE range.  terms (nullable) receives {bend, torsion, lj_intra, lj_inter,
 * fene}. */
double orc_energy(const orc_model* m, const double* xyz, double* terms);

/* Draw move number t of the walker with key `seed` (see orc_propose in the .c). */
void orc_propose(const orc_model* m, const orc_muca* mu, uint64_t seed, uint64_t t,
                 orc_move* mv, double* u_acc);

/* New coordinates of the moved monomers; xyz_new is a full copy of xyz with the
 * move applied.  Returns the number of moved monomers, 0 if degenerate. */
int orc_apply_move(const orc_model* m, const orc_move* mv, const double* xyz, double* xyz_new);

/* Hastings factor J of the move from xyz (1 except for bond-length moves). */
double orc_move_jacobian(const orc_model* m, const double* xyz, const orc_move* mv);

/* Energy change of the move by its affected terms only. */
double orc_delta_energy(const orc_model* m, const double* xyz, const orc_move* mv, double* xyz_new);

/* Magnitude of the terms a move changes (sum of absolute values before and
 * after): the scale for judging a reduced-precision dE. */
double orc_delta_scale(const orc_model* m, const double* xyz, const orc_move* mv);

/* Number of pair evaluations a move costs under the pair-evaluation count
 * defined in orc_pair_evals (.c). */
int64_t orc_pair_evals(const orc_model* m, const orc_move* mv);

/* Bin of energy E, or -1 if out of [e_min, e_min + n_bins * bin_width). */
int32_t orc_bin(const orc_muca* mu, double E);

/* One walker: run n_moves attempts starting at move index *t.  State: xyz
 * (in/out), *E, *bin, *t.  hist[n_bins] (uint64, in/out) gets +1 per attempt.
 * force (nullable, [n_moves]): -1 = own decision, 0/1 = impose this decision
 * (used to replay another sampler's trajectory).  rec (nullable, [n_moves]).
 * stats (nullable, [16]): attempts[6], accepts[6], pair_evals, n_recompute,
 * drift_max (as double bits), own_vs_forced_mismatches.
 * Returns 0, or -1 if the walker state is invalid (E out of range). */
int orc_sweep_walker(const orc_model* m, const orc_muca* mu, const double* lnW,
                     uint64_t seed, int64_t n_moves,
                     double* xyz, double* E, int32_t* bin, uint64_t* t,
                     uint64_t* hist, const int8_t* force, orc_record* rec, double* stats);

/* Berg's multicanonical recursion with accumulated error weights, one step.
 * H[K] histogram summed over walkers, lnW[K] in/out, g_acc[K-1] in/out.
 * flat_out[4] (nullable): n_visited, mean, c_Var, max |H-mean|/mean over visited bins. */
void orc_berg_update(int32_t K, double bin_width, const double* H, double* lnW,
                     double* g_acc, double* flat_out);

/* Microcanonical analysis, Eq. 4-6, plus canonical reweighting.
 * lnW[K]; Hb[n_blocks][K] (nullable: S from weights alone);
 * outputs S[K], beta[K], CV[K] (NaN where undefined), E_T[n_T], cV_T[n_T]
 * (c_V per monomer), peak[2] = {T_peak, cV_peak}. */
void orc_micro_analysis(int32_t K, double e_min, double bin_width, const double* lnW,
                        const double* H, int32_t fd_half_width, int32_t n_monomers,
                        int32_t n_T, const double* T,
                        double* S, double* beta, double* CV,
                        double* E_T, double* cV_T, double* peak);

/* Jackknife error (Sec. 4.1, error bars from data blocks) of an estimate from
 * its n leave-one-block-out replicates: rep [n][m], err [m] =
 * sqrt((n-1)/n sum_b (rep[b] - mean)^2) per column; NaN for n < 2. */
void orc_jackknife(int32_t n, int32_t m, const double* rep, double* err);

/* Binning over iterations (Sec. 4.1): rows i < n_it of lnW and H (nullable)
 * analysed one by one, each observable averaged over n_it / block blocks of
 * `block` consecutive iterations; values = mean of the block means, errors =
 * their standard error (NaN with fewer than 2 blocks). */
void orc_micro_binned(int32_t K, double e_min, double bin_width, const double* lnW, const double* H,
                      int32_t n_it, int32_t block, int32_t h, int32_t n_monomers, int32_t n_T, const double* T,
                      double* S, double* beta, double* CV, double* E_T, double* cV_T, double* peak,
                      double* S_err, double* beta_err, double* CV_err, double* E_T_err, double* cV_T_err,
                      double* peak_err);

/* Energy (returned) and its derivatives: gx [N*3] (nullable) with respect to
 * the coordinates, gp [5] (nullable) with respect to (C_AA, C_BB, C_AB, kappa,
 * kappa_C), each term of Eq. 2/3 and the torsion term differentiated by hand. */
double orc_energy_grad(const orc_model* m, const double* xyz, double* gx, double* gp);

/* Canonical <E>, c_V (per monomer) and their derivatives in a parameter lambda
 * at temperatures T[n_T], reweighted from n multicanonical samples with
 * energies E, derivatives D = dE/dlambda and sampling log-weights lnW. */
void orc_reweight_sensitivity(int64_t n, const double* E, const double* D, const double* lnW, int32_t n_monomers,
                              int32_t n_T, const double* T, double* E_T, double* cV_T, double* dE_T, double* dcV_T);

/* Free energy f_k = (E_k - S_k / beta_c) / N (Eq. 7, per monomer) and the
 * Maxwell construction on the caloric curve (see orc_maxwell in the .c for the
 * reading).  S [K] with NaN on unvisited bins; beta_c_in > 0 fixes beta_c (no
 * construction), 0 asks for it.  res[6] = {beta_c, eps_1, eps_2, latent heat,
 * barrier, found}; f_out [K] nullable. */
void orc_maxwell(int32_t K, double e_min, double bin_width, const double* S, int32_t n_monomers,
                 int32_t fd_half_width, double beta_c_in, double tol_beta, double tol_L, double* f_out,
                 double* res);

#ifdef __cplusplus
}
#endif
#endif
