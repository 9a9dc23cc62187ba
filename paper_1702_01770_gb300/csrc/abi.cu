// abi.cu -- host-side pieces of the C ABI: thread-local error messages,
// validation of the system / force-field / MUCA structs and their flattening
// into device descriptors, version.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "common.cuh"

static thread_local char g_err[512] = "";

int phast_set_error(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

extern "C" const char* phast_last_error(void) { return g_err; }
extern "C" int phast_version(void) { return PHAST_VERSION; }

int phast_build_desc(const phast_system* sys, const phast_ff* ff, const phast_muca_params* mp,
                     SysDesc* d, const char* what) {
    memset(d, 0, sizeof(*d));
    if (!sys || !ff) return phast_set_error(PHAST_EINVAL, "%s: NULL system or force field", what);
    if (sys->n_chains < 1 || sys->n_chains > PHAST_MAX_CHAINS)
        return phast_set_error(PHAST_EINVAL, "%s: n_chains %d outside [1, %d]", what, sys->n_chains,
                               PHAST_MAX_CHAINS);
    if (!sys->chain_len || !sys->seq)
        return phast_set_error(PHAST_EINVAL, "%s: NULL chain_len or seq", what);
    int N = 0, maxc = 0;
    for (int c = 0; c < sys->n_chains; ++c) {
        int n = sys->chain_len[c];
        if (n < 3) return phast_set_error(PHAST_EINVAL, "%s: chain %d has %d < 3 monomers", what, c, n);
        if (N + n > PHAST_MAX_MONOMERS)
            return phast_set_error(PHAST_EINVAL, "%s: more than %d monomers", what, PHAST_MAX_MONOMERS);
        d->chain_off[c] = N;
        for (int j = 0; j < n; ++j) {
            uint8_t s = sys->seq[N + j];
            if (s > 1) return phast_set_error(PHAST_EINVAL, "%s: sequence value %d not 0 (A) or 1 (B)", what, s);
            d->seq[N + j] = s;
            d->chain_of[N + j] = (uint8_t)c;
        }
        N += n;
        if (n > maxc) maxc = n;
    }
    d->chain_off[sys->n_chains] = N;
    d->n_a_before[0] = 0;
    for (int j = 0; j < N; ++j) d->n_a_before[j + 1] = (uint16_t)(d->n_a_before[j] + (d->seq[j] == 0));
    d->n_chains = sys->n_chains;
    d->N = N;
    d->max_chain = maxc;
    if (!(sys->box_L >= 0.0) || !isfinite(sys->box_L))
        return phast_set_error(PHAST_EINVAL, "%s: box_L must be finite and >= 0", what);
    d->box_L = sys->box_L;
    d->inv_L = sys->box_L > 0.0 ? 1.0 / sys->box_L : 0.0;
    if (!(sys->sphere_R >= 0.0) || !isfinite(sys->sphere_R))
        return phast_set_error(PHAST_EINVAL, "%s: sphere_R must be finite and >= 0", what);
    if (sys->sphere_R > 0.0 && sys->box_L > 0.0)
        return phast_set_error(PHAST_EINVAL, "%s: a spherical container and a periodic box exclude each other", what);
    d->sphere_R2 = sys->sphere_R * sys->sphere_R;
    d->has_sphere = sys->sphere_R > 0.0;
    d->sphere_R2_32 = (float)d->sphere_R2;
    d->k_bend = ff->k_bend;
    d->k_tors = ff->k_tors;
    d->k_lj_intra = ff->k_lj_intra;
    d->k_lj_inter = ff->k_lj_inter;
    for (int i = 0; i < 4; ++i) d->C[i] = ff->C[i];
    for (int i = 0; i < 4; ++i)
        if (!isfinite(d->C[i])) return phast_set_error(PHAST_EINVAL, "%s: non-finite coupling", what);
    if (!isfinite(d->k_bend) || !isfinite(d->k_tors) || !isfinite(d->k_lj_intra) || !isfinite(d->k_lj_inter))
        return phast_set_error(PHAST_EINVAL, "%s: non-finite force-field weight", what);
    d->k_fene = ff->k_fene;
    d->fene_r0 = ff->fene_r0;
    d->fene_R = ff->fene_R;
    for (int i = 0; i < 4; ++i) d->C_F[i] = ff->C_F[i];
    if (!isfinite(d->k_fene)) return phast_set_error(PHAST_EINVAL, "%s: non-finite k_fene", what);
    if (d->k_fene != 0.0) {
        if (!(d->fene_R > 0.0) || !isfinite(d->fene_R) || !(d->fene_r0 > 0.0) || !isfinite(d->fene_r0))
            return phast_set_error(PHAST_EINVAL, "%s: the FENE term needs finite fene_r0 > 0 and fene_R > 0", what);
        for (int i = 0; i < 4; ++i)
            if (!isfinite(d->C_F[i])) return phast_set_error(PHAST_EINVAL, "%s: non-finite C_F", what);
    }
    d->fene_kR2 = d->k_fene * (d->fene_R * d->fene_R);
    d->fene_r0_32 = (float)d->fene_r0;
    d->fene_iR32 = d->k_fene != 0.0 ? (float)(1.0 / d->fene_R) : 0.0f;
    d->fene_kR2_32 = (float)d->fene_kR2;
    for (int i = 0; i < 4; ++i) d->C_F32[i] = (float)d->C_F[i];
    for (int i = 0; i < 4; ++i) d->C32[i] = (float)d->C[i];
    d->L32 = (float)d->box_L;
    d->iL32 = (float)d->inv_L;
    d->kin32 = (float)d->k_lj_intra;
    d->kout32 = (float)d->k_lj_inter;
    d->kbend32 = (float)d->k_bend;
    d->ktors32 = (float)d->k_tors;
    d->pair_precision = 64;
    if (mp) {
        if (!(mp->bin_width > 0.0) || !isfinite(mp->e_min) || !isfinite(mp->bin_width))
            return phast_set_error(PHAST_EINVAL, "%s: bins need finite e_min and bin_width > 0", what);
        if (mp->n_bins < 1 || mp->n_bins > PHAST_MAX_BINS)
            return phast_set_error(PHAST_EINVAL, "%s: n_bins %d outside [1, %d]", what, mp->n_bins,
                                   PHAST_MAX_BINS);
        if (mp->recompute_every < 0)
            return phast_set_error(PHAST_EINVAL, "%s: recompute_every < 0", what);
        if (mp->pair_precision != 32 && mp->pair_precision != 64)
            return phast_set_error(PHAST_EINVAL, "%s: pair_precision must be 32 or 64", what);
        double sum = 0.0;
        for (int i = 0; i < PHAST_N_MOVES; ++i) {
            if (!(mp->p[i] >= 0.0)) return phast_set_error(PHAST_EINVAL, "%s: negative move probability", what);
            sum += mp->p[i];
        }
        if ((mp->p[PHAST_BOND] > 0.0 || mp->p[PHAST_CAP] > 0.0) && d->k_fene == 0.0)
            return phast_set_error(PHAST_EINVAL,
                                   "%s: bond-length and spherical-cap moves change bond lengths and need k_fene != 0", what);
        if (fabs(sum - 1.0) > 1e-9) return phast_set_error(PHAST_EINVAL, "%s: move probabilities sum to %.17g", what, sum);
        for (int i = 0; i < PHAST_N_MOVES; ++i) {
            if (!(mp->amax[i] >= 0.0) || !isfinite(mp->amax[i]))
                return phast_set_error(PHAST_EINVAL, "%s: amplitude %d must be finite and >= 0", what, i);
            if (i != PHAST_TRANS && i != PHAST_BOND && mp->amax[i] > PHAST_MAX_ANGLE)
                return phast_set_error(PHAST_EINVAL, "%s: rotation amplitude %g > %g rad", what, mp->amax[i],
                                       PHAST_MAX_ANGLE);
        }
        d->e_min = mp->e_min;
        d->bin_width = mp->bin_width;
        d->n_bins = mp->n_bins;
        d->recompute_every = mp->recompute_every;
        for (int i = 0; i < PHAST_N_MOVES; ++i) { d->p[i] = mp->p[i]; d->amax[i] = mp->amax[i]; }
        // integer move-type thresholds: u < cum_i  <=>  2n + 1 < ceil(cum_i 2^53) for u = (n + 1/2) 2^-52
        double cum = 0.0;
        d->last_type = 0;
        d->type_mask = 0;
        for (int i = 0; i < PHAST_N_MOVES; ++i) {
            cum = cum + mp->p[i];
            d->thr[i] = (uint64_t)ceil(cum * 9007199254740992.0);
            if (mp->p[i] > 0.0) { d->last_type = i; d->type_mask |= 1 << i; }
        }
        d->pair_precision = mp->pair_precision;
        for (int i = 0; i < PHAST_N_MOVES; ++i) d->amax32[i] = (float)mp->amax[i];
        d->iw32 = (float)(1.0 / mp->bin_width);
    }
    return PHAST_OK;
}
